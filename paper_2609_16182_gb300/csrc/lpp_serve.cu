// lpp_serve.cu -- the serving loop: continuous batching of presolve rounds.
//
// A server owns one arena (an Engine allocated once from the HBM budget) and
// a worker thread.  Every tick of the worker:
//   1. admits queued LPs, oldest first, while the arena's row / column /
//      nonzero capacity, the record space and a free slot allow: each is
//      checked, transposed and appended behind the LPs already resident;
//   2. runs ONE presolve round over every resident LP (Engine::step), each LP
//      counting rounds from its own admission;
//   3. hands finished LPs (no change in the round, a verdict, or the round
//      cap) to their tickets: their reduced LP is copied out of the arena and
//      they leave it at the next compaction.
// A row's or column's arithmetic never depends on the other LPs in the arena,
// so every LP gets the result lpp_presolve gives it alone.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "lpp_engine.h"
#include "ranges.h"

namespace lpp {

namespace {

__global__ void k_set_slot(int32_t *verdict, int32_t *round0, uint8_t *retired, double *offset, uint8_t *dropped_dev,
                           int32_t slot, int32_t r0, double off) {
    if (threadIdx.x < V_SLOTS) verdict[slot * V_SLOTS + threadIdx.x] = kNone;
    if (threadIdx.x == 0) {
        round0[slot] = r0;
        retired[slot] = 0;
        offset[slot] = off;
        (void)dropped_dev;
    }
}

struct AppendArgs {
    // the LP (checked, vectors already normalised into the arena)
    const int32_t *rp, *ci, *tp, *ti;
    const double *rv, *tv;
    int32_t m, n, nnz;
    // where it goes
    int32_t m0, n0, z0;  // arena sizes before the append
    int32_t rbase, cbase, slot;
    int32_t *a_rp, *a_ci, *a_tp, *a_ti, *a_rmap, *a_cmap, *a_lprow, *a_lpcol, *rec_rk, *rec_rr, *rec_ra, *rec_ck,
        *rec_cr;
    double *a_rv, *a_tv, *rec_rv, *rec_cv;
    uint8_t *a_rdirty;
};

__global__ void k_append(AppendArgs a) {
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = t0; i <= a.m; i += step) {
        a.a_rp[a.m0 + i] = a.z0 + a.rp[i];
        if (i < a.m) {
            a.a_rmap[a.m0 + i] = a.rbase + (int32_t)i;
            a.a_lprow[a.m0 + i] = a.slot;
            a.a_rdirty[a.m0 + i] = 1;
            a.rec_rk[a.rbase + i] = 0;
            a.rec_rr[a.rbase + i] = 0;
            a.rec_ra[a.rbase + i] = -1;
            a.rec_rv[a.rbase + i] = 0.0;
        }
    }
    for (int64_t j = t0; j <= a.n; j += step) {
        a.a_tp[a.n0 + j] = a.z0 + a.tp[j];
        if (j < a.n) {
            a.a_cmap[a.n0 + j] = a.cbase + (int32_t)j;
            a.a_lpcol[a.n0 + j] = a.slot;
            a.rec_ck[a.cbase + j] = 0;
            a.rec_cr[a.cbase + j] = 0;
            a.rec_cv[a.cbase + j] = 0.0;
        }
    }
    for (int64_t e = t0; e < a.nnz; e += step) {
        a.a_ci[a.z0 + e] = a.n0 + a.ci[e];
        a.a_rv[a.z0 + e] = a.rv[e];
        a.a_ti[a.z0 + e] = a.m0 + a.ti[e];
        a.a_tv[a.z0 + e] = a.tv[e];
    }
}

// per-slot first / last row and column of the arena (LPs are contiguous)
__global__ void k_bounds(const int32_t *lp, int32_t cnt, int32_t *first, int32_t *last) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int32_t k = lp[i];
    if (i == 0 || lp[i - 1] != k) first[k] = (int32_t)i;
    if (i == cnt - 1 || lp[i + 1] != k) last[k] = (int32_t)i + 1;
}

struct ExtractArgs {
    int32_t r0, mr, c0, nc, z0, nz, rbase, cbase, m0, n0, a0, na;
    const int32_t *rp, *ci, *tp, *ti, *rmap, *cmap, *act_rmap_src;
    const double *rv, *tv, *L, *U, *c;
    const double2 *lu, *act_src;
    const int2 *ninf_src;
    const int32_t *rec_rk, *rec_rr, *rec_ra, *rec_ck, *rec_cr;
    const double *rec_rv, *rec_cv;
    // outputs
    int32_t *o_rp, *o_ci, *o_tp, *o_ti, *o_rmap, *o_cmap, *o_rk, *o_rr, *o_ra, *o_ck, *o_cr, *o_dcmap, *o_armap;
    double *o_rv, *o_tv, *o_L, *o_U, *o_lb, *o_ub, *o_c, *o_rv2, *o_cv2;
    double2 *o_lu, *o_act;
    int2 *o_ninf;
};

__global__ void k_extract(ExtractArgs a) {
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = t0; i <= a.mr; i += step) {
        a.o_rp[i] = a.rp[a.r0 + i] - a.rp[a.r0];
        if (i < a.mr) {
            a.o_L[i] = a.L[a.r0 + i];
            a.o_U[i] = a.U[a.r0 + i];
            a.o_rmap[i] = a.rmap[a.r0 + i] - a.rbase;
        }
    }
    for (int64_t j = t0; j <= a.nc; j += step) {
        a.o_tp[j] = a.tp[a.c0 + j] - a.tp[a.c0];
        if (j < a.nc) {
            const double2 b = a.lu[a.c0 + j];
            a.o_lb[j] = b.x;
            a.o_ub[j] = b.y;
            a.o_lu[j] = b;
            a.o_c[j] = a.c[a.c0 + j];
            a.o_cmap[j] = a.cmap[a.c0 + j] - a.cbase;
            a.o_dcmap[j] = a.cmap[a.c0 + j] - a.cbase;
        }
    }
    for (int64_t e = t0; e < a.nz; e += step) {
        a.o_ci[e] = a.ci[a.z0 + e] - a.c0;
        a.o_rv[e] = a.rv[a.z0 + e];
        a.o_ti[e] = a.ti[a.z0 + e] - a.r0;
        a.o_tv[e] = a.tv[a.z0 + e];
    }
    for (int64_t i = t0; i < a.m0; i += step) {  // records, aux made local
        const int32_t k = a.rec_rk[a.rbase + i];
        const int32_t x = a.rec_ra[a.rbase + i];
        a.o_rk[i] = k;
        a.o_rr[i] = a.rec_rr[a.rbase + i];
        a.o_ra[i] = x < 0 ? -1 : (k == RK_SINGLETON ? x - a.cbase : x - a.rbase);
        a.o_rv2[i] = a.rec_rv[a.rbase + i];
    }
    for (int64_t j = t0; j < a.n0; j += step) {
        a.o_ck[j] = a.rec_ck[a.cbase + j];
        a.o_cr[j] = a.rec_cr[a.cbase + j];
        a.o_cv2[j] = a.rec_cv[a.cbase + j];
    }
    for (int64_t i = t0; i < a.na; i += step) {  // last round's activities
        a.o_act[i] = a.act_src[a.a0 + i];
        a.o_ninf[i] = a.ninf_src[a.a0 + i];
        a.o_armap[i] = a.act_rmap_src[a.a0 + i] - a.rbase;
    }
}

unsigned grid_for(int64_t cnt) {
    const int64_t b = (cnt + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

// ---------------------------------------------------------- engine additions
void Engine::init_empty() {
    fill_u64(cand_l, n0, kEncNegInf, s);
    fill_u64(cand_u, n0, kEncPosInf, s);
    LPP_CUDA(cudaMemsetAsync(ctouch, 0, sizeof(uint32_t) * (size_t)std::max(n0, 1), s));
    fill_u64(mL, m0, kEncNegInf, s);
    fill_u64(mU, m0, kEncPosInf, s);
    LPP_CUDA(cudaMemsetAsync(hasf, 0, (size_t)std::max(m0, 1), s));
    LPP_CUDA(cudaMemsetAsync(rwork, 0, (size_t)std::max(m0, 1), s));
    fill_i32(verdict, (int64_t)nlp * V_SLOTS, kNone, s);
    LPP_CUDA(cudaMemsetAsync(K.offset, 0, sizeof(double) * (size_t)nlp, s));
    lp_round0_dev = pool.alloc<int32_t>(nlp);
    lp_retired_dev = pool.alloc<uint8_t>(nlp);
    LPP_CUDA(cudaMemsetAsync(lp_round0_dev, 0, sizeof(int32_t) * (size_t)nlp, s));
    LPP_CUDA(cudaMemsetAsync(lp_retired_dev, 0, (size_t)nlp, s));
    K.lp_retired = lp_retired_dev;
    lp_dropped.assign(nlp, 1);
    m = n = 0;
    nnz = 0;
    cur = 0;
    LPP_CUDA(cudaMemsetAsync(rp[0], 0, sizeof(int32_t), s));
    LPP_CUDA(cudaMemsetAsync(tp[0], 0, sizeof(int32_t), s));
    LPP_CUDA(cudaMemsetAsync(&st->m_new, 0, sizeof(int32_t) * 2, s));  // m_new, n_new
    schedule_current();
    read_status();
    adopt_schedule();
}

void Engine::append(int32_t slot, const lpp_lp &in, int32_t rbase, int32_t cbase, int32_t round0) {
    const int32_t ml = in.m, nl = in.n, zl = (int32_t)in.nnz;
    DevPool tmp;  // staging of a host request: freed stream-ordered
    tmp.s = s;
    tmp.cache = false;
    const int32_t *rp_in = in.row_ptr, *ci_in = in.col_idx;
    const double *rv_in = in.val;
    const double *lhs = in.lhs, *rhs = in.rhs, *lb = in.lb, *ub = in.ub, *cc = in.c;
    if (!in.on_device) {
        int32_t *d_rp = tmp.alloc<int32_t>((size_t)ml + 1), *d_ci = tmp.alloc<int32_t>(zl);
        double *d_rv = tmp.alloc<double>(zl), *d_vec = tmp.alloc<double>(2 * (size_t)ml + 3 * (size_t)nl);
        auto up = [&](void *d, const void *h, size_t b) {
            if (b) LPP_CUDA(cudaMemcpyAsync(d, h, b, cudaMemcpyHostToDevice, s));
        };
        up(d_rp, in.row_ptr, 4 * ((size_t)ml + 1));
        up(d_ci, in.col_idx, 4 * (size_t)zl);
        up(d_rv, in.val, 8 * (size_t)zl);
        up(d_vec, in.lhs, 8 * (size_t)ml);
        up(d_vec + ml, in.rhs, 8 * (size_t)ml);
        up(d_vec + 2 * ml, in.lb, 8 * (size_t)nl);
        up(d_vec + 2 * ml + nl, in.ub, 8 * (size_t)nl);
        up(d_vec + 2 * ml + 2 * nl, in.c, 8 * (size_t)nl);
        rp_in = d_rp;
        ci_in = d_ci;
        rv_in = d_rv;
        lhs = d_vec;
        rhs = d_vec + ml;
        lb = d_vec + 2 * ml;
        ub = d_vec + 2 * ml + nl;
        cc = d_vec + 2 * ml + 2 * nl;
    }
    // checks (S0) and normalised vectors straight into the arena tail
    LPP_CUDA(cudaMemsetAsync(&st->err, 0, sizeof(int32_t), s));
    int32_t *row_of = tmp.alloc<int32_t>((size_t)zl + 1);
    int32_t *stmp = tmp.alloc<int32_t>(scan_tmp_elems(std::max<int64_t>({(int64_t)zl + 1, (int64_t)nl + 1, (int64_t)transpose_hist_elems(zl)})));
    check_csr(rp_in, ci_in, rv_in, ml, nl, zl, row_of, stmp, &st->err, s);
    ingest_vectors(lhs, rhs, lb, ub, cc, ml, nl, o.huge, L[cur] + m, U[cur] + m, lu[cur] + n, c[cur] + n, &st->err,
                   s);
    LPP_CUDA(cudaGetLastError());
    read_status();
    if (st_h->err) throw StatusError(LPP_ERR_INVALID, "invalid LP");
    // A^T of the new LP, then both matrices appended behind the arena
    TransposeBufs tb;
    tb.k0 = tmp.alloc<uint32_t>(zl);
    tb.k1 = tmp.alloc<uint32_t>(zl);
    tb.v0 = tmp.alloc<int32_t>(zl);
    tb.v1 = tmp.alloc<int32_t>(zl);
    tb.hist = tmp.alloc<int32_t>(transpose_hist_elems(zl));
    tb.tmp = stmp;
    int32_t *ttp = tmp.alloc<int32_t>((size_t)nl + 1), *tti = tmp.alloc<int32_t>(zl);
    double *ttv = tmp.alloc<double>(zl);
    transpose(rp_in, ci_in, rv_in, row_of + 1, ml, nl, zl, tb, ttp, tti, ttv, s);
    AppendArgs a;
    a.rp = rp_in;
    a.ci = ci_in;
    a.rv = rv_in;
    a.tp = ttp;
    a.ti = tti;
    a.tv = ttv;
    a.m = ml;
    a.n = nl;
    a.nnz = zl;
    a.m0 = m;
    a.n0 = n;
    a.z0 = (int32_t)nnz;
    a.rbase = rbase;
    a.cbase = cbase;
    a.slot = slot;
    a.a_rp = rp[cur];
    a.a_ci = ci[cur];
    a.a_tp = tp[cur];
    a.a_ti = ti[cur];
    a.a_rmap = rmap[cur];
    a.a_cmap = cmap[cur];
    a.a_lprow = lprow[cur];
    a.a_lpcol = lpcol[cur];
    a.rec_rk = rec_rk;
    a.rec_rr = rec_rr;
    a.rec_ra = rec_ra;
    a.rec_ck = rec_ck;
    a.rec_cr = rec_cr;
    a.a_rv = rv[cur];
    a.a_tv = tv[cur];
    a.rec_rv = rec_rv;
    a.rec_cv = rec_cv;
    a.a_rdirty = rdirty[cur];
    (k_append<<<grid_for(std::max<int64_t>({(int64_t)ml + 1, (int64_t)nl + 1, (int64_t)zl})), 256, 0, s>>>(a), note_launch());
    (k_set_slot<<<1, 32, 0, s>>>(verdict, lp_round0_dev, lp_retired_dev, K.offset, nullptr, slot, round0,
                                 in.obj_offset), note_launch());
    LPP_CUDA(cudaGetLastError());
    m += ml;
    n += nl;
    nnz += zl;
    lp_dropped[slot] = 0;
    LPP_CUDA(cudaStreamSynchronize(s));  // temporaries and host inputs outlive their use
}

void Engine::reschedule() {
    k_sizes_set(m, n);
    schedule_current();
    read_status();
    adopt_schedule();
}

}  // namespace lpp

using namespace lpp;

// ================================================================== server
struct lpp_server {
    Engine E;
    lpp_opts o{};
    size_t budget = 0;
    int32_t m_cap = 0, n_cap = 0, slots = 0;
    int64_t nnz_cap = 0;
    std::thread worker;
    std::mutex mu;
    std::mutex submit_mu;                 // one device copy of a request at a time
    cudaStream_t submit_stream = nullptr; // non-blocking: copies do not wait for the rounds
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::string fatal;
    uint64_t next_ticket = 1;
    struct Req {
        uint64_t ticket;
        lpp_lp lp;  // pointers into the owned copies below
        std::vector<int32_t> h_i;
        std::vector<double> h_d;
        void *dev = nullptr;  // device copy (device inputs)
        double t_submit;
    };
    std::deque<Req *> queue;
    struct Done {
        lpp_status st;
        lpp_reduced *red;
        lpp_postsolve *rec;
    };
    std::unordered_map<uint64_t, Done> done;
    struct Slot {
        bool used = false, retired = false;
        uint64_t ticket = 0;
        int32_t round0 = 0, rbase = 0, cbase = 0, m0 = 0, n0 = 0;
        int64_t nnz0 = 0, nnz_proc = 0, last_nnz = 0;
        double t_submit = 0, ms = 0;
    };
    std::vector<Slot> sl;
    Ranges rec_rows, rec_cols;
    lpp_server_stats stats{};
    int32_t tick = 0;
};

namespace {

void free_req(lpp_server::Req *q, cudaStream_t s) {
    if (q->dev) cudaFreeAsync(q->dev, s);
    delete q;
}

// device bytes of the arena per unit (both buffers of every array)
constexpr double kBytesNnz = 2 * 24 + 32;     // CSR + CSC twice, chunk partials, transpose room
constexpr double kBytesRow = 260;              // rows: sides, maps, results, flags, hash table, scans
constexpr double kBytesCol = 160;              // columns: bounds, costs, maps, candidates, scans

void finish_slot(lpp_server *S, int32_t k, const std::vector<int32_t> &rng, const std::vector<int32_t> &arng,
                 const std::vector<double> &offs) {
    Engine &E = S->E;
    lpp_server::Slot &Z = S->sl[k];
    const int32_t nl = E.nlp;
    const int32_t r0 = rng[k] < 0 ? 0 : rng[k], r1 = rng[nl + k] < 0 ? 0 : rng[nl + k];
    const int32_t c0 = rng[2 * nl + k] < 0 ? 0 : rng[2 * nl + k], c1 = rng[3 * nl + k] < 0 ? 0 : rng[3 * nl + k];
    const int32_t z0 = rng[4 * nl + k], z1 = rng[5 * nl + k];
    const int32_t a0 = arng[k] < 0 ? 0 : arng[k], a1 = arng[nl + k] < 0 ? 0 : arng[nl + k];
    const int32_t mr = r1 - r0, nc = c1 - c0, nz = z1 - z0, na = a1 - a0;
    auto *R = new lpp_reduced();
    auto D = std::make_shared<DeviceRecords>();
    auto own = [&](size_t bytes, std::vector<void *> &into) {
        void *p = nullptr;
        LPP_CUDA(cudaMallocAsync(&p, bytes ? bytes : 1, E.s));
        into.push_back(p);
        return p;
    };
    ExtractArgs a;
    std::memset(&a, 0, sizeof a);
    a.r0 = r0;
    a.mr = mr;
    a.c0 = c0;
    a.nc = nc;
    a.z0 = z0;
    a.nz = nz;
    a.rbase = Z.rbase;
    a.cbase = Z.cbase;
    a.m0 = Z.m0;
    a.n0 = Z.n0;
    a.a0 = a0;
    a.na = na;
    const int c = E.cur;
    a.rp = E.rp[c];
    a.ci = E.ci[c];
    a.tp = E.tp[c];
    a.ti = E.ti[c];
    a.rmap = E.rmap[c];
    a.cmap = E.cmap[c];
    a.act_rmap_src = E.rmap[E.act_buf];
    a.rv = E.rv[c];
    a.tv = E.tv[c];
    a.L = E.L[c];
    a.U = E.U[c];
    a.c = E.c[c];
    a.lu = E.lu[c];
    a.act_src = E.act[E.act_buf];
    a.ninf_src = E.ninf[E.act_buf];
    a.rec_rk = E.rec_rk;
    a.rec_rr = E.rec_rr;
    a.rec_ra = E.rec_ra;
    a.rec_ck = E.rec_ck;
    a.rec_cr = E.rec_cr;
    a.rec_rv = E.rec_rv;
    a.rec_cv = E.rec_cv;
    R->rp = a.o_rp = (int32_t *)own(4 * ((size_t)mr + 1), R->owned);
    R->ci = a.o_ci = (int32_t *)own(4 * (size_t)nz, R->owned);
    R->rv = a.o_rv = (double *)own(8 * (size_t)nz, R->owned);
    R->tp = a.o_tp = (int32_t *)own(4 * ((size_t)nc + 1), R->owned);
    R->ti = a.o_ti = (int32_t *)own(4 * (size_t)nz, R->owned);
    R->tv = a.o_tv = (double *)own(8 * (size_t)nz, R->owned);
    R->L = a.o_L = (double *)own(8 * (size_t)mr, R->owned);
    R->U = a.o_U = (double *)own(8 * (size_t)mr, R->owned);
    R->lb = a.o_lb = (double *)own(8 * (size_t)nc, R->owned);
    R->ub = a.o_ub = (double *)own(8 * (size_t)nc, R->owned);
    R->c = a.o_c = (double *)own(8 * (size_t)nc, R->owned);
    R->rmap = a.o_rmap = (int32_t *)own(4 * (size_t)mr, R->owned);
    R->cmap = a.o_cmap = (int32_t *)own(4 * (size_t)nc, R->owned);
    D->m0 = Z.m0;
    D->n0 = Z.n0;
    D->n_final = nc;
    D->act_m = na;
    D->rk = a.o_rk = (int32_t *)own(4 * (size_t)Z.m0, D->owned);
    D->rr = a.o_rr = (int32_t *)own(4 * (size_t)Z.m0, D->owned);
    D->ra = a.o_ra = (int32_t *)own(4 * (size_t)Z.m0, D->owned);
    D->rv = a.o_rv2 = (double *)own(8 * (size_t)Z.m0, D->owned);
    D->ck = a.o_ck = (int32_t *)own(4 * (size_t)Z.n0, D->owned);
    D->cr = a.o_cr = (int32_t *)own(4 * (size_t)Z.n0, D->owned);
    D->cv = a.o_cv2 = (double *)own(8 * (size_t)Z.n0, D->owned);
    D->lu = a.o_lu = (double2 *)own(16 * (size_t)nc, D->owned);
    D->cmap = a.o_dcmap = (int32_t *)own(4 * (size_t)nc, D->owned);
    D->act = a.o_act = (double2 *)own(16 * (size_t)na, D->owned);
    D->ninf = a.o_ninf = (int2 *)own(8 * (size_t)na, D->owned);
    D->act_rmap = a.o_armap = (int32_t *)own(4 * (size_t)na, D->owned);
    const int64_t span = std::max<int64_t>({(int64_t)mr + 1, (int64_t)nc + 1, (int64_t)nz, (int64_t)Z.m0,
                                            (int64_t)Z.n0, (int64_t)na});
    (k_extract<<<grid_for(span), 256, 0, E.s>>>(a), note_launch());
    LPP_CUDA(cudaGetLastError());
    LPP_CUDA(cudaStreamSynchronize(E.s));
    R->m = mr;
    R->n = nc;
    R->nnz = nz;
    R->obj_offset = offs[k];
    auto *P = new lpp_postsolve();
    P->dev = D;
    P->acnt = na;
    lpp_info &I = P->info;
    I.status = E.lp_status[k];
    I.where = E.lp_where[k];
    I.index = E.lp_index[k] < 0 ? -1 : E.lp_index[k] - (I.where == LPP_WHERE_ROW ? Z.rbase : Z.cbase);
    I.round = E.lp_round[k];
    I.rounds = E.lp_rounds[k];
    I.m = Z.m0;
    I.n = Z.n0;
    I.nnz = Z.nnz0;
    I.m_red = mr;
    I.n_red = nc;
    I.nnz_red = nz;
    I.obj_offset = offs[k];
    I.presolve_ms = Z.ms;
    I.nnz_processed = Z.nnz_proc;
    I.s5_left = -1;
    S->done[Z.ticket] = lpp_server::Done{(lpp_status)I.status, R, P};
}

// one tick of the worker (called with the lock released)
bool tick(lpp_server *S, std::vector<std::pair<int32_t, lpp_server::Req *>> &admit) {
    Engine &E = S->E;
    const int32_t nl = E.nlp;
    S->tick++;
    const int32_t r = S->tick;
    bool first = false;
    for (auto &pr : admit) {
        lpp_server::Slot &Z = S->sl[pr.first];
        try {
            E.append(pr.first, pr.second->lp, Z.rbase, Z.cbase, r);
            first = true;
        } catch (const StatusError &e) {
            std::lock_guard<std::mutex> g(S->mu);
            S->done[Z.ticket] = lpp_server::Done{e.st, nullptr, nullptr};
            S->rec_rows.give(Z.rbase, Z.m0);
            S->rec_cols.give(Z.cbase, Z.n0);
            Z = lpp_server::Slot();
        }
        free_req(pr.second, E.s);
    }
    if (first) E.reschedule();
    bool any = false, retired = false;
    for (int32_t k = 0; k < nl; k++) {
        any |= S->sl[k].used && !S->sl[k].retired;
        retired |= S->sl[k].retired;
    }
    if (!any && !retired) return false;
    // round start: every active LP's nonzeros count as processed
    for (int32_t k = 0; k < nl; k++)
        if (S->sl[k].used && !S->sl[k].retired) S->sl[k].nnz_proc += S->sl[k].last_nnz;
    const Engine::StepOut so = E.step(r, first, retired);
    S->stats.ticks++;
    // retired LPs have left the arena in this round's compaction
    if (so.structural) {
        std::lock_guard<std::mutex> g(S->mu);
        for (int32_t k = 0; k < nl; k++)
            if (S->sl[k].used && S->sl[k].retired) {
                S->rec_rows.give(S->sl[k].rbase, S->sl[k].m0);
                S->rec_cols.give(S->sl[k].cbase, S->sl[k].n0);
                S->sl[k] = lpp_server::Slot();
                E.lp_dropped[k] = 1;
            }
    }
    // per-slot ranges now and at the round start, objective constants
    int32_t *dr = E.pool.alloc<int32_t>(8 * (size_t)nl);
    fill_i32(dr, 8 * (int64_t)nl, -1, E.s);
    if (E.m > 0) (k_bounds<<<(E.m + 255) / 256, 256, 0, E.s>>>(E.lprow[E.cur], E.m, dr, dr + nl), note_launch());
    if (E.n > 0) (k_bounds<<<(E.n + 255) / 256, 256, 0, E.s>>>(E.lpcol[E.cur], E.n, dr + 2 * nl, dr + 3 * nl), note_launch());
    if (E.act_m > 0) (k_bounds<<<(E.act_m + 255) / 256, 256, 0, E.s>>>(E.lprow[E.act_buf], E.act_m, dr + 6 * nl,
                                                                        dr + 7 * nl), note_launch());
    std::vector<int32_t> h(8 * (size_t)nl), rp_h((size_t)E.m + 1);
    std::vector<double> offs(nl);
    LPP_CUDA(cudaMemcpyAsync(h.data(), dr, sizeof(int32_t) * h.size(), cudaMemcpyDeviceToHost, E.s));
    LPP_CUDA(cudaMemcpyAsync(rp_h.data(), E.rp[E.cur], sizeof(int32_t) * rp_h.size(), cudaMemcpyDeviceToHost, E.s));
    LPP_CUDA(cudaMemcpyAsync(offs.data(), E.K.offset, sizeof(double) * nl, cudaMemcpyDeviceToHost, E.s));
    LPP_CUDA(cudaStreamSynchronize(E.s));
    E.pool.forget(dr);
    cudaFreeAsync(dr, E.s);
    std::vector<int32_t> rng(6 * (size_t)nl), arng(2 * (size_t)nl);
    for (int32_t k = 0; k < nl; k++) {
        const int32_t f = h[k], l = h[nl + k];
        rng[k] = f;
        rng[nl + k] = l;
        rng[2 * nl + k] = h[2 * nl + k];
        rng[3 * nl + k] = h[3 * nl + k];
        rng[4 * nl + k] = f >= 0 ? rp_h[f] : 0;
        rng[5 * nl + k] = l >= 0 ? rp_h[l] : 0;
        arng[k] = h[6 * nl + k];
        arng[nl + k] = h[7 * nl + k];
    }
    // finished LPs: a verdict, no change, or the round cap
    for (int32_t k = 0; k < nl; k++) {
        lpp_server::Slot &Z = S->sl[k];
        if (!Z.used || Z.retired) continue;
        Z.ms += so.ms;
        Z.last_nnz = rng[5 * nl + k] - rng[4 * nl + k];
        const int32_t local = r - Z.round0 + 1;
        int v = 0;
        while (v < V_SLOTS && E.verdict_h[k * V_SLOTS + v] == kNone) v++;
        bool fin = false;
        if (v < V_SLOTS) {
            E.lp_status[k] = v == V_S6_COL ? LPP_UNBOUNDED : LPP_INFEASIBLE;
            E.lp_where[k] = (v == V_S2_ROW || v == V_S5_ROW) ? LPP_WHERE_ROW : LPP_WHERE_COL;
            E.lp_index[k] = E.verdict_h[k * V_SLOTS + v];
            E.lp_round[k] = local;
            fin = true;
        } else if (!E.changed_h[k] || local >= S->o.max_rounds) {
            E.lp_status[k] = LPP_OK;
            E.lp_where[k] = LPP_WHERE_NONE;
            E.lp_index[k] = -1;
            E.lp_round[k] = 0;
            fin = true;
        }
        E.lp_rounds[k] = local;
        if (!fin) continue;
        {
            std::lock_guard<std::mutex> g(S->mu);
            finish_slot(S, k, rng, arng, offs);
            S->stats.finished++;
        }
        Z.retired = true;
        const uint8_t one = 1;
        LPP_CUDA(cudaMemcpyAsync(E.lp_retired_dev + k, &one, 1, cudaMemcpyHostToDevice, E.s));
        LPP_CUDA(cudaStreamSynchronize(E.s));
    }
    S->cv_done.notify_all();
    return true;
}

// a request presolved alone on the worker's stream (lpp_presolve's engine)
// The longest queue an idle server still serves one request at a time (each
// presolved alone, back to back); a longer one joins the arena.  Served one
// by one a request waits for the ones before it; in the arena every resident
// LP advances one round per tick, which pays off only when enough of them
// share the ticks.
constexpr size_t kSoloQueue = 64;

void run_solo(lpp_server *S, lpp_server::Req *q) {
    lpp_opts o = S->o;
    o.stream = S->E.s;
    lpp_reduced *red = nullptr;
    lpp_postsolve *rec = nullptr;
    const lpp_status st = lpp_presolve(&q->lp, &o, &red, &rec);
    const uint64_t ticket = q->ticket;
    free_req(q, S->E.s);
    std::lock_guard<std::mutex> g(S->mu);
    S->done[ticket] = lpp_server::Done{st, red, rec};
    S->stats.finished++;
    S->stats.solo++;
    S->cv_done.notify_all();
}

void worker_main(lpp_server *S) {
    try {
        LPP_CUDA(cudaSetDevice(S->o.device));
        while (true) {
            std::vector<std::pair<int32_t, lpp_server::Req *>> admit;
            lpp_server::Req *solo = nullptr;
            {
                std::unique_lock<std::mutex> lk(S->mu);
                auto busy = [&] {
                    for (auto &z : S->sl)
                        if (z.used) return true;
                    return false;
                };
                S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || busy(); });
                if (S->stop) break;
                // an idle arena with a short queue: presolve the oldest at
                // once, rounds back to back, instead of one round per tick;
                // a queue longer than kSoloQueue (an overload) is batched
                if (!busy() && S->queue.size() <= kSoloQueue) {
                    solo = S->queue.front();
                    S->queue.pop_front();
                    S->stats.admitted++;
                }
                // admission, oldest first, while the arena and record space allow
                int64_t m = S->E.m, n = S->E.n, z = S->E.nnz;
                while (!solo && !S->queue.empty()) {
                    lpp_server::Req *q = S->queue.front();
                    const lpp_lp &lp = q->lp;
                    int32_t slot = -1;
                    for (int32_t k = 0; k < (int32_t)S->sl.size() && slot < 0; k++)
                        if (!S->sl[k].used) slot = k;
                    if (slot < 0 || m + lp.m > S->m_cap || n + lp.n > S->n_cap || z + lp.nnz > S->nnz_cap) break;
                    const int32_t rb = S->rec_rows.take(lp.m);
                    if (rb < 0) break;
                    const int32_t cb = S->rec_cols.take(lp.n);
                    if (cb < 0) {
                        S->rec_rows.give(rb, lp.m);
                        break;
                    }
                    S->queue.pop_front();
                    lpp_server::Slot &Z = S->sl[slot];
                    Z = lpp_server::Slot();
                    Z.used = true;
                    Z.ticket = q->ticket;
                    Z.round0 = S->tick + 1;
                    Z.rbase = rb;
                    Z.cbase = cb;
                    Z.m0 = lp.m;
                    Z.n0 = lp.n;
                    Z.nnz0 = lp.nnz;
                    Z.last_nnz = lp.nnz;
                    Z.t_submit = q->t_submit;
                    m += lp.m;
                    n += lp.n;
                    z += lp.nnz;
                    admit.emplace_back(slot, q);
                    S->stats.admitted++;
                }
            }
            if (solo) {
                run_solo(S, solo);
                continue;
            }
            const bool ran = tick(S, admit);
            std::lock_guard<std::mutex> g(S->mu);
            int32_t live = 0;
            int64_t res = 0;
            for (auto &zz : S->sl)
                if (zz.used) {
                    live++;
                    res += (int64_t)(zz.m0 * kBytesRow + zz.n0 * kBytesCol + zz.nnz0 * kBytesNnz);
                }
            S->stats.max_concurrent = std::max<int32_t>(S->stats.max_concurrent, live);
            S->stats.resident_bytes = res;
            S->stats.peak_resident_bytes = std::max<int64_t>(S->stats.peak_resident_bytes, res);
            (void)ran;
        }
    } catch (const std::exception &e) {
        std::lock_guard<std::mutex> g(S->mu);
        S->fatal = e.what();
        S->stop = true;
        S->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

lpp_status lpp_server_create(size_t hbm_budget, const lpp_opts *opts, lpp_server **srv) {
    if (!srv) return lpp_noalloc_fail(LPP_ERR_INVALID, "srv is NULL");
    *srv = nullptr;
    lpp_opts o;
    if (opts) o = *opts;
    else lpp_opts_default(&o);
    if (hbm_budget < (size_t)(1 << 20)) return lpp_noalloc_fail(LPP_ERR_BUDGET, "budget below 1 MiB");
    if (o.parallel_cols != 0 || o.col_singletons != 0 || o.doubletons != 0 || o.dual_records != 0 || o.dep_rows != 0)
        return lpp_noalloc_fail(LPP_ERR_INVALID,
                                "parallel_cols, col_singletons, doubletons, dual_records: lpp_presolve and "
                                "lpp_presolve_batch only; dep_rows: lpp_presolve only");
    auto *S = new lpp_server();
    try {
        S->o = o;
        S->o.stream = nullptr;  // the worker owns its stream
        S->o.timing = 0;
        S->budget = hbm_budget;
        // the budget is split between nonzeros (55%), rows (25%) and columns (20%)
        S->nnz_cap = std::min<int64_t>(2147483000LL, (int64_t)(0.55 * hbm_budget / kBytesNnz));
        S->m_cap = (int32_t)std::min<int64_t>(1 << 30, (int64_t)(0.25 * hbm_budget / (kBytesRow + 20)));
        S->n_cap = (int32_t)std::min<int64_t>(1 << 30, (int64_t)(0.20 * hbm_budget / (kBytesCol + 16)));
        S->slots = 4096;
        S->sl.resize(S->slots);
        S->rec_rows.init(S->m_cap);
        S->rec_cols.init(S->n_cap);
        Member cap{S->m_cap, S->n_cap, S->nnz_cap, 0, 0, 0, 0.0};
        S->E.setup(S->o, S->slots, {cap});
        S->E.lp_rounds.assign(S->slots, 0);
        S->E.lp_status.assign(S->slots, LPP_OK);
        S->E.lp_where.assign(S->slots, 0);
        S->E.lp_index.assign(S->slots, -1);
        S->E.lp_round.assign(S->slots, 0);
        S->E.init_empty();
        LPP_CUDA(cudaStreamCreateWithFlags(&S->submit_stream, cudaStreamNonBlocking));
        S->worker = std::thread(worker_main, S);
    } catch (const StatusError &e) {
        delete S;
        return lpp_noalloc_fail(e.st, e.what());
    } catch (const std::exception &e) {
        delete S;
        return lpp_noalloc_fail(LPP_ERR_CUDA, e.what());
    }
    *srv = S;
    return LPP_OK;
}

lpp_status lpp_server_submit(lpp_server *S, const lpp_lp *lp, uint64_t *ticket) {
    if (!S || !lp || !ticket) return lpp_noalloc_fail(LPP_ERR_INVALID, "NULL argument");
    if (lp->m < 0 || lp->n < 0 || lp->nnz < 0 || !lp->row_ptr) return lpp_noalloc_fail(LPP_ERR_INVALID, "bad LP");
    if (lp->m > S->m_cap || lp->n > S->n_cap || lp->nnz > S->nnz_cap)
        return lpp_noalloc_fail(LPP_ERR_BUDGET, "LP larger than the server's budget allows");
    auto *q = new lpp_server::Req();
    q->lp = *lp;
    const size_t m = lp->m, n = lp->n, z = (size_t)lp->nnz;
    if (!lp->on_device) {
        // host inputs are copied now; the worker uploads them at admission
        q->h_i.resize(m + 1 + z);
        q->h_d.resize(z + 2 * m + 3 * n);
        std::memcpy(q->h_i.data(), lp->row_ptr, 4 * (m + 1));
        if (z) std::memcpy(q->h_i.data() + m + 1, lp->col_idx, 4 * z);
        double *d = q->h_d.data();
        if (z) std::memcpy(d, lp->val, 8 * z);
        if (m) std::memcpy(d + z, lp->lhs, 8 * m);
        if (m) std::memcpy(d + z + m, lp->rhs, 8 * m);
        if (n) std::memcpy(d + z + 2 * m, lp->lb, 8 * n);
        if (n) std::memcpy(d + z + 2 * m + n, lp->ub, 8 * n);
        if (n) std::memcpy(d + z + 2 * m + 2 * n, lp->c, 8 * n);
        q->lp.row_ptr = q->h_i.data();
        q->lp.col_idx = q->h_i.data() + m + 1;
        q->lp.val = d;
        q->lp.lhs = d + z;
        q->lp.rhs = d + z + m;
        q->lp.lb = d + z + 2 * m;
        q->lp.ub = d + z + 2 * m + n;
        q->lp.c = d + z + 2 * m + 2 * n;
    } else {
        // the copy is made on the server's submit stream (which does not wait
        // for the worker's rounds) from its stream-ordered memory pool
        const size_t ibytes = 4 * (m + 1 + z), doff = (ibytes + 7) / 8 * 8;
        const size_t bytes = doff + 8 * (z + 2 * m + 3 * n);
        std::lock_guard<std::mutex> sg(S->submit_mu);
        cudaStream_t ss = S->submit_stream;
        if (cudaMallocAsync(&q->dev, bytes, ss) != cudaSuccess) {
            delete q;
            return lpp_noalloc_fail(LPP_ERR_OOM, "device copy of the request failed");
        }
        char *p = static_cast<char *>(q->dev);
        bool copy_ok = true;
        auto cp = [&](const void *src, size_t b) {
            void *dst = p;
            if (b && cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToDevice, ss) != cudaSuccess) copy_ok = false;
            p += b;
            return dst;
        };
        q->lp.row_ptr = (const int32_t *)cp(lp->row_ptr, 4 * (m + 1));
        q->lp.col_idx = (const int32_t *)cp(lp->col_idx, 4 * z);
        p = static_cast<char *>(q->dev) + doff;
        q->lp.val = (const double *)cp(lp->val, 8 * z);
        q->lp.lhs = (const double *)cp(lp->lhs, 8 * m);
        q->lp.rhs = (const double *)cp(lp->rhs, 8 * m);
        q->lp.lb = (const double *)cp(lp->lb, 8 * n);
        q->lp.ub = (const double *)cp(lp->ub, 8 * n);
        q->lp.c = (const double *)cp(lp->c, 8 * n);
        if (!copy_ok || cudaStreamSynchronize(ss) != cudaSuccess) {
            cudaFreeAsync(q->dev, ss);
            delete q;
            return lpp_noalloc_fail(LPP_ERR_CUDA, "device copy of the request failed");
        }
    }
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stop) {
            free_req(q, S->submit_stream);
            return lpp_noalloc_fail(LPP_ERR_CUDA, S->fatal.empty() ? "server stopped" : S->fatal.c_str());
        }
        q->ticket = S->next_ticket++;
        q->t_submit = now_s();
        *ticket = q->ticket;
        S->queue.push_back(q);
        S->stats.submitted++;
    }
    S->cv_work.notify_one();
    return LPP_OK;
}

lpp_status lpp_server_take(lpp_server *S, uint64_t ticket, int32_t wait_ms, lpp_reduced **out, lpp_postsolve **rec) {
    if (!S || !out || !rec) return lpp_noalloc_fail(LPP_ERR_INVALID, "NULL argument");
    *out = nullptr;
    *rec = nullptr;
    std::unique_lock<std::mutex> lk(S->mu);
    auto ready = [&] { return S->done.count(ticket) > 0 || S->stop; };
    if (wait_ms < 0) S->cv_done.wait(lk, ready);
    else S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
    auto it = S->done.find(ticket);
    if (it == S->done.end()) {
        if (S->stop && !S->fatal.empty()) return lpp_noalloc_fail(LPP_ERR_CUDA, S->fatal.c_str());
        return lpp_noalloc_fail(LPP_ERR_TIMEOUT, "result not ready");
    }
    const lpp_server::Done d = it->second;
    S->done.erase(it);
    S->stats.taken++;
    if (d.st < 0) return lpp_noalloc_fail(d.st, "request failed");
    *out = d.red;
    *rec = d.rec;
    return d.st;
}

lpp_status lpp_server_stats_get(lpp_server *S, lpp_server_stats *st) {
    if (!S || !st) return lpp_noalloc_fail(LPP_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> g(S->mu);
    *st = S->stats;
    return LPP_OK;
}

void lpp_server_destroy(lpp_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto *q : S->queue) free_req(q, S->submit_stream);
    for (auto &kv : S->done) {
        lpp_free_reduced(kv.second.red);
        lpp_free_postsolve(kv.second.rec);
    }
    if (S->submit_stream) {
        cudaStreamSynchronize(S->submit_stream);
        cudaStreamDestroy(S->submit_stream);
    }
    delete S;
}

}  // extern "C"
