// lpp_api.cu -- the C ABI of lpp.h: argument checks, engine runs, result objects.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>

#include "lpp_engine.h"
#include "postsolve.h"

using namespace lpp;

namespace {

thread_local std::string g_err;

lpp_status set_err(lpp_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

template <class F>
lpp_status guarded(F &&f) {
    try {
        return f();
    } catch (const StatusError &e) {
        return set_err(e.st, e.what());
    } catch (const CudaError &e) {
        return set_err(LPP_ERR_CUDA, e.what());
    } catch (const std::bad_alloc &) {
        return set_err(LPP_ERR_OOM, "host allocation failed");
    } catch (const std::exception &e) {
        return set_err(LPP_ERR_CUDA, e.what());
    }
}

void check_lp_shape(const lpp_lp *in) {
    if (!in) throw StatusError(LPP_ERR_INVALID, "lp is NULL");
    if (in->m < 0 || in->n < 0 || in->nnz < 0) throw StatusError(LPP_ERR_INVALID, "negative size");
    if (in->nnz >= 2147483647LL) throw StatusError(LPP_ERR_INVALID, "nnz must be < 2^31");
    if (!in->row_ptr) throw StatusError(LPP_ERR_INVALID, "row_ptr is NULL");
    if (in->nnz > 0 && (!in->col_idx || !in->val)) throw StatusError(LPP_ERR_INVALID, "col_idx/val is NULL");
    if (in->m > 0 && (!in->lhs || !in->rhs)) throw StatusError(LPP_ERR_INVALID, "lhs/rhs is NULL");
    if (in->n > 0 && (!in->lb || !in->ub || !in->c)) throw StatusError(LPP_ERR_INVALID, "lb/ub/c is NULL");
    if (in->nnz > 0 && in->n == 0) throw StatusError(LPP_ERR_INVALID, "entries but no columns");
    if (in->m == 0 && in->nnz != 0) throw StatusError(LPP_ERR_INVALID, "entries but no rows");
}

lpp_opts resolve_opts(const lpp_opts *opts) {
    lpp_opts o;
    if (opts) o = *opts;
    else lpp_opts_default(&o);
    if (o.max_rounds < 0 || o.par_max_iter < 1 || !(o.feas_tol >= 0) || !(o.bound_tol >= 0) || !(o.huge > 0) ||
        !(o.max_implied > 0) || !(o.par_tol >= 0) || (o.parallel_cols != 0 && o.parallel_cols != 1) ||
        (o.col_singletons != 0 && o.col_singletons != 1) || (o.dual_fixing != 0 && o.dual_fixing != 1) ||
        (o.doubletons != 0 && o.doubletons != 1) || (o.batch_persistent != 0 && o.batch_persistent != 1) ||
        (o.dual_records != 0 && o.dual_records != 1) || (o.dep_rows != 0 && o.dep_rows != 1))
        throw StatusError(LPP_ERR_INVALID, "bad options");
    return o;
}

__global__ void k_count_lp(const int32_t *lprow, const int32_t *rp, int32_t m, const int32_t *lpcol, int32_t n,
                           int32_t *rows, int32_t *cols, int32_t *nnz) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) {
        atomicAdd(&rows[lprow[t]], 1);
        atomicAdd(&nnz[lprow[t]], rp[t + 1] - rp[t]);
    }
    if (t < n) atomicAdd(&cols[lpcol[t]], 1);
}

// arena -> per-LP local numbering: ptr arrays get one extra entry per LP
__global__ void k_rebase_rows(const int32_t *rp, const int32_t *lprow, const int32_t *rmap, int32_t m,
                              const int32_t *nnz_start, const int32_t *row_orig, int32_t *rp_out, int32_t *rmap_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int32_t lp = lprow[i];
    rp_out[i + lp] = rp[i] - nnz_start[lp];
    rmap_out[i] = rmap[i] - row_orig[lp];
}
__global__ void k_rebase_cols(const int32_t *tp, const int32_t *lpcol, const int32_t *cmap, int32_t n,
                              const int32_t *nnz_start, const int32_t *col_orig, int32_t *tp_out, int32_t *cmap_out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int32_t lp = lpcol[j];
    tp_out[j + lp] = tp[j] - nnz_start[lp];
    cmap_out[j] = cmap[j] - col_orig[lp];
}
__global__ void k_ptr_tails(const int32_t *row_start, const int32_t *rows, const int32_t *col_start,
                            const int32_t *cols, const int32_t *nnz, int32_t nlp, int32_t *rp_out, int32_t *tp_out) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nlp) return;
    rp_out[row_start[k] + rows[k] + k] = nnz[k];
    tp_out[col_start[k] + cols[k] + k] = nnz[k];
}
// entries: column index (CSR) / row index (CSC) made local to the LP
__global__ void k_rebase_idx(int32_t *idx, const int32_t *ptr, const int32_t *lp_of_seg, int32_t segs,
                             const int32_t *start) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= segs) return;
    const int32_t d = start[lp_of_seg[i]];
    for (int32_t k = ptr[i]; k < ptr[i + 1]; k++) idx[k] -= d;
}

__global__ void k_count_rows_lp(const int32_t *lprow, int32_t m, int32_t *rows) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) atomicAdd(&rows[lprow[t]], 1);
}

unsigned nblk(int64_t cnt) { return (unsigned)((cnt + 255) / 256 > 0 ? (cnt + 255) / 256 : 1); }

// Moves the record arrays of a finished run into a DeviceRecords object
// (ownership leaves the engine's pool) together with copies of the final
// bounds and column map and the last round's activities.
std::shared_ptr<DeviceRecords> take_records(Engine &E) {
    auto D = std::make_shared<DeviceRecords>();
    D->m0 = E.m0;
    D->n0 = E.n0;
    D->n_final = E.n;
    D->act_m = E.act_m;
    D->rk = E.rec_rk;
    D->rr = E.rec_rr;
    D->ra = E.rec_ra;
    D->rv = E.rec_rv;
    D->ck = E.rec_ck;
    D->cr = E.rec_cr;
    D->cv = E.rec_cv;
    D->ca = E.rec_ca;
    D->cp = E.rec_cp;
    D->cm = E.rec_cm;
    D->sb = E.rec_sb;
    D->sl = E.rec_sl;
    D->srhs = E.rec_srhs;
    D->scol = E.rec_scol;
    D->sval = E.rec_sval;
    D->bs = E.rec_bs;
    if (E.sub_used) {
        unsigned long long used = 0;
        LPP_CUDA(cudaMemcpyAsync(&used, E.sub_used, sizeof used, cudaMemcpyDeviceToHost, E.s));
        LPP_CUDA(cudaStreamSynchronize(E.s));
        D->sub_used = (int64_t)used;
    }
    D->lu = E.lu[E.cur];
    D->act = E.act_rec ? E.act_rec : E.act[E.act_buf];
    D->ninf = E.ninf_rec ? E.ninf_rec : E.ninf[E.act_buf];
    for (void *p : {(void *)D->rk, (void *)D->rr, (void *)D->ra, (void *)D->rv, (void *)D->ck, (void *)D->cr,
                    (void *)D->cv, (void *)D->lu, (void *)D->act, (void *)D->ninf, (void *)D->ca, (void *)D->cp,
                    (void *)D->cm, (void *)D->sb, (void *)D->sl, (void *)D->srhs, (void *)D->scol,
                    (void *)D->sval, (void *)D->bs}) {
        if (!p) continue;
        E.pool.forget(p);
        D->owned.push_back(p);
    }
    // maps may belong to the reduced LP: copy them
    D->cmap = E.pool.alloc<int32_t>(E.n);
    D->act_rmap = E.pool.alloc<int32_t>(E.act_m);
    E.pool.forget(D->cmap);
    E.pool.forget(D->act_rmap);
    D->owned.push_back(D->cmap);
    D->owned.push_back(D->act_rmap);
    if (E.n) LPP_CUDA(cudaMemcpyAsync(D->cmap, E.cmap[E.cur], 4 * (size_t)E.n, cudaMemcpyDeviceToDevice, E.s));
    if (E.act_m)
        LPP_CUDA(cudaMemcpyAsync(D->act_rmap, E.rmap_rec ? E.rmap_rec : E.rmap[E.act_buf], 4 * (size_t)E.act_m,
                                 cudaMemcpyDeviceToDevice, E.s));
    return D;
}

// Postsolve record of LP k: verdict and counters now, the rest on first access.
lpp_postsolve *make_postsolve(Engine &E, const std::shared_ptr<DeviceRecords> &D, int32_t k, int32_t m_red,
                              int32_t n_red, int64_t nnz_red, double offset, int32_t cstart, int32_t astart,
                              int32_t acnt) {
    auto *P = new lpp_postsolve();
    const Member &mm = E.mem[k];
    P->dev = D;
    P->huge = E.o.huge;
    P->r0 = mm.row_off;
    P->c0 = mm.col_off;
    P->cstart = cstart;
    P->astart = astart;
    P->acnt = acnt;
    lpp_info &I = P->info;
    I.status = E.lp_status[k];
    I.where = E.lp_where[k];
    I.index = E.lp_index[k] < 0 ? -1 : E.lp_index[k] - (I.where == LPP_WHERE_ROW ? P->r0 : P->c0);
    I.round = E.lp_round[k];
    I.rounds = E.lp_rounds[k];
    I.m = mm.m;
    I.n = mm.n;
    I.nnz = mm.nnz;
    I.m_red = m_red;
    I.n_red = n_red;
    I.nnz_red = nnz_red;
    I.obj_offset = offset;
    I.presolve_ms = E.loop_ms;
    I.nnz_processed = E.nnz_processed;
    I.launches = launch_count() - E.launches0;
    I.s5_left = E.s5_left;
    I.dep_pivots = E.dep_pivots;
    I.dep_peeled = E.dep_peeled;
    I.dep_rows = E.dep_found;
    I.dep_stopped = E.dep_stopped;
    P->r_nnz = E.r_nnz;
    P->r_rows = E.r_rows;
    P->r_cols = E.r_cols;
    P->r_bounds = E.r_bounds;
    P->r_ms = E.r_ms;
    if (E.o.timing) {
        std::vector<lpp_kernel_stat> ks(F_NUM);
        for (int f = 0; f < F_NUM; f++) {
            std::memset(&ks[f], 0, sizeof(lpp_kernel_stat));
            std::snprintf(ks[f].name, sizeof ks[f].name, "%s", fam_name(f));
        }
        for (auto &mk : E.marks) {
            float ms = 0.f;
            LPP_CUDA(cudaEventElapsedTime(&ms, mk.a, mk.b));
            ks[mk.fam].launches++;
            ks[mk.fam].ms += ms;
            ks[mk.fam].bytes += mk.bytes;
            ks[mk.fam].fp64_ops += mk.ops;
        }
        P->kstats = ks;
    }
    return P;
}

template <class T>
void d2h_slice(std::vector<T> &h, const T *d, size_t off, size_t cnt) {
    h.resize(cnt);
    if (cnt) LPP_CUDA(cudaMemcpy(h.data(), d + off, sizeof(T) * cnt, cudaMemcpyDeviceToHost));
}

// host copies of this LP's records, bounds and activities
void materialize(lpp_postsolve *P) {
    if (P->host_ready) return;
    const DeviceRecords &D = *P->dev;
    const int32_t m = P->info.m, n = P->info.n, r0 = P->r0, c0 = P->c0;
    d2h_slice(P->row_kind, D.rk, r0, m);
    d2h_slice(P->row_round, D.rr, r0, m);
    d2h_slice(P->row_aux, D.ra, r0, m);
    d2h_slice(P->row_val, D.rv, r0, m);
    d2h_slice(P->col_kind, D.ck, c0, n);
    d2h_slice(P->col_round, D.cr, c0, n);
    d2h_slice(P->col_val, D.cv, c0, n);
    for (int32_t i = 0; i < m; i++) {
        const int32_t a = P->row_aux[i];
        if (a >= 0)  // singleton and substitution rows name a column, parallel rows a row
            P->row_aux[i] = (P->row_kind[i] == LPP_ROW_SINGLETON || P->row_kind[i] == LPP_ROW_SUBST ||
                             P->row_kind[i] == LPP_ROW_DOUBLETON)
                                ? a - c0
                                : a - r0;
    }
    std::vector<int32_t> cm;
    std::vector<double2> lu;
    d2h_slice(cm, D.cmap, P->cstart, P->info.n_red);
    d2h_slice(lu, D.lu, P->cstart, P->info.n_red);
    P->col_map.resize(cm.size());
    P->col_lb.assign(n, NAN);
    P->col_ub.assign(n, NAN);
    for (size_t k = 0; k < cm.size(); k++) {
        const int32_t o = cm[k] - c0;
        P->col_map[k] = o;
        if (o >= 0 && o < n) {
            P->col_lb[o] = lu[k].x;
            P->col_ub[o] = lu[k].y;
        }
    }
    for (int32_t j = 0; j < n; j++)
        if (P->col_kind[j] == LPP_COL_FIXED || P->col_kind[j] == LPP_COL_EMPTY)
            P->col_lb[j] = P->col_ub[j] = P->col_val[j];
    if (D.ca) {
        d2h_slice(P->col_aux, D.ca, c0, n);
        d2h_slice(P->col_pass, D.cp, c0, n);
        d2h_slice(P->col_mrg, D.cm, 4 * (size_t)c0, 4 * (size_t)n);
        for (int32_t j = 0; j < n; j++)
            if (P->col_aux[j] >= 0) P->col_aux[j] -= c0;
    } else {
        P->col_aux.assign(n, -1);
        P->col_pass.assign(n, 0);
        P->col_mrg.assign(4 * (size_t)n, NAN);
    }
    if (D.bs) {  // bound sources: LP-local rows, round 0 where the side has no source
        std::vector<int4> bs;
        d2h_slice(bs, D.bs, c0, n);
        P->col_lsrc.resize(n);
        P->col_lrnd.resize(n);
        P->col_usrc.resize(n);
        P->col_urnd.resize(n);
        for (int32_t j = 0; j < n; j++) {
            P->col_lsrc[j] = bs[j].x >= 0 ? bs[j].x - r0 : bs[j].x;
            P->col_lrnd[j] = bs[j].x == -1 ? 0 : bs[j].y;
            P->col_usrc[j] = bs[j].z >= 0 ? bs[j].z - r0 : bs[j].z;
            P->col_urnd[j] = bs[j].z == -1 ? 0 : bs[j].w;
        }
    }
    // substitutions: this LP's rows and their entries, the store compacted to
    // them (LP-local column indices)
    P->sub_beg.assign(m, 0);
    P->sub_len.assign(m, 0);
    P->sub_rhs.assign(m, 0.0);
    P->sub_col.clear();
    P->sub_val.clear();
    if (D.sb) {
        DeviceRecords &DM = const_cast<DeviceRecords &>(D);
        std::call_once(DM.store_once, [&DM]() {
            d2h_slice(DM.h_scol, DM.scol, 0, (size_t)DM.sub_used);
            d2h_slice(DM.h_sval, DM.sval, 0, (size_t)DM.sub_used);
        });
        std::vector<long long> sb;
        std::vector<int32_t> sl;
        d2h_slice(sb, D.sb, r0, m);
        d2h_slice(sl, D.sl, r0, m);
        d2h_slice(P->sub_rhs, D.srhs, r0, m);
        for (int32_t i = 0; i < m; i++) {
            if (P->row_kind[i] != LPP_ROW_SUBST && P->row_kind[i] != LPP_ROW_DOUBLETON) {
                P->sub_rhs[i] = 0.0;
                continue;
            }
            if (sb[i] < 0 || sl[i] < 0 || sb[i] + sl[i] > DM.sub_used)
                throw StatusError(LPP_ERR_CUDA, "internal: substitution record out of range");
            P->sub_beg[i] = (int64_t)P->sub_col.size();
            P->sub_len[i] = sl[i];
            for (long long q = sb[i]; q < sb[i] + sl[i]; q++) {
                P->sub_col.push_back(DM.h_scol[(size_t)q] - c0);
                P->sub_val.push_back(DM.h_sval[(size_t)q]);
            }
        }
    }
    std::vector<double2> act;
    std::vector<int2> ni;
    std::vector<int32_t> am;
    d2h_slice(act, D.act, P->astart, P->acnt);
    d2h_slice(ni, D.ninf, P->astart, P->acnt);
    d2h_slice(am, D.act_rmap, P->astart, P->acnt);
    P->act_min.assign(m, NAN);
    P->act_max.assign(m, NAN);
    P->ninf_min.assign(m, -1);
    P->ninf_max.assign(m, -1);
    for (int32_t i = 0; i < P->acnt; i++) {
        const int32_t o = am[i] - r0;
        if (o >= 0 && o < m) {
            P->act_min[o] = act[i].x;
            P->act_max[o] = act[i].y;
            P->ninf_min[o] = ni[i].x;
            P->ninf_max[o] = ni[i].y;
        }
    }
    P->host_ready = true;
}

// Host copies of a reduced LP live in one pinned block (from the pinned
// cache, sized for every array); each group is copied on its first request
// with async copies and one synchronisation: 0 = the LP (CSR, c, sides,
// bounds), 1 = the index maps, 2 = the CSC.
void materialize_host(lpp_reduced *R, int group) {
    if (R->host_done & (1 << group)) return;
    const size_t m = (size_t)R->m, n = (size_t)R->n, z = (size_t)R->nnz;
    struct Part {
        int group;
        void **dst;
        const void *src;
        size_t bytes;
    };
    const Part parts[] = {{0, (void **)&R->h_rp, R->rp, 4 * (m + 1)}, {0, (void **)&R->h_ci, R->ci, 4 * z},
                          {0, (void **)&R->h_rv, R->rv, 8 * z},       {0, (void **)&R->h_c, R->c, 8 * n},
                          {0, (void **)&R->h_L, R->L, 8 * m},         {0, (void **)&R->h_U, R->U, 8 * m},
                          {0, (void **)&R->h_lb, R->lb, 8 * n},       {0, (void **)&R->h_ub, R->ub, 8 * n},
                          {1, (void **)&R->h_rmap, R->rmap, 4 * m},   {1, (void **)&R->h_cmap, R->cmap, 4 * n},
                          {2, (void **)&R->h_tp, R->tp, 4 * (n + 1)}, {2, (void **)&R->h_ti, R->ti, 4 * z},
                          {2, (void **)&R->h_tv, R->tv, 8 * z}};
    auto up = [](size_t b) { return (b + 63) & ~(size_t)63; };
    if (!R->hblock) {
        size_t total = 0;
        for (const Part &p : parts) total += up(p.bytes);
        R->hblock = pinned_get_sized(total);
    }
    char *blk = static_cast<char *>(R->hblock);
    size_t off = 0;
    for (const Part &p : parts) {
        if (p.group == group) {
            *p.dst = blk + off;
            if (p.bytes && p.src) LPP_CUDA(cudaMemcpyAsync(blk + off, p.src, p.bytes, cudaMemcpyDeviceToHost, 0));
        }
        off += up(p.bytes);
    }
    LPP_CUDA(cudaStreamSynchronize(0));
    R->host_done |= 1 << group;
}

// ------------------------------------------------ batch: the persistent kernel
// Launch geometry of the persistent batch kernel -- threads per block and
// resident blocks per SM -- chosen per kind of batch (log2 of the LP count
// and of the mean nonzeros per LP, dual fixing on or off) by measurement: the
// first calls of a kind run each candidate once and record its kernel time,
// later calls use the fastest.  Fewer resident blocks keep the LPs being
// presolved inside L2; more hide more latency.  Every candidate gives the
// same results (the lanes per row do not depend on it).
struct FusedTuner {
    static constexpr int kN = 6;
    static constexpr int kThreads[kN] = {256, 256, 256, 512, 512, 128};
    static constexpr int kPerSm[kN] = {1, 2, 4, 1, 2, 8};
    struct Entry {
        float ms[kN] = {-1.f, -1.f, -1.f, -1.f, -1.f, -1.f};
    };
    std::mutex mu;
    std::map<uint64_t, Entry> tab;
    int pick(uint64_t key) {
        std::lock_guard<std::mutex> g(mu);
        Entry &e = tab[key];
        int best = -1;
        for (int c = 0; c < kN; c++) {
            if (e.ms[c] < 0.f) return c;  // not tried yet
            if (best < 0 || e.ms[c] < e.ms[best]) best = c;
        }
        return best;
    }
    void record(uint64_t key, int c, float ms) {
        std::lock_guard<std::mutex> g(mu);
        Entry &e = tab[key];
        if (e.ms[c] < 0.f || ms < e.ms[c]) e.ms[c] = ms;
    }
};
FusedTuner g_tuner;
constexpr int FusedTuner::kThreads[FusedTuner::kN];
constexpr int FusedTuner::kPerSm[FusedTuner::kN];

uint64_t tuner_key(int32_t count, int64_t nnz, int32_t dualfix) {
    int a = 0, b = 0;
    while ((1LL << (a + 1)) <= count) a++;
    const int64_t per = nnz / std::max<int32_t>(count, 1);
    while ((1LL << (b + 1)) <= per) b++;
    return ((uint64_t)a << 32) | ((uint64_t)b << 1) | (uint64_t)(dualfix != 0);
}

// Runs the batch in the persistent kernel when every LP qualifies (no row or
// column beyond 4096 entries, none of the steps it does not carry); returns
// false, with nothing done, otherwise.  E is prepared (ingested, checked,
// transposed); the results are handed out as the per-round path does.
bool batch_fused(Engine &E, const std::vector<Member> &mem, int32_t count, lpp_reduced **outs, lpp_postsolve **recs,
                 lpp_status *per_lp) {
    const lpp_opts &o = E.o;
    if (!o.batch_persistent || o.parallel_cols || o.col_singletons || o.doubletons || o.dual_records || o.timing ||
        o.max_rounds <= 0)
        return false;
    if (E.A.cls_start[7] != E.A.cls_start[6] || E.T.cls_start[7] != E.T.cls_start[6]) return false;
    cudaStream_t s = E.s;
    const int32_t m0 = E.m0, n0 = E.n0;
    const int64_t nnz0 = E.nnz0;
    const int32_t R = std::max(0, o.max_rounds);
    // per-LP table: ranges, S5 table region; the queue, largest LP first
    std::vector<FusedLP> lps(count);
    int64_t tab = 0;
    for (int32_t k = 0; k < count; k++) {
        const Member &mm = mem[k];
        int64_t tcap = 2;
        while (tcap < 2 * (int64_t)std::max(mm.m, 1)) tcap <<= 1;
        lps[k] = FusedLP{mm.row_off, mm.col_off, (int32_t)mm.nnz_off, mm.m, mm.n, (int32_t)mm.nnz, (int32_t)tab,
                         (int32_t)tcap};
        tab += tcap;
        if (tab >= 2147483647LL) return false;
    }
    std::vector<int32_t> queue(count);
    for (int32_t k = 0; k < count; k++) queue[k] = k;
    std::stable_sort(queue.begin(), queue.end(), [&](int32_t a, int32_t b) { return mem[a].nnz > mem[b].nnz; });
    DevPool &P = E.pool;
    FusedArgs F;
    std::memset(&F, 0, sizeof F);
    F.base = E.ctx(1);
    F.base.t_orig = 0;  // each block compacts its LP's CSC itself
    F.base.rinv = F.base.cinv = F.base.clen = nullptr;
    F.K = E.K;
    F.K.rinv = F.K.cinv = nullptr;
    for (int b = 0; b < 2; b++) {
        F.frp[b] = P.alloc<int32_t>((size_t)m0 + count + 1);
        F.ftp[b] = P.alloc<int32_t>((size_t)n0 + count + 1);
        F.ci[b] = E.ci[b];
        F.ti[b] = E.ti[b];
        F.rv[b] = E.rv[b];
        F.tv[b] = E.tv[b];
        F.L[b] = E.L[b];
        F.U[b] = E.U[b];
        F.c[b] = E.c[b];
        F.lu[b] = E.lu[b];
        F.rmap[b] = E.rmap[b];
        F.cmap[b] = E.cmap[b];
        F.list[b] = E.s5_list[b];
        F.act[b] = E.act[b];
        F.ninf[b] = E.ninf[b];
        F.hrow[b] = E.hrow[b];
        F.rdirty[b] = E.rdirty[b];
    }
    F.rp0 = E.rp[0];
    F.tp0 = E.tp[0];
    F.order = P.alloc<int32_t>(m0);
    F.tkey = P.alloc<unsigned long long>((size_t)tab);
    F.tlead = P.alloc<unsigned long long>((size_t)tab);
    F.st = P.alloc<DevStatus>(count);
    F.cnt = P.alloc<int32_t>(4 * (size_t)count);
    F.dead = P.alloc<uint8_t>(count);
    FusedLP *d_lps = P.alloc<FusedLP>(count);
    int32_t *d_queue = P.alloc<int32_t>(count);
    F.lps = d_lps;
    F.queue = d_queue;
    F.next = P.alloc<int32_t>(1);
    F.count = count;
    F.max_rounds = R;
    F.par_max_iter = o.par_max_iter;
    F.out = P.alloc<FusedOut>(count);
    F.rstat = P.alloc<int32_t>(4 * (size_t)count * (size_t)R);
    // outputs: moved to the reduced LPs' shared store and the records below
    F.o_rp = P.alloc<int32_t>((size_t)m0 + count);
    F.o_tp = P.alloc<int32_t>((size_t)n0 + count);
    F.o_ci = P.alloc<int32_t>(nnz0);
    F.o_ti = P.alloc<int32_t>(nnz0);
    F.o_rv = P.alloc<double>(nnz0);
    F.o_tv = P.alloc<double>(nnz0);
    F.o_L = P.alloc<double>(m0);
    F.o_U = P.alloc<double>(m0);
    F.o_rmap = P.alloc<int32_t>(m0);
    F.o_c = P.alloc<double>(n0);
    F.o_lb = P.alloc<double>(n0);
    F.o_ub = P.alloc<double>(n0);
    F.o_cmap = P.alloc<int32_t>(n0);
    F.o_fcmap = P.alloc<int32_t>(n0);
    F.o_lu = P.alloc<double2>(n0);
    F.o_act = P.alloc<double2>(m0);
    F.o_ninf = P.alloc<int2>(m0);
    F.o_armap = P.alloc<int32_t>(m0);
    LPP_CUDA(cudaMemcpyAsync(d_lps, lps.data(), sizeof(FusedLP) * lps.size(), cudaMemcpyHostToDevice, s));
    LPP_CUDA(cudaMemcpyAsync(d_queue, queue.data(), sizeof(int32_t) * queue.size(), cudaMemcpyHostToDevice, s));
    LPP_CUDA(cudaMemsetAsync(F.tkey, 0, sizeof(unsigned long long) * (size_t)tab, s));
    LPP_CUDA(cudaMemsetAsync(F.tlead, 0xff, sizeof(unsigned long long) * (size_t)tab, s));
    LPP_CUDA(cudaMemsetAsync(F.dead, 0, (size_t)count, s));
    LPP_CUDA(cudaMemsetAsync(F.next, 0, sizeof(int32_t), s));
    LPP_CUDA(cudaMemsetAsync(F.rstat, 0, sizeof(int32_t) * 4 * (size_t)count * (size_t)R, s));
    // launch geometry: the tuner's block size, as many blocks as stay resident
    const uint64_t key = tuner_key(count, nnz0, o.dual_fixing);
    const int cand = g_tuner.pick(key);
    const int threads = FusedTuner::kThreads[cand];
    int sms = 0;
    LPP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o.device));
    const int per_sm = std::max(1, std::min(FusedTuner::kPerSm[cand], batch_fused_blocks_per_sm(threads)));
    const int blocks = (int)std::min<int64_t>(count, (int64_t)sms * per_sm);
    cudaEvent_t e0, e1;
    LPP_CUDA(cudaEventCreate(&e0));
    LPP_CUDA(cudaEventCreate(&e1));
    E.spare_events.push_back(e0);
    E.spare_events.push_back(e1);
    LPP_CUDA(cudaEventRecord(e0, s));
    launch_batch_fused(F, threads, blocks, s);
    LPP_CUDA(cudaGetLastError());
    LPP_CUDA(cudaEventRecord(e1, s));
    std::vector<FusedOut> out(count);
    std::vector<int32_t> rstat(4 * (size_t)count * (size_t)R);
    std::vector<double> offs(count);
    LPP_CUDA(cudaMemcpyAsync(out.data(), F.out, sizeof(FusedOut) * out.size(), cudaMemcpyDeviceToHost, s));
    LPP_CUDA(cudaMemcpyAsync(rstat.data(), F.rstat, sizeof(int32_t) * rstat.size(), cudaMemcpyDeviceToHost, s));
    LPP_CUDA(cudaMemcpyAsync(offs.data(), E.K.offset, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
    std::vector<DevStatus> sts(count);
    LPP_CUDA(cudaMemcpyAsync(sts.data(), F.st, sizeof(DevStatus) * count, cudaMemcpyDeviceToHost, s));
    LPP_CUDA(cudaStreamSynchronize(s));
    for (auto &x : sts)
        if (x.err) throw StatusError(LPP_ERR_CUDA, "internal: S5 hash table overflow (batch)");
    float ms = 0.f;
    LPP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    g_tuner.record(key, cand, ms);
    E.loop_ms = ms;
    // per-LP verdicts and counters for the records
    E.lp_status.assign(count, LPP_OK);
    E.lp_where.assign(count, LPP_WHERE_NONE);
    E.lp_index.assign(count, -1);
    E.lp_round.assign(count, 0);
    E.lp_rounds.assign(count, 0);
    int64_t proc = 0;
    for (int32_t k = 0; k < count; k++) {
        E.lp_status[k] = out[k].status;
        E.lp_where[k] = out[k].where;
        E.lp_index[k] = out[k].index;
        E.lp_round[k] = out[k].round;
        E.lp_rounds[k] = out[k].rounds;
        for (int32_t r = 0; r < out[k].rounds; r++) proc += rstat[4 * ((size_t)k * R + r)];
    }
    E.nnz_processed = proc;
    // records: the engine's record arrays, the fused outputs for bounds, maps
    // and activities (each LP's at its own ranges)
    auto D = std::make_shared<DeviceRecords>();
    D->m0 = m0;
    D->n0 = n0;
    D->n_final = n0;
    D->act_m = m0;
    D->rk = E.rec_rk;
    D->rr = E.rec_rr;
    D->ra = E.rec_ra;
    D->rv = E.rec_rv;
    D->ck = E.rec_ck;
    D->cr = E.rec_cr;
    D->cv = E.rec_cv;
    D->lu = F.o_lu;
    D->cmap = F.o_fcmap;
    D->act = F.o_act;
    D->ninf = F.o_ninf;
    D->act_rmap = F.o_armap;
    for (void *p : {(void *)D->rk, (void *)D->rr, (void *)D->ra, (void *)D->rv, (void *)D->ck, (void *)D->cr,
                    (void *)D->cv, (void *)D->lu, (void *)D->cmap, (void *)D->act, (void *)D->ninf,
                    (void *)D->act_rmap}) {
        P.forget(p);
        D->owned.push_back(p);
    }
    auto store = std::make_shared<SharedStore>();
    for (void *p : {(void *)F.o_rp, (void *)F.o_tp, (void *)F.o_ci, (void *)F.o_ti, (void *)F.o_rv, (void *)F.o_tv,
                    (void *)F.o_L, (void *)F.o_U, (void *)F.o_rmap, (void *)F.o_c, (void *)F.o_lb, (void *)F.o_ub,
                    (void *)F.o_cmap}) {
        P.forget(p);
        store->ptrs.push_back(p);
    }
    for (int32_t k = 0; k < count; k++) {
        const FusedLP &L = lps[k];
        auto *Rd = new lpp_reduced();
        Rd->m = out[k].m;
        Rd->n = out[k].n;
        Rd->nnz = out[k].nnz;
        Rd->obj_offset = offs[k];
        Rd->rp = F.o_rp + L.row_off + k;
        Rd->tp = F.o_tp + L.col_off + k;
        Rd->ci = F.o_ci + L.nnz_off;
        Rd->rv = F.o_rv + L.nnz_off;
        Rd->ti = F.o_ti + L.nnz_off;
        Rd->tv = F.o_tv + L.nnz_off;
        Rd->L = F.o_L + L.row_off;
        Rd->U = F.o_U + L.row_off;
        Rd->c = F.o_c + L.col_off;
        Rd->lb = F.o_lb + L.col_off;
        Rd->ub = F.o_ub + L.col_off;
        Rd->rmap = F.o_rmap + L.row_off;
        Rd->cmap = F.o_cmap + L.col_off;
        Rd->shared = store;
        outs[k] = Rd;
        lpp_postsolve *Pk = make_postsolve(E, D, k, Rd->m, Rd->n, Rd->nnz, offs[k], L.col_off, L.row_off, out[k].act_m);
        const int32_t rk = out[k].rounds;
        Pk->r_nnz.assign(rk, 0);
        Pk->r_rows.assign(rk, 0);
        Pk->r_cols.assign(rk, 0);
        Pk->r_bounds.assign(rk, 0);
        Pk->r_ms.assign(rk, 0.f);
        for (int32_t r = 0; r < rk; r++) {
            const int32_t *q = &rstat[4 * ((size_t)k * R + r)];
            Pk->r_nnz[r] = q[0];
            Pk->r_rows[r] = q[1];
            Pk->r_cols[r] = q[2];
            Pk->r_bounds[r] = q[3];
        }
        Pk->info.s5_left = out[k].s5_left;
        recs[k] = Pk;
        per_lp[k] = (lpp_status)Pk->info.status;
    }
    return true;
}

}  // namespace

lpp_status lpp_noalloc_fail(lpp_status st, const char *msg) { return set_err(st, msg); }

extern "C" {

void lpp_opts_default(lpp_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->feas_tol = 1e-9;
    o->bound_tol = 1e-6;
    o->huge = 1e20;
    o->max_implied = 1e10;
    o->par_tol = 1e-12;
    o->max_rounds = 20;
    o->dual_reductions = 1;
    o->par_max_iter = 16;
    o->parallel_cols = 0;
    o->col_singletons = 0;
    o->dual_fixing = 0;
    o->doubletons = 0;
    o->batch_persistent = 1;
    o->dual_records = 0;
    o->dep_rows = 0;
    o->timing = 0;
    o->device = 0;
    o->stream = nullptr;
}

const char *lpp_last_error(void) { return g_err.c_str(); }

lpp_status lpp_presolve(const lpp_lp *in, const lpp_opts *opts, lpp_reduced **out, lpp_postsolve **rec) {
    return guarded([&]() -> lpp_status {
        if (!out || !rec) throw StatusError(LPP_ERR_INVALID, "out/rec is NULL");
        *out = nullptr;
        *rec = nullptr;
        check_lp_shape(in);
        const lpp_opts o = resolve_opts(opts);
        auto E = std::make_unique<Engine>();
        Member mm{in->m, in->n, in->nnz, 0, 0, 0, in->obj_offset};
        E->lazy_req = true;  // the CSC is compacted once, at the end, when no step reads it
        E->setup(o, 1, {mm});
        // ingest: checks, copies, CSC, schedules (bytes: the input once, the CSC written)
        E->tbegin(F_INGEST, 24.0 * in->nnz + 48.0 * in->m + 40.0 * in->n);
        E->ingest_plain(*in);
        E->prepare();
        E->tend();
        E->run();
        E->tbegin(F_FINISH, 0.0);  // records and the reduced LP handed over
        double offset = 0.0;
        LPP_CUDA(cudaMemcpyAsync(&offset, E->K.offset, sizeof(double), cudaMemcpyDeviceToHost, E->s));
        auto D = take_records(*E);
        // the reduced LP takes the current buffers
        auto *R = new lpp_reduced();
        const int c = E->cur;
        R->m = E->m;
        R->n = E->n;
        R->nnz = E->nnz;
        R->rp = E->rp[c];
        R->ci = E->ci[c];
        R->rv = E->rv[c];
        R->tp = E->tp[c];
        R->ti = E->ti[c];
        R->tv = E->tv[c];
        R->L = E->L[c];
        R->U = E->U[c];
        R->c = E->c[c];
        R->rmap = E->rmap[c];
        R->cmap = E->cmap[c];
        for (void *p : {(void *)R->rp, (void *)R->ci, (void *)R->rv, (void *)R->tp, (void *)R->ti, (void *)R->tv,
                        (void *)R->L, (void *)R->U, (void *)R->c, (void *)R->rmap, (void *)R->cmap}) {
            E->pool.forget(p);
            R->owned.push_back(p);
        }
        R->lb = E->pool.alloc<double>(R->n);
        R->ub = E->pool.alloc<double>(R->n);
        E->pool.forget(R->lb);
        E->pool.forget(R->ub);
        R->owned.push_back(R->lb);
        R->owned.push_back(R->ub);
        split_lu(D->lu, R->n, R->lb, R->ub, E->s);
        E->tend();
        LPP_CUDA(cudaStreamSynchronize(E->s));
        R->obj_offset = offset;
        lpp_postsolve *P = make_postsolve(*E, D, 0, R->m, R->n, R->nnz, offset, 0, 0, E->act_m);
        *out = R;
        *rec = P;
        return (lpp_status)P->info.status;
    });
}

lpp_status lpp_presolve_batch(const lpp_lp *ins, int32_t count, const lpp_opts *opts, lpp_reduced **outs,
                              lpp_postsolve **recs, lpp_status *per_lp) {
    return guarded([&]() -> lpp_status {
        if (count < 0 || (count > 0 && (!ins || !outs || !recs || !per_lp)))
            throw StatusError(LPP_ERR_INVALID, "bad batch arguments");
        if (count == 0) return LPP_OK;
        for (int32_t k = 0; k < count; k++) {
            outs[k] = nullptr;
            recs[k] = nullptr;
            per_lp[k] = LPP_ERR_INVALID;
        }
        const lpp_opts o = resolve_opts(opts);
        if (o.dep_rows) throw StatusError(LPP_ERR_INVALID, "dep_rows: lpp_presolve only");
        std::vector<Member> mem(count);
        int64_t ro = 0, co = 0, zo = 0;
        for (int32_t k = 0; k < count; k++) {
            check_lp_shape(&ins[k]);
            mem[k] = Member{ins[k].m, ins[k].n, ins[k].nnz, (int32_t)ro, (int32_t)co, zo, ins[k].obj_offset};
            ro += ins[k].m;
            co += ins[k].n;
            zo += ins[k].nnz;
            if (ro >= 2147483647LL || co >= 2147483647LL || zo >= 2147483647LL)
                throw StatusError(LPP_ERR_INVALID, "batch too large for int32 indices");
        }
        auto E = std::make_unique<Engine>();
        E->lazy_req = true;  // the CSC is compacted once, at the end, when no step reads it
        E->setup(o, count, mem);
        E->ingest_batch(ins, count);
        E->prepare();
        if (batch_fused(*E, mem, count, outs, recs, per_lp)) return LPP_OK;
        E->run();
        cudaStream_t s = E->s;
        const int c = E->cur;
        std::vector<double> offs(count);
        LPP_CUDA(cudaMemcpyAsync(offs.data(), E->K.offset, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
        // rows of each LP in the numbering of the last round's start (activities)
        int32_t *acnt = E->pool.alloc<int32_t>(count);
        LPP_CUDA(cudaMemsetAsync(acnt, 0, sizeof(int32_t) * (size_t)count, s));
        if (E->act_m > 0) (k_count_rows_lp<<<nblk(E->act_m), 256, 0, s>>>(E->lprow[E->act_buf], E->act_m, acnt), note_launch());
        std::vector<int32_t> acnt_h(count);
        LPP_CUDA(cudaMemcpyAsync(acnt_h.data(), acnt, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, s));
        auto D = take_records(*E);
        // per-LP sizes of the reduced arena
        int32_t *cnt = E->pool.alloc<int32_t>(3 * (size_t)count);
        LPP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * 3 * (size_t)count, s));
        (k_count_lp<<<nblk(std::max(E->m, E->n)), 256, 0, s>>>(E->lprow[c], E->rp[c], E->m, E->lpcol[c], E->n, cnt,
                                                                cnt + count, cnt + 2 * count), note_launch());
        std::vector<int32_t> hc(3 * (size_t)count);
        LPP_CUDA(cudaMemcpyAsync(hc.data(), cnt, sizeof(int32_t) * hc.size(), cudaMemcpyDeviceToHost, s));
        LPP_CUDA(cudaStreamSynchronize(s));
        // tables: row/col/nnz starts (reduced) and original offsets
        std::vector<int32_t> tab(5 * (size_t)count);
        int32_t rs = 0, cs = 0, zs = 0;
        for (int32_t k = 0; k < count; k++) {
            tab[k] = rs;
            tab[count + k] = cs;
            tab[2 * count + k] = zs;
            tab[3 * count + k] = mem[k].row_off;
            tab[4 * count + k] = mem[k].col_off;
            rs += hc[k];
            cs += hc[count + k];
            zs += hc[2 * count + k];
        }
        int32_t *dtab = E->pool.alloc<int32_t>(tab.size());
        LPP_CUDA(cudaMemcpyAsync(dtab, tab.data(), sizeof(int32_t) * tab.size(), cudaMemcpyHostToDevice, s));
        const int32_t *row_start = dtab, *col_start = dtab + count, *nnz_start = dtab + 2 * count;
        const int32_t *row_orig = dtab + 3 * count, *col_orig = dtab + 4 * count;
        int32_t *rows = cnt, *cols = cnt + count, *nnzs = cnt + 2 * count;
        // shared storage of all reduced LPs
        auto store = std::make_shared<SharedStore>();
        int32_t *rp_out = E->pool.alloc<int32_t>((size_t)E->m + count);
        int32_t *tp_out = E->pool.alloc<int32_t>((size_t)E->n + count);
        int32_t *rmap_out = E->pool.alloc<int32_t>(E->m);
        int32_t *cmap_out = E->pool.alloc<int32_t>(E->n);
        double *lb = E->pool.alloc<double>(E->n), *ub = E->pool.alloc<double>(E->n);
        if (E->m > 0)
            (k_rebase_rows<<<nblk(E->m), 256, 0, s>>>(E->rp[c], E->lprow[c], E->rmap[c], E->m, nnz_start, row_orig,
                                                     rp_out, rmap_out), note_launch());
        if (E->n > 0)
            (k_rebase_cols<<<nblk(E->n), 256, 0, s>>>(E->tp[c], E->lpcol[c], E->cmap[c], E->n, nnz_start, col_orig,
                                                     tp_out, cmap_out), note_launch());
        (k_ptr_tails<<<nblk(count), 256, 0, s>>>(row_start, rows, col_start, cols, nnzs, count, rp_out, tp_out), note_launch());
        if (E->m > 0) (k_rebase_idx<<<nblk(E->m), 256, 0, s>>>(E->ci[c], E->rp[c], E->lprow[c], E->m, col_start), note_launch());
        if (E->n > 0) (k_rebase_idx<<<nblk(E->n), 256, 0, s>>>(E->ti[c], E->tp[c], E->lpcol[c], E->n, row_start), note_launch());
        split_lu(E->lu[c], E->n, lb, ub, s);
        LPP_CUDA(cudaGetLastError());
        LPP_CUDA(cudaStreamSynchronize(s));
        for (void *p : {(void *)rp_out, (void *)tp_out, (void *)rmap_out, (void *)cmap_out, (void *)lb, (void *)ub,
                        (void *)E->ci[c], (void *)E->rv[c], (void *)E->ti[c], (void *)E->tv[c], (void *)E->L[c],
                        (void *)E->U[c], (void *)E->c[c]}) {
            E->pool.forget(p);
            store->ptrs.push_back(p);
        }
        int32_t astart = 0;
        for (int32_t k = 0; k < count; k++) {
            auto *R = new lpp_reduced();
            const int32_t r0 = tab[k], c0 = tab[count + k], z0 = tab[2 * count + k];
            R->m = hc[k];
            R->n = hc[count + k];
            R->nnz = hc[2 * count + k];
            R->obj_offset = offs[k];
            R->rp = rp_out + r0 + k;
            R->tp = tp_out + c0 + k;
            R->ci = E->ci[c] + z0;
            R->rv = E->rv[c] + z0;
            R->ti = E->ti[c] + z0;
            R->tv = E->tv[c] + z0;
            R->L = E->L[c] + r0;
            R->U = E->U[c] + r0;
            R->c = E->c[c] + c0;
            R->lb = lb + c0;
            R->ub = ub + c0;
            R->rmap = rmap_out + r0;
            R->cmap = cmap_out + c0;
            R->shared = store;
            outs[k] = R;
            recs[k] = make_postsolve(*E, D, k, R->m, R->n, R->nnz, offs[k], c0, astart, acnt_h[k]);
            astart += acnt_h[k];
            per_lp[k] = (lpp_status)recs[k]->info.status;
        }
        return LPP_OK;
    });
}

lpp_status lpp_reduced_view(lpp_reduced *R, lpp_lp *v, int32_t on_device) {
    return guarded([&]() -> lpp_status {
        if (!R || !v) throw StatusError(LPP_ERR_INVALID, "NULL argument");
        std::memset(v, 0, sizeof *v);
        v->m = R->m;
        v->n = R->n;
        v->nnz = R->nnz;
        v->obj_offset = R->obj_offset;
        if (on_device) {
            v->row_ptr = R->rp;
            v->col_idx = R->ci;
            v->val = R->rv;
            v->c = R->c;
            v->lhs = R->L;
            v->rhs = R->U;
            v->lb = R->lb;
            v->ub = R->ub;
            v->on_device = 1;
            return LPP_OK;
        }
        materialize_host(R, 0);
        v->row_ptr = R->h_rp;
        v->col_idx = R->h_ci;
        v->val = R->h_rv;
        v->c = R->h_c;
        v->lhs = R->h_L;
        v->rhs = R->h_U;
        v->lb = R->h_lb;
        v->ub = R->h_ub;
        v->on_device = 0;
        return LPP_OK;
    });
}

lpp_status lpp_reduced_csc(lpp_reduced *R, const int32_t **col_ptr, const int32_t **row_idx, const double **val,
                           int32_t on_device) {
    return guarded([&]() -> lpp_status {
        if (!R) throw StatusError(LPP_ERR_INVALID, "NULL reduced");
        if (on_device) {
            if (col_ptr) *col_ptr = R->tp;
            if (row_idx) *row_idx = R->ti;
            if (val) *val = R->tv;
        } else {
            materialize_host(R, 2);
            if (col_ptr) *col_ptr = R->h_tp;
            if (row_idx) *row_idx = R->h_ti;
            if (val) *val = R->h_tv;
        }
        return LPP_OK;
    });
}

lpp_status lpp_reduced_maps(lpp_reduced *R, const int32_t **row_map, const int32_t **col_map, int32_t on_device) {
    return guarded([&]() -> lpp_status {
        if (!R) throw StatusError(LPP_ERR_INVALID, "NULL reduced");
        if (on_device) {
            if (row_map) *row_map = R->rmap;
            if (col_map) *col_map = R->cmap;
        } else {
            materialize_host(R, 1);
            if (row_map) *row_map = R->h_rmap;
            if (col_map) *col_map = R->h_cmap;
        }
        return LPP_OK;
    });
}

lpp_status lpp_result_info(const lpp_postsolve *P, lpp_info *info) {
    if (!P || !info) return set_err(LPP_ERR_INVALID, "NULL argument");
    *info = P->info;
    return LPP_OK;
}

lpp_status lpp_result_rows(const lpp_postsolve *Pc, int32_t *kind, int32_t *round, int32_t *aux, double *val) {
    if (!Pc) return set_err(LPP_ERR_INVALID, "NULL record");
    lpp_postsolve *P = const_cast<lpp_postsolve *>(Pc);
    const lpp_status st = guarded([&]() -> lpp_status { materialize(P); return LPP_OK; });
    if (st != LPP_OK) return st;
    const size_t m = P->row_kind.size();
    if (kind && m) std::memcpy(kind, P->row_kind.data(), 4 * m);
    if (round && m) std::memcpy(round, P->row_round.data(), 4 * m);
    if (aux && m) std::memcpy(aux, P->row_aux.data(), 4 * m);
    if (val && m) std::memcpy(val, P->row_val.data(), 8 * m);
    return LPP_OK;
}

lpp_status lpp_result_cols(const lpp_postsolve *Pc, int32_t *kind, int32_t *round, double *val, double *lb,
                           double *ub) {
    if (!Pc) return set_err(LPP_ERR_INVALID, "NULL record");
    lpp_postsolve *P = const_cast<lpp_postsolve *>(Pc);
    const lpp_status st = guarded([&]() -> lpp_status { materialize(P); return LPP_OK; });
    if (st != LPP_OK) return st;
    const size_t n = P->col_kind.size();
    if (kind && n) std::memcpy(kind, P->col_kind.data(), 4 * n);
    if (round && n) std::memcpy(round, P->col_round.data(), 4 * n);
    if (val && n) std::memcpy(val, P->col_val.data(), 8 * n);
    if (lb && n) std::memcpy(lb, P->col_lb.data(), 8 * n);
    if (ub && n) std::memcpy(ub, P->col_ub.data(), 8 * n);
    return LPP_OK;
}

lpp_status lpp_result_merges(const lpp_postsolve *Pc, int32_t *leader, int32_t *pass, double *bounds) {
    if (!Pc) return set_err(LPP_ERR_INVALID, "NULL record");
    lpp_postsolve *P = const_cast<lpp_postsolve *>(Pc);
    const lpp_status st = guarded([&]() -> lpp_status { materialize(P); return LPP_OK; });
    if (st != LPP_OK) return st;
    const size_t n = P->col_kind.size();
    if (leader && n) std::memcpy(leader, P->col_aux.data(), 4 * n);
    if (pass && n) std::memcpy(pass, P->col_pass.data(), 4 * n);
    if (bounds && n) std::memcpy(bounds, P->col_mrg.data(), 32 * n);
    return LPP_OK;
}

lpp_status lpp_result_bound_sources(const lpp_postsolve *Pc, int32_t *lsrc, int32_t *lrnd, int32_t *usrc,
                                    int32_t *urnd) {
    if (!Pc) return set_err(LPP_ERR_INVALID, "NULL record");
    lpp_postsolve *P = const_cast<lpp_postsolve *>(Pc);
    const lpp_status st = guarded([&]() -> lpp_status { materialize(P); return LPP_OK; });
    if (st != LPP_OK) return st;
    const size_t n = P->col_kind.size();
    if (P->col_lsrc.size() != n || !P->dev->bs)
        return set_err(LPP_ERR_INVALID, "no bound sources: the presolve ran without opts.dual_records");
    if (lsrc && n) std::memcpy(lsrc, P->col_lsrc.data(), 4 * n);
    if (lrnd && n) std::memcpy(lrnd, P->col_lrnd.data(), 4 * n);
    if (usrc && n) std::memcpy(usrc, P->col_usrc.data(), 4 * n);
    if (urnd && n) std::memcpy(urnd, P->col_urnd.data(), 4 * n);
    return LPP_OK;
}

lpp_status lpp_result_substitutions(const lpp_postsolve *Pc, int64_t *beg, int32_t *len, double *rhs, int64_t cap,
                                    int32_t *col, double *val, int64_t *total) {
    if (!Pc || cap < 0) return set_err(LPP_ERR_INVALID, "bad argument");
    lpp_postsolve *P = const_cast<lpp_postsolve *>(Pc);
    const lpp_status st = guarded([&]() -> lpp_status { materialize(P); return LPP_OK; });
    if (st != LPP_OK) return st;
    const size_t m = P->sub_beg.size();
    const int64_t T = (int64_t)P->sub_col.size();
    if (beg && m) std::memcpy(beg, P->sub_beg.data(), 8 * m);
    if (len && m) std::memcpy(len, P->sub_len.data(), 4 * m);
    if (rhs && m) std::memcpy(rhs, P->sub_rhs.data(), 8 * m);
    const int64_t w = std::min(cap, T);
    if (col && w) std::memcpy(col, P->sub_col.data(), 4 * (size_t)w);
    if (val && w) std::memcpy(val, P->sub_val.data(), 8 * (size_t)w);
    if (total) *total = T;
    return LPP_OK;
}

lpp_status lpp_result_activity(const lpp_postsolve *Pc, double *act_min, double *act_max, int32_t *ninf_min,
                               int32_t *ninf_max) {
    if (!Pc) return set_err(LPP_ERR_INVALID, "NULL record");
    lpp_postsolve *P = const_cast<lpp_postsolve *>(Pc);
    const lpp_status st = guarded([&]() -> lpp_status { materialize(P); return LPP_OK; });
    if (st != LPP_OK) return st;
    const size_t m = P->act_min.size();
    if (act_min && m) std::memcpy(act_min, P->act_min.data(), 8 * m);
    if (act_max && m) std::memcpy(act_max, P->act_max.data(), 8 * m);
    if (ninf_min && m) std::memcpy(ninf_min, P->ninf_min.data(), 4 * m);
    if (ninf_max && m) std::memcpy(ninf_max, P->ninf_max.data(), 4 * m);
    return LPP_OK;
}

lpp_status lpp_result_rounds(const lpp_postsolve *P, int32_t cap, int64_t *nnz, int32_t *rows_removed,
                             int32_t *cols_fixed, int32_t *bounds_changed, float *ms, int32_t *rounds) {
    if (!P || cap < 0) return set_err(LPP_ERR_INVALID, "bad argument");
    const int32_t R = (int32_t)P->r_nnz.size();
    if (rounds) *rounds = R;
    for (int32_t r = 0; r < R && r < cap; r++) {
        if (nnz) nnz[r] = P->r_nnz[r];
        if (rows_removed) rows_removed[r] = P->r_rows[r];
        if (cols_fixed) cols_fixed[r] = P->r_cols[r];
        if (bounds_changed) bounds_changed[r] = P->r_bounds[r];
        if (ms) ms[r] = P->r_ms[r];
    }
    return LPP_OK;
}

lpp_status lpp_result_kernels(const lpp_postsolve *P, int32_t cap, lpp_kernel_stat *stats, int32_t *count) {
    if (!P || cap < 0) return set_err(LPP_ERR_INVALID, "bad argument");
    const int32_t K = (int32_t)P->kstats.size();
    if (count) *count = K;
    for (int32_t k = 0; k < K && k < cap && stats; k++) stats[k] = P->kstats[k];
    return LPP_OK;
}

lpp_status lpp_postsolve_primal(const lpp_postsolve *Pc, const double *x_red, double *x_orig) {
    if (!Pc || !x_orig) return set_err(LPP_ERR_INVALID, "NULL argument");
    lpp_postsolve *P = const_cast<lpp_postsolve *>(Pc);
    const lpp_status st = guarded([&]() -> lpp_status { materialize(P); return LPP_OK; });
    if (st != LPP_OK) return st;
    if (!x_red && !P->col_map.empty()) return set_err(LPP_ERR_INVALID, "NULL argument");
    PostsolveRecords R;
    R.n = (int64_t)P->col_kind.size();
    R.m = (int64_t)P->row_kind.size();
    R.n_red = (int64_t)P->col_map.size();
    R.col_kind = P->col_kind.data();
    R.col_round = P->col_round.data();
    R.col_aux = P->col_aux.data();
    R.col_map = P->col_map.data();
    R.col_val = P->col_val.data();
    R.col_mrg = P->col_mrg.data();
    R.row_kind = P->row_kind.data();
    R.row_round = P->row_round.data();
    R.row_aux = P->row_aux.data();
    R.row_val = P->row_val.data();
    R.sub_beg = P->sub_beg.data();
    R.sub_len = P->sub_len.data();
    R.sub_col = P->sub_col.data();
    R.sub_rhs = P->sub_rhs.data();
    R.sub_val = P->sub_val.data();
    R.sub_size = (int64_t)P->sub_col.size();
    const char *err = postsolve_primal(R, x_red, x_orig);
    return err ? set_err(LPP_ERR_INVALID, err) : LPP_OK;
}

lpp_status lpp_postsolve_dual(const lpp_postsolve *Pc, const lpp_lp *lp, const double *x_red, const double *y_red,
                              double *x_orig, double *y_orig, double *z_orig) {
    if (!Pc || !lp) return set_err(LPP_ERR_INVALID, "NULL argument");
    lpp_postsolve *P = const_cast<lpp_postsolve *>(Pc);
    const lpp_status st = guarded([&]() -> lpp_status { materialize(P); return LPP_OK; });
    if (st != LPP_OK) return st;
    if (!P->dev->bs || P->col_lsrc.size() != P->col_kind.size())
        return set_err(LPP_ERR_INVALID, "no bound sources: the presolve ran without opts.dual_records");
    if (P->info.status != LPP_OK) return set_err(LPP_ERR_INVALID, "the presolve did not end with LPP_OK");
    const int64_t m = P->info.m, n = P->info.n;
    if (lp->on_device) return set_err(LPP_ERR_INVALID, "lpp_postsolve_dual reads the LP from host memory");
    if (lp->m != m || lp->n != n) return set_err(LPP_ERR_INVALID, "the LP's sizes differ from the presolved LP's");
    if ((m && (!lp->row_ptr || !lp->lhs || !lp->rhs || !y_orig)) || (n && (!lp->c || !x_orig || !z_orig)) ||
        (lp->nnz && (!lp->col_idx || !lp->val)))
        return set_err(LPP_ERR_INVALID, "NULL argument");
    if ((P->info.m_red && !y_red) || (P->info.n_red && !x_red)) return set_err(LPP_ERR_INVALID, "NULL argument");
    if (m && (lp->row_ptr[0] != 0 || lp->row_ptr[m] != lp->nnz))
        return set_err(LPP_ERR_INVALID, "the LP's row pointers do not match its nonzero count");
    for (int64_t i = 0; i < m; i++)
        if (lp->row_ptr[i + 1] < lp->row_ptr[i]) return set_err(LPP_ERR_INVALID, "row pointers decrease");
    for (int64_t k = 0; k < lp->nnz; k++)
        if (lp->col_idx[k] < 0 || lp->col_idx[k] >= n) return set_err(LPP_ERR_INVALID, "column index out of range");
    // the reduced rows are the kept rows in their input order
    std::vector<int32_t> row_map;
    row_map.reserve((size_t)P->info.m_red);
    for (int64_t i = 0; i < m; i++)
        if (P->row_kind[i] == LPP_ROW_KEPT) row_map.push_back((int32_t)i);
    if ((int64_t)row_map.size() != P->info.m_red) return set_err(LPP_ERR_INVALID, "corrupt row records");
    const lpp_status ps = lpp_postsolve_primal(Pc, x_red, x_orig);
    if (ps != LPP_OK) return ps;
    DualRecords D;
    D.m = m;
    D.n = n;
    D.m_red = P->info.m_red;
    D.row_ptr = lp->row_ptr;
    D.col_idx = lp->col_idx;
    D.val = lp->val;
    D.c = lp->c;
    D.lhs = lp->lhs;
    D.rhs = lp->rhs;
    D.huge = P->huge;
    D.row_map = row_map.data();
    D.row_kind = P->row_kind.data();
    D.row_round = P->row_round.data();
    D.row_aux = P->row_aux.data();
    D.row_val = P->row_val.data();
    D.col_kind = P->col_kind.data();
    D.lsrc = P->col_lsrc.data();
    D.lrnd = P->col_lrnd.data();
    D.usrc = P->col_usrc.data();
    D.urnd = P->col_urnd.data();
    const char *err = nullptr;
    const lpp_status gs = guarded([&]() -> lpp_status {
        err = postsolve_dual(D, x_orig, y_red, y_orig, z_orig);
        return LPP_OK;
    });
    if (gs != LPP_OK) return gs;
    return err ? set_err(LPP_ERR_INVALID, err) : LPP_OK;
}

void lpp_free_reduced(lpp_reduced *R) {
    if (!R) return;
    if (R->hblock) pinned_put(R->hblock);
    for (void *p : R->owned) cudaFree(p);
    delete R;
}

void lpp_free_postsolve(lpp_postsolve *P) { delete P; }

void lpp_free_results(lpp_reduced *const *reds, lpp_postsolve *const *recs, int32_t count) {
    for (int32_t k = 0; k < count; k++) {
        if (reds) lpp_free_reduced(reds[k]);
        if (recs) lpp_free_postsolve(recs[k]);
    }
}

}  // extern "C"
