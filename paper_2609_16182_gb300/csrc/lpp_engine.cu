// lpp_engine.cu -- device state and the round loop (S0 .. S8) of the presolve.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>

#include "lpp_engine.h"
#include "deprows.h"

namespace lpp {

void cuda_check(cudaError_t e, const char *expr, const char *file, int line) {
    if (e == cudaSuccess) return;
    char buf[512];
    std::snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", expr, cudaGetErrorString(e), file, line);
    if (e == cudaErrorMemoryAllocation) throw StatusError(LPP_ERR_OOM, buf);
    throw CudaError(e, buf);
}

void DevPool::forget(void *p) {
    auto it = std::find(ptrs.begin(), ptrs.end(), p);
    if (it != ptrs.end()) {
        sizes.erase(sizes.begin() + (it - ptrs.begin()));
        ptrs.erase(it);
    }
}
void DevPool::release() {
    if (ptrs.empty()) return;
    const bool done = cache && cudaStreamSynchronize(s) == cudaSuccess;
    for (size_t k = 0; k < ptrs.size(); k++) {
        if (done) dev_cache_put(ptrs[k], sizes[k], s);
        else cudaFreeAsync(ptrs[k], s);
    }
    ptrs.clear();
    sizes.clear();
}

namespace {
std::mutex g_dev_mu;
std::multimap<std::pair<int, size_t>, void *> g_dev_free;
size_t g_dev_free_bytes = 0;
constexpr size_t kDevCacheMax = size_t(16) << 30;  // beyond this, released blocks are freed
}  // namespace

void *dev_cache_take(size_t bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> g(g_dev_mu);
    auto it = g_dev_free.find({dev, bytes});
    if (it == g_dev_free.end()) return nullptr;
    void *p = it->second;
    g_dev_free.erase(it);
    g_dev_free_bytes -= bytes;
    return p;
}

void dev_cache_put(void *p, size_t bytes, cudaStream_t s) {
    int dev = 0;
    bool keep = cudaGetDevice(&dev) == cudaSuccess;
    {
        std::lock_guard<std::mutex> g(g_dev_mu);
        keep = keep && g_dev_free_bytes + bytes <= kDevCacheMax;
        if (keep) {
            g_dev_free.emplace(std::make_pair(dev, bytes), p);
            g_dev_free_bytes += bytes;
        }
    }
    if (!keep) cudaFreeAsync(p, s);
}

// Pinned host buffers (status mirrors, host copies of reduced LPs) are reused
// across presolves: pinning memory costs far more than the rounds of a small LP.
static std::mutex g_pin_mu;
static std::vector<std::pair<size_t, void *>> g_pin_free;

// best fit among the free buffers, and none more than 4x (+ 1 MiB) the
// request: a status mirror must not take the block a reduced LP needs next
static void *pinned_get(size_t bytes) {
    bytes = std::max<size_t>(bytes, 64);
    {
        std::lock_guard<std::mutex> g(g_pin_mu);
        size_t best = g_pin_free.size();
        for (size_t k = 0; k < g_pin_free.size(); k++) {
            const size_t cap = g_pin_free[k].first;
            if (cap >= bytes && cap <= 4 * bytes + (1u << 20) &&
                (best == g_pin_free.size() || cap < g_pin_free[best].first))
                best = k;
        }
        if (best < g_pin_free.size()) {
            void *p = g_pin_free[best].second;
            g_pin_free.erase(g_pin_free.begin() + (long)best);
            return p;
        }
    }
    void *p = nullptr;
    LPP_CUDA(cudaMallocHost(&p, bytes));
    std::memset(p, 0, bytes);
    return p;
}

// remembers a pinned buffer's capacity so it can be handed out again
static std::mutex g_cap_mu;
static std::vector<std::pair<void *, size_t>> g_pin_cap;

void *pinned_get_sized(size_t bytes) {
    bytes = std::max<size_t>(bytes, 64);
    void *p = pinned_get(bytes);
    std::lock_guard<std::mutex> g(g_cap_mu);
    bool known = false;
    for (auto &e : g_pin_cap)
        if (e.first == p) known = true;
    if (!known) g_pin_cap.emplace_back(p, bytes);
    return p;
}

void pinned_put(void *p) {
    if (!p) return;
    size_t cap = 0;
    {
        std::lock_guard<std::mutex> g(g_cap_mu);
        for (auto &e : g_pin_cap)
            if (e.first == p) cap = e.second;
    }
    std::lock_guard<std::mutex> g(g_pin_mu);
    g_pin_free.emplace_back(cap, p);
}

namespace {

// Freed device memory stays in the device's default pool (stream-ordered
// allocations are then reused by the next presolve instead of being mapped
// again); set once per device.
std::mutex g_pool_mu;
bool g_pool_done[256] = {};

void keep_pool_memory(int dev) {
    std::lock_guard<std::mutex> g(g_pool_mu);
    if (dev < 0 || dev >= 256 || g_pool_done[dev]) return;
    cudaMemPool_t mp;
    if (cudaDeviceGetDefaultMemPool(&mp, dev) == cudaSuccess) {
        uint64_t thr = ~0ULL;
        cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    g_pool_done[dev] = true;
}

int32_t pow2_at_least(int64_t v) {
    int64_t p = 2;
    while (p < v) p <<= 1;
    return (int32_t)p;
}

// batch ingest from device inputs: one block row per LP copies and rebases
struct SrcDesc {
    const int32_t *rp, *ci;
    const double *v, *c, *lhs, *rhs, *lb, *ub;
    int32_t m, n;
    int64_t nnz;
    int32_t row_off, col_off;
    int64_t nnz_off;
};

__global__ void k_gather_lps(const SrcDesc *d, int32_t *rp, int32_t *ci, double *v, double *lhs, double *rhs,
                             double *lb, double *ub, double *c, int32_t *lprow, int32_t *lpcol, int32_t *err) {
    const SrcDesc D = d[blockIdx.y];
    const int32_t k = blockIdx.y;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = t0; i < D.m; i += step) {
        const int32_t p = D.rp[i];
        if (p < 0 || p > D.nnz) atomicOr(err, 1);
        rp[D.row_off + i] = (int32_t)(D.nnz_off + p);
        lhs[D.row_off + i] = D.lhs[i];
        rhs[D.row_off + i] = D.rhs[i];
        lprow[D.row_off + i] = k;
    }
    if (t0 == 0 && (D.rp[0] != 0 || D.rp[D.m] != D.nnz)) atomicOr(err, 1);
    for (int64_t j = t0; j < D.n; j += step) {
        lb[D.col_off + j] = D.lb[j];
        ub[D.col_off + j] = D.ub[j];
        c[D.col_off + j] = D.c[j];
        lpcol[D.col_off + j] = k;
    }
    for (int64_t e = t0; e < D.nnz; e += step) {
        const int32_t j = D.ci[e];
        if (j < 0 || j >= D.n) atomicOr(err, 2);
        ci[D.nnz_off + e] = D.col_off + j;
        v[D.nnz_off + e] = D.v[e];
    }
}

__global__ void k_set_i32(int32_t *p, int32_t v) { *p = v; }
__global__ void k_csc_sizes(const CompactCtx K, int32_t n, DevStatus *st) {
    st->n_new = K.c_pos[n];
    st->nnz_new_t = K.c_off[n];
}

// cols_in_place: the column slots stay (n), the CSC is not compacted
__global__ void k_sizes(const CompactCtx K, int32_t m, int32_t n, int32_t cols_in_place, DevStatus *st) {
    st->m_new = K.r_pos[m];
    st->nnz_new = K.r_off[m];
    st->n_new = cols_in_place ? n : K.c_pos[n];
    st->nnz_new_t = cols_in_place ? K.r_off[m] : K.c_off[n];
}

const char *kFamNames[F_NUM] = {"prop",     "colfin",   "s5",     "compact_count", "scan", "compact_scatter",
                                "schedule", "ingest",   "finish", "s5c", "s5d", "s5e"};

}  // namespace

Engine::~Engine() {
    for (auto &mk : marks) {
        cudaEventDestroy(mk.a);
        cudaEventDestroy(mk.b);
    }
    for (auto e : spare_events) cudaEventDestroy(e);
    for (auto e : ev_round)
        if (e) cudaEventDestroy(e);
    if (s2) cudaStreamSynchronize(s2);  // vector copies still in flight after an error
    if (s_long) {
        cudaStreamSynchronize(s_long);
        cudaStreamDestroy(s_long);
    }
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    pool.release();
    if (s) cudaStreamSynchronize(s);
    pinned_put(st_h);
    pinned_put(verdict_h);
    pinned_put(changed_h);
    pinned_put(s5_left_h);
    pinned_put(de_cnt_h);
    if (own_stream && s) cudaStreamDestroy(s);
    if (ev_mat) cudaEventDestroy(ev_mat);
    if (ev_vec) cudaEventDestroy(ev_vec);
    if (s2) cudaStreamDestroy(s2);
}

void Engine::tbegin(int fam, double bytes) {
    if (!o.timing) return;
    Tmark mk;
    mk.fam = fam;
    mk.bytes = bytes;
    mk.ops = 0.0;
    LPP_CUDA(cudaEventCreate(&mk.a));
    LPP_CUDA(cudaEventCreate(&mk.b));
    LPP_CUDA(cudaEventRecord(mk.a, s));
    marks.push_back(mk);
}
void Engine::tend() {
    if (!o.timing) return;
    LPP_CUDA(cudaEventRecord(marks.back().b, s));
}

void Engine::setup(const lpp_opts &opts, int32_t nlp_, const std::vector<Member> &members) {
    o = opts;
    nlp = nlp_;
    mem = members;
    launches0 = launch_count();
    m0 = n0 = 0;
    nnz0 = 0;
    for (const Member &x : mem) {
        m0 += x.m;
        n0 += x.n;
        nnz0 += x.nnz;
    }
    if (nnz0 >= 2147483647LL) throw StatusError(LPP_ERR_INVALID, "nnz must be < 2^31");
    LPP_CUDA(cudaSetDevice(o.device));
    if (o.stream) {
        s = static_cast<cudaStream_t>(o.stream);
    } else {
        LPP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        own_stream = true;
    }
    pool.s = s;
    keep_pool_memory(o.device);
    st_h = static_cast<DevStatus *>(pinned_get_sized(sizeof(DevStatus)));
    verdict_h = static_cast<int32_t *>(pinned_get_sized(sizeof(int32_t) * (size_t)nlp * V_SLOTS));
    changed_h = static_cast<uint8_t *>(pinned_get_sized((size_t)nlp));
    s5_left_h = static_cast<int32_t *>(pinned_get_sized(sizeof(int32_t)));
    const bool arena = nlp > 1;
    for (int b = 0; b < 2; b++) {
        rp[b] = pool.alloc<int32_t>(m0 + 1);
        ci[b] = pool.alloc<int32_t>(nnz0);
        rv[b] = pool.alloc<double>(nnz0);
        tp[b] = pool.alloc<int32_t>(n0 + 1);
        ti[b] = pool.alloc<int32_t>(nnz0);
        tv[b] = pool.alloc<double>(nnz0);
        L[b] = pool.alloc<double>(m0);
        U[b] = pool.alloc<double>(m0);
        rmap[b] = pool.alloc<int32_t>(m0);
        lu[b] = pool.alloc<double2>(n0);
        c[b] = pool.alloc<double>(n0);
        cmap[b] = pool.alloc<int32_t>(n0);
        lprow[b] = arena ? pool.alloc<int32_t>(m0) : nullptr;
        lpcol[b] = arena ? pool.alloc<int32_t>(n0) : nullptr;
    }
    cap_long_a = sched_cap_long(nnz0);
    cap_long_t = cap_long_a;
    const int64_t cap_chunk = nnz0 / kChunk + cap_long_a + 1;
    const int64_t max_scan = std::max<int64_t>({nnz0 + 1, (int64_t)transpose_hist_elems(nnz0),
                                                (int64_t)sched_tile_hist_elems(std::max(m0, n0)), m0 + 1, n0 + 1,
                                                (int64_t)cap_long_a + 1});
    scan_tmp = pool.alloc<int32_t>(scan_tmp_elems(max_scan));
    for (int w = 0; w < 2; w++) {
        SchedBufs &b = w == 0 ? sa : sb;
        const int32_t cnt = w == 0 ? m0 : n0;
        b.order = pool.alloc<int32_t>(cnt);
        b.chunks = pool.alloc<Chunk>(cap_chunk);
        b.lfirst = pool.alloc<int32_t>(cap_long_a + 1);
        b.nch = pool.alloc<int32_t>(cap_long_a + 1);
        b.tile_hist = pool.alloc<int32_t>(sched_tile_hist_elems(cnt));
        b.tmp = scan_tmp;
    }
    for (int b = 0; b < 2; b++) {
        act[b] = pool.alloc<double2>(m0);
        ninf[b] = pool.alloc<int2>(m0);
        hrow[b] = pool.alloc<unsigned long long>(m0);
        rdirty[b] = pool.alloc<uint8_t>(m0);
    }
    rdnext = pool.alloc<uint8_t>(m0);
    cchg = pool.alloc<uint8_t>(n0);
    t_orig = lazy_req && !o.parallel_cols && !o.col_singletons && !o.dual_fixing && !o.doubletons;
    t_fixed = false;
    if (t_orig) {
        rinv = pool.alloc<int32_t>(m0);
        cinv = pool.alloc<int32_t>(n0);
        clive = pool.alloc<int32_t>(n0);
        rleft = pool.alloc<uint8_t>(m0);
    }
    rkind = pool.alloc<uint8_t>(m0);
    rwork = pool.alloc<uint8_t>(m0);
    hasf = pool.alloc<uint8_t>(m0);
    mL = pool.alloc<unsigned long long>(m0);
    mU = pool.alloc<unsigned long long>(m0);
    rslot = pool.alloc<int32_t>(m0);
    cand_l = pool.alloc<unsigned long long>(n0);
    cand_u = pool.alloc<unsigned long long>(n0);
    ctouch = pool.alloc<uint32_t>(n0);
    tl_list = pool.alloc<int32_t>(n0);
    cl_list = pool.alloc<int32_t>(n0);
    col_cnt = pool.alloc<int32_t>(3);
    ckind = pool.alloc<uint8_t>(n0);
    fixv = pool.alloc<double>(n0);
    tcap_max = pow2_at_least(2 * (int64_t)std::max(m0, 1));
    tkey = pool.alloc<unsigned long long>(tcap_max);
    tlead = pool.alloc<unsigned long long>(tcap_max);
    s5_list[0] = pool.alloc<int32_t>(m0);
    s5_list[1] = pool.alloc<int32_t>(m0);
    s5_cnt = pool.alloc<int32_t>((size_t)o.par_max_iter + 2);
    s5_bar = pool.alloc<unsigned>(2);
    LPP_CUDA(cudaMemsetAsync(s5_bar, 0, 2 * sizeof(unsigned), s));
    ch_act = pool.alloc<double2>(cap_chunk);
    ch_ninf = pool.alloc<int2>(cap_chunk);
    ch_hash = pool.alloc<unsigned long long>(cap_chunk);
    lneed = pool.alloc<uint8_t>(cap_long_a + 1);
    verdict = pool.alloc<int32_t>((size_t)nlp * V_SLOTS);
    lp_changed = pool.alloc<uint8_t>(nlp);
    lp_dead = pool.alloc<uint8_t>(nlp);
    std::memset(&K, 0, sizeof K);
    K.r_keep = pool.alloc<int32_t>(m0 + 1);
    K.r_len = pool.alloc<int32_t>(m0 + 1);
    K.r_pos = pool.alloc<int32_t>(m0 + 1);
    K.r_off = pool.alloc<int32_t>(m0 + 1);
    K.c_keep = pool.alloc<int32_t>(n0 + 1);
    K.c_len = pool.alloc<int32_t>(n0 + 1);
    K.c_pos = pool.alloc<int32_t>(n0 + 1);
    K.c_off = pool.alloc<int32_t>(n0 + 1);
    K.shift = pool.alloc<double>(m0);
    K.chr_cnt = pool.alloc<int32_t>(cap_chunk);
    K.chr_off = pool.alloc<int32_t>(cap_chunk);
    K.chr_shift = pool.alloc<double>(cap_chunk);
    K.cht_cnt = pool.alloc<int32_t>(cap_chunk);
    K.cht_off = pool.alloc<int32_t>(cap_chunk);
    K.contrib = pool.alloc<double>(n0);
    K.offset = pool.alloc<double>(nlp);
    K.offset_part = pool.alloc<double>(n0 / kScanTile + 2);
    K.lp_first = pool.alloc<int32_t>(nlp);
    K.lp_last = pool.alloc<int32_t>(nlp);
    K.lp_dead = lp_dead;
    K.tile_a = pool.alloc<int32_t>(nnz0 / kFlatTile + 2);
    K.tile_t = pool.alloc<int32_t>(nnz0 / kFlatTile + 2);
    K.r_ch0 = pool.alloc<int32_t>(m0 + 1);
    K.c_ch0 = pool.alloc<int32_t>(n0 + 1);
    K.r_new = pool.alloc<int32_t>(m0 + 1);
    K.c_new = pool.alloc<int32_t>(n0 + 1);
    K.c_lock = o.dual_fixing ? pool.alloc<int32_t>(n0 + 1) : nullptr;
    rec_rk = pool.alloc<int32_t>(m0);
    rec_rr = pool.alloc<int32_t>(m0);
    rec_ra = pool.alloc<int32_t>(m0);
    rec_rv = pool.alloc<double>(m0);
    rec_ck = pool.alloc<int32_t>(n0);
    rec_cr = pool.alloc<int32_t>(n0);
    rec_cv = pool.alloc<double>(n0);
    if (o.dual_records) {
        rec_bs = pool.alloc<int4>(n0);
        bsrc = pool.alloc<int2>(n0);
    }
    if (o.parallel_cols) {
        cslot = pool.alloc<int32_t>(n0);
        ctcap_max = pow2_at_least(2 * (int64_t)std::max(n0, 1));
        ctkey = pool.alloc<unsigned long long>(ctcap_max);
        ctcnt = pool.alloc<int32_t>(ctcap_max);
        ctnew = pool.alloc<int32_t>(ctcap_max);
        pkey = pool.alloc<unsigned long long>(n0);
        pcnt = pool.alloc<int32_t>(n0);
        plen = pool.alloc<int32_t>(n0);
        pc_cnt = pool.alloc<int32_t>(4);
        pc_mem = pool.alloc<unsigned char>(s5c_mem_bytes() * (size_t)std::max(n0, 1));
        pc_flags = pool.alloc<int32_t>(n0 + 1);
        pc_pos = pool.alloc<int32_t>(n0 + 1);
        pc_slot = pool.alloc<uint32_t>(n0);
        pc_col = pool.alloc<int32_t>(n0);
        pc_sort.k0 = pool.alloc<uint32_t>(n0);
        pc_sort.k1 = pool.alloc<uint32_t>(n0);
        pc_sort.v0 = pool.alloc<int32_t>(n0);
        pc_sort.v1 = pool.alloc<int32_t>(n0);
        pc_sort.hist = pool.alloc<int32_t>(transpose_hist_elems(n0));
        pc_scan = pool.alloc<int32_t>(scan_tmp_elems(std::max<int64_t>(n0 + 1, transpose_hist_elems(n0))));
        pc_sort.tmp = pc_scan;
        pc_alive = pool.alloc<uint8_t>(n0);
        pc_glist = pool.alloc<int2>(n0 / 2 + 1);  // groups on blocks: two columns or more each
        rec_ca = pool.alloc<int32_t>(n0);
        rec_cp = pool.alloc<int32_t>(n0);
        rec_cm = pool.alloc<double>(4 * (int64_t)n0);
    }
    if (o.col_singletons) {
        cs_rcand = pool.alloc<int32_t>(m0);
        cs_cmin = pool.alloc<int32_t>(n0);
        cs_relig = pool.alloc<uint8_t>(m0);
        cs_tasks = pool.alloc<int32_t>(m0);
        cs_ntask = pool.alloc<int32_t>(1);
        cs_a = pool.alloc<double>(m0);
    }
    if (o.doubletons) {
        de.dk = pool.alloc<int32_t>(m0);
        de.rmin = pool.alloc<int32_t>(m0);
        de.cmin = pool.alloc<int32_t>(n0);
        de.dj = pool.alloc<int32_t>(m0);
        de.dmj = pool.alloc<int32_t>(m0);
        de.dmk = pool.alloc<int32_t>(m0);
        de.dpk = pool.alloc<int32_t>(m0);
        de.dpj = pool.alloc<int32_t>(m0);
        de.jlist = pool.alloc<int32_t>(n0);
        de.cnt = pool.alloc<int32_t>(2);
        de.dsel = pool.alloc<uint8_t>(m0);
        de.dfl = pool.alloc<uint8_t>(m0);
        de.df = pool.alloc<double>(m0);
        de.dg = pool.alloc<double>(m0);
        de.dmd = pool.alloc<double>(m0);
        de.dnv = pool.alloc<double>(m0);
        de_cnt_h = static_cast<int32_t *>(pinned_get_sized(2 * sizeof(int32_t)));
    }
    if (o.col_singletons || o.doubletons) {
        // each row is stored at most once, with fewer entries than it has
        // (rows never grow: a doubleton swaps x_k for x_j at most)
        rec_sb = pool.alloc<long long>(m0);
        rec_sl = pool.alloc<int32_t>(m0);
        rec_srhs = pool.alloc<double>(m0);
        rec_scol = pool.alloc<int32_t>(nnz0);  // each row is stored at most once
        rec_sval = pool.alloc<double>(nnz0);
        sub_used = pool.alloc<unsigned long long>(1);
    }
    st = pool.alloc<DevStatus>(1);
    LPP_CUDA(cudaMemsetAsync(st, 0, sizeof(DevStatus), s));
}

void Engine::ingest_plain(const lpp_lp &in) {
    const cudaMemcpyKind kind = in.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    LPP_CUDA(cudaMemcpyAsync(rp[0], in.row_ptr, sizeof(int32_t) * (size_t)(in.m + 1), kind, s));
    if (in.nnz > 0) {
        LPP_CUDA(cudaMemcpyAsync(ci[0], in.col_idx, sizeof(int32_t) * (size_t)in.nnz, kind, s));
        LPP_CUDA(cudaMemcpyAsync(rv[0], in.val, sizeof(double) * (size_t)in.nnz, kind, s));
    }
    // vectors: staged in the second buffers, checked and normalised into the
    // first.  From the host they are copied on a second stream after the
    // matrix, while the matrix checks and the transpose run (prepare then
    // checks them); device inputs are copied and checked at once.
    double *slhs = L[1], *srhs = U[1], *slb = reinterpret_cast<double *>(lu[1]), *sub = slb + n0, *sc = c[1];
    cudaStream_t sv = s;
    if (!in.on_device) {
        if (!s2) {
            LPP_CUDA(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
            LPP_CUDA(cudaEventCreateWithFlags(&ev_mat, cudaEventDisableTiming));
            LPP_CUDA(cudaEventCreateWithFlags(&ev_vec, cudaEventDisableTiming));
        }
        LPP_CUDA(cudaEventRecord(ev_mat, s));
        LPP_CUDA(cudaStreamWaitEvent(s2, ev_mat, 0));
        sv = s2;
    }
    if (in.m > 0) {
        LPP_CUDA(cudaMemcpyAsync(slhs, in.lhs, sizeof(double) * (size_t)in.m, kind, sv));
        LPP_CUDA(cudaMemcpyAsync(srhs, in.rhs, sizeof(double) * (size_t)in.m, kind, sv));
    }
    if (in.n > 0) {
        LPP_CUDA(cudaMemcpyAsync(slb, in.lb, sizeof(double) * (size_t)in.n, kind, sv));
        LPP_CUDA(cudaMemcpyAsync(sub, in.ub, sizeof(double) * (size_t)in.n, kind, sv));
        LPP_CUDA(cudaMemcpyAsync(sc, in.c, sizeof(double) * (size_t)in.n, kind, sv));
    }
    if (sv == s) {
        ingest_vectors(slhs, srhs, slb, sub, sc, m0, n0, o.huge, L[0], U[0], lu[0], c[0], &st->err, s);
    } else {
        LPP_CUDA(cudaEventRecord(ev_vec, s2));
        vec_pending = true;
    }
}

void Engine::ingest_batch(const lpp_lp *ins, int32_t count) {
    double *slhs = L[1], *srhs = U[1], *slb = reinterpret_cast<double *>(lu[1]), *sub = slb + n0, *sc = c[1];
    const bool dev = ins[0].on_device != 0;
    for (int32_t k = 0; k < count; k++)
        if ((ins[k].on_device != 0) != dev) throw StatusError(LPP_ERR_INVALID, "batch mixes host and device inputs");
    if (dev) {
        std::vector<SrcDesc> d(count);
        for (int32_t k = 0; k < count; k++) {
            const lpp_lp &x = ins[k];
            d[k] = SrcDesc{x.row_ptr, x.col_idx, x.val, x.c, x.lhs, x.rhs, x.lb, x.ub, x.m, x.n, x.nnz,
                           mem[k].row_off, mem[k].col_off, mem[k].nnz_off};
        }
        SrcDesc *dd = pool.alloc<SrcDesc>(count);
        LPP_CUDA(cudaMemcpyAsync(dd, d.data(), sizeof(SrcDesc) * count, cudaMemcpyHostToDevice, s));
        // the host vector must outlive the copy
        LPP_CUDA(cudaStreamSynchronize(s));
        dim3 grid(8, (unsigned)count);
        (k_gather_lps<<<grid, 256, 0, s>>>(dd, rp[0], ci[0], rv[0], slhs, srhs, slb, sub, sc, lprow[0], lpcol[0],
                                          &st->err), note_launch());
        LPP_CUDA(cudaGetLastError());
    } else {
        // pack on the host into pinned staging, then one copy per array
        std::vector<int32_t> h_rp((size_t)m0 + 1), h_ci((size_t)nnz0), h_lr((size_t)m0), h_lc((size_t)n0);
        std::vector<double> h_v((size_t)nnz0), h_l((size_t)m0), h_r((size_t)m0), h_lb((size_t)n0),
            h_ub((size_t)n0), h_c((size_t)n0);
        for (int32_t k = 0; k < count; k++) {
            const lpp_lp &x = ins[k];
            const Member &mm = mem[k];
            if (x.m > 0 && (x.row_ptr[0] != 0 || x.row_ptr[x.m] != x.nnz))
                throw StatusError(LPP_ERR_INVALID, "row_ptr does not match nnz");
            for (int32_t i = 0; i < x.m; i++) {
                h_rp[mm.row_off + i] = (int32_t)(mm.nnz_off + x.row_ptr[i]);
                h_l[mm.row_off + i] = x.lhs[i];
                h_r[mm.row_off + i] = x.rhs[i];
                h_lr[mm.row_off + i] = k;
            }
            for (int32_t j = 0; j < x.n; j++) {
                h_lb[mm.col_off + j] = x.lb[j];
                h_ub[mm.col_off + j] = x.ub[j];
                h_c[mm.col_off + j] = x.c[j];
                h_lc[mm.col_off + j] = k;
            }
            for (int64_t e = 0; e < x.nnz; e++) {
                const int32_t j = x.col_idx[e];
                if (j < 0 || j >= x.n) throw StatusError(LPP_ERR_INVALID, "column index out of range");
                h_ci[mm.nnz_off + e] = mm.col_off + j;
                h_v[mm.nnz_off + e] = x.val[e];
            }
        }
        h_rp[m0] = (int32_t)nnz0;
        auto up = [&](void *dst, const void *src, size_t bytes) {
            if (bytes) LPP_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
        };
        up(rp[0], h_rp.data(), sizeof(int32_t) * h_rp.size());
        up(ci[0], h_ci.data(), sizeof(int32_t) * h_ci.size());
        up(rv[0], h_v.data(), sizeof(double) * h_v.size());
        up(slhs, h_l.data(), sizeof(double) * h_l.size());
        up(srhs, h_r.data(), sizeof(double) * h_r.size());
        up(slb, h_lb.data(), sizeof(double) * h_lb.size());
        up(sub, h_ub.data(), sizeof(double) * h_ub.size());
        up(sc, h_c.data(), sizeof(double) * h_c.size());
        up(lprow[0], h_lr.data(), sizeof(int32_t) * h_lr.size());
        up(lpcol[0], h_lc.data(), sizeof(int32_t) * h_lc.size());
        LPP_CUDA(cudaStreamSynchronize(s));  // pageable staging must outlive the copies
    }
    (k_set_i32<<<1, 1, 0, s>>>(rp[0] + m0, (int32_t)nnz0), note_launch());
    ingest_vectors(slhs, srhs, slb, sub, sc, m0, n0, o.huge, L[0], U[0], lu[0], c[0], &st->err, s);
}

void Engine::prepare() {
    // S0: checks, then A^T by a stable transpose
    int32_t *row_of = pool.alloc<int32_t>(nnz0 + 1);
    check_csr(rp[0], ci[0], rv[0], m0, n0, nnz0, row_of, scan_tmp, &st->err, s);
    LPP_CUDA(cudaGetLastError());
    read_status();
    if (st_h->err) {
        char buf[160];
        std::snprintf(buf, sizeof buf,
                      "invalid LP (checks failed: %s%s%s%s%s)", (st_h->err & 1) ? "row_ptr " : "",
                      (st_h->err & 2) ? "col_idx-range " : "", (st_h->err & 4) ? "val-not-finite-or-zero " : "",
                      (st_h->err & 8) ? "col_idx-not-increasing " : "", (st_h->err & 16) ? "vectors" : "");
        throw StatusError(LPP_ERR_INVALID, buf);
    }
    TransposeBufs tb;
    tb.k0 = reinterpret_cast<uint32_t *>(ci[1]);
    tb.k1 = reinterpret_cast<uint32_t *>(ti[1]);
    tb.v0 = reinterpret_cast<int32_t *>(rv[1]);
    tb.v1 = reinterpret_cast<int32_t *>(rv[1]) + nnz0;
    tb.hist = pool.alloc<int32_t>(transpose_hist_elems(nnz0));
    tb.tmp = scan_tmp;
    t_hist = tb.hist;  // S5e transposes its rewritten matrices with it
    transpose(rp[0], ci[0], rv[0], row_of + 1, m0, n0, nnz0, tb, tp[0], ti[0], tv[0], s);
    LPP_CUDA(cudaGetLastError());
    if (vec_pending) {  // the vectors' copies overlapped the checks and the transpose
        vec_pending = false;
        LPP_CUDA(cudaStreamWaitEvent(s, ev_vec, 0));
        double *slb = reinterpret_cast<double *>(lu[1]);
        ingest_vectors(L[1], U[1], slb, slb + n0, c[1], m0, n0, o.huge, L[0], U[0], lu[0], c[0], &st->err, s);
    }
    iota(rmap[0], m0, 0, s);
    iota(cmap[0], n0, 0, s);
    if (t_orig) {
        iota(rinv, m0, 0, s);
        iota(cinv, n0, 0, s);
        ptr_diff(tp[0], n0, clive, s);
        // every column starts kept at its own slot, with no contribution
        fill_i32(K.c_keep, n0, 1, s);
        iota(K.c_new, n0, 0, s);
        LPP_CUDA(cudaMemsetAsync(K.contrib, 0, sizeof(double) * (size_t)std::max(n0, 1), s));
    }
    fill_u64(cand_l, n0, kEncNegInf, s);
    fill_u64(cand_u, n0, kEncPosInf, s);
    LPP_CUDA(cudaMemsetAsync(ctouch, 0, sizeof(uint32_t) * (size_t)std::max(n0, 1), s));
    fill_u64(mL, m0, kEncNegInf, s);
    fill_u64(mU, m0, kEncPosInf, s);
    LPP_CUDA(cudaMemsetAsync(hasf, 0, (size_t)std::max(m0, 1), s));
    LPP_CUDA(cudaMemsetAsync(rdirty[0], 1, (size_t)std::max(m0, 1), s));  // round 1 evaluates every row
    LPP_CUDA(cudaMemsetAsync(rwork, 0, (size_t)std::max(m0, 1), s));
    fill_i32(verdict, (int64_t)nlp * V_SLOTS, kNone, s);
    LPP_CUDA(cudaMemsetAsync(rec_rk, 0, sizeof(int32_t) * (size_t)std::max(m0, 1), s));
    LPP_CUDA(cudaMemsetAsync(rec_rr, 0, sizeof(int32_t) * (size_t)std::max(m0, 1), s));
    fill_i32(rec_ra, m0, -1, s);
    LPP_CUDA(cudaMemsetAsync(rec_rv, 0, sizeof(double) * (size_t)std::max(m0, 1), s));
    LPP_CUDA(cudaMemsetAsync(rec_ck, 0, sizeof(int32_t) * (size_t)std::max(n0, 1), s));
    LPP_CUDA(cudaMemsetAsync(rec_cr, 0, sizeof(int32_t) * (size_t)std::max(n0, 1), s));
    LPP_CUDA(cudaMemsetAsync(rec_cv, 0, sizeof(double) * (size_t)std::max(n0, 1), s));
    if (o.dual_records) {  // no source (-1, round -1: read as 0); no candidate row yet
        fill_i32(reinterpret_cast<int32_t *>(rec_bs), 4 * (int64_t)n0, -1, s);
        fill_i32(reinterpret_cast<int32_t *>(bsrc), 2 * (int64_t)n0, INT32_MAX, s);
    }
    if (o.parallel_cols) {
        // an empty column table: no key, no column
        LPP_CUDA(cudaMemsetAsync(ctkey, 0, sizeof(unsigned long long) * (size_t)ctcap_max, s));
        LPP_CUDA(cudaMemsetAsync(ctcnt, 0, sizeof(int32_t) * (size_t)ctcap_max, s));
        LPP_CUDA(cudaMemsetAsync(ctnew, 0, sizeof(int32_t) * (size_t)ctcap_max, s));
        // no column has been through S5c: key 0 is never a key, size 0 never a group's
        LPP_CUDA(cudaMemsetAsync(pkey, 0, sizeof(unsigned long long) * (size_t)std::max(n0, 1), s));
        LPP_CUDA(cudaMemsetAsync(pcnt, 0, sizeof(int32_t) * (size_t)std::max(n0, 1), s));
        LPP_CUDA(cudaMemsetAsync(plen, 0, sizeof(int32_t) * (size_t)std::max(n0, 1), s));  // no key stored
        fill_i32(rec_ca, n0, -1, s);
        LPP_CUDA(cudaMemsetAsync(rec_cp, 0, sizeof(int32_t) * (size_t)std::max(n0, 1), s));
        fill_u64(reinterpret_cast<unsigned long long *>(rec_cm), 4 * (int64_t)n0, 0x7ff8000000000000ULL, s);  // NaN
    }
    if (o.col_singletons || o.doubletons) {
        LPP_CUDA(cudaMemsetAsync(rec_sb, 0, sizeof(long long) * (size_t)std::max(m0, 1), s));
        LPP_CUDA(cudaMemsetAsync(rec_sl, 0, sizeof(int32_t) * (size_t)std::max(m0, 1), s));
        LPP_CUDA(cudaMemsetAsync(rec_srhs, 0, sizeof(double) * (size_t)std::max(m0, 1), s));
        LPP_CUDA(cudaMemsetAsync(sub_used, 0, sizeof(unsigned long long), s));
    }
    std::vector<double> offs(nlp);
    for (int32_t k = 0; k < nlp; k++) offs[k] = mem[k].obj_offset;
    LPP_CUDA(cudaMemcpyAsync(K.offset, offs.data(), sizeof(double) * nlp, cudaMemcpyHostToDevice, s));
    m = m0;
    n = n0;
    nnz = nnz0;
    cur = 0;
    (k_set_i32<<<1, 1, 0, s>>>(&st->m_new, m0), note_launch());
    (k_set_i32<<<1, 1, 0, s>>>(&st->n_new, n0), note_launch());
    schedule_current();
    read_status();  // also keeps offs alive until its copy is done
    if (st_h->err) throw StatusError(LPP_ERR_INVALID, "invalid LP (checks failed: vectors)");
    adopt_schedule();
    t_fixed = t_orig;  // from here on T and its schedule stay the input's
}

// Launches the schedule builds of the current CSR and CSC (not of a CSC kept
// as the input's); the segment counts are read from st->m_new / st->n_new on
// the device (m, n bound them).
void Engine::schedule_current() {
    build_schedule(rp[cur], &st->m_new, m, nnz, sa, st->cls_r, &st->nchunk_r, s);
    if (!t_fixed) build_schedule(tp[cur], &st->n_new, n, nnz, sb, st->cls_c, &st->nchunk_c, s);
    LPP_CUDA(cudaGetLastError());
}

// After read_status(): the host copies of the current schedules.
void Engine::adopt_schedule() {
    A.ptr = rp[cur];
    A.idx = ci[cur];
    A.val = rv[cur];
    A.order = sa.order;
    A.chunks = sa.chunks;
    A.lfirst = sa.lfirst;
    A.cnt = m;
    segmat_from_counts(A, st_h->cls_r, st_h->nchunk_r);
    if (t_fixed) {
        if (A.cls_start[kNumClass] != m) throw StatusError(LPP_ERR_CUDA, "internal: schedule does not cover every segment");
        return;
    }
    T.ptr = tp[cur];
    T.idx = ti[cur];
    T.val = tv[cur];
    T.order = sb.order;
    T.chunks = sb.chunks;
    T.lfirst = sb.lfirst;
    T.cnt = n;
    segmat_from_counts(T, st_h->cls_c, st_h->nchunk_c);
    if (A.cls_start[kNumClass] != m || T.cls_start[kNumClass] != n)
        throw StatusError(LPP_ERR_CUDA, "internal: schedule does not cover every segment");
}

void Engine::read_status() {
    LPP_CUDA(cudaMemcpyAsync(st_h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    LPP_CUDA(cudaMemcpyAsync(verdict_h, verdict, sizeof(int32_t) * (size_t)nlp * V_SLOTS, cudaMemcpyDeviceToHost, s));
    LPP_CUDA(cudaMemcpyAsync(changed_h, lp_changed, (size_t)nlp, cudaMemcpyDeviceToHost, s));
    LPP_CUDA(cudaStreamSynchronize(s));
}

Ctx Engine::ctx(int32_t round) const {
    Ctx C;
    std::memset(&C, 0, sizeof C);
    C.A = A;
    C.T = T;
    C.m = m;
    C.n = n;
    C.nlp = nlp;
    C.round = round;
    C.L = L[cur];
    C.U = U[cur];
    C.rmap = rmap[cur];
    C.lp_row = lprow[cur];
    C.lu = lu[cur];
    C.c = c[cur];
    C.cmap = cmap[cur];
    C.lp_col = lpcol[cur];
    C.t_orig = t_orig ? 1 : 0;
    C.rinv = rinv;
    C.cinv = cinv;
    C.clen = t_orig ? clive : nullptr;
    C.act = act[cur];
    C.ninf = ninf[cur];
    C.rdirty = rdirty[cur];
    C.rdnext = rdnext;
    C.cchg = cchg;
    C.rkind = rkind;
    C.rwork = rwork;
    C.hrow = hrow[cur];
    C.rslot = rslot;
    C.mL = mL;
    C.mU = mU;
    C.hasf = hasf;
    C.cand_l = cand_l;
    C.cand_u = cand_u;
    C.ctouch = ctouch;
    C.tl_list = tl_list;
    C.tl_cnt = col_cnt;
    C.cl_list = cl_list;
    C.cl_cnt = col_cnt + 1;
    C.cl_nnz = col_cnt + 2;
    C.ckind = ckind;
    C.fixv = fixv;
    C.tkey = tkey;
    C.tlead = tlead;
    C.tcap = 2;
    C.ch_act = ch_act;
    C.ch_ninf = ch_ninf;
    C.ch_hash = ch_hash;
    C.lneed = lneed;
    C.rec_rk = rec_rk;
    C.rec_rr = rec_rr;
    C.rec_ra = rec_ra;
    C.rec_rv = rec_rv;
    C.rec_ck = rec_ck;
    C.rec_cr = rec_cr;
    C.rec_cv = rec_cv;
    C.rec_ca = rec_ca;
    C.rec_cp = rec_cp;
    C.rec_cm = rec_cm;
    C.rec_sb = rec_sb;
    C.rec_sl = rec_sl;
    C.rec_srhs = rec_srhs;
    C.rec_scol = rec_scol;
    C.rec_sval = rec_sval;
    C.sub_used = sub_used;
    C.cslot = cslot;
    C.ctkey = ctkey;
    C.ctcnt = ctcnt;
    C.ctnew = ctnew;
    C.pkey = pkey;
    C.pcnt = pcnt;
    C.plen = plen;
    C.ctcap = 2;
    C.lp_round0 = lp_round0_dev;
    C.verdict = verdict;
    C.lp_changed = lp_changed;
    C.st = st;
    C.feas_tol = o.feas_tol;
    C.bound_tol = o.bound_tol;
    C.max_implied = o.max_implied;
    C.par_tol = o.par_tol;
    C.dual = o.dual_reductions;
    C.dualfix = o.dual_fixing;
    C.count_work = o.timing ? 1 : 0;
    C.list_touched = 1;
    C.dual_rec = o.dual_records ? 1 : 0;
    C.bsrc = bsrc;
    C.rec_bs = rec_bs;
    return C;
}

void Engine::compact(int32_t round) {
    const int nx = cur ^ 1;
    K.rp2 = rp[nx];
    K.ci2 = ci[nx];
    K.rv2 = rv[nx];
    K.cp2 = t_orig ? nullptr : tp[nx];
    K.ri2 = t_orig ? nullptr : ti[nx];
    K.cv2 = t_orig ? nullptr : tv[nx];
    K.rinv = t_orig ? rinv : nullptr;
    K.cinv = t_orig ? cinv : nullptr;
    K.L2 = L[nx];
    K.U2 = U[nx];
    K.rmap2 = rmap[nx];
    K.lp_row2 = lprow[nx];
    K.lu2 = lu[nx];
    K.c2 = c[nx];
    K.cmap2 = cmap[nx];
    K.lp_col2 = lpcol[nx];
    K.rdirty2 = rdirty[nx];
    K.act2 = act[nx];
    K.ninf2 = ninf[nx];
    K.hrow2 = hrow[nx];
    const Ctx C = ctx(round);
    // columns kept in place (t_orig): their counts are updated in place, no
    // column scan, no column vectors moved; the slots of the columns that
    // leave are marked (cinv) and dropped once, at the end
    int32_t *own_clen = K.c_len;
    if (t_orig) K.c_len = clive;
    tbegin(F_COUNT, 4.0 * nnz * 2 + 8.0 * nnz + 24.0 * m + 40.0 * n);
    ensure_side_stream();
    const SideStream side{s_long, ev_fork, ev_join};
    launch_compact_counts(C, K, s, &side);
    tend();
    tbegin(F_SCAN, 16.0 * (m + (t_orig ? 0 : n)) * 2);
    scan_excl2(K.r_keep, K.r_len, K.r_pos, K.r_off, m, scan_tmp, s);
    if (!t_orig) scan_excl2(K.c_keep, K.c_len, K.c_pos, K.c_off, n, scan_tmp, s);
    tend();
    // the objective constant of the columns that left: with the columns in
    // place (t_orig) each slot's contribution stays until one sum at the end
    if (!t_orig) launch_offset(C, K, s);
    (k_sizes<<<1, 1, 0, s>>>(K, m, n, t_orig ? 1 : 0, st), note_launch());
    tbegin(F_SCATTER, 24.0 * nnz * 2 + 48.0 * (m + n));
    launch_compact_scatter(C, K, (int32_t)nnz, s);
    tend();
    LPP_CUDA(cudaGetLastError());
    K.c_len = own_clen;
    // the next buffers become current; sizes and schedules are read back at
    // the end of the round (one host sync per round)
    if (t_orig) {  // the column vectors stay where they are: they move with cur
        std::swap(lu[cur], lu[nx]);
        std::swap(c[cur], c[nx]);
        std::swap(cmap[cur], cmap[nx]);
        std::swap(lpcol[cur], lpcol[nx]);
    }
    cur = nx;
    tbegin(F_SCHED, 8.0 * (m + n));
    schedule_current();
    tend();
}

// The second stream for the long rows' kernels (made on first use).
void Engine::ensure_side_stream() {
    if (s_long) return;
    LPP_CUDA(cudaStreamCreateWithFlags(&s_long, cudaStreamNonBlocking));
    LPP_CUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
    LPP_CUDA(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
}

// One round (S1 .. S8) over the whole arena.  first_round: some LP is in
// its first round (S6 must then run on its input columns); force: compact even
// if nothing was removed (to drop retired LPs).
Engine::StepOut Engine::step(int32_t r, bool first_round, bool force) {
    StepOut out;
    if (!ev_round[0]) {
        LPP_CUDA(cudaEventCreate(&ev_round[0]));
        LPP_CUDA(cudaEventCreate(&ev_round[1]));
    }
    act_m = m;
    act_buf = cur;
    r_nnz.push_back(nnz);
    nnz_processed += nnz;
    LPP_CUDA(cudaEventRecord(ev_round[0], s));
    LPP_CUDA(cudaMemsetAsync(st, 0, 8 * sizeof(int32_t), s));
    LPP_CUDA(cudaMemsetAsync(lp_changed, 0, (size_t)nlp, s));
    if (m > 0) LPP_CUDA(cudaMemsetAsync(rdnext, 0, (size_t)m, s));
    // the column lists of S3' start empty; outside a first round only listed
    // columns are finalised, the others keep kind KEPT and no change flag
    LPP_CUDA(cudaMemsetAsync(col_cnt, 0, 3 * sizeof(int32_t), s));
    if (!first_round && n > 0) {
        LPP_CUDA(cudaMemsetAsync(ckind, 0, (size_t)n, s));
        LPP_CUDA(cudaMemsetAsync(cchg, 0, (size_t)n, s));
    }
    Ctx C = ctx(r);
    C.list_touched = first_round ? 0 : 1;  // a first round's S3' checks every column
    tbegin(F_PROP, 0.0);  // bytes and ops set once the evaluated nonzeros are known
    const size_t prop_mark = marks.size();
    // the long rows' chunk kernels on a second stream, beside the short
    // rows' kernel, joined before S3'
    const bool long_rows = prop_has_long(C);
    if (long_rows) {
        ensure_side_stream();
        LPP_CUDA(cudaEventRecord(ev_fork, s));
        LPP_CUDA(cudaStreamWaitEvent(s_long, ev_fork, 0));
        launch_prop_long(C, s_long);
        LPP_CUDA(cudaEventRecord(ev_join, s_long));
    }
    launch_prop_short(C, s);
    if (long_rows) LPP_CUDA(cudaStreamWaitEvent(s, ev_join, 0));
    tend();
    tbegin(F_COLFIN, 33.0 * n);
    if (o.dual_records) launch_bound_src(C, s);
    launch_colfin(C, first_round, s);
    launch_mark_dirty(C, nnz, s);
    tend();
    LPP_CUDA(cudaGetLastError());
    // S5: leader passes.  Skipped when the last S5 resolved every key group
    // (no row left unmatched at the pass cap) and no row lost an entry since:
    // its survivors are pairwise not parallel, so it would remove nothing.
    const bool run_s5 = first_round || !s5_clean;
    int32_t tcap = std::min(tcap_max, pow2_at_least(2 * (int64_t)std::max(m, 1)));
    tbegin(F_S5, run_s5 ? 16.0 * tcap + 12.0 * m : 0.0);
    if (run_s5) {
        LPP_CUDA(cudaMemsetAsync(tkey, 0, sizeof(unsigned long long) * tcap, s));
        LPP_CUDA(cudaMemsetAsync(tlead, 0xff, sizeof(unsigned long long) * tcap, s));
        C.tcap = tcap;
        LPP_CUDA(cudaMemsetAsync(s5_cnt, 0, sizeof(int32_t) * (size_t)(o.par_max_iter + 2), s));
        C.s5_out = s5_list[0];
        C.s5_out_cnt = s5_cnt + 1;
        launch_s5_pass(C, s);
    }
    tend();
    LPP_CUDA(cudaGetLastError());
    read_status();
    r_eval.push_back(st_h->nnz_eval);
    if (o.timing && prop_mark > 0) {
        // S1-S3 algorithmic work: per evaluated nonzero its 12 bytes and two
        // FMAs (activities), per tested entry side two FMAs (the residual and
        // the sign test); per row ptr, sides, results (4 + 16 + 33 bytes), the
        // bounds once
        Tmark &pm = marks[prop_mark - 1];
        pm.bytes = 12.0 * st_h->nnz_eval + 53.0 * m + 16.0 * n;
        pm.ops = 2.0 * st_h->nnz_eval + 2.0 * st_h->sides_tested;
    }
    // later passes on the list of unmatched rows, without a host sync per
    // pass: one block for a short list, else one cooperative launch with grid
    // barriers (launched chunks of 2, 4, 8, ... passes if that launch is not
    // possible), then one read of the list size
    const int32_t n1 = run_s5 ? st_h->unmatched : 0;
    bool resolved = n1 == 0;
    if (n1 > 0 && o.par_max_iter > 1) {
        tbegin(F_S5, 0.0);
        tcap = std::min(tcap_max, pow2_at_least(2 * (int64_t)n1));
        LPP_CUDA(cudaMemsetAsync(tkey, 0, sizeof(unsigned long long) * tcap, s));
        LPP_CUDA(cudaMemsetAsync(tlead, 0xff, sizeof(unsigned long long) * tcap, s));
        C.tcap = tcap;
        int32_t chunk = 2, left = n1;
        for (int32_t pass = 1; pass < o.par_max_iter;) {
            if (left <= kTailBlockRows) {  // the remaining passes in one block, one read
                launch_s5_tail_block(C, s5_list[0], s5_list[1], s5_cnt, pass, o.par_max_iter, s);
                LPP_CUDA(cudaGetLastError());
                LPP_CUDA(cudaMemcpyAsync(s5_left_h, s5_cnt + o.par_max_iter, sizeof(int32_t),
                                         cudaMemcpyDeviceToHost, s));
                LPP_CUDA(cudaMemcpyAsync(st_h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
                LPP_CUDA(cudaStreamSynchronize(s));
                resolved = *s5_left_h == 0;
                break;
            }
            if (launch_s5_tail_grid(C, s5_list[0], s5_list[1], s5_cnt, pass, o.par_max_iter, left, s5_bar, s)) {
                // the remaining passes in one cooperative launch, one read
                LPP_CUDA(cudaGetLastError());
                LPP_CUDA(cudaMemcpyAsync(s5_left_h, s5_cnt + o.par_max_iter, sizeof(int32_t),
                                         cudaMemcpyDeviceToHost, s));
                LPP_CUDA(cudaMemcpyAsync(st_h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
                LPP_CUDA(cudaStreamSynchronize(s));
                if (st_h->err & 4) throw StatusError(LPP_ERR_CUDA, "internal: S5 pass barrier timed out");
                resolved = *s5_left_h == 0;
                break;
            }
            cudaGetLastError();  // no cooperative launch: launched passes
            const int32_t end = std::min<int32_t>(pass + chunk, o.par_max_iter);
            for (int32_t q = pass; q < end; q++)
                launch_s5_tail(C, s5_list[(q - 1) & 1], s5_cnt + q, s5_list[q & 1], s5_cnt + q + 1, n1, s);
            LPP_CUDA(cudaGetLastError());
            LPP_CUDA(cudaMemcpyAsync(s5_left_h, s5_cnt + end, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            // the status with the rows these passes removed (the round's
            // removals decide whether it compacts)
            LPP_CUDA(cudaMemcpyAsync(st_h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
            LPP_CUDA(cudaStreamSynchronize(s));
            if (*s5_left_h == 0) {
                resolved = true;
                break;
            }
            left = *s5_left_h;
            pass = end;
            chunk *= 2;
        }
        tend();
    }
    if (run_s5) s5_clean = resolved;
    if (run_s5 && !resolved) s5_left += o.par_max_iter > 1 ? *s5_left_h : n1;
    if (st_h->err) throw StatusError(LPP_ERR_CUDA, "internal: S5 hash table overflow");
    if (run_s5) launch_s5_leader(C, s);
    LPP_CUDA(cudaGetLastError());
    // S5c (opt-in) on the round-start columns.  Skipped when no row was
    // removed and no column fixed or merged since the last S5c and S4 fixed
    // none this round: every group is then the one the last S5c left, with
    // the same leaders and no parallel pair.
    if (o.parallel_cols && (first_round || s5c_dirty || st_h->cols_fixed > 0)) {
        run_s5c(C);
        s5c_dirty = false;
    }
    // S5d (opt-in) on the rows kept so far and the columns left
    if (o.col_singletons) run_s5d(C);
    // S5e (opt-in) on the rows and columns left; may rewrite the matrices
    if (o.doubletons) run_s5e(C);
    bool newly_dead = false;
    for (int32_t k = 0; k < nlp; k++) {
        if (lp_dropped[k]) continue;
        for (int v = 0; v < V_SLOTS; v++) newly_dead |= verdict_h[k * V_SLOTS + v] != kNone;
    }
    out.structural = first_round || force || st_h->rows_removed > 0 || st_h->cols_fixed > 0 || newly_dead;
    const int32_t rows_removed = st_h->rows_removed, bounds = st_h->bounds_changed;
    if (out.structural) compact(r);
    else std::swap(rdirty[cur], rdnext);  // same numbering: next round's flags
    LPP_CUDA(cudaEventRecord(ev_round[1], s));
    read_status();
    if (st_h->err) throw StatusError(LPP_ERR_CUDA, "internal: S5 hash table overflow");
    if (st_h->cols_fixed > 0) s5_clean = false;  // rows lost entries (S4 or S6 fixings, S5c merges)
    if (rows_removed > 0 || st_h->cols_fixed > 0) s5c_dirty = true;
    if (out.structural) {
        const int32_t m_new = st_h->m_new, n_new = st_h->n_new, nnz_new = st_h->nnz_new;
        if (nnz_new != st_h->nnz_new_t || m_new < 0 || m_new > m || n_new < 0 || n_new > n || nnz_new > nnz)
            throw StatusError(LPP_ERR_CUDA, "internal: compaction sizes disagree");
        m = m_new;
        n = n_new;
        nnz = nnz_new;
        adopt_schedule();
    }
    LPP_CUDA(cudaEventElapsedTime(&out.ms, ev_round[0], ev_round[1]));
    r_ms.push_back(out.ms);
    r_rows.push_back(rows_removed);
    r_cols.push_back(st_h->cols_fixed);
    r_bounds.push_back(bounds);
    rounds = r;
    return out;
}

// S5c: keys into the column table, the columns of the changed groups in
// column order, sorted by slot, then every such group's passes on the
// device.  Two host reads: the number of grouped columns (sizes the sort),
// then the status.  Refreshes st_h, whose column count then includes the
// merges.
void Engine::run_s5c(const Ctx &C0) {
    Ctx C = C0;
    tbegin(F_S5C, 0.0);
    LPP_CUDA(cudaMemsetAsync(pc_cnt, 0, 4 * sizeof(int32_t), s));
    C.ctcap = std::min(ctcap_max, pow2_at_least(2 * (int64_t)std::max(n, 1)));
    launch_s5c_keys(C, s);
    launch_s5c_members(C, pc_flags, pc_pos, pc_scan, pc_slot, pc_col, s);
    LPP_CUDA(cudaGetLastError());
    LPP_CUDA(cudaMemcpyAsync(s5_left_h, pc_pos + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LPP_CUDA(cudaStreamSynchronize(s));
    const int32_t F = n > 0 ? *s5_left_h : 0;
    if (F > 0) {
        int bits = 0;
        while (((int64_t)1 << bits) < (int64_t)C.ctcap) bits++;
        const uint32_t *ks = nullptr;
        const int32_t *vs = nullptr;
        sort_pairs(pc_slot, pc_col, F, bits, pc_sort, &ks, &vs, s);
        launch_s5c_groups(C, ks, vs, F, pc_mem, pc_alive, pc_glist, pc_cnt, o.par_max_iter, s);
    }
    // the table slots of this round, emptied for the next
    LPP_CUDA(cudaMemsetAsync(ctkey, 0, sizeof(unsigned long long) * (size_t)C.ctcap, s));
    LPP_CUDA(cudaMemsetAsync(ctcnt, 0, sizeof(int32_t) * (size_t)C.ctcap, s));
    LPP_CUDA(cudaMemsetAsync(ctnew, 0, sizeof(int32_t) * (size_t)C.ctcap, s));
    LPP_CUDA(cudaGetLastError());
    tend();
    LPP_CUDA(cudaMemcpyAsync(st_h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    LPP_CUDA(cudaStreamSynchronize(s));
    if (st_h->err) throw StatusError(LPP_ERR_CUDA, "internal: S5c hash table overflow");
}

// S5d: the column-singleton kernels, then a read of the status (its counts
// decide whether the round compacts)
void Engine::run_s5d(const Ctx &C) {
    tbegin(F_S5D, 0.0);
    if (m > 0 && n > 0) {
        fill_i32(cs_rcand, m, kNone, s);
        fill_i32(cs_cmin, n, kNone, s);
        LPP_CUDA(cudaMemsetAsync(cs_relig, 0, (size_t)m, s));
        LPP_CUDA(cudaMemsetAsync(cs_ntask, 0, sizeof(int32_t), s));
        launch_s5d(C, cs_rcand, cs_relig, cs_cmin, cs_tasks, cs_ntask, cs_a, s);
        LPP_CUDA(cudaGetLastError());
    }
    tend();
    LPP_CUDA(cudaMemcpyAsync(st_h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    LPP_CUDA(cudaStreamSynchronize(s));
}

// S5e: candidates, claims, the applied doubletons, a status read.  When any
// applied, the CSR is rewritten into the other buffers (lengths, a scan, one
// read of the new size, the placement) and the CSC rebuilt from it by the
// ingest transpose; the old matrices, dead by then, lend the transpose its
// scratch (the old CSC the row of each entry).  The buffers swap roles, the
// schedules are rebuilt, and the rows of every x_j are marked for the next
// round.  S6 and the compaction of the round then see the rewritten LP.
void Engine::run_s5e(const Ctx &C) {
    tbegin(F_S5E, 0.0);
    int32_t applied = 0, nj = 0;
    if (m > 0 && n > 0) {
        fill_i32(de.rmin, m, kNone, s);
        fill_i32(de.cmin, n, kNone, s);
        LPP_CUDA(cudaMemsetAsync(de.cnt, 0, 2 * sizeof(int32_t), s));
        launch_s5e(C, de, s);
        LPP_CUDA(cudaGetLastError());
        LPP_CUDA(cudaMemcpyAsync(de_cnt_h, de.cnt, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LPP_CUDA(cudaStreamSynchronize(s));
        applied = de_cnt_h[0];
        nj = de_cnt_h[1];
    }
    if (applied > 0) {
        const int nx = cur ^ 1;
        launch_s5e_rowlen(C, de, K.r_len, s);
        scan_excl(K.r_len, rp[nx], m, scan_tmp, s);
        LPP_CUDA(cudaGetLastError());
        LPP_CUDA(cudaMemcpyAsync(de_cnt_h, rp[nx] + m, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LPP_CUDA(cudaStreamSynchronize(s));
        const int32_t nnz2 = de_cnt_h[0];
        if (nnz2 < 0 || nnz2 > nnz) throw StatusError(LPP_ERR_CUDA, "internal: S5e rewrite grew the matrix");
        int32_t *row_of = ti[cur];
        launch_s5e_scatter(C, de, rp[nx], ci[nx], rv[nx], row_of, nnz, s);
        TransposeBufs tb;
        tb.k0 = reinterpret_cast<uint32_t *>(ci[cur]);
        tb.k1 = reinterpret_cast<uint32_t *>(rv[cur]);
        tb.v0 = reinterpret_cast<int32_t *>(rv[cur]) + nnz0;
        tb.v1 = reinterpret_cast<int32_t *>(tv[cur]);
        tb.hist = t_hist;
        tb.tmp = scan_tmp;
        transpose(rp[nx], ci[nx], rv[nx], row_of, m, n, nnz2, tb, tp[nx], ti[nx], tv[nx], s);
        LPP_CUDA(cudaGetLastError());
        std::swap(rp[0], rp[1]);
        std::swap(ci[0], ci[1]);
        std::swap(rv[0], rv[1]);
        std::swap(tp[0], tp[1]);
        std::swap(ti[0], ti[1]);
        std::swap(tv[0], tv[1]);
        nnz = nnz2;
        schedule_current();
        read_status();
        if (st_h->err) throw StatusError(LPP_ERR_CUDA, "internal: S5e rewrite placed an entry outside its row");
        adopt_schedule();
        launch_s5e_mark(ctx(C.round), de, nj, s);
        LPP_CUDA(cudaGetLastError());
    }
    tend();
    read_status();
}

void Engine::run() {
    const int32_t R = std::max(0, o.max_rounds);
    s5_clean = false;
    s5c_dirty = true;
    s5_left = 0;
    lp_rounds.assign(nlp, 0);
    lp_status.assign(nlp, LPP_OK);
    lp_where.assign(nlp, LPP_WHERE_NONE);
    lp_index.assign(nlp, -1);
    lp_round.assign(nlp, 0);
    lp_done.assign(nlp, 0);
    lp_dropped.assign(nlp, 0);
    cudaEvent_t eloop, eend;
    LPP_CUDA(cudaEventCreate(&eloop));
    LPP_CUDA(cudaEventCreate(&eend));
    spare_events.push_back(eloop);
    spare_events.push_back(eend);
    LPP_CUDA(cudaEventRecord(eloop, s));
    int32_t live = nlp;
    for (int32_t r = 1; r <= R && live > 0; r++) {
        const StepOut so = step(r, r == 1, false);
        for (int32_t k = 0; k < nlp; k++) {
            if (lp_done[k]) {
                if (so.structural && lp_status[k] != LPP_OK) lp_dropped[k] = 1;
                continue;
            }
            int v = 0;
            while (v < V_SLOTS && verdict_h[k * V_SLOTS + v] == kNone) v++;
            if (v < V_SLOTS) {
                lp_status[k] = v == V_S6_COL ? LPP_UNBOUNDED : LPP_INFEASIBLE;
                lp_where[k] = (v == V_S2_ROW || v == V_S5_ROW) ? LPP_WHERE_ROW : LPP_WHERE_COL;
                lp_index[k] = verdict_h[k * V_SLOTS + v];
                lp_round[k] = r;
                lp_rounds[k] = r;
                lp_done[k] = 1;
                if (so.structural) lp_dropped[k] = 1;
                live--;
            } else if (!changed_h[k]) {
                lp_rounds[k] = r;
                lp_done[k] = 1;
                live--;
            } else {
                lp_rounds[k] = r;
            }
        }
    }
    if (o.dep_rows && nlp == 1 && lp_status[0] == LPP_OK) remove_dependent();
    if (t_orig) {
        launch_offset(ctx(rounds), K, s);  // every slot's contribution, once, in column order
        finish_cols();
        finish_csc();
    }
    float lms = 0.f;
    LPP_CUDA(cudaEventRecord(eend, s));
    LPP_CUDA(cudaEventSynchronize(eend));
    LPP_CUDA(cudaEventElapsedTime(&lms, eloop, eend));
    loop_ms = lms;
}

// The dependent-row step (Sec. 5, the hybrid design): the current CSR and
// sides go to the host, the peeling and elimination of deprows.h run there,
// and the
// rows it finds are removed on the device by one more compaction, whose S6
// fixes the columns that then have no entry left (or every column no kept
// row locks, with dual fixing).  Its records carry round rounds + 1; a
// contradiction is a verdict of that round.
void Engine::remove_dependent() {
    const int32_t r = rounds + 1;
    // host copies, left uninitialised until the copies fill them
    std::unique_ptr<int32_t[]> hp(new int32_t[(size_t)m + 1]), hi(new int32_t[(size_t)nnz + 1]),
        hrmap(new int32_t[(size_t)m + 1]);
    std::unique_ptr<double[]> hv(new double[(size_t)nnz + 1]), hL(new double[(size_t)m + 1]),
        hU(new double[(size_t)m + 1]);
    LPP_CUDA(cudaMemcpyAsync(hp.get(), rp[cur], 4 * ((size_t)m + 1), cudaMemcpyDeviceToHost, s));
    if (nnz) {
        LPP_CUDA(cudaMemcpyAsync(hi.get(), ci[cur], 4 * (size_t)nnz, cudaMemcpyDeviceToHost, s));
        LPP_CUDA(cudaMemcpyAsync(hv.get(), rv[cur], 8 * (size_t)nnz, cudaMemcpyDeviceToHost, s));
    }
    if (m) {
        LPP_CUDA(cudaMemcpyAsync(hL.get(), L[cur], 8 * (size_t)m, cudaMemcpyDeviceToHost, s));
        LPP_CUDA(cudaMemcpyAsync(hU.get(), U[cur], 8 * (size_t)m, cudaMemcpyDeviceToHost, s));
        LPP_CUDA(cudaMemcpyAsync(hrmap.get(), rmap[cur], 4 * (size_t)m, cudaMemcpyDeviceToHost, s));
    }
    LPP_CUDA(cudaStreamSynchronize(s));
    int64_t eq_nnz = 0;
    for (int64_t i = 0; i < m; i++)
        if (std::isfinite(hL[i]) && hL[i] == hU[i]) eq_nnz += hp[i + 1] - hp[i];
    DepRowsIn in{m, n, hp.get(), hi.get(), hv.get(), hL.get(), hU.get(), o.feas_tol,
                 std::max<int64_t>(8 * eq_nnz, (int64_t)1 << 24)};
    DepRowsOut out;
    dependent_rows(in, out);
    dep_pivots = out.pivots;
    dep_peeled = out.peeled;
    dep_stopped = out.stopped ? 1 : 0;
    if (out.bad >= 0) {
        lp_status[0] = LPP_INFEASIBLE;
        lp_where[0] = LPP_WHERE_ROW;
        lp_index[0] = hrmap[out.bad];
        lp_round[0] = r;
        return;
    }
    dep_found = (int32_t)out.dep.size();
    if (out.dep.empty()) return;
    int32_t *list = pool.alloc<int32_t>((int64_t)out.dep.size());
    LPP_CUDA(cudaMemcpyAsync(list, out.dep.data(), 4 * out.dep.size(), cudaMemcpyHostToDevice, s));
    LPP_CUDA(cudaMemsetAsync(st, 0, 8 * sizeof(int32_t), s));
    LPP_CUDA(cudaMemsetAsync(rkind, 0, (size_t)std::max<int32_t>(m, 1), s));
    if (n > 0) {
        LPP_CUDA(cudaMemsetAsync(ckind, 0, (size_t)n, s));
        LPP_CUDA(cudaMemsetAsync(cchg, 0, (size_t)n, s));
    }
    if (act_buf != cur) {
        // the last round compacted: its activities and row map (the records'
        // last-round activities) sit in the buffers this compaction writes,
        // which therefore get fresh ones
        act_rec = act[act_buf];
        ninf_rec = ninf[act_buf];
        rmap_rec = rmap[act_buf];
        act[act_buf] = pool.alloc<double2>(m0);
        ninf[act_buf] = pool.alloc<int2>(m0);
        rmap[act_buf] = pool.alloc<int32_t>(m0);
    }
    const Ctx C = ctx(r);
    launch_mark_dependent(C, list, (int32_t)out.dep.size(), s);
    compact(r);
    read_status();
    if (st_h->err) throw StatusError(LPP_ERR_CUDA, "internal: compaction error");
    const int32_t m_new = st_h->m_new, n_new = st_h->n_new, nnz_new = st_h->nnz_new;
    if (nnz_new != st_h->nnz_new_t || m_new < 0 || m_new > m || n_new < 0 || n_new > n || nnz_new > nnz)
        throw StatusError(LPP_ERR_CUDA, "internal: compaction sizes disagree");
    m = m_new;
    n = n_new;
    nnz = nnz_new;
    adopt_schedule();
    for (int v = 0; v < V_SLOTS; v++)
        if (verdict_h[v] != kNone) {  // S6 found an unbounded column
            lp_status[0] = v == V_S6_COL ? LPP_UNBOUNDED : LPP_INFEASIBLE;
            lp_where[0] = (v == V_S2_ROW || v == V_S5_ROW) ? LPP_WHERE_ROW : LPP_WHERE_COL;
            lp_index[0] = verdict_h[v];
            lp_round[0] = r;
            break;
        }
}

// The columns' one compaction when the rounds kept them in place: the
// slots still in the LP, in order, into the other buffers (which then become
// the current ones), the CSR's column indices renumbered, cinv to the final
// indices.
void Engine::finish_cols() {
    tbegin(F_SCATTER, 4.0 * nnz * 2 + 72.0 * n);
    launch_cols_alive(cinv, n, K.c_keep, s);
    scan_excl(K.c_keep, K.c_pos, n, scan_tmp, s);
    const int nx = cur ^ 1;
    K.lu2 = lu[nx];
    K.c2 = c[nx];
    K.cmap2 = cmap[nx];
    K.lp_col2 = lpcol[nx];
    const Ctx C = ctx(rounds);
    launch_cols_final(C, K, n, cinv, ci[cur], nnz, s);
    (k_csc_sizes<<<1, 1, 0, s>>>(K, n, st), note_launch());  // n_new: the columns left
    LPP_CUDA(cudaGetLastError());
    tend();
    read_status();
    const int32_t n_new = st_h->n_new;
    if (n_new < 0 || n_new > n) throw StatusError(LPP_ERR_CUDA, "internal: column compaction size");
    std::swap(lu[cur], lu[nx]);
    std::swap(c[cur], c[nx]);
    std::swap(cmap[cur], cmap[nx]);
    std::swap(lpcol[cur], lpcol[nx]);
    n = n_new;
}

// The result's CSC when the rounds kept the input's: one compaction of the
// input CSC (slot 0) to the rows and columns still in the LP, renumbered,
// into the other slot, which then becomes the current one.  Its sizes must
// be the current CSR's.
void Engine::finish_csc() {
    tbegin(F_SCATTER, 24.0 * nnz0 + 12.0 * nnz + 16.0 * (m0 + n0));
    launch_rows_left(rinv, m0, rleft, s);
    Ctx C0 = ctx(rounds);
    C0.rkind = rleft;
    C0.m = m0;
    C0.n = n0;
    launch_csc_from_input_counts(C0, K, s);
    scan_excl2(K.c_keep, K.c_len, K.c_pos, K.c_off, n0, scan_tmp, s);
    const int o = 1;  // the slot not holding the input CSC
    launch_csc_from_input_scatter(C0, K, nnz0, tp[o], ti[o], tv[o], s);
    (k_csc_sizes<<<1, 1, 0, s>>>(K, n0, st), note_launch());
    LPP_CUDA(cudaGetLastError());
    tend();
    read_status();
    if (st_h->n_new != n || st_h->nnz_new_t != nnz)
        throw StatusError(LPP_ERR_CUDA, "internal: result CSC sizes disagree with the CSR");
    if (cur != o) {
        std::swap(tp[0], tp[1]);
        std::swap(ti[0], ti[1]);
        std::swap(tv[0], tv[1]);
    }
    T.ptr = tp[cur];
    T.idx = ti[cur];
    T.val = tv[cur];
}

const char *fam_name(int f) { return kFamNames[f]; }

void Engine::k_sizes_set(int32_t m_, int32_t n_) {
    (k_set_i32<<<1, 1, 0, s>>>(&st->m_new, m_), note_launch());
    (k_set_i32<<<1, 1, 0, s>>>(&st->n_new, n_), note_launch());
}

}  // namespace lpp
