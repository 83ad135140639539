// k_parcols.cu -- S5c, parallel columns (Sec. 3.2, parallel columns; opt-in).
//
// Columns j and k are parallel when A_:j = lam A_:k and c_j = lam c_k.  They
// are found, like parallel rows, by hashing keys and checking candidates
// against a leader, here on the columns of [c; A] (the CSR of A^T at the
// round start, rows removed earlier in the round included):
//   key      length, row pattern, whether each coefficient's sign differs
//            from the first one's, sign of c_j times the first coefficient's
//            (equal for parallel columns whatever lam);
//   group    the columns of one key, in column order;
//   pass     the group's first live column k leads and leaves the group;
//            every live column j parallel to it (entries and cost within
//            par_tol, lam = a_j,first / a_k,first) merges into it, one after
//            the other in column order:
//              y = x_k + lam x_j,  lam > 0: [l_y + lam l_j, u_y + lam u_j]
//                                  lam < 0: [l_y + lam u_j, u_y + lam l_j],
//            and column j leaves the LP (no side shift, no objective
//            constant); at most par_max_iter passes, while two columns live.
// Only columns S4 left unfixed take part.
//
// GPU layout: a hash table counts the columns per key; the columns of keys
// with two or more are compacted in column order and sorted stably by slot,
// so each group is a contiguous run in column order.  A group none of whose
// columns changed its key since its last S5c, and whose size is the one that
// S5c left, is skipped: it would yield the same leaders and no merge.  One warp runs all
// passes of a group of at most 256 columns; larger groups (singleton columns
// of long rows reach thousands) get a thread block, whose threads check the
// members in parallel while one warp applies the chain of merges in order.
#include <algorithm>

#include "lpp_launch.h"

namespace lpp {

namespace {

constexpr int kWarpGroupMax = 256;  // larger groups run on a block,
constexpr int kWarpLenMax = 256;    // and so do groups of longer columns
constexpr int kLargeThreads = 512;

__device__ __forceinline__ unsigned long long cost_hash(int cs) {
    return mix64(0x2d358dccaa6c78a5ULL + (unsigned long long)(cs + 1));
}

// Inserts column j with key hash `key` into the column table of capacity
// cap (a power of two) and counts it; a key other than the column's key at
// its last S5c marks the slot changed.  Returns the slot, -1 if the table is
// full (an internal error: the capacity is at least twice the columns).
__device__ __forceinline__ int32_t s5c_insert(const Ctx &C, int32_t j, unsigned long long key, uint32_t cap) {
    if (key == 0) key = 1;
    const int32_t o = C.cmap[j];
    const bool changed = C.pkey[o] != key;
    C.pkey[o] = key;
    uint32_t sl = (uint32_t)(key ^ (key >> 32)) & (cap - 1u);
    for (uint32_t probe = 0; probe < cap; probe++) {
        const unsigned long long prev = atomicCAS(&C.ctkey[sl], 0ULL, key);
        if (prev == 0ULL || prev == key) {
            atomicAdd(&C.ctcnt[sl], 1);
            if (changed) C.ctnew[sl] = 1;
            return (int32_t)sl;
        }
        sl = (sl + 1u) & (cap - 1u);
    }
    atomicOr(&C.st->err, 1);
    return -1;
}

// final key hash of column j from the sum of its entry hashes
__device__ __forceinline__ unsigned long long s5c_key(const Ctx &C, int32_t j, int32_t len, bool neg0,
                                                      unsigned long long h) {
    const double cj = C.c[j];
    const int cs = (cj > 0.0) - (cj < 0.0);
    return h + len_hash(len) + cost_hash(neg0 ? -cs : cs);
}

// The key hashes the original row indices, so that a column keeps its key
// from round to round until it loses an entry (rows are renumbered by every
// compaction; the grouping is the same, the order of rows being kept).  A
// column whose length is the one its last S5c saw has the same entries
// (entries are only ever removed) and reuses its stored key.
__device__ __forceinline__ bool s5c_reuse(const Ctx &C, int32_t o, int32_t len) { return C.plen[o] == len; }

// columns of classes 0..5: W lanes per column hash its entries
template <int W>
__device__ __forceinline__ void s5c_key_group(const Ctx &C, int32_t j, bool valid) {
    const unsigned mask = group_mask<W>();
    const int lane = threadIdx.x & (W - 1);
    bool act = valid && C.ckind[j] == CK_KEPT;
    int32_t beg = 0, end = 0, o = 0;
    if (act) {
        beg = C.T.ptr[j];
        end = C.T.ptr[j + 1];
        act = end > beg;
        o = C.cmap[j];
    }
    const bool reuse = act && s5c_reuse(C, o, end - beg);  // the same in the whole lane group
    const bool neg0 = act && !reuse ? is_neg(C.T.val[beg]) : false;
    unsigned long long h = 0;
    if (act && !reuse)
        for (int32_t k = beg + lane; k < end; k += W)
            h += entry_hash(C.rmap[C.T.idx[k]], is_neg(C.T.val[k]) != neg0);
    h = group_sum<W>(h, mask);
    if (valid && lane == 0) {
        int32_t sl = -1;
        if (act) {
            const unsigned long long key = reuse ? C.pkey[o] : s5c_key(C, j, end - beg, neg0, h);
            C.plen[o] = end - beg;
            sl = s5c_insert(C, j, key, (uint32_t)C.ctcap);
        }
        C.cslot[j] = sl;
    }
}

__global__ void __launch_bounds__(kBlock) k_s5c_key_groups(Ctx C, GroupGrid g) {
    const int c = grid_class(g, blockIdx.x);
    const int W = 1 << c;
    const int32_t pos = C.T.cls_start[c] + (blockIdx.x - g.blk_start[c]) * (kBlock / W) + threadIdx.x / W;
    const bool valid = pos < C.T.cls_start[c + 1];
    const int32_t j = valid ? C.T.order[pos] : 0;
    switch (c) {
        case 0: s5c_key_group<1>(C, j, valid); break;
        case 1: s5c_key_group<2>(C, j, valid); break;
        case 2: s5c_key_group<4>(C, j, valid); break;
        case 3: s5c_key_group<8>(C, j, valid); break;
        case 4: s5c_key_group<16>(C, j, valid); break;
        default: s5c_key_group<32>(C, j, valid); break;
    }
}

// long columns (class 6): one block per chunk sums its entry hashes
__global__ void __launch_bounds__(kBlock) k_s5c_key_long_partial(Ctx C) {
    __shared__ unsigned long long s_h[kBlock / 32];
    const Chunk ch = C.T.chunks[blockIdx.x];
    const int32_t j = ch.seg, beg = C.T.ptr[j];
    if (C.ckind[j] != CK_KEPT || s5c_reuse(C, C.cmap[j], C.T.ptr[j + 1] - beg)) return;  // block-uniform
    const bool neg0 = is_neg(C.T.val[beg]);
    unsigned long long h = 0;
    for (int32_t k = ch.begin + threadIdx.x; k < ch.end; k += kBlock)
        h += entry_hash(C.rmap[C.T.idx[k]], is_neg(C.T.val[k]) != neg0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if ((threadIdx.x & 31) == 0) s_h[threadIdx.x >> 5] = h;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kBlock / 32; w++) t += s_h[w];
        C.ch_hash[blockIdx.x] = t;
    }
}

// one warp per long column: its chunk sums (or its stored key), then the insert
__global__ void __launch_bounds__(kBlock) k_s5c_key_long(Ctx C) {
    const int32_t t = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int32_t nlong = C.T.cls_start[7] - C.T.cls_start[6];
    if (t < nlong) {  // the same t in the whole warp
        const int32_t j = C.T.order[C.T.cls_start[6] + t];
        const int32_t beg = C.T.ptr[j], len = C.T.ptr[j + 1] - beg, o = C.cmap[j];
        const bool act = C.ckind[j] == CK_KEPT;
        const bool reuse = act && s5c_reuse(C, o, len);
        unsigned long long h = 0;
        if (act && !reuse)
            for (int32_t q = C.T.lfirst[t] + lane; q < C.T.lfirst[t + 1]; q += 32) h += C.ch_hash[q];
        h = group_sum<32>(h, 0xffffffffu);
        if (lane == 0) {
            int32_t sl = -1;
            if (act) {
                const unsigned long long key = reuse ? C.pkey[o] : s5c_key(C, j, len, is_neg(C.T.val[beg]), h);
                C.plen[o] = len;
                sl = s5c_insert(C, j, key, (uint32_t)C.ctcap);
            }
            C.cslot[j] = sl;
        }
    }
}

// A group whose columns all kept their keys and whose size is the one its
// last S5c left has the same leaders and no parallel pair: its passes would
// merge nothing (coefficients and costs never change, a removed row changes
// the key).  Mark the other groups: a key changed (at insert) or the size.
__global__ void __launch_bounds__(kBlock) k_s5c_mark(Ctx C) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= C.n) return;
    const int32_t sl = C.cslot[j];
    if (sl >= 0 && C.ctcnt[sl] != C.pcnt[C.cmap[j]]) C.ctnew[sl] = 1;
}

// 1 for a column of a changed group of two or more columns; the others keep
// their group's size as the size after this S5c
__global__ void __launch_bounds__(kBlock) k_s5c_flags(Ctx C, int32_t *flags) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= C.n) return;
    const int32_t sl = C.cslot[j];
    const bool f = sl >= 0 && C.ctcnt[sl] >= 2 && C.ctnew[sl];
    if (sl >= 0 && !f) C.pcnt[C.cmap[j]] = C.ctcnt[sl];
    flags[j] = f;
}

__global__ void __launch_bounds__(kBlock) k_s5c_compact(Ctx C, const int32_t *flags, const int32_t *pos,
                                                       uint32_t *slot, int32_t *col) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= C.n || !flags[j]) return;
    slot[pos[j]] = (uint32_t)C.cslot[j];
    col[pos[j]] = j;
}

// entry q of columns j (first entry bj) and k (first entry bk): same row and
// a_j = lam a_k within par_tol
__device__ __forceinline__ bool s5c_same(const Ctx &C, int32_t bj, int32_t bk, int32_t q, double lam) {
    const double aj = C.T.val[bj + q], la = lam * C.T.val[bk + q];
    return C.T.idx[bj + q] == C.T.idx[bk + q] && fabs(aj - la) <= C.par_tol * fmax(fabs(aj), fabs(la));
}

// What the checks read of a grouped column, gathered once per round at its
// sorted position: first entry, length, first coefficient, cost, and the
// filter key r (below).
struct Mem {
    double a0, c;
    unsigned long long r;
    int32_t bj, len;
};
constexpr unsigned long long kNoFilter = ~0ULL;

// Cost filter.  For parallel columns c_j / a_j,first = c_k / a_k,first
// (= c_k lam / (a_k,first lam)), and the cost test accepts only costs whose
// ratios agree to relative par_tol plus a few roundings, i.e. within
// (par_tol + 8u) 2^53 + 2 units in the last place (u = 2^-53) as long as no
// quotient or product leaves the normal range.  r = enc(c / a_first) when
// |a_first| and |c| (or c = 0) have binary exponents in [-323, 317], else
// kNoFilter; two columns whose r differ by more than `ulps` (twice that
// bound plus 64) fail the cost test, and only the others are tested.
__device__ __forceinline__ bool mid_range(double x) {
    const int e = (int)((dbits(x) >> 52) & 0x7ff);
    return e >= 700 && e <= 1340;
}
__device__ __forceinline__ bool s5c_filtered(unsigned long long ra, unsigned long long rb, long long ulps) {
    if (ulps < 0 || ra == kNoFilter || rb == kNoFilter) return false;
    const unsigned long long d = ra > rb ? ra - rb : rb - ra;
    return d > (unsigned long long)ulps;
}

__global__ void __launch_bounds__(kBlock) k_s5c_gather(Ctx C, const int32_t *col, int32_t F, Mem *mem) {
    const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= F) return;
    const int32_t j = col[p];
    Mem m;
    m.bj = C.T.ptr[j];
    m.len = C.T.ptr[j + 1] - m.bj;
    m.a0 = C.T.val[m.bj];
    m.c = C.c[j];
    m.r = mid_range(m.a0) && (m.c == 0.0 || mid_range(m.c)) ? enc_dbl(m.c / m.a0) : kNoFilter;
    mem[p] = m;
}

// the leader of a pass, as read by every checker
struct Lead {
    int32_t k, bk, len;
    double a0, c;
    unsigned long long r;
};
__device__ __forceinline__ Lead s5c_lead(int32_t k, const Mem &m) {
    Lead L;
    L.k = k;
    L.bk = m.bj;
    L.len = m.len;
    L.a0 = m.a0;
    L.c = m.c;
    L.r = m.r;
    return L;
}

// length and cost test of a column against the leader (lam = a_j,first / a_k,first)
__device__ __forceinline__ bool s5c_head(const Ctx &C, const Lead &L, const Mem &m, long long ulps, double &lam) {
    if (m.len != L.len || s5c_filtered(m.r, L.r, ulps)) return false;
    lam = m.a0 / L.a0;
    const double lc = lam * L.c;
    return fabs(m.c - lc) <= C.par_tol * fmax(fabs(m.c), fabs(lc));
}

// Merge of column j (with factor lam) into the running y of leader k:
// records the bounds before it, returns the new ones.
__device__ __forceinline__ double2 s5c_merge(const Ctx &C, int32_t k, int32_t j, double lam, double2 y,
                                             int32_t pass) {
    const double2 bj = C.lu[j];
    double2 ny;
    if (lam > 0.0) {
        ny.x = y.x + lam * bj.x;
        ny.y = y.y + lam * bj.y;
    } else {
        ny.x = y.x + lam * bj.y;
        ny.y = y.y + lam * bj.x;
    }
    C.ckind[j] = CK_PARALLEL;
    C.fixv[j] = 0.0;
    const int32_t lp = lp_of_col(C, j);
    const int32_t o = C.cmap[j];
    C.rec_ck[o] = CK_PARALLEL;
    C.rec_cr[o] = lp_round(C, lp);
    C.rec_cv[o] = lam;
    C.rec_ca[o] = C.cmap[k];
    C.rec_cp[o] = pass;
    double *r = C.rec_cm + 4 * (int64_t)o;
    r[0] = y.x;
    r[1] = y.y;
    r[2] = bj.x;
    r[3] = bj.y;
    return ny;
}

// All passes of one group (G members at sorted positions 0..G: columns cols,
// cached data mem, live flags alive) by one warp.  Returns the merges (the
// same in every lane).
__device__ int32_t s5c_group_warp(const Ctx &C, const int32_t *cols, const Mem *mem, int32_t G, uint8_t *alive,
                                  int32_t max_iter, long long ulps, int32_t *unresolved) {
    const int lane = threadIdx.x & 31;
    for (int32_t t = lane; t < G; t += 32) alive[t] = 1;
    __syncwarp();
    int32_t live = G, merged = 0, lead = -1;
    for (int32_t it = 0; it < max_iter && live >= 2; it++) {
        // the first live column after the last leader (live >= 2: there is one)
        int32_t nl = -1;
        for (int32_t b0 = lead + 1; b0 < G && nl < 0; b0 += 32) {
            const int32_t q = b0 + lane;
            const unsigned b = __ballot_sync(0xffffffffu, q < G && alive[q]);
            if (b) nl = b0 + __ffs(b) - 1;
        }
        if (nl < 0) break;  // cannot happen while live >= 2; guards the index
        lead = nl;
        if (lane == 0) alive[lead] = 0;
        __syncwarp();
        live--;
        const Lead L = s5c_lead(cols[lead], mem[lead]);
        double2 y = C.lu[L.k];
        int32_t nm = 0;
        for (int32_t b0 = lead + 1; b0 < G; b0 += 32) {
            const int32_t q = b0 + lane;
            int32_t bj = 0, len = 0;
            double lam = 0.0;
            bool ok = false;
            if (q < G && alive[q]) {
                const Mem m = mem[q];
                bj = m.bj;
                len = m.len;
                ok = s5c_head(C, L, m, ulps, lam);
            }
            if (ok && len <= 32)
                for (int32_t e = 0; e < len && ok; e++) ok = s5c_same(C, bj, L.bk, e, lam);
            unsigned todo = __ballot_sync(0xffffffffu, ok && len > 32);
            while (todo) {  // long columns: the whole warp checks one at a time
                const int src = __ffs(todo) - 1;
                todo &= todo - 1u;
                const int32_t sbj = __shfl_sync(0xffffffffu, bj, src), slen = __shfl_sync(0xffffffffu, len, src);
                const double slam = __shfl_sync(0xffffffffu, lam, src);
                bool sok = true;
                for (int32_t e = lane; e < slen; e += 32) sok = sok && s5c_same(C, sbj, L.bk, e, slam);
                sok = __all_sync(0xffffffffu, sok) != 0;
                if (lane == src) ok = sok;
            }
            unsigned mb = __ballot_sync(0xffffffffu, ok);
            nm += __popc(mb);
            while (mb) {  // the chain, in column order
                const int src = __ffs(mb) - 1;
                mb &= mb - 1u;
                double2 ny = y;
                if (lane == src) {
                    ny = s5c_merge(C, L.k, cols[q], lam, y, it);
                    alive[q] = 0;
                }
                y.x = __shfl_sync(0xffffffffu, ny.x, src);
                y.y = __shfl_sync(0xffffffffu, ny.y, src);
            }
        }
        __syncwarp();
        if (nm > 0 && lane == 0) {
            C.lu[L.k] = y;
            mark_lp_changed(C, lp_of_col(C, L.k));
        }
        live -= nm;
        merged += nm;
    }
    if (live >= 2 && lane == 0) atomicAdd(unresolved, 1);
    for (int32_t t = lane; t < G; t += 32) C.pcnt[C.cmap[cols[t]]] = G - merged;
    return merged;
}

// One warp per 32 sorted positions runs the groups that start there.
__global__ void __launch_bounds__(kBlock) k_s5c_small(Ctx C, const uint32_t *slot, const int32_t *col, const Mem *mem,
                                                     int32_t F, uint8_t *alive, int2 *glist, int32_t *ctr,
                                                     int32_t max_iter, long long ulps) {
    const int lane = threadIdx.x & 31;
    const int64_t p0 = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * 32;
    int32_t merged = 0;
    if (p0 < F) {  // the same p0 in the whole warp
        const int64_t p = p0 + lane;
        unsigned starts = __ballot_sync(0xffffffffu, p < F && (p == 0 || slot[p] != slot[p - 1]));
        while (starts) {
            const int src = __ffs(starts) - 1;
            starts &= starts - 1u;
            const int32_t s0 = (int32_t)p0 + src;
            const int32_t G = C.ctcnt[slot[s0]];  // every column of the slot is in the run
            if (G > kWarpGroupMax || mem[s0].len > kWarpLenMax) {
                if (lane == 0) glist[atomicAdd(&ctr[1], 1)] = make_int2(s0, G);
            } else {
                merged += s5c_group_warp(C, col + s0, mem + s0, G, alive + s0, max_iter, ulps, &ctr[0]);
            }
        }
    }
    block_add(lane == 0 ? merged : 0, &C.st->cols_fixed);
}

// Large groups, one thread block each (grid-stride over the list): every
// pass the threads check the live members against the leader in parallel
// (alive = 2 marks a parallel one), then warp 0 applies the marked merges in
// column order.  The live flags and filter keys of the first kLargeCache
// members sit in shared memory (most members of a large group fail the cost
// filter against every leader, so a pass mostly reads those two).
constexpr int32_t kLargeCache = 12288;
constexpr size_t kLargeSmem = (size_t)kLargeCache * (sizeof(unsigned long long) + 1);

struct LiveView {
    uint8_t *sh, *gl;
    int32_t cached;
    __device__ __forceinline__ uint8_t get(int32_t q) const { return q < cached ? sh[q] : gl[q]; }
    __device__ __forceinline__ void set(int32_t q, uint8_t v) const {
        if (q < cached) sh[q] = v;
        else gl[q] = v;
    }
};

__global__ void __launch_bounds__(kLargeThreads) k_s5c_large(Ctx C, const int32_t *col, const Mem *mem_all,
                                                            uint8_t *alive_all, const int2 *glist, int32_t *ctr,
                                                            int32_t max_iter, long long ulps) {
    extern __shared__ unsigned long long s_r[];  // [kLargeCache] filter keys, then the live flags
    __shared__ int32_t s_min, s_cnt;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t ng = ctr[1];
    int32_t merged_blk = 0;
    for (int32_t g = blockIdx.x; g < ng; g += gridDim.x) {
        const int32_t s0 = glist[g].x, G = glist[g].y;
        const int32_t *cols = col + s0;
        const Mem *mem = mem_all + s0;
        const LiveView alive{reinterpret_cast<uint8_t *>(s_r + kLargeCache), alive_all + s0,
                             G < kLargeCache ? G : kLargeCache};
        for (int32_t t = threadIdx.x; t < G; t += kLargeThreads) {
            alive.set(t, 1);
            if (t < alive.cached) s_r[t] = mem[t].r;
        }
        __syncthreads();
        int32_t live = G, lead = -1, merged_g = 0;
        for (int32_t it = 0; it < max_iter && live >= 2; it++) {
            // next leader: the first live column after the last one
            int32_t nl = -1;
            for (int32_t b0 = lead + 1; b0 < G && nl < 0; b0 += kLargeThreads) {
                if (threadIdx.x == 0) s_min = kNone;
                __syncthreads();
                const int32_t q = b0 + threadIdx.x;
                if (q < G && alive.get(q)) atomicMin(&s_min, q);
                __syncthreads();
                nl = s_min == kNone ? -1 : s_min;
                __syncthreads();
            }
            if (nl < 0) break;  // cannot happen while live >= 2; guards the index
            lead = nl;
            const Lead L = s5c_lead(cols[lead], mem[lead]);
            if (threadIdx.x == 0) {
                alive.set(lead, 0);
                s_cnt = 0;
            }
            __syncthreads();
            live--;
            int32_t cnt = 0;
            if (L.len > kWarpLenMax) {
                // long columns: one member at a time, its entries spread over the block
                for (int32_t q = lead + 1; q < G; q++) {
                    if (alive.get(q) != 1) continue;  // the same in every thread
                    const Mem m = mem[q];
                    double lam = 0.0;
                    bool ok = s5c_head(C, L, m, ulps, lam);
                    if (ok) {
                        bool mine = true;
                        for (int32_t e = threadIdx.x; e < m.len; e += kLargeThreads)
                            mine = mine && s5c_same(C, m.bj, L.bk, e, lam);
                        ok = __syncthreads_and(mine) != 0;
                    }
                    if (ok && threadIdx.x == 0) {
                        alive.set(q, 2);
                        cnt++;
                    }
                }
            } else {
                for (int32_t q = lead + 1 + threadIdx.x; q < G; q += kLargeThreads) {
                    if (alive.get(q) != 1) continue;
                    if (s5c_filtered(q < alive.cached ? s_r[q] : mem[q].r, L.r, ulps)) continue;
                    const Mem m = mem[q];
                    double lam = 0.0;
                    bool ok = s5c_head(C, L, m, ulps, lam);
                    for (int32_t e = 0; e < m.len && ok; e++) ok = s5c_same(C, m.bj, L.bk, e, lam);
                    if (ok) {
                        alive.set(q, 2);
                        cnt++;
                    }
                }
            }
            if (cnt) atomicAdd(&s_cnt, cnt);
            __syncthreads();
            const int32_t nm = s_cnt;
            if (nm > 0 && warp == 0) {
                double2 y = C.lu[L.k];
                for (int32_t b0 = lead + 1; b0 < G; b0 += 32) {
                    const int32_t q = b0 + lane;
                    const bool mine = q < G && alive.get(q) == 2;
                    unsigned mb = __ballot_sync(0xffffffffu, mine);
                    const double lam = mine ? mem[q].a0 / L.a0 : 0.0;
                    while (mb) {
                        const int src = __ffs(mb) - 1;
                        mb &= mb - 1u;
                        double2 ny = y;
                        if (lane == src) {
                            ny = s5c_merge(C, L.k, cols[q], lam, y, it);
                            alive.set(q, 0);
                        }
                        y.x = __shfl_sync(0xffffffffu, ny.x, src);
                        y.y = __shfl_sync(0xffffffffu, ny.y, src);
                    }
                }
                if (lane == 0) {
                    C.lu[L.k] = y;
                    mark_lp_changed(C, lp_of_col(C, L.k));
                }
            }
            __syncthreads();
            live -= nm;
            merged_g += nm;
            merged_blk += nm;
        }
        if (threadIdx.x == 0 && live >= 2) atomicAdd(&ctr[0], 1);
        for (int32_t t = threadIdx.x; t < G; t += kLargeThreads) C.pcnt[C.cmap[cols[t]]] = G - merged_g;
        __syncthreads();
    }
    if (threadIdx.x == 0 && merged_blk) atomicAdd(&C.st->cols_fixed, merged_blk);
}

inline unsigned blocks_for(int64_t cnt, int threads) {
    return (unsigned)((cnt + threads - 1) / threads > 0 ? (cnt + threads - 1) / threads : 1);
}

}  // namespace

void launch_s5c_keys(const Ctx &C, cudaStream_t s) {
    if (C.n <= 0) return;
    const GroupGrid g = group_grid(C.T);
    if (g.blk_start[6] > 0) (k_s5c_key_groups<<<g.blk_start[6], kBlock, 0, s>>>(C, g), note_launch());
    const int32_t nlong = C.T.cls_start[7] - C.T.cls_start[6];
    if (nlong > 0 && C.T.nchunks > 0) {
        (k_s5c_key_long_partial<<<C.T.nchunks, kBlock, 0, s>>>(C), note_launch());
        (k_s5c_key_long<<<blocks_for((int64_t)nlong * 32, kBlock), kBlock, 0, s>>>(C), note_launch());
    }
}

void launch_s5c_members(const Ctx &C, int32_t *flags, int32_t *pos, int32_t *scan_tmp, uint32_t *slot, int32_t *col,
                        cudaStream_t s) {
    if (C.n <= 0) {
        cudaMemsetAsync(pos, 0, sizeof(int32_t), s);
        return;
    }
    (k_s5c_mark<<<blocks_for(C.n, kBlock), kBlock, 0, s>>>(C), note_launch());
    (k_s5c_flags<<<blocks_for(C.n, kBlock), kBlock, 0, s>>>(C, flags), note_launch());
    scan_excl(flags, pos, C.n, scan_tmp, s);
    (k_s5c_compact<<<blocks_for(C.n, kBlock), kBlock, 0, s>>>(C, flags, pos, slot, col), note_launch());
}

size_t s5c_mem_bytes() { return sizeof(Mem); }

void launch_s5c_groups(const Ctx &C, const uint32_t *slot, const int32_t *col, int32_t F, void *mem, uint8_t *alive,
                       int2 *glist, int32_t *ctr, int32_t max_iter, cudaStream_t s) {
    if (F <= 0) return;
    // the cost filter's window, 2 (par_tol 2^53 + 8) + 64 units in the last
    // place; off for tolerances of 1e-6 and more
    const long long ulps = C.par_tol < 1e-6 ? (long long)(2.0 * (C.par_tol * 9007199254740992.0 + 8.0)) + 64 : -1;
    Mem *m = static_cast<Mem *>(mem);
    (k_s5c_gather<<<blocks_for(F, kBlock), kBlock, 0, s>>>(C, col, F, m), note_launch());
    (k_s5c_small<<<blocks_for((int64_t)F, kBlock), kBlock, 0, s>>>(C, slot, col, m, F, alive, glist, ctr, max_iter,
                                                                   ulps),
     note_launch());
    // at most F / 2 groups go to blocks (more than 256 columns, or longer
    // columns); two blocks per SM take them in turn
    const int32_t nlarge_max = F / 2;
    if (nlarge_max > 0) {
        // shared memory above 48 KB is an opt-in of the current device (a
        // refusal shows as the launch's error)
        cudaFuncSetAttribute(k_s5c_large, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLargeSmem);
        (k_s5c_large<<<std::min<int32_t>(nlarge_max, 2 * 152), kLargeThreads, kLargeSmem, s>>>(
             C, col, m, alive, glist, ctr, max_iter, ulps),
         note_launch());
    }
}

}  // namespace lpp
