// k_parcols.cu -- S5c, parallel columns (Sec. 3.2, parallel columns; opt-in).
//
// Columns j and k are parallel when A_:j = lam A_:k and c_j = lam c_k.  They
// are found, like parallel rows, by hashing keys and checking candidates
// against a leader, here on the columns of [c; A] (the CSR of A^T at the
// round start, rows removed earlier in the round included):
//   key      length, row pattern, whether each coefficient's sign differs
//            from the first one's, sign of c_j times the first coefficient's
//            (equal for parallel columns whatever lam);
//   leader   the smallest column index of the key (the first column);
//   pass     every other column of the key is checked against the leader
//            (entries and cost within par_tol, lam = a_j,first / a_k,first);
//            the smallest parallel one merges into the leader:
//              y = x_k + lam x_j,  lam > 0: [l_k + lam l_j, u_k + lam u_j]
//                                  lam < 0: [l_k + lam u_j, u_k + lam l_j],
//            and column j leaves the LP (no side shift, no objective
//            constant).  A leader with no parallel column leaves the key;
//            the others take part in the next pass, at most par_max_iter.
// One merge per leader and pass keeps every bound update a single write.
// Only columns S4 left unfixed take part.
#include <algorithm>

#include "lpp_launch.h"

namespace lpp {

namespace {

__device__ __forceinline__ unsigned long long cost_hash(int cs) {
    return mix64(0x2d358dccaa6c78a5ULL + (unsigned long long)(cs + 1));
}

// Inserts column j with key hash `key` into the column table of capacity
// cap (a power of two) and elects the smallest index as the key's leader.
// Returns the slot, -1 if the table is full (an internal error: the capacity
// is at least twice the columns inserted).
__device__ __forceinline__ int32_t s5c_insert(const Ctx &C, int32_t j, unsigned long long key, uint32_t cap) {
    if (key == 0) key = 1;
    uint32_t sl = (uint32_t)(key ^ (key >> 32)) & (cap - 1u);
    for (uint32_t probe = 0; probe < cap; probe++) {
        const unsigned long long prev = atomicCAS(&C.ctkey[sl], 0ULL, key);
        if (prev == 0ULL || prev == key) {
            atomicMin(&C.ctlead[sl], (unsigned long long)(uint32_t)j);
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

// first pass, columns of classes 0..5: W lanes per column hash its entries
template <int W>
__device__ __forceinline__ bool s5c_key_group(const Ctx &C, int32_t j, bool valid) {
    const unsigned mask = group_mask<W>();
    const int lane = threadIdx.x & (W - 1);
    bool act = valid && C.ckind[j] == CK_KEPT;
    int32_t beg = 0, end = 0;
    if (act) {
        beg = C.T.ptr[j];
        end = C.T.ptr[j + 1];
        act = end > beg;
    }
    const bool neg0 = act ? is_neg(C.T.val[beg]) : false;
    unsigned long long h = 0;
    for (int32_t k = beg + lane; k < end; k += W) h += entry_hash(C.T.idx[k], is_neg(C.T.val[k]) != neg0);
    h = group_sum<W>(h, mask);
    bool part = false;
    if (valid && lane == 0) {
        int32_t sl = -1;
        if (act) {
            const unsigned long long key = s5c_key(C, j, end - beg, neg0, h);
            C.hcol[j] = key;
            sl = s5c_insert(C, j, key, (uint32_t)C.ctcap);
        }
        C.cslot[j] = sl;
        part = sl >= 0;
    }
    return part;
}

__global__ void __launch_bounds__(kBlock) k_s5c_key_groups(Ctx C, GroupGrid g, int32_t *list, int32_t *cnt) {
    const int c = grid_class(g, blockIdx.x);
    const int W = 1 << c;
    const int32_t pos = C.T.cls_start[c] + (blockIdx.x - g.blk_start[c]) * (kBlock / W) + threadIdx.x / W;
    const bool valid = pos < C.T.cls_start[c + 1];
    const int32_t j = valid ? C.T.order[pos] : 0;
    bool part;
    switch (c) {
        case 0: part = s5c_key_group<1>(C, j, valid); break;
        case 1: part = s5c_key_group<2>(C, j, valid); break;
        case 2: part = s5c_key_group<4>(C, j, valid); break;
        case 3: part = s5c_key_group<8>(C, j, valid); break;
        case 4: part = s5c_key_group<16>(C, j, valid); break;
        default: part = s5c_key_group<32>(C, j, valid); break;
    }
    block_append(part, j, cnt, list);
}

// long columns (class 6): one block per chunk sums its entry hashes
__global__ void __launch_bounds__(kBlock) k_s5c_key_long_partial(Ctx C) {
    __shared__ unsigned long long s_h[kBlock / 32];
    const Chunk ch = C.T.chunks[blockIdx.x];
    const bool neg0 = is_neg(C.T.val[C.T.ptr[ch.seg]]);
    unsigned long long h = 0;
    for (int32_t k = ch.begin + threadIdx.x; k < ch.end; k += kBlock)
        h += entry_hash(C.T.idx[k], is_neg(C.T.val[k]) != neg0);
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

// one warp per long column: its chunk sums, then the insert
__global__ void __launch_bounds__(kBlock) k_s5c_key_long(Ctx C, int32_t *list, int32_t *cnt) {
    const int32_t t = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int32_t nlong = C.T.cls_start[7] - C.T.cls_start[6];
    bool part = false;
    int32_t j = 0;
    if (t < nlong) {  // the same t in the whole warp
        j = C.T.order[C.T.cls_start[6] + t];
        unsigned long long h = 0;
        for (int32_t q = C.T.lfirst[t] + lane; q < C.T.lfirst[t + 1]; q += 32) h += C.ch_hash[q];
        h = group_sum<32>(h, 0xffffffffu);
        if (lane == 0) {
            int32_t sl = -1;
            if (C.ckind[j] == CK_KEPT) {
                const int32_t beg = C.T.ptr[j];
                const unsigned long long key = s5c_key(C, j, C.T.ptr[j + 1] - beg, is_neg(C.T.val[beg]), h);
                C.hcol[j] = key;
                sl = s5c_insert(C, j, key, (uint32_t)C.ctcap);
            }
            C.cslot[j] = sl;
            part = sl >= 0;
        }
    }
    block_append(part, j, cnt, list);
}

// later passes: the listed columns are inserted again with their stored keys
__global__ void __launch_bounds__(kBlock) k_s5c_insert(Ctx C, const int32_t *list, const int32_t *cnt) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *cnt) return;
    const int32_t j = list[t];
    C.cslot[j] = s5c_insert(C, j, C.hcol[j], (uint32_t)C.ctcap);
}

// entry q of columns j (first entry bj) and k (first entry bk): same row and
// a_j = lam a_k within par_tol
__device__ __forceinline__ bool s5c_same(const Ctx &C, int32_t bj, int32_t bk, int32_t q, double lam) {
    const double aj = C.T.val[bj + q], la = lam * C.T.val[bk + q];
    return C.T.idx[bj + q] == C.T.idx[bk + q] && fabs(aj - la) <= C.par_tol * fmax(fabs(aj), fabs(la));
}

// One thread per listed column checks it against its key's leader (columns
// longer than 32 entries are checked by the whole warp in turn); parallel
// columns bid for the leader with atomicMin on their index.
__global__ void __launch_bounds__(kBlock) k_s5c_match(Ctx C, const int32_t *list, const int32_t *cnt) {
    const int32_t n = *cnt;
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool ok = false;
    int32_t j = -1, k = -1, sl = -1, bj = 0, bk = 0, len = 0;
    double lam = 0.0;
    if (t < n) {
        j = list[t];
        sl = C.cslot[j];
        if (sl >= 0) {
            k = (int32_t)(uint32_t)C.ctlead[sl];
            if (k != j) {
                bj = C.T.ptr[j];
                bk = C.T.ptr[k];
                len = C.T.ptr[j + 1] - bj;
                lam = C.T.val[bj] / C.T.val[bk];
                const double cj = C.c[j], lc = lam * C.c[k];
                ok = C.T.ptr[k + 1] - bk == len && fabs(cj - lc) <= C.par_tol * fmax(fabs(cj), fabs(lc));
            }
        }
    }
    if (ok && len <= 32)
        for (int32_t q = 0; q < len && ok; q++) ok = s5c_same(C, bj, bk, q, lam);
    unsigned todo = __ballot_sync(0xffffffffu, ok && len > 32);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1u;
        const int32_t sbj = __shfl_sync(0xffffffffu, bj, src), sbk = __shfl_sync(0xffffffffu, bk, src);
        const int32_t slen = __shfl_sync(0xffffffffu, len, src);
        const double slam = __shfl_sync(0xffffffffu, lam, src);
        bool sok = true;
        for (int32_t q = lane; q < slen; q += 32) sok = sok && s5c_same(C, sbj, sbk, q, slam);
        sok = __all_sync(0xffffffffu, sok) != 0;
        if (lane == src) ok = sok;
    }
    if (ok) atomicMin(&C.ctfol[sl], j);
}

// The winning follower of each key merges into the leader (the only write to
// the leader's bounds in the pass); the leader stays while it merged, the
// columns that lost the bid or were not parallel stay too.
__global__ void __launch_bounds__(kBlock) k_s5c_merge(Ctx C, const int32_t *list, const int32_t *cnt, int32_t pass,
                                                     int32_t *out, int32_t *out_cnt) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    bool stay = false;
    int32_t j = -1, merged = 0;
    if (t < *cnt) {
        j = list[t];
        const int32_t sl = C.cslot[j];
        if (sl >= 0) {
            const int32_t k = (int32_t)(uint32_t)C.ctlead[sl], f = C.ctfol[sl];
            if (j == f) {
                const double lam = C.T.val[C.T.ptr[j]] / C.T.val[C.T.ptr[k]];
                const double2 bk = C.lu[k], bj = C.lu[j];
                double2 y;
                if (lam > 0.0) {
                    y.x = bk.x + lam * bj.x;
                    y.y = bk.y + lam * bj.y;
                } else {
                    y.x = bk.x + lam * bj.y;
                    y.y = bk.y + lam * bj.x;
                }
                C.lu[k] = y;
                C.ckind[j] = CK_PARALLEL;
                C.fixv[j] = 0.0;
                const int32_t lp = lp_of_col(C, j);
                const int32_t o = C.cmap[j];
                C.rec_ck[o] = CK_PARALLEL;
                C.rec_cr[o] = lp_round(C, lp);
                C.rec_cv[o] = lam;
                C.rec_ca[o] = C.cmap[k];
                C.rec_cp[o] = pass;
                C.rec_cm[4 * (int64_t)o] = bk.x;
                C.rec_cm[4 * (int64_t)o + 1] = bk.y;
                C.rec_cm[4 * (int64_t)o + 2] = bj.x;
                C.rec_cm[4 * (int64_t)o + 3] = bj.y;
                C.lp_changed[lp] = 1;
                merged = 1;
            } else {
                stay = j != k || f != kNone;
            }
        }
    }
    block_add(merged, &C.st->cols_fixed);
    block_append(stay, j, out_cnt, out);
}

// empties the slots the pass used (the table is empty between passes)
__global__ void __launch_bounds__(kBlock) k_s5c_clear(Ctx C, const int32_t *list, const int32_t *cnt) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *cnt) return;
    const int32_t sl = C.cslot[list[t]];
    if (sl >= 0) {
        C.ctkey[sl] = 0ULL;
        C.ctlead[sl] = ~0ULL;
        C.ctfol[sl] = kNone;
    }
}

inline unsigned blocks_for(int64_t cnt, int threads) {
    return (unsigned)((cnt + threads - 1) / threads > 0 ? (cnt + threads - 1) / threads : 1);
}

}  // namespace

void launch_s5c_keys(const Ctx &C, int32_t *list, int32_t *cnt, cudaStream_t s) {
    if (C.n <= 0) return;
    const GroupGrid g = group_grid(C.T);
    if (g.blk_start[6] > 0) (k_s5c_key_groups<<<g.blk_start[6], kBlock, 0, s>>>(C, g, list, cnt), note_launch());
    const int32_t nlong = C.T.cls_start[7] - C.T.cls_start[6];
    if (nlong > 0 && C.T.nchunks > 0) {
        (k_s5c_key_long_partial<<<C.T.nchunks, kBlock, 0, s>>>(C), note_launch());
        (k_s5c_key_long<<<blocks_for((int64_t)nlong * 32, kBlock), kBlock, 0, s>>>(C, list, cnt), note_launch());
    }
}

void launch_s5c_pass(const Ctx &C, const int32_t *list, const int32_t *cnt, int32_t pass, int32_t *out,
                     int32_t *out_cnt, int32_t max_cols, bool insert, cudaStream_t s) {
    if (max_cols <= 0) return;
    const unsigned b = blocks_for(max_cols, kBlock);
    if (insert) (k_s5c_insert<<<b, kBlock, 0, s>>>(C, list, cnt), note_launch());
    (k_s5c_match<<<b, kBlock, 0, s>>>(C, list, cnt), note_launch());
    (k_s5c_merge<<<b, kBlock, 0, s>>>(C, list, cnt, pass, out, out_cnt), note_launch());
    (k_s5c_clear<<<b, kBlock, 0, s>>>(C, list, cnt), note_launch());
}

}  // namespace lpp
