// k_compact.cu -- S6 (empty columns) and S7 (compaction) of a round.
//
// After S5 every row is kept or removed and every column kept or fixed.  The
// compaction keeps the relative order of rows, columns and entries:
//   1. per column (CSC): entries left in kept rows; a column with none left
//      is fixed at the bound its cost prefers (S6, dual rule);
//   2. per row (CSR): entries left in kept columns, and the shift
//      sum_j a_ij v_j over its fixed columns;
//   3. four exclusive scans: new row / column index, new row / column offset;
//   4. row and column vectors are gathered into the next buffers, the kept
//      sides shifted by their fixed columns (L -= shift, U -= shift);
//   5. entries are scattered into the next CSR and CSC, renumbered.
// Long segments use the chunk lists of the schedule: a chunk counts its kept
// entries, the chunks of a segment are prefix-summed in order, and each chunk
// then writes its entries from its own offset.
#include <algorithm>

#include "compact_dev.cuh"
#include "lpp_launch.h"

namespace lpp {

namespace {

__global__ void k_lp_dead(Ctx C, CompactCtx K) {
    const int32_t lp = blockIdx.x * blockDim.x + threadIdx.x;
    if (lp >= C.nlp) return;
    bool d = K.lp_retired ? K.lp_retired[lp] != 0 : false;
    for (int v = 0; v < V_SLOTS; v++) d |= C.verdict[lp * V_SLOTS + v] != kNone;
    K.lp_dead[lp] = d;
}

// warp-group count of the entries of one segment that satisfy `keep`
template <int W, class Keep>
__device__ __forceinline__ int32_t group_count(const int32_t *idx, int32_t beg, int32_t end, Keep keep) {
    const int lane = threadIdx.x & (W - 1);
    int32_t c = 0;
    for (int32_t k = beg + lane; k < end; k += W) c += keep(idx[k]) ? 1 : 0;
    return group_sum<W>(c, group_mask<W>());
}

// The flat scatter's tile t starts at entry t * kFlatTile; the segment (or
// chunk) [b, e) that holds that entry records itself.  Segments and chunks
// are at most kFlatTile long, so each holds at most one tile start.
__device__ __forceinline__ void mark_tile(int32_t *tile, int32_t b, int32_t e, int32_t seg) {
    const int64_t t = ((int64_t)b + kFlatTile - 1) / kFlatTile;
    if (t * kFlatTile < e) tile[t] = seg;
}

// ---------------------------------------------------------------- CSC count
template <int W>
__device__ __forceinline__ void csc_count_group(const Ctx &C, const CompactCtx &K, int32_t j, bool valid) {
    int32_t beg = 0, end = 0;
    if (valid) {
        beg = C.T.ptr[j];
        end = C.T.ptr[j + 1];
    }
    const uint8_t *rk = C.rkind;
    const int32_t cnt = group_count<W>(C.T.idx, beg, end, [rk](int32_t r) { return rk[r] == RK_KEPT; });
    if (valid && (threadIdx.x & (W - 1)) == 0) {
        K.c_len[j] = cnt;
        mark_tile(K.tile_t, beg, end, j);
    }
}

__global__ void __launch_bounds__(kBlock) k_csc_count_groups(Ctx C, CompactCtx K, GroupGrid g) {
    const int c = grid_class(g, blockIdx.x);
    const int W = 1 << c;
    const int32_t pos = C.T.cls_start[c] + (blockIdx.x - g.blk_start[c]) * (kBlock / W) + threadIdx.x / W;
    const bool valid = pos < C.T.cls_start[c + 1];
    const int32_t j = valid ? C.T.order[pos] : 0;
    switch (c) {
        case 0: csc_count_group<1>(C, K, j, valid); break;
        case 1: csc_count_group<2>(C, K, j, valid); break;
        case 2: csc_count_group<4>(C, K, j, valid); break;
        case 3: csc_count_group<8>(C, K, j, valid); break;
        case 4: csc_count_group<16>(C, K, j, valid); break;
        default: csc_count_group<32>(C, K, j, valid); break;
    }
}

__device__ __forceinline__ int32_t block_sum_int(int32_t v) {
    __shared__ int32_t s_w[kBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    int32_t t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kBlock / 32; w++) t += s_w[w];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(kBlock) k_csc_count_long(Ctx C, CompactCtx K) {
    const Chunk ch = C.T.chunks[blockIdx.x];
    int32_t c = 0;
    for (int32_t k = ch.begin + threadIdx.x; k < ch.end; k += kBlock) c += C.rkind[C.T.idx[k]] == RK_KEPT;
    c = block_sum_int(c);
    if (threadIdx.x == 0) {
        K.cht_cnt[blockIdx.x] = c;
        mark_tile(K.tile_t, ch.begin, ch.end, ch.seg);
        if (ch.begin == C.T.ptr[ch.seg]) K.c_ch0[ch.seg] = blockIdx.x;
    }
}

// per long segment (one warp): chunk offsets (prefix in chunk order), the
// total, and the sum of the chunks' side shifts (lane-strided, then a butterfly)
__global__ void k_long_prefix(const SegMat M, const int32_t *ch_cnt, int32_t *ch_off, int32_t *len_out,
                              const double *ch_shift, double *shift_out) {
    const int32_t t = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int32_t nlong = M.cls_start[7] - M.cls_start[6];
    if (t >= nlong) return;  // the same t in the whole warp
    const int32_t q1 = M.lfirst[t + 1];
    int32_t carry = 0;
    double sh = 0.0;
    for (int32_t q0 = M.lfirst[t]; q0 < q1; q0 += 32) {
        const int32_t q = q0 + lane;
        const int32_t c = q < q1 ? ch_cnt[q] : 0;
        int32_t inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (q < q1) {
            ch_off[q] = carry + inc - c;
            if (ch_shift) sh += ch_shift[q];
        }
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sh += __shfl_xor_sync(0xffffffffu, sh, o);
    if (lane == 0) {
        const int32_t seg = M.order[M.cls_start[6] + t];
        len_out[seg] = carry;
        if (shift_out) shift_out[seg] = sh;
    }
}

template <int W>
__device__ __forceinline__ void lock_group(const Ctx &C, const CompactCtx &K, int32_t j, bool valid) {
    const unsigned mask = group_mask<W>();
    const int lane = threadIdx.x & (W - 1);
    int32_t beg = 0, end = 0, lk = 0;
    if (valid) {
        beg = C.T.ptr[j];
        end = C.T.ptr[j + 1];
    }
    for (int32_t k = beg + lane; k < end; k += W) lk |= entry_locks(C, C.T.idx[k], C.T.val[k]);
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) lk |= __shfl_xor_sync(mask, lk, o, W);
    if (valid && lane == 0) K.c_lock[j] = lk;
}

__global__ void __launch_bounds__(kBlock) k_locks_groups(Ctx C, CompactCtx K, GroupGrid g) {
    const int c = grid_class(g, blockIdx.x);
    const int W = 1 << c;
    const int32_t pos = C.T.cls_start[c] + (blockIdx.x - g.blk_start[c]) * (kBlock / W) + threadIdx.x / W;
    const bool valid = pos < C.T.cls_start[c + 1];
    const int32_t j = valid ? C.T.order[pos] : 0;
    switch (c) {
        case 0: lock_group<1>(C, K, j, valid); break;
        case 1: lock_group<2>(C, K, j, valid); break;
        case 2: lock_group<4>(C, K, j, valid); break;
        case 3: lock_group<8>(C, K, j, valid); break;
        case 4: lock_group<16>(C, K, j, valid); break;
        default: lock_group<32>(C, K, j, valid); break;
    }
}

// long columns: one block per chunk, OR-ed into the column (zero before)
__global__ void __launch_bounds__(kBlock) k_locks_long(Ctx C, CompactCtx K) {
    const Chunk ch = C.T.chunks[blockIdx.x];
    int32_t lk = 0;
    for (int32_t k = ch.begin + threadIdx.x; k < ch.end; k += kBlock) lk |= entry_locks(C, C.T.idx[k], C.T.val[k]);
    lk = __reduce_or_sync(0xffffffffu, (unsigned)lk);
    if ((threadIdx.x & 31) == 0 && lk) atomicOr(&K.c_lock[ch.seg], lk);
}

// ------------------------------------------------------- S6 + column keep
// With the input CSC kept (Ctx::t_orig) the columns also stay in place: a
// column that left in an earlier round (cinv < 0) is skipped, the others
// keep their index (c_new = j), and one that leaves now gets cinv = -1.
// (grid-stride over a grid of at most 8 blocks per SM: one block sum per block)
__global__ void __launch_bounds__(kBlock) k_colkeep(Ctx C, CompactCtx K) {
    int32_t fixed = 0;
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < C.n; j += gridDim.x * blockDim.x) {
        if (C.t_orig && (C.cinv[j] < 0 || (C.ckind[j] == CK_KEPT && K.c_len[j] > 0 && !K.lp_dead[lp_of_col(C, j)]))) {
            // columns in place: one that left earlier keeps the flags it got
            // then (its contribution was consumed by the objective sum), and a
            // kept column with entries that S4 did not fix stays as it is
            // (no S6 test applies to it, its contribution is zero)
        } else {
            fixed += colkeep_one(C, K, j);
            if (C.t_orig) {
                const bool kp = K.c_keep[j] != 0;
                K.c_new[j] = kp ? j : -1;
                if (!kp) K.cinv[j] = -1;
            }
        }
    }
    block_add(fixed, &C.st->cols_fixed);
}

// --------------------------------------------------------------- CSR count
template <int W>
__device__ __forceinline__ void csr_count_group(const Ctx &C, const CompactCtx &K, int32_t i, bool valid) {
    if (valid && (threadIdx.x & (W - 1)) == 0) mark_tile(K.tile_a, C.A.ptr[i], C.A.ptr[i + 1], i);
    csr_count_row<W>(C, K, i, valid, valid && C.rkind[i] == RK_KEPT && !K.lp_dead[lp_of_row(C, i)]);
}

__global__ void __launch_bounds__(kBlock) k_csr_count_groups(Ctx C, CompactCtx K, GroupGrid g) {
    const int c = grid_class(g, blockIdx.x);
    const int W = 1 << c;
    const int32_t pos = C.A.cls_start[c] + (blockIdx.x - g.blk_start[c]) * (kBlock / W) + threadIdx.x / W;
    const bool valid = pos < C.A.cls_start[c + 1];
    const int32_t i = valid ? C.A.order[pos] : 0;
    switch (c) {
        case 0: csr_count_group<1>(C, K, i, valid); break;
        case 1: csr_count_group<2>(C, K, i, valid); break;
        case 2: csr_count_group<4>(C, K, i, valid); break;
        case 3: csr_count_group<8>(C, K, i, valid); break;
        case 4: csr_count_group<16>(C, K, i, valid); break;
        default: csr_count_group<32>(C, K, i, valid); break;
    }
}

__device__ __forceinline__ double block_sum_dbl(double v) {
    __shared__ double s_w[kBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kBlock / 32; w++) t += s_w[w];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(kBlock) k_csr_count_long(Ctx C, CompactCtx K) {
    const Chunk ch = C.A.chunks[blockIdx.x];
    const int32_t i = ch.seg;
    const bool keep = C.rkind[i] == RK_KEPT && !K.lp_dead[lp_of_row(C, i)];
    int32_t cnt = 0;
    double sh = 0.0;
    if (keep) {  // eight entries per thread and step in flight; the shift in entry order
        for (int32_t k0 = ch.begin + threadIdx.x; k0 < ch.end; k0 += 8 * kBlock) {
            int32_t jq[8], kq[8];
#pragma unroll
            for (int q = 0; q < 8; q++) jq[q] = k0 + q * kBlock < ch.end ? C.A.idx[k0 + q * kBlock] : 0;
#pragma unroll
            for (int q = 0; q < 8; q++) kq[q] = k0 + q * kBlock < ch.end ? K.c_keep[jq[q]] : 1;
#pragma unroll
            for (int q = 0; q < 8; q++) {
                if (k0 + q * kBlock >= ch.end) break;
                if (kq[q]) cnt++;
                else sh = fma(C.A.val[k0 + q * kBlock], C.fixv[jq[q]], sh);
            }
        }
    }
    cnt = block_sum_int(cnt);
    sh = block_sum_dbl(sh);
    if (threadIdx.x == 0) {
        K.chr_cnt[blockIdx.x] = cnt;
        K.chr_shift[blockIdx.x] = sh;
        mark_tile(K.tile_a, ch.begin, ch.end, i);
        if (ch.begin == C.A.ptr[i]) {  // the first chunk writes the flag
            K.r_keep[i] = keep;
            K.r_ch0[i] = blockIdx.x;
        }
    }
}

// ------------------------------------- column counts with the input CSC kept
// When T is the input's A^T (Ctx::t_orig) the entries per current column in
// the kept rows are the previous counts less the entries of the rows this
// round removed: their CSR entries, one atomic each (K.c_len holds the
// previous counts on entry).
template <int W>
__device__ __forceinline__ void clen_dec_group(const Ctx &C, const CompactCtx &K, int32_t i, bool valid) {
    const int lane = threadIdx.x & (W - 1);
    int32_t beg = 0, end = 0;
    if (valid && C.rkind[i] != RK_KEPT) {
        beg = C.A.ptr[i];
        end = C.A.ptr[i + 1];
    }
    for (int32_t k = beg + lane; k < end; k += W) atomicSub(&K.c_len[C.A.idx[k]], 1);
}

__global__ void __launch_bounds__(kBlock) k_clen_dec_groups(Ctx C, CompactCtx K, GroupGrid g) {
    const int c = grid_class(g, blockIdx.x);
    const int W = 1 << c;
    const int32_t pos = C.A.cls_start[c] + (blockIdx.x - g.blk_start[c]) * (kBlock / W) + threadIdx.x / W;
    const bool valid = pos < C.A.cls_start[c + 1];
    const int32_t i = valid ? C.A.order[pos] : 0;
    switch (c) {
        case 0: clen_dec_group<1>(C, K, i, valid); break;
        case 1: clen_dec_group<2>(C, K, i, valid); break;
        case 2: clen_dec_group<4>(C, K, i, valid); break;
        case 3: clen_dec_group<8>(C, K, i, valid); break;
        case 4: clen_dec_group<16>(C, K, i, valid); break;
        default: clen_dec_group<32>(C, K, i, valid); break;
    }
}

__global__ void __launch_bounds__(kBlock) k_clen_dec_long(Ctx C, CompactCtx K) {
    const Chunk ch = C.A.chunks[blockIdx.x];
    if (C.rkind[ch.seg] == RK_KEPT) return;  // block-uniform
    for (int32_t k = ch.begin + threadIdx.x; k < ch.end; k += kBlock) atomicSub(&K.c_len[C.A.idx[k]], 1);
}

// ------------------------------------- the columns' one compaction (t_orig)
// keep flag of each column slot: still in the LP
__global__ void k_cols_alive(const int32_t *cinv, int32_t n, int32_t *keep) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) keep[j] = cinv[j] >= 0;
}
// the kept columns' vectors to their compacted positions; cinv then maps
// an input column to its final index
__global__ void k_cols_final(const Ctx C, const CompactCtx K, int32_t n, int32_t *cinv) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (!K.c_keep[j]) return;  // cinv already -1
    const int32_t p = K.c_pos[j];
    K.lu2[p] = C.lu[j];
    K.c2[p] = C.c[j];
    K.cmap2[p] = C.cmap[j];
    if (C.lp_col) K.lp_col2[p] = C.lp_col[j];
    cinv[C.cmap[j]] = p;
}
// the CSR's column indices renumbered in place
__global__ void k_idx_renumber(int32_t *idx, int64_t nnz, const int32_t *pos) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nnz) idx[k] = pos[idx[k]];
}

// input rows / columns still in the LP, as a row kind (KEPT or not) and a
// keep flag for the compaction of the input CSC into the result's
__global__ void k_rows_left(const int32_t *rinv, int32_t m, uint8_t *rk) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) rk[i] = rinv[i] >= 0 ? (uint8_t)RK_KEPT : (uint8_t)RK_EMPTY;
}
__global__ void k_cols_left(const int32_t *cinv, int32_t n, int32_t *keep, int32_t *len) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    keep[j] = cinv[j] >= 0;
    if (cinv[j] < 0) len[j] = 0;
}
// the result CSC's pointers from the kept input columns' offsets
__global__ void k_cols_ptr(const CompactCtx K, int32_t n, int32_t *ptr) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) ptr[K.c_pos[n]] = K.c_off[n];
    if (j < n && K.c_keep[j]) ptr[K.c_pos[j]] = K.c_off[j];
}

// ---------------------------------------------------------- vector gathers
__global__ void __launch_bounds__(kBlock) k_rowvec(Ctx C, CompactCtx K) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C.m) return;
    if (i == C.m - 1) K.rp2[K.r_pos[C.m]] = K.r_off[C.m];
    const int32_t p = K.r_pos[i];
    K.r_new[i] = K.r_keep[i] ? p : -1;
    if (K.rinv) K.rinv[C.rmap[i]] = K.r_keep[i] ? p : -1;
    if (!K.r_keep[i]) return;
    const double sh = K.shift[i];
    const double Lv = C.L[i], Uv = C.U[i];
    K.L2[p] = is_fin(Lv) ? Lv - sh : Lv;
    K.U2[p] = is_fin(Uv) ? Uv - sh : Uv;
    K.rmap2[p] = C.rmap[i];
    if (C.lp_row) K.lp_row2[p] = C.lp_row[i];
    K.rp2[p] = K.r_off[i];
    // a row that lost entries (fixed columns) changed: evaluate it next round;
    // an unchanged row's S5 key is taken again when columns were dropped (the
    // key hashes column indices, which the compaction renumbers)
    const bool lost = K.r_len[i] != C.A.ptr[i + 1] - C.A.ptr[i];
    K.rdirty2[p] = (C.rdnext[i] | lost) ? 1 : (!C.t_orig && K.c_pos[C.n] != C.n ? 2 : 0);
    K.act2[p] = C.act[i];
    K.ninf2[p] = C.ninf[i];
    K.hrow2[p] = C.hrow[i];
}

__global__ void __launch_bounds__(kBlock) k_colvec(Ctx C, CompactCtx K) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= C.n) return;
    if (j == C.n - 1) K.cp2[K.c_pos[C.n]] = K.c_off[C.n];
    const int32_t p = K.c_pos[j];
    K.c_new[j] = K.c_keep[j] ? p : -1;
    if (!K.c_keep[j]) return;
    K.lu2[p] = C.lu[j];
    K.c2[p] = C.c[j];
    K.cmap2[p] = C.cmap[j];
    if (C.lp_col) K.lp_col2[p] = C.lp_col[j];
    K.cp2[p] = K.c_off[j];
}

// empty matrices still need ptr[0] = 0
__global__ void k_zero_ptr(int32_t *p) { p[0] = 0; }

// ---------------------------------------------------------------- scatter
// Flat ordered compaction of all entries.  Segments of at most kFlatTile
// entries, and the chunks of kChunk entries of the long ones, are the units.
// Block t takes the entries [t T, t T + T) of the matrix, T = kFlatTile:
//   1. one thread per segment between the segments of the entries t T and
//      (t + 1) T (coalesced, independent loads) marks the first in-tile entry
//      of each of its units in the tile, with a keep bit and the unit's base;
//      a block max-scan of the marks gives every entry the first in-tile
//      entry of its unit, or -1 if its segment is dropped;
//   2. striped (coalesced): keep = unit kept and the other index kept (one
//      gather of its new index, -1 if dropped); one ballot per warp and
//      step, exclusive scan of the counts;
//   3. striped: a kept entry x of unit s goes to
//         off[s] + (kept entries of s before x),
//      where the second term is scan(x) - scan(first in-tile entry of s) plus,
//      for a unit that started in an earlier tile, len[s] minus its kept
//      entries in this tile (it ends in this tile: it has at most T entries).
struct FlatArgs {
    const int32_t *ptr, *idx;
    const double *val;
    int32_t nnz, cnt, ntiles;
    const int32_t *seg_keep, *seg_off, *seg_len;  // per segment: kept, new offset, kept entries
    const int32_t *seg_ch0;                       // per long segment: its first chunk
    const int32_t *ch_off, *ch_cnt;               // per chunk: kept entries of its segment before it, its own
    const int32_t *oth_new;                       // per index of the other dimension: new index, -1 if dropped
    const int32_t *tile_seg;                      // per tile: segment of its first entry
    int32_t *out_idx;
    double *out_val;
};

constexpr int kFlatPer = kFlatTile / kBlock;  // entries per thread
constexpr int kFlatWords = kFlatTile / 32;    // ballot words per tile

__global__ void __launch_bounds__(kBlock) k_scatter_flat(FlatArgs F) {
    __shared__ __align__(16) int16_t s_start[kFlatTile];
    __shared__ int32_t s_raw[kFlatTile];
    __shared__ unsigned s_bal[kFlatWords + 1];
    __shared__ int32_t s_cb[kFlatWords + 1];
    __shared__ int32_t s_wmax[kBlock / 32];
    __shared__ int32_t s_re;
    __shared__ int32_t s_fp;
    const int t = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t k0 = (int32_t)((int64_t)t * kFlatTile);
    const int32_t len = F.nnz - k0 < kFlatTile ? F.nnz - k0 : kFlatTile;

    // 1a. no marks; 1b. one thread per segment marks its units
    {
        int4 *w = reinterpret_cast<int4 *>(s_start);
        for (int q = tid; q < kFlatTile / 8; q += kBlock) w[q] = make_int4(-1, -1, -1, -1);
    }
    if (tid == 0) s_fp = 0;
    __syncthreads();
    const int32_t lo = F.tile_seg[t];
    const int32_t hi = t + 1 < F.ntiles ? F.tile_seg[t + 1] : F.cnt - 1;
    const int32_t k1 = k0 + len;
    for (int32_t r = lo + tid; r <= hi; r += kBlock) {
        const int32_t pb = __ldg(F.ptr + r), pe = __ldg(F.ptr + r + 1);
        if (pe <= pb || pb >= k1) continue;  // empty, or after the tile
        const bool emit = F.seg_keep[r] != 0;
        // units of r that meet the tile: the segment, or chunks q0..q1
        int32_t q0 = 0, q1 = 0;
        const bool lng = pe - pb >= kLongMin;
        if (lng) {
            q0 = ((pb > k0 ? pb : k0) - pb) / kChunk;
            q1 = ((pe < k1 ? pe : k1) - 1 - pb) / kChunk;
        }
        for (int32_t q = q0; q <= q1; q++) {
            const int32_t vb = pb + q * kChunk;
            const int32_t ve = lng ? min(vb + kChunk, pe) : pe;
            const int32_t xs = vb > k0 ? vb - k0 : 0;
            s_start[xs] = (int16_t)(2 * xs + (emit ? 1 : 0));
            if (emit) {
                int32_t raw, ln;
                if (lng) {
                    const int32_t ch = F.seg_ch0[r] + q;
                    raw = F.seg_off[r] + F.ch_off[ch];
                    ln = F.ch_cnt[ch];
                } else {
                    raw = F.seg_off[r];
                    ln = F.seg_len[r];
                }
                if (vb < k0) {  // the unit holding entry k0
                    raw += ln;
                    s_re = ve - k0;
                    s_fp = 1;
                }
                s_raw[xs] = raw;
            }
        }
    }
    __syncthreads();
    // 1c. inclusive max-scan of the marks (blocked, 16 per thread)
    {
        const int x0 = tid * kFlatPer;
        int4 *w = reinterpret_cast<int4 *>(s_start + x0);
        int4 a = w[0], b = w[1];
        int16_t v[kFlatPer];
        memcpy(v, &a, 16);
        memcpy(v + 8, &b, 16);
        int32_t run = -1;
#pragma unroll
        for (int e = 0; e < kFlatPer; e++) {
            run = v[e] > run ? v[e] : run;
        }
        int32_t inc = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o && y > inc) inc = y;
        }
        if (lane == 31) s_wmax[warp] = inc;
        int32_t prev = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane == 0) prev = -1;
        __syncthreads();
        for (int q = 0; q < warp; q++) prev = s_wmax[q] > prev ? s_wmax[q] : prev;
        run = prev;
#pragma unroll
        for (int e = 0; e < kFlatPer; e++) {
            run = v[e] > run ? v[e] : run;
            v[e] = (x0 + e < len && (run & 1)) ? (int16_t)(run >> 1) : (int16_t)-1;
        }
        memcpy(&a, v, 16);
        memcpy(&b, v + 8, 16);
        w[0] = a;
        w[1] = b;
    }
    __syncthreads();

    // 2. keep flags, striped
    int32_t jn[kFlatPer];
#pragma unroll
    for (int i = 0; i < kFlatPer; i++) {
        const int x = i * kBlock + tid;
        jn[i] = -1;
        if (x < len && s_start[x] >= 0) jn[i] = F.idx[k0 + x];
    }
#pragma unroll
    for (int i = 0; i < kFlatPer; i++) {
        if (jn[i] >= 0) jn[i] = F.oth_new[jn[i]];
        const unsigned bal = __ballot_sync(0xffffffffu, jn[i] >= 0);
        if (lane == 0) s_bal[i * (kBlock / 32) + warp] = bal;
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the ballot counts
        constexpr int per = kFlatWords / 32;
        int32_t c[per], tot = 0;
#pragma unroll
        for (int q = 0; q < per; q++) {
            c[q] = __popc(s_bal[lane * per + q]);
            tot += c[q];
        }
        int32_t inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        int32_t acc = inc - tot;
#pragma unroll
        for (int q = 0; q < per; q++) {
            s_cb[lane * per + q] = acc;
            acc += c[q];
        }
        if (lane == 31) {
            s_cb[kFlatWords] = inc;
            s_bal[kFlatWords] = 0u;
        }
    }
    __syncthreads();

    // 3. positions and copies, striped
    auto scan_at = [&](int y) {  // kept entries of the tile before position y (0 <= y <= T)
        const int q = y >> 5;
        return s_cb[q] + __popc(s_bal[q] & ((1u << (y & 31)) - 1u));
    };
    const int32_t fix = s_fp ? scan_at(s_re) : 0;
#pragma unroll
    for (int i = 0; i < kFlatPer; i++) {
        if (jn[i] < 0) continue;
        const int x = i * kBlock + tid;
        const int xs = s_start[x];
        int32_t p = s_raw[xs] - scan_at(xs) + scan_at(x);
        if (xs == 0) p -= fix;
        F.out_idx[p] = jn[i];
        F.out_val[p] = F.val[k0 + x];
    }
}

// ---------------------------------------------------------- objective constant
// one LP: tiles of kScanTile columns summed in a fixed order, then the tiles
// the contributions are consumed: reset to zero once read (a column whose
// flags are not recomputed in a later round then contributes nothing)
__global__ void __launch_bounds__(kBlock) k_offset_tiles(double *contrib, int32_t n, double *part) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    double s = 0.0;
    for (int t = threadIdx.x; t < kScanTile; t += kBlock) {
        const int64_t j = base + t;
        if (j < n) {
            const double v = contrib[j];
            s += v;
            if (v != 0.0) contrib[j] = 0.0;
        }
    }
    s = block_sum_dbl(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}
// one block: thread t adds tiles t, t+256, ... in order, then the fixed-order block sum
__global__ void __launch_bounds__(kBlock) k_offset_final(const double *part, int32_t ntiles, double *offset) {
    double s = 0.0;
    for (int32_t t = threadIdx.x; t < ntiles; t += kBlock) s += part[t];
    s = block_sum_dbl(s);
    if (threadIdx.x == 0) offset[0] += s;
}
// many LPs: column range of each LP, then one warp per LP
__global__ void k_lp_ranges(const int32_t *lp_col, int32_t n, int32_t *first, int32_t *last) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int32_t lp = lp_col[j];
    if (j == 0 || lp_col[j - 1] != lp) first[lp] = j;
    if (j == n - 1 || lp_col[j + 1] != lp) last[lp] = j + 1;
}
__global__ void k_offset_lps(double *contrib, const int32_t *first, const int32_t *last, int32_t nlp,
                             double *offset) {
    const int32_t lp = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (lp >= nlp) return;
    double s = 0.0;
    for (int32_t j = first[lp] + lane; j < last[lp]; j += 32) {  // consumed as in k_offset_tiles
        const double v = contrib[j];
        s += v;
        if (v != 0.0) contrib[j] = 0.0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) offset[lp] += s;
}

inline unsigned blocks_for(int64_t cnt, int threads) {
    return (unsigned)std::max<int64_t>(1, (cnt + threads - 1) / threads);
}

}  // namespace

void launch_compact_counts(const Ctx &C, const CompactCtx &K, cudaStream_t s, const SideStream *side) {
    (k_lp_dead<<<blocks_for(C.nlp, 256), 256, 0, s>>>(C, K), note_launch());
    // 1. column counts over kept rows, then S6 and the column keep flags
    const GroupGrid ga = group_grid(C.A);
    const int32_t along = C.A.cls_start[7] - C.A.cls_start[6];
    if (C.t_orig) {  // the previous counts less the removed rows' entries
        if (C.n > 0 && K.c_len != C.clen)
            cudaMemcpyAsync(K.c_len, C.clen, sizeof(int32_t) * (size_t)C.n, cudaMemcpyDeviceToDevice, s);
        if (ga.blk_start[6] > 0) (k_clen_dec_groups<<<ga.blk_start[6], kBlock, 0, s>>>(C, K, ga), note_launch());
        if (along > 0 && C.A.nchunks > 0) (k_clen_dec_long<<<C.A.nchunks, kBlock, 0, s>>>(C, K), note_launch());
    }
    const GroupGrid gt = group_grid(C.T);
    if (!C.t_orig && gt.blk_start[6] > 0) (k_csc_count_groups<<<gt.blk_start[6], kBlock, 0, s>>>(C, K, gt), note_launch());
    const int32_t tlong = C.T.cls_start[7] - C.T.cls_start[6];
    if (!C.t_orig && tlong > 0 && C.T.nchunks > 0) {
        (k_csc_count_long<<<C.T.nchunks, kBlock, 0, s>>>(C, K), note_launch());
        (k_long_prefix<<<blocks_for((int64_t)tlong * 32, 128), 128, 0, s>>>(C.T, K.cht_cnt, K.cht_off, K.c_len, nullptr,
                                                                             nullptr), note_launch());
    }
    if (C.dualfix && C.n > 0) {
        cudaMemsetAsync(K.c_lock, 0, sizeof(int32_t) * (size_t)C.n, s);
        if (gt.blk_start[6] > 0) (k_locks_groups<<<gt.blk_start[6], kBlock, 0, s>>>(C, K, gt), note_launch());
        if (tlong > 0 && C.T.nchunks > 0) (k_locks_long<<<C.T.nchunks, kBlock, 0, s>>>(C, K), note_launch());
    }
    if (C.n > 0) (k_colkeep<<<std::min<unsigned>(blocks_for(C.n, kBlock), 8u * 152u), kBlock, 0, s>>>(C, K), note_launch());
    // 2. row counts over kept columns and the side shifts; the long rows'
    // chunks (and their prefix) on the side stream when one is given: the
    // two touch disjoint rows, and each tile start lies in one row
    const bool long_rows = along > 0 && C.A.nchunks > 0;
    const bool fork = long_rows && side && side->s;
    cudaStream_t sl = s;
    if (fork) {
        cudaEventRecord(side->fork, s);
        cudaStreamWaitEvent(side->s, side->fork, 0);
        sl = side->s;
    }
    if (long_rows) {
        (k_csr_count_long<<<C.A.nchunks, kBlock, 0, sl>>>(C, K), note_launch());
        (k_long_prefix<<<blocks_for((int64_t)along * 32, 128), 128, 0, sl>>>(C.A, K.chr_cnt, K.chr_off, K.r_len,
                                                                              K.chr_shift, K.shift), note_launch());
    }
    if (ga.blk_start[6] > 0) (k_csr_count_groups<<<ga.blk_start[6], kBlock, 0, s>>>(C, K, ga), note_launch());
    if (fork) {
        cudaEventRecord(side->join, side->s);
        cudaStreamWaitEvent(s, side->join, 0);
    }
}

void launch_compact_scatter(const Ctx &C, const CompactCtx &K, int32_t nnz, cudaStream_t s) {
    (k_zero_ptr<<<1, 1, 0, s>>>(K.rp2), note_launch());
    if (!C.t_orig) (k_zero_ptr<<<1, 1, 0, s>>>(K.cp2), note_launch());
    if (C.m > 0) (k_rowvec<<<blocks_for(C.m, kBlock), kBlock, 0, s>>>(C, K), note_launch());
    if (C.n > 0 && !C.t_orig) (k_colvec<<<blocks_for(C.n, kBlock), kBlock, 0, s>>>(C, K), note_launch());
    const int32_t ntiles = (int32_t)(((int64_t)nnz + kFlatTile - 1) / kFlatTile);
    if (ntiles > 0) {
        FlatArgs fa{C.A.ptr, C.A.idx, C.A.val, nnz, C.m, ntiles, K.r_keep, K.r_off, K.r_len, K.r_ch0,
                    K.chr_off, K.chr_cnt, K.c_new, K.tile_a, K.ci2, K.rv2};
        (k_scatter_flat<<<ntiles, kBlock, 0, s>>>(fa), note_launch());
        if (!C.t_orig) {
            FlatArgs ft{C.T.ptr, C.T.idx, C.T.val, nnz, C.n, ntiles, K.c_keep, K.c_off, K.c_len, K.c_ch0,
                        K.cht_off, K.cht_cnt, K.r_new, K.tile_t, K.ri2, K.cv2};
            (k_scatter_flat<<<ntiles, kBlock, 0, s>>>(ft), note_launch());
        }
    }
}

// The result's CSC from the input CSC C.T (input numbering, Ctx::t_orig):
// C.rkind marks the input rows still in the LP, keep / len the input
// columns still in it and their entries left; the one compaction of the
// kept columns' kept entries, renumbered by rinv, into ptr / idx / val
// (K.c_pos / c_off: the column scan, done by the caller between the two
// calls).
void launch_csc_from_input_counts(const Ctx &C, const CompactCtx &K, cudaStream_t s) {
    const GroupGrid gt = group_grid(C.T);
    if (gt.blk_start[6] > 0) (k_csc_count_groups<<<gt.blk_start[6], kBlock, 0, s>>>(C, K, gt), note_launch());
    const int32_t tlong = C.T.cls_start[7] - C.T.cls_start[6];
    if (tlong > 0 && C.T.nchunks > 0) {
        (k_csc_count_long<<<C.T.nchunks, kBlock, 0, s>>>(C, K), note_launch());
        (k_long_prefix<<<blocks_for((int64_t)tlong * 32, 128), 128, 0, s>>>(C.T, K.cht_cnt, K.cht_off, K.c_len, nullptr,
                                                                             nullptr), note_launch());
    }
    if (C.n > 0) (k_cols_left<<<blocks_for(C.n, kBlock), kBlock, 0, s>>>(C.cinv, C.n, K.c_keep, K.c_len), note_launch());
}

void launch_csc_from_input_scatter(const Ctx &C, const CompactCtx &K, int64_t nnz, int32_t *ptr, int32_t *idx,
                                   double *val, cudaStream_t s) {
    (k_cols_ptr<<<blocks_for(std::max(C.n, 1), kBlock), kBlock, 0, s>>>(K, C.n, ptr), note_launch());
    const int32_t ntiles = (int32_t)((nnz + kFlatTile - 1) / kFlatTile);
    if (ntiles > 0) {
        FlatArgs ft{C.T.ptr, C.T.idx, C.T.val, (int32_t)nnz, C.n, ntiles, K.c_keep, K.c_off, K.c_len, K.c_ch0,
                    K.cht_off, K.cht_cnt, C.rinv, K.tile_t, idx, val};
        (k_scatter_flat<<<ntiles, kBlock, 0, s>>>(ft), note_launch());
    }
}

void launch_cols_alive(const int32_t *cinv, int32_t n, int32_t *keep, cudaStream_t s) {
    if (n > 0) (k_cols_alive<<<blocks_for(n, kBlock), kBlock, 0, s>>>(cinv, n, keep), note_launch());
}
void launch_cols_final(const Ctx &C, const CompactCtx &K, int32_t n, int32_t *cinv, int32_t *idx, int64_t nnz,
                       cudaStream_t s) {
    if (n > 0) (k_cols_final<<<blocks_for(n, kBlock), kBlock, 0, s>>>(C, K, n, cinv), note_launch());
    if (nnz > 0) (k_idx_renumber<<<blocks_for(nnz, kBlock), kBlock, 0, s>>>(idx, nnz, K.c_pos), note_launch());
}

void launch_rows_left(const int32_t *rinv, int32_t m, uint8_t *rk, cudaStream_t s) {
    if (m > 0) (k_rows_left<<<blocks_for(m, kBlock), kBlock, 0, s>>>(rinv, m, rk), note_launch());
}

void launch_offset(const Ctx &C, const CompactCtx &K, cudaStream_t s) {
    if (C.n == 0) return;
    if (C.nlp == 1) {
        const int32_t ntiles = (int32_t)((C.n + kScanTile - 1) / kScanTile);
        (k_offset_tiles<<<ntiles, kBlock, 0, s>>>(K.contrib, C.n, K.offset_part), note_launch());
        (k_offset_final<<<1, kBlock, 0, s>>>(K.offset_part, ntiles, K.offset), note_launch());
    } else {
        cudaMemsetAsync(K.lp_first, 0, sizeof(int32_t) * (size_t)C.nlp, s);
        cudaMemsetAsync(K.lp_last, 0, sizeof(int32_t) * (size_t)C.nlp, s);
        (k_lp_ranges<<<blocks_for(C.n, 256), 256, 0, s>>>(C.lp_col, C.n, K.lp_first, K.lp_last), note_launch());
        (k_offset_lps<<<blocks_for((int64_t)C.nlp * 32, 256), 256, 0, s>>>(K.contrib, K.lp_first, K.lp_last, C.nlp,
                                                                           K.offset), note_launch());
    }
}

}  // namespace lpp
