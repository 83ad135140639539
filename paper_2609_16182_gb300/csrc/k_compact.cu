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
    if (valid && (threadIdx.x & (W - 1)) == 0) K.c_len[j] = cnt;
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
    if (threadIdx.x == 0) K.cht_cnt[blockIdx.x] = c;
}

// per long segment: chunk offsets (prefix in chunk order) and the total
__global__ void k_long_prefix(const SegMat M, const int32_t *ch_cnt, int32_t *ch_off, int32_t *len_out,
                              const double *ch_shift, double *shift_out) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t nlong = M.cls_start[7] - M.cls_start[6];
    if (t >= nlong) return;
    int32_t acc = 0;
    double sh = 0.0;
    for (int32_t q = M.lfirst[t]; q < M.lfirst[t + 1]; q++) {
        ch_off[q] = acc;
        acc += ch_cnt[q];
        if (ch_shift) sh += ch_shift[q];
    }
    const int32_t seg = M.order[M.cls_start[6] + t];
    len_out[seg] = acc;
    if (shift_out) shift_out[seg] = sh;
}

// ------------------------------------------------------- S6 + column keep
__global__ void __launch_bounds__(kBlock) k_colkeep(Ctx C, CompactCtx K) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t fixed = 0;
    if (j < C.n) {
        const int32_t lp = lp_of_col(C, j);
        const bool dead = K.lp_dead[lp];
        uint8_t kind = C.ckind[j];
        double contrib = 0.0;
        if (!dead && kind == CK_KEPT && C.dual && K.c_len[j] == 0) {
            const double2 b = C.lu[j];
            const double cj = C.c[j];
            double v;
            if (cj > 0.0) v = b.x;
            else if (cj < 0.0) v = b.y;
            else v = is_fin(b.x) ? b.x : (is_fin(b.y) ? b.y : 0.0);
            if (!is_fin(v)) {
                atomicMin(&C.verdict[lp * V_SLOTS + V_S6_COL], C.cmap[j]);
            } else {
                kind = CK_EMPTY;
                C.ckind[j] = kind;
                C.fixv[j] = v;
                const int32_t o = C.cmap[j];
                C.rec_ck[o] = CK_EMPTY;
                C.rec_cr[o] = lp_round(C, lp);
                C.rec_cv[o] = v;
                C.lp_changed[lp] = 1;
                fixed = 1;
            }
        }
        if (!dead && kind != CK_KEPT) contrib = C.c[j] * C.fixv[j];
        const bool keep = !dead && kind == CK_KEPT;
        K.c_keep[j] = keep;
        if (!keep) K.c_len[j] = 0;
        K.contrib[j] = contrib;
    }
    block_add(fixed, &C.st->cols_fixed);
}

// --------------------------------------------------------------- CSR count
template <int W>
__device__ __forceinline__ void csr_count_group(const Ctx &C, const CompactCtx &K, int32_t i, bool valid) {
    const unsigned mask = group_mask<W>();
    const int lane = threadIdx.x & (W - 1);
    int32_t beg = 0, end = 0;
    bool keep = false;
    if (valid) {
        keep = C.rkind[i] == RK_KEPT && !K.lp_dead[lp_of_row(C, i)];
        if (keep) {
            beg = C.A.ptr[i];
            end = C.A.ptr[i + 1];
        }
    }
    int32_t cnt = 0;
    double sh = 0.0;
    for (int32_t k = beg + lane; k < end; k += W) {
        const int32_t j = C.A.idx[k];
        if (K.c_keep[j]) cnt++;
        else sh = fma(C.A.val[k], C.fixv[j], sh);
    }
    cnt = group_sum<W>(cnt, mask);
    sh = group_sum<W>(sh, mask);
    if (valid && lane == 0) {
        K.r_keep[i] = keep;
        K.r_len[i] = cnt;
        K.shift[i] = sh;
    }
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
    if (keep) {
        for (int32_t k = ch.begin + threadIdx.x; k < ch.end; k += kBlock) {
            const int32_t j = C.A.idx[k];
            if (K.c_keep[j]) cnt++;
            else sh = fma(C.A.val[k], C.fixv[j], sh);
        }
    }
    cnt = block_sum_int(cnt);
    sh = block_sum_dbl(sh);
    if (threadIdx.x == 0) {
        K.chr_cnt[blockIdx.x] = cnt;
        K.chr_shift[blockIdx.x] = sh;
        if (ch.begin == C.A.ptr[i]) K.r_keep[i] = keep;  // first chunk writes the flag
    }
}

// ---------------------------------------------------------- vector gathers
__global__ void __launch_bounds__(kBlock) k_rowvec(Ctx C, CompactCtx K) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C.m) return;
    if (i == C.m - 1) K.rp2[K.r_pos[C.m]] = K.r_off[C.m];
    if (!K.r_keep[i]) return;
    const int32_t p = K.r_pos[i];
    const double sh = K.shift[i];
    const double Lv = C.L[i], Uv = C.U[i];
    K.L2[p] = is_fin(Lv) ? Lv - sh : Lv;
    K.U2[p] = is_fin(Uv) ? Uv - sh : Uv;
    K.rmap2[p] = C.rmap[i];
    if (C.lp_row) K.lp_row2[p] = C.lp_row[i];
    K.rp2[p] = K.r_off[i];
    // a row that lost entries (fixed columns) changed: evaluate it next round
    const bool lost = K.r_len[i] != C.A.ptr[i + 1] - C.A.ptr[i];
    K.rdirty2[p] = (uint8_t)(C.rdnext[i] | lost);
    K.act2[p] = C.act[i];
    K.ninf2[p] = C.ninf[i];
    K.hrow2[p] = C.hrow[i];
}

__global__ void __launch_bounds__(kBlock) k_colvec(Ctx C, CompactCtx K) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= C.n) return;
    if (j == C.n - 1) K.cp2[K.c_pos[C.n]] = K.c_off[C.n];
    if (!K.c_keep[j]) return;
    const int32_t p = K.c_pos[j];
    K.lu2[p] = C.lu[j];
    K.c2[p] = C.c[j];
    K.cmap2[p] = C.cmap[j];
    if (C.lp_col) K.lp_col2[p] = C.lp_col[j];
    K.cp2[p] = K.c_off[j];
}

// empty matrices still need ptr[0] = 0
__global__ void k_zero_ptr(int32_t *p) { p[0] = 0; }

// ---------------------------------------------------------------- scatter
// ordered compaction of the kept entries of one segment by a lane group
template <int W, class Keep, class Emit>
__device__ __forceinline__ void group_scatter(const int32_t *idx, int32_t beg, int32_t end, int32_t out0, Keep keep,
                                              Emit emit) {
    const unsigned mask = group_mask<W>();
    const int lane = threadIdx.x & (W - 1);
    int32_t base = out0;
    for (int32_t k0 = beg; k0 < end; k0 += W) {
        const int32_t k = k0 + lane;
        const bool in = k < end;
        const int32_t t = in ? idx[k] : 0;
        const bool kp = in && keep(t);
        const unsigned b = group_bits<W>(__ballot_sync(mask, kp));
        if (kp) emit(k, t, base + __popc(b & ((1u << lane) - 1u)));
        base += __popc(b);
    }
}

template <int W>
__device__ __forceinline__ void csr_scatter_group(const Ctx &C, const CompactCtx &K, int32_t i, bool valid) {
    int32_t beg = 0, end = 0, out0 = 0;
    if (valid && K.r_keep[i]) {
        beg = C.A.ptr[i];
        end = C.A.ptr[i + 1];
        out0 = K.r_off[i];
    }
    const int32_t *ck = K.c_keep;
    const int32_t *cpos = K.c_pos;
    const double *val = C.A.val;
    int32_t *ci2 = K.ci2;
    double *rv2 = K.rv2;
    group_scatter<W>(C.A.idx, beg, end, out0, [ck](int32_t j) { return ck[j] != 0; },
                     [=](int32_t k, int32_t j, int32_t p) {
                         ci2[p] = cpos[j];
                         rv2[p] = val[k];
                     });
}

template <int W>
__device__ __forceinline__ void csc_scatter_group(const Ctx &C, const CompactCtx &K, int32_t j, bool valid) {
    int32_t beg = 0, end = 0, out0 = 0;
    if (valid && K.c_keep[j]) {
        beg = C.T.ptr[j];
        end = C.T.ptr[j + 1];
        out0 = K.c_off[j];
    }
    const int32_t *rk = K.r_keep;
    const int32_t *rpos = K.r_pos;
    const double *val = C.T.val;
    int32_t *ri2 = K.ri2;
    double *cv2 = K.cv2;
    group_scatter<W>(C.T.idx, beg, end, out0, [rk](int32_t r) { return rk[r] != 0; },
                     [=](int32_t k, int32_t r, int32_t p) {
                         ri2[p] = rpos[r];
                         cv2[p] = val[k];
                     });
}

__global__ void __launch_bounds__(kBlock) k_csr_scatter_groups(Ctx C, CompactCtx K, GroupGrid g) {
    const int c = grid_class(g, blockIdx.x);
    const int W = 1 << c;
    const int32_t pos = C.A.cls_start[c] + (blockIdx.x - g.blk_start[c]) * (kBlock / W) + threadIdx.x / W;
    const bool valid = pos < C.A.cls_start[c + 1];
    const int32_t i = valid ? C.A.order[pos] : 0;
    switch (c) {
        case 0: csr_scatter_group<1>(C, K, i, valid); break;
        case 1: csr_scatter_group<2>(C, K, i, valid); break;
        case 2: csr_scatter_group<4>(C, K, i, valid); break;
        case 3: csr_scatter_group<8>(C, K, i, valid); break;
        case 4: csr_scatter_group<16>(C, K, i, valid); break;
        default: csr_scatter_group<32>(C, K, i, valid); break;
    }
}

__global__ void __launch_bounds__(kBlock) k_csc_scatter_groups(Ctx C, CompactCtx K, GroupGrid g) {
    const int c = grid_class(g, blockIdx.x);
    const int W = 1 << c;
    const int32_t pos = C.T.cls_start[c] + (blockIdx.x - g.blk_start[c]) * (kBlock / W) + threadIdx.x / W;
    const bool valid = pos < C.T.cls_start[c + 1];
    const int32_t j = valid ? C.T.order[pos] : 0;
    switch (c) {
        case 0: csc_scatter_group<1>(C, K, j, valid); break;
        case 1: csc_scatter_group<2>(C, K, j, valid); break;
        case 2: csc_scatter_group<4>(C, K, j, valid); break;
        case 3: csc_scatter_group<8>(C, K, j, valid); break;
        case 4: csc_scatter_group<16>(C, K, j, valid); break;
        default: csc_scatter_group<32>(C, K, j, valid); break;
    }
}

// ordered compaction of one chunk by a whole block
template <class Keep, class Emit>
__device__ __forceinline__ void block_scatter(const int32_t *idx, int32_t beg, int32_t end, int32_t out0, Keep keep,
                                              Emit emit) {
    __shared__ int32_t s_w[kBlock / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t base = out0;
    for (int32_t k0 = beg; k0 < end; k0 += kBlock) {
        const int32_t k = k0 + threadIdx.x;
        const bool in = k < end;
        const int32_t t = in ? idx[k] : 0;
        const bool kp = in && keep(t);
        const unsigned b = __ballot_sync(0xffffffffu, kp);
        if (lane == 0) s_w[warp] = __popc(b);
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t acc = 0;
            for (int w = 0; w < kBlock / 32; w++) {
                const int32_t v = s_w[w];
                s_w[w] = acc;
                acc += v;
            }
            s_w[kBlock / 32] = acc;
        }
        __syncthreads();
        if (kp) emit(k, t, base + s_w[warp] + __popc(b & ((1u << lane) - 1u)));
        base += s_w[kBlock / 32];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBlock) k_csr_scatter_long(Ctx C, CompactCtx K) {
    const Chunk ch = C.A.chunks[blockIdx.x];
    if (!K.r_keep[ch.seg]) return;
    const int32_t out0 = K.r_off[ch.seg] + K.chr_off[blockIdx.x];
    const int32_t *ck = K.c_keep;
    const int32_t *cpos = K.c_pos;
    const double *val = C.A.val;
    int32_t *ci2 = K.ci2;
    double *rv2 = K.rv2;
    block_scatter(C.A.idx, ch.begin, ch.end, out0, [ck](int32_t j) { return ck[j] != 0; },
                  [=](int32_t k, int32_t j, int32_t p) {
                      ci2[p] = cpos[j];
                      rv2[p] = val[k];
                  });
}

__global__ void __launch_bounds__(kBlock) k_csc_scatter_long(Ctx C, CompactCtx K) {
    const Chunk ch = C.T.chunks[blockIdx.x];
    if (!K.c_keep[ch.seg]) return;
    const int32_t out0 = K.c_off[ch.seg] + K.cht_off[blockIdx.x];
    const int32_t *rk = K.r_keep;
    const int32_t *rpos = K.r_pos;
    const double *val = C.T.val;
    int32_t *ri2 = K.ri2;
    double *cv2 = K.cv2;
    block_scatter(C.T.idx, ch.begin, ch.end, out0, [rk](int32_t r) { return rk[r] != 0; },
                  [=](int32_t k, int32_t r, int32_t p) {
                      ri2[p] = rpos[r];
                      cv2[p] = val[k];
                  });
}

// ---------------------------------------------------------- objective constant
// one LP: tiles of kScanTile columns summed in a fixed order, then the tiles
__global__ void __launch_bounds__(kBlock) k_offset_tiles(const double *contrib, int32_t n, double *part) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    double s = 0.0;
    for (int t = threadIdx.x; t < kScanTile; t += kBlock) {
        const int64_t j = base + t;
        if (j < n) s += contrib[j];
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
__global__ void k_offset_lps(const double *contrib, const int32_t *first, const int32_t *last, int32_t nlp,
                             double *offset) {
    const int32_t lp = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (lp >= nlp) return;
    double s = 0.0;
    for (int32_t j = first[lp] + lane; j < last[lp]; j += 32) s += contrib[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) offset[lp] += s;
}

inline unsigned blocks_for(int64_t cnt, int threads) {
    return (unsigned)std::max<int64_t>(1, (cnt + threads - 1) / threads);
}

}  // namespace

void launch_compact_counts(const Ctx &C, const CompactCtx &K, cudaStream_t s) {
    (k_lp_dead<<<blocks_for(C.nlp, 256), 256, 0, s>>>(C, K), note_launch());
    // 1. column counts over kept rows, then S6 and the column keep flags
    const GroupGrid gt = group_grid(C.T);
    if (gt.blk_start[6] > 0) (k_csc_count_groups<<<gt.blk_start[6], kBlock, 0, s>>>(C, K, gt), note_launch());
    const int32_t tlong = C.T.cls_start[7] - C.T.cls_start[6];
    if (tlong > 0 && C.T.nchunks > 0) {
        (k_csc_count_long<<<C.T.nchunks, kBlock, 0, s>>>(C, K), note_launch());
        (k_long_prefix<<<blocks_for(tlong, 128), 128, 0, s>>>(C.T, K.cht_cnt, K.cht_off, K.c_len, nullptr, nullptr), note_launch());
    }
    if (C.n > 0) (k_colkeep<<<blocks_for(C.n, kBlock), kBlock, 0, s>>>(C, K), note_launch());
    // 2. row counts over kept columns and the side shifts
    const GroupGrid ga = group_grid(C.A);
    if (ga.blk_start[6] > 0) (k_csr_count_groups<<<ga.blk_start[6], kBlock, 0, s>>>(C, K, ga), note_launch());
    const int32_t along = C.A.cls_start[7] - C.A.cls_start[6];
    if (along > 0 && C.A.nchunks > 0) {
        (k_csr_count_long<<<C.A.nchunks, kBlock, 0, s>>>(C, K), note_launch());
        (k_long_prefix<<<blocks_for(along, 128), 128, 0, s>>>(C.A, K.chr_cnt, K.chr_off, K.r_len, K.chr_shift,
                                                               K.shift), note_launch());
    }
}

void launch_compact_scatter(const Ctx &C, const CompactCtx &K, int32_t m_new, int32_t n_new, cudaStream_t s) {
    (void)m_new;
    (void)n_new;
    (k_zero_ptr<<<1, 1, 0, s>>>(K.rp2), note_launch());
    (k_zero_ptr<<<1, 1, 0, s>>>(K.cp2), note_launch());
    if (C.m > 0) (k_rowvec<<<blocks_for(C.m, kBlock), kBlock, 0, s>>>(C, K), note_launch());
    if (C.n > 0) (k_colvec<<<blocks_for(C.n, kBlock), kBlock, 0, s>>>(C, K), note_launch());
    const GroupGrid ga = group_grid(C.A);
    if (ga.blk_start[6] > 0) (k_csr_scatter_groups<<<ga.blk_start[6], kBlock, 0, s>>>(C, K, ga), note_launch());
    if (C.A.cls_start[7] > C.A.cls_start[6] && C.A.nchunks > 0)
        (k_csr_scatter_long<<<C.A.nchunks, kBlock, 0, s>>>(C, K), note_launch());
    const GroupGrid gt = group_grid(C.T);
    if (gt.blk_start[6] > 0) (k_csc_scatter_groups<<<gt.blk_start[6], kBlock, 0, s>>>(C, K, gt), note_launch());
    if (C.T.cls_start[7] > C.T.cls_start[6] && C.T.nchunks > 0)
        (k_csc_scatter_long<<<C.T.nchunks, kBlock, 0, s>>>(C, K), note_launch());
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
