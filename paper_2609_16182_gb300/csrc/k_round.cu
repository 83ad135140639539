// k_round.cu -- the kernels of one presolve round up to compaction:
//   S1 activities, S2 row classes, S3 implied bounds (fused, one pass over the
//   CSR), S3'/S4 bound finalisation and fixing, S5 parallel rows.
//
// Load balance (Sec. 3.1, "length-based load balancing"): rows are grouped
// by length class.  Class c <= 5 gives each row a group of W = 2^c lanes of a
// warp (lane t walks entries t, t+W, ...; the group then reduces with an xor
// butterfly), class 6 (more than 4096 entries) splits the row into chunks of
// 4096 entries, one thread block each, whose partial results are combined in
// chunk order.  The order of every floating-point sum depends only on the
// row's own length.
//
// Bound tightening follows Sec. 3.1 in Jacobi form: activities and the
// acceptance tests read the bounds of the round start, accepted implied
// bounds are combined with atomicMin / atomicMax on an order-preserving
// integer encoding, which is exact and independent of the order of updates.
//
// FP64 is scarce on this GPU (about two DFMA per SM and clock), so every
// per-entry sign, finiteness and max(1,|x|) test runs on integer pipes, the
// activity sums are fused multiply-adds, and an implied bound is divided out
// only after an exact FMA sign test (x - thr*a) says it will be accepted.
#include <algorithm>

#include "lpp_launch.h"
#include "round_dev.cuh"

namespace lpp {

namespace {

__global__ void __launch_bounds__(kBlock, 4) k_prop_groups(Ctx C, GroupGrid g) {
    __shared__ double s_qx[kBlock / 32][kQueueCap], s_qa[kBlock / 32][kQueueCap];
    __shared__ int32_t s_qj[kBlock / 32][kQueueCap], s_qk[kBlock / 32][kQueueCap];
    __shared__ double s_ta[kBlock / 32][kQueueCap], s_ts[kBlock / 32][kQueueCap], s_tb[kBlock / 32][kQueueCap],
        s_to[kBlock / 32][kQueueCap];
    __shared__ int32_t s_tj[kBlock / 32][kQueueCap], s_tf[kBlock / 32][kQueueCap];
    const int warp = threadIdx.x >> 5;
    CandQueue q{s_qx[warp], s_qa[warp], s_qj[warp], s_qk[warp], 0};
    TestQueue tq{s_ta[warp], s_ts[warp], s_tb[warp], s_to[warp], s_tj[warp], s_tf[warp], 0};
    const int c = grid_class(g, blockIdx.x);
    const int32_t lb = blockIdx.x - g.blk_start[c];
    int32_t removed = 0, evaluated = 0, tested = 0;
    const int W = prop_lanes(c);
    const int32_t pos = C.A.cls_start[c] + lb * (kBlock / W) + threadIdx.x / W;
    const bool valid = pos < C.A.cls_start[c + 1];
    const int32_t i = valid ? C.A.order[pos] : 0;
    switch (c) {
        case 0:
        case 1:
        case 2: prop_group<1>(C, i, valid, removed, evaluated, tested, q, tq); break;
        case 3: prop_group<8>(C, i, valid, removed, evaluated, tested, q, tq); break;
        case 4: prop_group<16>(C, i, valid, removed, evaluated, tested, q, tq); break;
        default: prop_group<32>(C, i, valid, removed, evaluated, tested, q, tq); break;
    }
    tq_flush(C, tq, q);
    cq_flush(C, q);
    block_add(removed, &C.st->rows_removed);
    if (C.count_work) {  // statistics of a timed run only: each block_add is two block barriers
        block_add(evaluated, &C.st->nnz_eval);
        block_add(tested, &C.st->sides_tested);
    }
}

// fixed-order block reduction (warp butterflies, then warps in order)
template <typename T>
__device__ __forceinline__ T block_reduce_ordered(T v, T *s_w) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = T(0);
    if (threadIdx.x == 0)
        for (int w = 0; w < kBlock / 32; w++) t += s_w[w];
    __syncthreads();
    return t;  // thread 0
}

// ------------------------------------------------------------ long rows
__global__ void __launch_bounds__(kBlock) k_prop_long_partial(Ctx C, unsigned long long *ch_hash) {
    __shared__ double s_d[kBlock / 32];
    __shared__ int s_i[kBlock / 32];
    __shared__ unsigned long long s_h[kBlock / 32];
    const Chunk ch = C.A.chunks[blockIdx.x];
    if (!C.rdirty[ch.seg]) return;  // block-uniform
    const bool neg0 = is_neg(C.A.val[C.A.ptr[ch.seg]]);
    double smin = 0.0, smax = 0.0;
    int nmin = 0, nmax = 0;
    unsigned long long h = 0;
#pragma unroll 4
    for (int32_t k = ch.begin + threadIdx.x; k < ch.end; k += kBlock) {
        const int32_t j = __ldcs(C.A.idx + k);  // streamed once: evict first, keep the bounds cached
        const double a = __ldcs(C.A.val + k);
        const double2 b = C.lu[j];
        const bool neg = is_neg(a);
        const double bmin = neg ? b.y : b.x, bmax = neg ? b.x : b.y;
        if (is_fin(bmin)) smin = fma(a, bmin, smin);
        else nmin++;
        if (is_fin(bmax)) smax = fma(a, bmax, smax);
        else nmax++;
        h += entry_hash(j, neg != neg0);
    }
    smin = block_reduce_ordered(smin, s_d);
    smax = block_reduce_ordered(smax, s_d);
    nmin = block_reduce_ordered(nmin, s_i);
    nmax = block_reduce_ordered(nmax, s_i);
    h = block_reduce_ordered(h, s_h);
    if (threadIdx.x == 0) {
        C.ch_act[blockIdx.x] = make_double2(smin, smax);
        C.ch_ninf[blockIdx.x] = make_int2(nmin, nmax);
        ch_hash[blockIdx.x] = h;
    }
}

// one warp per long row: the chunk partials, lane-strided then a butterfly
__global__ void __launch_bounds__(kBlock) k_prop_long_combine(Ctx C, const unsigned long long *ch_hash) {
    const int32_t t = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int32_t nlong = C.A.cls_start[7] - C.A.cls_start[6];
    int32_t removed = 0, evaluated = 0;
    if (t < nlong) {  // the same t in the whole warp
        const int32_t i = C.A.order[C.A.cls_start[6] + t];
        if (!C.rdirty[i]) {
            if (lane == 0) {
                C.rkind[i] = RK_KEPT;
                C.lneed[t] = 0;
            }
        } else {
            double smin = 0.0, smax = 0.0;
            int nmin = 0, nmax = 0;
            unsigned long long h = 0;
            for (int32_t q = C.A.lfirst[t] + lane; q < C.A.lfirst[t + 1]; q += 32) {
                const double2 a = C.ch_act[q];
                const int2 c = C.ch_ninf[q];
                smin += a.x;
                smax += a.y;
                nmin += c.x;
                nmax += c.y;
                h += ch_hash[q];
            }
            smin = group_sum<32>(smin, 0xffffffffu);
            smax = group_sum<32>(smax, 0xffffffffu);
            nmin = group_sum<32>(nmin, 0xffffffffu);
            nmax = group_sum<32>(nmax, 0xffffffffu);
            h = group_sum<32>(h, 0xffffffffu);
            if (lane == 0) {
                const int32_t beg = C.A.ptr[i], len = C.A.ptr[i + 1] - beg;
                h += len_hash(len);
                const double Lv = C.L[i], Uv = C.U[i];
                uint8_t kind;
                double sa = 0.0;
                int32_t sj = -1;  // long rows are never singletons
                removed = finish_row(C, i, beg, len, Lv, Uv, smin, smax, nmin, nmax, h, kind, sa, sj);
                evaluated = len;
                C.lneed[t] = kind == RK_KEPT && ((is_fin(Uv) && nmin <= 1) || (is_fin(Lv) && nmax <= 1));
            }
        }
    }
    block_add(removed, &C.st->rows_removed);
    block_add(evaluated, &C.st->nnz_eval);
}

__global__ void __launch_bounds__(kBlock) k_prop_long_tighten(Ctx C) {
    const Chunk ch = C.A.chunks[blockIdx.x];
    if (!C.lneed[ch.lidx]) return;
    const int32_t i = ch.seg;
    const double Lv = C.L[i], Uv = C.U[i];
    const double2 act = C.act[i];
    const int2 ni = C.ninf[i];
    const bool up_row = is_fin(Uv) && ni.x <= 1, lo_row = is_fin(Lv) && ni.y <= 1;
    const double dU = Uv - act.x, dL = Lv - act.y;
    int32_t tested = 0;
    for (int32_t k = ch.begin + threadIdx.x; k < ch.end; k += kBlock)
        tighten_entry(C, C.A.idx[k], C.A.val[k], up_row, lo_row, dU, dL, ni.x, ni.y, tested);
    block_add(tested, &C.st->sides_tested);  // the whole block returned above or reaches here
}

// ------------------------------------------ S3 bound sources (dual records)
// The dual postsolve moves a reduced cost on a tightened bound to the row
// that implied it, so each accepted candidate needs its row.  Between S3 and
// S3', every row S1-S3 evaluated this round (a dirty flag) runs over its
// entries again, row by row as S3 does: an entry whose column received a
// candidate re-derives its implied bound (or the singleton row's bound) on
// the stored activities with the activity kernels' arithmetic, and a value
// equal to the accepted candidate (encoded values compared: bit for bit)
// offers its original row index to the column's side (atomicMin: the
// smallest row wins).
__device__ __forceinline__ void bsrc_offer(const Ctx &C, int32_t j, double x, double a, bool upper, bool capped,
                                           unsigned long long el, unsigned long long eu, int32_t o) {
    if (capped && gt0(fma(-C.max_implied, fabs(a), fabs(x)))) return;
    const double v = x / a;
    if (!is_fin(v)) return;
    const unsigned long long e = enc_dbl(v);
    if (upper) {
        if (e == eu) atomicMin(&C.bsrc[j].y, o);
    } else if (e == el) {
        atomicMin(&C.bsrc[j].x, o);
    }
}

// entries [k0, k1) of row i, every step-th from k0
__device__ __forceinline__ void bsrc_row(const Ctx &C, int32_t i, int32_t k0, int32_t k1, int32_t step) {
    const uint8_t kind = C.rkind[i];
    const int32_t len = C.A.ptr[i + 1] - C.A.ptr[i];
    if (!(kind == RK_SINGLETON || (kind == RK_KEPT && len >= 2))) return;
    const double Lv = C.L[i], Uv = C.U[i];
    const int32_t o = C.rmap[i];
    const double2 act = C.act[i];
    const int2 ni = C.ninf[i];
    const bool up_row = is_fin(Uv) && ni.x <= 1, lo_row = is_fin(Lv) && ni.y <= 1;
    const double dU = Uv - act.x, dL = Lv - act.y;
    for (int32_t k = k0; k < k1; k += step) {
        const int32_t j = C.A.idx[k];
        if (C.ctouch[j] == 0u) continue;  // no candidate this round (one 4-byte gather)
        const unsigned long long el = C.cand_l[j], eu = C.cand_u[j];
        if (el == kEncNegInf && eu == kEncPosInf) continue;
        const double a = C.A.val[k];
        const bool neg = is_neg(a);
        if (kind == RK_SINGLETON) {  // L <= a x_j <= U: bounds L/a and U/a (a < 0 swaps them), no cap
            if (is_fin(Lv)) bsrc_offer(C, j, Lv, a, neg, false, el, eu, o);
            if (is_fin(Uv)) bsrc_offer(C, j, Uv, a, !neg, false, el, eu, o);
            continue;
        }
        const double2 b = C.lu[j];
        const double bmin = neg ? b.y : b.x, bmax = neg ? b.x : b.y;
        const bool fmn = is_fin(bmin), fmx = is_fin(bmax);
        if (up_row && (fmn ? ni.x == 0 : ni.x == 1))  // a x_j <= U - (min activity of the others)
            bsrc_offer(C, j, fmn ? fma(a, bmin, dU) : dU, a, !neg, true, el, eu, o);
        if (lo_row && (fmx ? ni.y == 0 : ni.y == 1))  // a x_j >= L - (max activity of the others)
            bsrc_offer(C, j, fmx ? fma(a, bmax, dL) : dL, a, neg, true, el, eu, o);
    }
}

// rows of classes 0..5, 1 << class lanes per row (the grid of group_grid)
__global__ void __launch_bounds__(kBlock) k_bsrc_groups(Ctx C, GroupGrid g) {
    const int c = grid_class(g, blockIdx.x);
    const int W = 1 << c;
    const int32_t pos = C.A.cls_start[c] + (blockIdx.x - g.blk_start[c]) * (kBlock / W) + threadIdx.x / W;
    if (pos >= C.A.cls_start[c + 1]) return;
    const int32_t i = C.A.order[pos];
    if (C.rdirty[i] == 0) return;
    bsrc_row(C, i, C.A.ptr[i] + (int32_t)(threadIdx.x & (W - 1)), C.A.ptr[i + 1], W);
}

// the chunks of the long rows, a block per chunk
__global__ void __launch_bounds__(kBlock) k_bsrc_chunks(Ctx C) {
    const Chunk ch = C.A.chunks[blockIdx.x];
    if (C.rdirty[ch.seg] == 0) return;
    bsrc_row(C, ch.seg, ch.begin + threadIdx.x, ch.end, kBlock);
}

// ---------------------------------------- dependent equality rows (Sec. 5)
// the rows the host found dependent leave with their records (the row kinds
// of every other row were reset to kept before)
__global__ void __launch_bounds__(kBlock) k_mark_dependent(Ctx C, const int32_t *list, int32_t cnt) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int32_t i = list[t];
    C.rkind[i] = RK_DEPENDENT;
    const int32_t o = C.rmap[i];
    C.rec_rk[o] = RK_DEPENDENT;
    C.rec_rr[o] = C.round;
    C.rec_ra[o] = -1;
    C.rec_rv[o] = 0.0;
}

// ------------------------------------------------- S3' finalise + S4 fixing
// every column (some LP in its first round)
// (grid-stride over a grid of at most 8 blocks per SM: the block sums run
// once per block, not once per 256 columns)
__global__ void __launch_bounds__(kBlock) k_colfin(Ctx C) {
    int32_t changed = 0, fixed = 0, chg_nnz = 0;
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < C.n; j += gridDim.x * blockDim.x)
        colfin_one(C, j, true, changed, fixed, chg_nnz);
    block_add(changed, &C.st->bounds_changed);
    block_add(fixed, &C.st->cols_fixed);
    block_add(chg_nnz, C.cl_nnz);
}

// the columns that received a candidate (the others keep their bounds; their
// kind and change flag were reset at the start of the round)
__global__ void __launch_bounds__(kBlock) k_colfin_list(Ctx C) {
    const int32_t cnt = *C.tl_cnt;
    int32_t changed = 0, fixed = 0, chg_nnz = 0;
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x)
        colfin_one(C, C.tl_list[t], false, changed, fixed, chg_nnz);
    block_add(changed, &C.st->bounds_changed);
    block_add(fixed, &C.st->cols_fixed);
    block_add(chg_nnz, C.cl_nnz);
}

// ------------------------------------------------------------ S5 parallel rows
// first pass: rows kept by S2 with >= 2 entries take part
// (grid-stride, one block sum per block)
__global__ void __launch_bounds__(kBlock) k_s5_insert(Ctx C) {
    int32_t part = 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < C.m; i += gridDim.x * blockDim.x) {
        int32_t slot = -1;
        if (C.rkind[i] == RK_KEPT && C.A.ptr[i + 1] - C.A.ptr[i] >= 2) slot = s5_insert_row(C, i, (uint32_t)C.tcap);
        C.rslot[i] = slot;
        C.rwork[i] = slot >= 0 ? 1 : 0;
        part += slot >= 0;
    }
    block_add(part, &C.st->participants);
}

__global__ void __launch_bounds__(kBlock) k_s5_match_groups(Ctx C, GroupGrid g) {
    const int c = grid_class(g, blockIdx.x);
    const int32_t lb = blockIdx.x - g.blk_start[c];
    int32_t removed = 0, unmatched = 0;
    const int W = 1 << c;
    const int32_t pos = C.A.cls_start[c] + lb * (kBlock / W) + threadIdx.x / W;
    const bool valid = pos < C.A.cls_start[c + 1];
    const int32_t i = valid ? C.A.order[pos] : 0;
    bool left;
    switch (c) {
        case 0: left = match_group<1>(C, i, valid, removed, unmatched); break;
        case 1: left = match_group<2>(C, i, valid, removed, unmatched); break;
        case 2: left = match_group<4>(C, i, valid, removed, unmatched); break;
        case 3: left = match_group<8>(C, i, valid, removed, unmatched); break;
        case 4: left = match_group<16>(C, i, valid, removed, unmatched); break;
        default: left = match_group<32>(C, i, valid, removed, unmatched); break;
    }
    block_add(removed, &C.st->rows_removed);
    block_add(unmatched, &C.st->unmatched);
    block_append(left, i, C.s5_out_cnt, C.s5_out);
}

// long rows: one block per row of class 6 (parallel long rows are rare)
__global__ void __launch_bounds__(kBlock) k_s5_match_long(Ctx C) {
    const int32_t t = blockIdx.x;
    const int32_t i = C.A.order[C.A.cls_start[6] + t];
    bool act = C.rwork[i] == 1;
    int32_t li = -1;
    if (act) {
        li = (int32_t)(uint32_t)(C.tlead[C.rslot[i]] & 0xffffffffULL);
        if (li == i) act = false;
    }
    int32_t bi = 0, bl = 0, len = 0;
    bool ok = false;
    double lam = 0.0;
    if (act) {
        bi = C.A.ptr[i];
        bl = C.A.ptr[li];
        len = C.A.ptr[i + 1] - bi;
        ok = (C.A.ptr[li + 1] - bl) == len;
        lam = C.A.val[bi] / C.A.val[bl];
    }
    if (ok) {
        for (int32_t k = threadIdx.x; k < len; k += kBlock) {
            const double ai = C.A.val[bi + k], al = C.A.val[bl + k];
            const double la = lam * al;
            if (!(C.A.idx[bi + k] == C.A.idx[bl + k] && fabs(ai - la) <= C.par_tol * fmax(fabs(ai), fabs(la))))
                ok = false;
        }
    }
    ok = __syncthreads_and(ok) != 0;
    int32_t removed = 0, unmatched = 0;
    if (threadIdx.x == 0) {
        if (act && ok) {
            s5_accept(C, i, li, lam);
            C.rwork[i] = 0;
            removed = 1;
        } else if (act) {
            C.rwork[i] = 2;
            unmatched = 1;
            C.s5_out[atomicAdd(C.s5_out_cnt, 1)] = i;
        } else {
            C.rwork[i] = 0;
        }
    }
    block_add(removed, &C.st->rows_removed);
    block_add(unmatched, &C.st->unmatched);
}

// Later passes run on the list of rows the previous pass left unmatched
// (count *cnt, at most the launch's grid): insert, match against the new
// leader (one warp per row; unmatched rows go to the next list), then clear
// the slots used so that the table is empty for the next pass.  The table
// capacity of a pass is the power of two >= 2 * count, at most C.tcap.
__global__ void __launch_bounds__(kBlock) k_s5_tail_insert(Ctx C, const int32_t *list, const int32_t *cnt) {
    const int32_t n = *cnt;
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int32_t i = list[t];
    C.rslot[i] = s5_insert_row(C, i, s5_tail_cap(C, n));
}

// one thread per listed row; rows longer than 32 entries are checked by the
// whole warp in turn
__global__ void __launch_bounds__(kBlock) k_s5_tail_match(Ctx C, const int32_t *list, const int32_t *cnt,
                                                         int32_t *out, int32_t *out_cnt) {
    const int32_t n = *cnt;
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t removed, i;
    bool left;
    s5_tail_match_one(C, list, n, t, removed, left, i);
    block_add(removed, &C.st->rows_removed);
    block_append(left, i, out_cnt, out);
}

__global__ void __launch_bounds__(kBlock) k_s5_tail_clear(Ctx C, const int32_t *list, const int32_t *cnt) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *cnt) return;
    const int32_t sl = C.rslot[list[t]];
    if (sl >= 0) {
        C.tkey[sl] = 0ULL;
        C.tlead[sl] = ~0ULL;
    }
}

// All remaining later passes in one block, for a short list: the passes
// above (insert, match, clear) separated by block barriers instead of
// launches, with no host read between them.  Starts at pass p0 from list
// lists[(p0 - 1) & 1] of cnt[p0] rows, runs passes p0 .. max_iter - 1 (fewer
// once no row is left) and writes the rows left after the last one to
// cnt[max_iter].  The next list of a pass is written in the order the rows
// are left (unspecified, as in the launched form; the leaders of a pass do
// not depend on it).
constexpr int kTailBlock = 1024;
__global__ void __launch_bounds__(kTailBlock) k_s5_tail_block(Ctx C, int32_t *l0, int32_t *l1, int32_t *cnt,
                                                              int32_t p0, int32_t max_iter) {
    __shared__ int32_t s_n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int32_t n = cnt[p0], from = (p0 - 1) & 1, rem = 0;
    for (int32_t p = p0; p < max_iter && n > 0; p++) {
        const int32_t *lst = from ? l1 : l0;
        int32_t *nxt = from ? l0 : l1;
        const uint32_t cap = s5_tail_cap(C, n);
        for (int32_t t = tid; t < n; t += kTailBlock) C.rslot[lst[t]] = s5_insert_row(C, lst[t], cap);
        if (tid == 0) s_n = 0;
        __syncthreads();
        for (int32_t tb = warp * 32; tb < n; tb += kTailBlock) {  // warp-uniform: every lane calls the match
            int32_t rm, i;
            bool left;
            s5_tail_match_one(C, lst, n, tb + lane, rm, left, i);
            rem += rm;
            if (left) nxt[atomicAdd(&s_n, 1)] = i;
        }
        __syncthreads();
        for (int32_t t = tid; t < n; t += kTailBlock) {
            const int32_t sl = C.rslot[lst[t]];
            if (sl >= 0) {
                C.tkey[sl] = 0ULL;
                C.tlead[sl] = ~0ULL;
            }
        }
        __syncthreads();
        n = s_n;
        from ^= 1;
        __syncthreads();  // every thread has read s_n before the next pass resets it
    }
    block_add(rem, &C.st->rows_removed);
    if (tid == 0) cnt[max_iter] = n;
}

// All remaining later passes of a long list in one cooperative launch (every
// block resident): the passes of the launched form, separated by grid
// barriers.  Mutable data (lists, slots, leaders, counts) is read at L2.  A
// barrier that waits too long (it cannot, with every block resident) sets
// st->err bit 4 and the kernel returns.  Same starting point and result
// slot as k_s5_tail_block.
constexpr long long kBarSpins = 1LL << 22;
__device__ bool grid_barrier(unsigned *bar, int32_t *err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        volatile int32_t *verr = err;
        const unsigned g = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(bar, 1u) + 1u == gridDim.x) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            for (long long spins = 0; *gen == g; spins++) {
                if (spins > kBarSpins || (*verr & 4)) {
                    atomicOr(err, 4);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__global__ void __launch_bounds__(kBlock) k_s5_tail_grid(Ctx C, int32_t *l0, int32_t *l1, int32_t *cnt, int32_t p0,
                                                        int32_t max_iter, unsigned *bar) {
    const int lane = threadIdx.x & 31;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gstride = (int64_t)gridDim.x * blockDim.x;
    const int64_t gwarp = gtid >> 5;
    int32_t n = __ldcg(cnt + p0), from = (p0 - 1) & 1, rem = 0;
    bool ok = true;
    int32_t p = p0;
    for (; p < max_iter && n > 0 && ok; p++) {
        const int32_t *lst = from ? l1 : l0;
        int32_t *nxt = from ? l0 : l1;
        const uint32_t cap = s5_tail_cap(C, n);
        for (int64_t t = gtid; t < n; t += gstride) {
            const int32_t i = __ldcg(lst + t);
            C.rslot[i] = s5_insert_row(C, i, cap);
        }
        if (!(ok = grid_barrier(bar, &C.st->err))) break;
        for (int64_t tb = gwarp * 32; tb < n; tb += gstride) {  // warp-uniform: every lane calls the match
            int32_t rm, i;
            bool left;
            s5_tail_match_one(C, lst, n, (int32_t)(tb + lane), rm, left, i);
            rem += rm;
            const unsigned want = __ballot_sync(0xffffffffu, left);
            int32_t base = 0;
            if (lane == 0 && want) base = atomicAdd(cnt + p + 1, __popc(want));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (left) nxt[base + __popc(want & ((1u << lane) - 1u))] = i;
        }
        if (!(ok = grid_barrier(bar, &C.st->err))) break;
        for (int64_t t = gtid; t < n; t += gstride) {
            const int32_t sl = __ldcg(C.rslot + __ldcg(lst + t));
            if (sl >= 0) {
                C.tkey[sl] = 0ULL;
                C.tlead[sl] = ~0ULL;
            }
        }
        if (!(ok = grid_barrier(bar, &C.st->err))) break;
        n = __ldcg(cnt + p + 1);
        from ^= 1;
    }
    block_add(rem, &C.st->rows_removed);
    if (blockIdx.x == 0 && threadIdx.x == 0 && ok) cnt[max_iter] = n;
}

__global__ void __launch_bounds__(kBlock) k_s5_leader(Ctx C) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C.m || !C.hasf[i]) return;
    s5_leader_one(C, i);
}

// row r of a T entry (an input row when T is not compacted: its current
// index, none once it left) is evaluated next round
__device__ __forceinline__ void mark_row_of(const Ctx &C, int32_t r) {
    if (C.t_orig) r = C.rinv[r];
    if (r >= 0) C.rdnext[r] = 1;
}

// rows of the changed short columns need their activities next round: one
// thread per listed column; columns longer than 32 entries are walked by the
// whole warp in turn.  When the changed columns hold at least an eighth of the
// nonzeros, every row is marked instead (re-evaluating a row whose inputs did
// not change finds nothing new).
__global__ void __launch_bounds__(kBlock) k_mark_list(Ctx C, int64_t nnz) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (8 * (int64_t)*C.cl_nnz >= nnz) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < C.m; i += stride) C.rdnext[i] = 1;
        return;
    }
    const int32_t cnt = *C.cl_cnt;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < cnt; base += stride) {
        const int64_t t = base + lane;
        int32_t b = 0, e = 0;
        if (t < cnt) {
            const int32_t j = C.cl_list[t];
            const int32_t jt = C.t_orig ? C.cmap[j] : j;
            b = C.T.ptr[jt];
            e = C.T.ptr[jt + 1];
        }
        if (e - b <= 32)
            for (int32_t k = b; k < e; k++) mark_row_of(C, C.T.idx[k]);
        unsigned todo = __ballot_sync(0xffffffffu, e - b > 32);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1u;
            const int32_t sb = __shfl_sync(0xffffffffu, b, src), se = __shfl_sync(0xffffffffu, e, src);
            for (int32_t k = sb + lane; k < se; k += 32) mark_row_of(C, C.T.idx[k]);
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_mark_long(Ctx C, int64_t nnz) {
    const Chunk ch = C.T.chunks[blockIdx.x];
    const int32_t j = C.t_orig ? C.cinv[ch.seg] : ch.seg;
    if (j < 0 || !C.cchg[j] || 8 * (int64_t)*C.cl_nnz >= nnz) return;
    for (int32_t k = ch.begin + threadIdx.x; k < ch.end; k += kBlock) mark_row_of(C, C.T.idx[k]);
}

inline unsigned blocks_for(int64_t cnt, int threads) {
    return (unsigned)((cnt + threads - 1) / threads > 0 ? (cnt + threads - 1) / threads : 1);
}

}  // namespace

void launch_prop_short(const Ctx &C, cudaStream_t s) {
    GroupGrid g;  // blocks per class at prop_lanes(c) lanes per row
    int32_t acc = 0;
    for (int c = 0; c < 6; c++) {
        g.blk_start[c] = acc;
        const int32_t per = kBlock / prop_lanes(c);
        acc += (C.A.cls_start[c + 1] - C.A.cls_start[c] + per - 1) / per;
    }
    g.blk_start[6] = acc;
    if (g.blk_start[6] > 0) (k_prop_groups<<<g.blk_start[6], kBlock, 0, s>>>(C, g), note_launch());
}

bool prop_has_long(const Ctx &C) { return C.A.cls_start[7] > C.A.cls_start[6] && C.A.nchunks > 0; }

void launch_prop_long(const Ctx &C, cudaStream_t s) {
    const int32_t nlong = C.A.cls_start[7] - C.A.cls_start[6];
    if (nlong <= 0 || C.A.nchunks <= 0) return;
    (k_prop_long_partial<<<C.A.nchunks, kBlock, 0, s>>>(C, C.ch_hash), note_launch());
    (k_prop_long_combine<<<blocks_for((int64_t)nlong * 32, kBlock), kBlock, 0, s>>>(C, C.ch_hash), note_launch());
    (k_prop_long_tighten<<<C.A.nchunks, kBlock, 0, s>>>(C), note_launch());
}

void launch_bound_src(const Ctx &C, cudaStream_t s) {
    if (C.m <= 0 || C.n <= 0) return;
    const GroupGrid g = group_grid(C.A);
    if (g.blk_start[6] > 0) (k_bsrc_groups<<<g.blk_start[6], kBlock, 0, s>>>(C, g), note_launch());
    if (C.A.cls_start[7] > C.A.cls_start[6] && C.A.nchunks > 0)
        (k_bsrc_chunks<<<C.A.nchunks, kBlock, 0, s>>>(C), note_launch());
}

void launch_mark_dependent(const Ctx &C, const int32_t *list, int32_t cnt, cudaStream_t s) {
    if (cnt > 0) (k_mark_dependent<<<blocks_for(cnt, kBlock), kBlock, 0, s>>>(C, list, cnt), note_launch());
}

void launch_colfin(const Ctx &C, bool full, cudaStream_t s) {
    if (C.n <= 0) return;
    if (full) (k_colfin<<<std::min<unsigned>(blocks_for(C.n, kBlock), 8u * 152u), kBlock, 0, s>>>(C), note_launch());
    else (k_colfin_list<<<std::min<unsigned>(blocks_for(C.n, kBlock), 8u * 152u), kBlock, 0, s>>>(C), note_launch());
}

void launch_mark_dirty(const Ctx &C, int64_t nnz, cudaStream_t s) {
    if (C.n <= 0) return;
    (k_mark_list<<<std::min<unsigned>(blocks_for(std::max(C.n, C.m), kBlock), 8u * 152u), kBlock, 0, s>>>(C, nnz),
     note_launch());
    if (C.T.cls_start[7] > C.T.cls_start[6] && C.T.nchunks > 0) (k_mark_long<<<C.T.nchunks, kBlock, 0, s>>>(C, nnz), note_launch());
}

void launch_s5_pass(const Ctx &C, cudaStream_t s) {
    if (C.m == 0) return;
    (k_s5_insert<<<std::min<unsigned>(blocks_for(C.m, kBlock), 8u * 152u), kBlock, 0, s>>>(C), note_launch());
    const GroupGrid g = group_grid(C.A);
    if (g.blk_start[6] > 0) (k_s5_match_groups<<<g.blk_start[6], kBlock, 0, s>>>(C, g), note_launch());
    const int32_t nlong = C.A.cls_start[7] - C.A.cls_start[6];
    if (nlong > 0) (k_s5_match_long<<<nlong, kBlock, 0, s>>>(C), note_launch());
}

void launch_s5_tail(const Ctx &C, const int32_t *list, const int32_t *cnt, int32_t *out, int32_t *out_cnt,
                    int32_t max_rows, cudaStream_t s) {
    if (max_rows <= 0) return;
    (k_s5_tail_insert<<<blocks_for(max_rows, kBlock), kBlock, 0, s>>>(C, list, cnt), note_launch());
    (k_s5_tail_match<<<blocks_for(max_rows, kBlock), kBlock, 0, s>>>(C, list, cnt, out, out_cnt), note_launch());
    (k_s5_tail_clear<<<blocks_for(max_rows, kBlock), kBlock, 0, s>>>(C, list, cnt), note_launch());
}

void launch_s5_tail_block(const Ctx &C, int32_t *l0, int32_t *l1, int32_t *cnt, int32_t p0, int32_t max_iter,
                          cudaStream_t s) {
    (k_s5_tail_block<<<1, kTailBlock, 0, s>>>(C, l0, l1, cnt, p0, max_iter), note_launch());
}

// cooperative launch of k_s5_tail_grid, at most one block per SM and
// resident block slot, no more than the first list needs; false if the
// device cannot take a cooperative launch (the caller then launches passes)
bool launch_s5_tail_grid(const Ctx &C, int32_t *l0, int32_t *l1, int32_t *cnt, int32_t p0, int32_t max_iter,
                         int32_t rows, unsigned *bar, cudaStream_t s) {
    static int per_sm = -1, sms = 0;
    if (per_sm < 0) {
        int dev = 0, coop = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int nb = 0;
        if (coop) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_s5_tail_grid, kBlock, 0);
        per_sm = coop ? nb : 0;
    }
    if (per_sm <= 0 || sms <= 0) return false;
    const int64_t want = std::max<int64_t>(1, ((int64_t)rows + kBlock - 1) / kBlock);
    const unsigned grid = (unsigned)std::min<int64_t>(want, (int64_t)per_sm * sms);
    Ctx Cv = C;
    void *args[] = {&Cv, &l0, &l1, &cnt, &p0, &max_iter, &bar};
    if (cudaLaunchCooperativeKernel((const void *)k_s5_tail_grid, dim3(grid), dim3(kBlock), args, 0, s) != cudaSuccess)
        return false;
    note_launch();
    return true;
}

void launch_s5_leader(const Ctx &C, cudaStream_t s) {
    if (C.m > 0) (k_s5_leader<<<blocks_for(C.m, kBlock), kBlock, 0, s>>>(C), note_launch());
}

}  // namespace lpp
