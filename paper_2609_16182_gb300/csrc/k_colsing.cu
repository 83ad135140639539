// k_colsing.cu -- S5d, free column singletons (Sec. 3.2, column singletons;
// opt-in).
//
// A column j with one entry in the round-start matrix, unfixed and unmerged,
// in a kept row i with sides [L_i, U_i] reads the row as the equality
// a_ij x_j + sum_k a_ik x_k = b at one side: the side its cost pushes a_ij x_j
// to (L_i when c_j a_ij > 0, U_i when c_j a_ij < 0; L_i = U_i for an
// equality), for c_j = 0 L_i if finite, else U_i.  With b finite it is a
// candidate of row i, whose candidate is the smallest such column.  It is eliminated when it is free
// or implied free: the range the row gives x_j under the current bounds of
// the other columns,
//   [(b - max rest) / a_ij, (b - min rest) / a_ij]   (ends swapped if a_ij < 0),
// lies within [l_j - d(l_j), u_j + d(u_j)] on each finite side, with
// d(x) = feas_tol max(1, |x|).  Substitutions of one round change each cost
// at most once: a row whose column j has a nonzero cost applies only when it
// is the first such eligible row in each of its columns (atomicMin per
// column); a row whose column j costs 0 changes no cost (it writes none, so
// it never races with a bidding row) and always applies.
// Applying row i: t = c_j / a_ij, c_k <- c_k - t a_ik, column j takes the
// value b / a_ij for the objective constant (as a fixed column does), row i
// and column j leave the LP, and the row's other entries and b are stored
// for the postsolve.  Columns merged in S5c are part of
// their leader's column and are skipped.
//
// Rows of at most kShortRow entries run one per thread, summing in row
// order; longer rows are deferred as tasks, one thread block each (the
// paper's design for long rows), summing with a fixed-order block reduction
// and storing the entries in row order through a block scan; rows of more
// than 4096 entries are split into their 4096-entry chunks, one block each,
// whose partial results one warp per row combines in chunk order.
#include <algorithm>

#include "lpp_launch.h"

namespace lpp {

namespace {

constexpr int kShortRow = 64;
constexpr int kTaskThreads = 256;

__device__ __forceinline__ bool s5d_skip(const Ctx &C, int32_t k, int32_t j) {
    return k == j || C.ckind[k] == CK_PARALLEL;
}

// the side b of row i that column j (coefficient a) is substituted at
__device__ __forceinline__ double s5d_side(const Ctx &C, int32_t i, int32_t j, double a) {
    const double cj = C.c[j];
    if (cj != 0.0) return (cj > 0.0) == (a > 0.0) ? C.L[i] : C.U[i];
    return is_fin(C.L[i]) ? C.L[i] : C.U[i];
}

// one column per thread: the singleton columns bid for their row
__global__ void __launch_bounds__(kBlock) k_s5d_detect(Ctx C, int32_t *rcand) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= C.n) return;
    const int32_t b = C.T.ptr[j];
    if (C.T.ptr[j + 1] - b != 1 || C.ckind[j] != CK_KEPT) return;
    const int32_t i = C.T.idx[b];
    if (C.rkind[i] != RK_KEPT || !is_fin(s5d_side(C, i, j, C.T.val[b]))) return;
    atomicMin(&rcand[i], j);
}

// the eligibility test from the rest activities (nmn / nmx infinite terms)
__device__ __forceinline__ bool s5d_eligible(const Ctx &C, int32_t j, double a, double b, double mnr, double mxr,
                                             int32_t nmn, int32_t nmx) {
    double lo, hi;
    if (a > 0.0) {
        lo = nmx == 0 ? (b - mxr) / a : ninf_();
        hi = nmn == 0 ? (b - mnr) / a : pinf();
    } else {
        lo = nmn == 0 ? (b - mnr) / a : ninf_();
        hi = nmx == 0 ? (b - mxr) / a : pinf();
    }
    const double2 bj = C.lu[j];
    if (is_fin(bj.x)) {
        const double thr = bj.x - C.feas_tol * fmax(1.0, fabs(bj.x));
        if (!(is_fin(lo) && lo >= thr)) return false;
    }
    if (is_fin(bj.y)) {
        const double thr = bj.y + C.feas_tol * fmax(1.0, fabs(bj.y));
        if (!(is_fin(hi) && hi <= thr)) return false;
    }
    return true;
}

// a column's term in the rest activities
__device__ __forceinline__ void s5d_term(const Ctx &C, int32_t k, double a, double &mnr, double &mxr, int32_t &nmn,
                                         int32_t &nmx) {
    const double2 bk = C.lu[k];
    const double bmn = a > 0.0 ? bk.x : bk.y, bmx = a > 0.0 ? bk.y : bk.x;
    if (is_fin(bmn)) mnr = mnr + a * bmn;
    else nmn++;
    if (is_fin(bmx)) mxr = mxr + a * bmx;
    else nmx++;
}

// Short candidate rows, one per thread (row order: the same sums as a
// sequential walk); long ones go to the task list.
__global__ void __launch_bounds__(kBlock) k_s5d_check(Ctx C, const int32_t *rcand, uint8_t *relig, int32_t *cmin,
                                                     int32_t *tasks, int32_t *ntask) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C.m) return;
    const int32_t j = rcand[i];
    if (j == kNone) return;
    const int32_t beg = C.A.ptr[i], end = C.A.ptr[i + 1];
    if (end - beg >= kLongMin) return;  // chunked
    if (end - beg > kShortRow) {
        tasks[atomicAdd(ntask, 1)] = i;
        return;
    }
    double a = 0.0, mnr = 0.0, mxr = 0.0;
    int32_t nmn = 0, nmx = 0;
    for (int32_t q = beg; q < end; q++) {
        const int32_t k = C.A.idx[q];
        if (k == j) a = C.A.val[q];
        if (s5d_skip(C, k, j)) continue;
        s5d_term(C, k, C.A.val[q], mnr, mxr, nmn, nmx);
    }
    if (!s5d_eligible(C, j, a, s5d_side(C, i, j, a), mnr, mxr, nmn, nmx)) return;
    relig[i] = 1;
    if (C.c[j] == 0.0) return;  // changes no cost: no bid
    for (int32_t q = beg; q < end; q++) {
        const int32_t k = C.A.idx[q];
        if (!s5d_skip(C, k, j)) atomicMin(&cmin[k], i);
    }
}

// block-wide exclusive scan of one flag per thread (kTaskThreads threads)
__device__ __forceinline__ int32_t block_rank(bool f, int32_t *s_w, int32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned b = __ballot_sync(0xffffffffu, f);
    if (lane == 0) s_w[warp] = __popc(b);
    __syncthreads();
    int32_t pre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kTaskThreads / 32; w++) {
        const int32_t c = s_w[w];
        pre += w < warp ? c : 0;
        tot += c;
    }
    __syncthreads();
    total = tot;
    return pre + __popc(b & ((1u << lane) - 1u));
}

template <typename T>
__device__ __forceinline__ T block_sum_ordered(T v, T *s_w) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = T(0);
#pragma unroll
    for (int w = 0; w < kTaskThreads / 32; w++) t += s_w[w];  // every thread, the same order
    __syncthreads();
    return t;
}

// long candidate rows, one block per task
__global__ void __launch_bounds__(kTaskThreads) k_s5d_check_long(Ctx C, const int32_t *rcand, uint8_t *relig,
                                                                int32_t *cmin, const int32_t *tasks,
                                                                const int32_t *ntask) {
    __shared__ double s_d[kTaskThreads / 32];
    __shared__ int32_t s_i[kTaskThreads / 32];
    __shared__ double s_a;
    const int32_t nt = *ntask;
    for (int32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const int32_t i = tasks[t], j = rcand[i];
        const int32_t beg = C.A.ptr[i], end = C.A.ptr[i + 1];
        double mnr = 0.0, mxr = 0.0;
        int32_t nmn = 0, nmx = 0;
        for (int32_t q = beg + threadIdx.x; q < end; q += kTaskThreads) {
            const int32_t k = C.A.idx[q];
            if (k == j) s_a = C.A.val[q];
            if (s5d_skip(C, k, j)) continue;
            s5d_term(C, k, C.A.val[q], mnr, mxr, nmn, nmx);
        }
        mnr = block_sum_ordered(mnr, s_d);
        mxr = block_sum_ordered(mxr, s_d);
        nmn = block_sum_ordered(nmn, s_i);
        nmx = block_sum_ordered(nmx, s_i);
        const bool ok = s5d_eligible(C, j, s_a, s5d_side(C, i, j, s_a), mnr, mxr, nmn, nmx);  // block-uniform
        if (ok) {
            if (threadIdx.x == 0) relig[i] = 1;
            if (C.c[j] != 0.0) {  // changes a cost: bid
                for (int32_t q = beg + threadIdx.x; q < end; q += kTaskThreads) {
                    const int32_t k = C.A.idx[q];
                    if (!s5d_skip(C, k, j)) atomicMin(&cmin[k], i);
                }
            }
        }
        __syncthreads();
    }
}

// records of an applied row (its entries are stored by the caller)
__device__ __forceinline__ void s5d_record(const Ctx &C, int32_t i, int32_t j, double a, double b,
                                           unsigned long long pos, int32_t cnt) {
    const int32_t lp = lp_of_row(C, i);
    const int32_t oi = C.rmap[i], oj = C.cmap[j];
    C.rkind[i] = RK_SUBST;
    C.rec_rk[oi] = RK_SUBST;
    C.rec_rr[oi] = lp_round(C, lp);
    C.rec_ra[oi] = oj;
    C.rec_rv[oi] = a;
    C.rec_sb[oi] = (long long)pos;
    C.rec_sl[oi] = cnt;
    C.rec_srhs[oi] = b;
    C.ckind[j] = CK_SUBST;
    C.fixv[j] = b / a;
    C.rec_ck[oj] = CK_SUBST;
    C.rec_cr[oj] = lp_round(C, lp);
    C.rec_cv[oj] = b / a;
    mark_lp_changed(C, lp);
}

// short eligible rows: applied when first in each of their columns
__global__ void __launch_bounds__(kBlock) k_s5d_apply(Ctx C, const int32_t *rcand, const uint8_t *relig,
                                                     const int32_t *cmin) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t applied = 0;
    if (i < C.m && relig[i]) {
        const int32_t j = rcand[i];
        const int32_t beg = C.A.ptr[i], end = C.A.ptr[i + 1];
        if (end - beg <= kShortRow) {
            const bool bids = C.c[j] != 0.0;
            bool sel = true;
            int32_t cnt = 0;
            double a = 0.0;
            for (int32_t q = beg; q < end; q++) {
                const int32_t k = C.A.idx[q];
                if (k == j) a = C.A.val[q];
                if (s5d_skip(C, k, j)) continue;
                sel = sel && (!bids || cmin[k] == i);
                cnt++;
            }
            if (sel) {
                const double b = s5d_side(C, i, j, a), t = C.c[j] / a;
                unsigned long long pos = atomicAdd(C.sub_used, (unsigned long long)cnt);
                s5d_record(C, i, j, a, b, pos, cnt);
                for (int32_t q = beg; q < end; q++) {
                    const int32_t k = C.A.idx[q];
                    if (s5d_skip(C, k, j)) continue;
                    const double ak = C.A.val[q];
                    if (bids) C.c[k] = C.c[k] - t * ak;  // a row that did not bid writes no cost
                    C.rec_scol[pos] = C.cmap[k];
                    C.rec_sval[pos] = ak;
                    pos++;
                }
                applied = 1;
            }
        }
    }
    block_add(applied, &C.st->rows_removed);
    block_add(applied, &C.st->cols_fixed);
}

// long eligible rows, one block per task: the selection test, then the cost
// updates and the entries in row order
__global__ void __launch_bounds__(kTaskThreads) k_s5d_apply_long(Ctx C, const int32_t *rcand, const uint8_t *relig,
                                                                const int32_t *cmin, const int32_t *tasks,
                                                                const int32_t *ntask) {
    __shared__ int32_t s_w[kTaskThreads / 32];
    __shared__ double s_a;
    __shared__ unsigned long long s_pos;
    const int32_t nt = *ntask;
    int32_t applied = 0;
    for (int32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const int32_t i = tasks[t];
        if (!relig[i]) continue;  // the same in every thread
        const int32_t j = rcand[i];
        const int32_t beg = C.A.ptr[i], end = C.A.ptr[i + 1];
        const bool bids = C.c[j] != 0.0;
        bool sel = true;
        int32_t cnt = 0;
        for (int32_t q = beg + threadIdx.x; q < end; q += kTaskThreads) {
            const int32_t k = C.A.idx[q];
            if (k == j) s_a = C.A.val[q];
            if (s5d_skip(C, k, j)) continue;
            sel = sel && (!bids || cmin[k] == i);
            cnt++;
        }
        sel = __syncthreads_and(sel) != 0;
        cnt = block_sum_ordered(cnt, s_w);
        if (!sel) continue;
        const double a = s_a, b = s5d_side(C, i, j, a), tj = C.c[j] / a;
        if (threadIdx.x == 0) {
            s_pos = atomicAdd(C.sub_used, (unsigned long long)cnt);
            s5d_record(C, i, j, a, b, s_pos, cnt);
        }
        __syncthreads();
        unsigned long long base = s_pos;
        for (int32_t q0 = beg; q0 < end; q0 += kTaskThreads) {
            const int32_t q = q0 + threadIdx.x;
            const int32_t k = q < end ? C.A.idx[q] : j;
            const bool keep = q < end && !s5d_skip(C, k, j);
            int32_t tot;
            const int32_t r = block_rank(keep, s_w, tot);
            if (keep) {
                const double ak = C.A.val[q];
                if (bids) C.c[k] = C.c[k] - tj * ak;  // a row that did not bid writes no cost
                C.rec_scol[base + r] = C.cmap[k];
                C.rec_sval[base + r] = ak;
            }
            base += tot;
        }
        applied++;
    }
    if (threadIdx.x == 0 && applied) {
        atomicAdd(&C.st->rows_removed, applied);
        atomicAdd(&C.st->cols_fixed, applied);
    }
}

// ---------------------------------------------- rows of more than 4096 entries
// per chunk of a candidate row: partial rest sums (ch_act, ch_ninf) and the
// coefficient of the candidate column (cs_a)
__global__ void __launch_bounds__(kTaskThreads) k_s5d_chunk_sums(Ctx C, const int32_t *rcand, double *cs_a) {
    __shared__ double s_d[kTaskThreads / 32];
    __shared__ int32_t s_i[kTaskThreads / 32];
    const Chunk ch = C.A.chunks[blockIdx.x];
    const int32_t i = ch.seg, j = rcand[i];
    if (j == kNone) return;  // block-uniform
    double mnr = 0.0, mxr = 0.0;
    int32_t nmn = 0, nmx = 0;
    for (int32_t q = ch.begin + threadIdx.x; q < ch.end; q += kTaskThreads) {
        const int32_t k = C.A.idx[q];
        if (k == j) cs_a[i] = C.A.val[q];
        if (s5d_skip(C, k, j)) continue;
        s5d_term(C, k, C.A.val[q], mnr, mxr, nmn, nmx);
    }
    mnr = block_sum_ordered(mnr, s_d);
    mxr = block_sum_ordered(mxr, s_d);
    nmn = block_sum_ordered(nmn, s_i);
    nmx = block_sum_ordered(nmx, s_i);
    if (threadIdx.x == 0) {
        C.ch_act[blockIdx.x] = make_double2(mnr, mxr);
        C.ch_ninf[blockIdx.x] = make_int2(nmn, nmx);
    }
}

// one warp per long row: the chunk sums in chunk order, then the test
__global__ void __launch_bounds__(kBlock) k_s5d_chunk_elig(Ctx C, const int32_t *rcand, const double *cs_a,
                                                          uint8_t *relig) {
    const int32_t t = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int32_t nlong = C.A.cls_start[7] - C.A.cls_start[6];
    if (t >= nlong) return;  // the same t in the whole warp
    const int32_t i = C.A.order[C.A.cls_start[6] + t], j = rcand[i];
    if (j == kNone) return;
    double mnr = 0.0, mxr = 0.0;
    int32_t nmn = 0, nmx = 0;
    for (int32_t q = C.A.lfirst[t] + lane; q < C.A.lfirst[t + 1]; q += 32) {
        const double2 a = C.ch_act[q];
        const int2 c = C.ch_ninf[q];
        mnr += a.x;
        mxr += a.y;
        nmn += c.x;
        nmx += c.y;
    }
    mnr = group_sum<32>(mnr, 0xffffffffu);
    mxr = group_sum<32>(mxr, 0xffffffffu);
    nmn = group_sum<32>(nmn, 0xffffffffu);
    nmx = group_sum<32>(nmx, 0xffffffffu);
    if (lane == 0 && s5d_eligible(C, j, cs_a[i], s5d_side(C, i, j, cs_a[i]), mnr, mxr, nmn, nmx)) relig[i] = 1;
}

// per chunk of an eligible row whose column costs something: the bids
__global__ void __launch_bounds__(kTaskThreads) k_s5d_chunk_bid(Ctx C, const int32_t *rcand, const uint8_t *relig,
                                                               int32_t *cmin) {
    const Chunk ch = C.A.chunks[blockIdx.x];
    const int32_t i = ch.seg;
    if (!relig[i]) return;
    const int32_t j = rcand[i];
    if (C.c[j] == 0.0) return;
    for (int32_t q = ch.begin + threadIdx.x; q < ch.end; q += kTaskThreads) {
        const int32_t k = C.A.idx[q];
        if (!s5d_skip(C, k, j)) atomicMin(&cmin[k], i);
    }
}

// per chunk of an eligible row: does it win every column (ch_ninf.x) and how
// many entries does it store (ch_ninf.y)
__global__ void __launch_bounds__(kTaskThreads) k_s5d_chunk_sel(Ctx C, const int32_t *rcand, const uint8_t *relig,
                                                               const int32_t *cmin) {
    __shared__ int32_t s_w[kTaskThreads / 32];
    const Chunk ch = C.A.chunks[blockIdx.x];
    const int32_t i = ch.seg;
    if (!relig[i]) return;
    const int32_t j = rcand[i];
    const bool bids = C.c[j] != 0.0;
    bool sel = true;
    int32_t cnt = 0;
    for (int32_t q = ch.begin + threadIdx.x; q < ch.end; q += kTaskThreads) {
        const int32_t k = C.A.idx[q];
        if (s5d_skip(C, k, j)) continue;
        sel = sel && (!bids || cmin[k] == i);
        cnt++;
    }
    sel = __syncthreads_and(sel) != 0;
    cnt = block_sum_ordered(cnt, s_w);
    if (threadIdx.x == 0) C.ch_ninf[blockIdx.x] = make_int2(sel ? 1 : 0, cnt);
}

// one warp per long eligible row: selected when every chunk won; then the
// store range (chunk bases in chunk order, in ch_hash) and the records
__global__ void __launch_bounds__(kBlock) k_s5d_chunk_row(Ctx C, const int32_t *rcand, const double *cs_a,
                                                         uint8_t *relig) {
    const int32_t t = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int32_t nlong = C.A.cls_start[7] - C.A.cls_start[6];
    int32_t applied = 0;
    if (t < nlong) {  // the same t in the whole warp
        const int32_t i = C.A.order[C.A.cls_start[6] + t];
        if (relig[i]) {
            const int32_t q0 = C.A.lfirst[t], q1 = C.A.lfirst[t + 1];
            bool sel = true;
            int32_t carry = 0;
            for (int32_t b0 = q0; b0 < q1; b0 += 32) {
                const int32_t q = b0 + lane;
                const int2 v = q < q1 ? C.ch_ninf[q] : make_int2(1, 0);
                sel = sel && v.x != 0;
                int32_t inc = v.y;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += y;
                }
                if (q < q1) C.ch_hash[q] = (unsigned long long)(carry + inc - v.y);  // offset within the row
                carry += __shfl_sync(0xffffffffu, inc, 31);
            }
            sel = __all_sync(0xffffffffu, sel) != 0;
            if (sel) {
                unsigned long long pos = 0;
                if (lane == 0) {
                    pos = atomicAdd(C.sub_used, (unsigned long long)carry);
                    const int32_t j = rcand[i];
                    s5d_record(C, i, j, cs_a[i], s5d_side(C, i, j, cs_a[i]), pos, carry);
                    relig[i] = 2;  // applied: the chunks write their entries
                }
                pos = __shfl_sync(0xffffffffu, pos, 0);
                for (int32_t q = q0 + lane; q < q1; q += 32) C.ch_hash[q] += pos;
                applied = lane == 0;
            }
        }
    }
    block_add(applied, &C.st->rows_removed);
    block_add(applied, &C.st->cols_fixed);
}

// per chunk of an applied row: cost updates and its entries at its base
__global__ void __launch_bounds__(kTaskThreads) k_s5d_chunk_apply(Ctx C, const int32_t *rcand, const double *cs_a,
                                                                 const uint8_t *relig) {
    __shared__ int32_t s_w[kTaskThreads / 32];
    const Chunk ch = C.A.chunks[blockIdx.x];
    const int32_t i = ch.seg;
    if (relig[i] != 2) return;
    const int32_t j = rcand[i];
    const bool bids = C.c[j] != 0.0;
    const double tj = C.c[j] / cs_a[i];
    unsigned long long base = C.ch_hash[blockIdx.x];
    for (int32_t q0 = ch.begin; q0 < ch.end; q0 += kTaskThreads) {
        const int32_t q = q0 + threadIdx.x;
        const int32_t k = q < ch.end ? C.A.idx[q] : j;
        const bool keep = q < ch.end && !s5d_skip(C, k, j);
        int32_t tot;
        const int32_t r = block_rank(keep, s_w, tot);
        if (keep) {
            const double ak = C.A.val[q];
            if (bids) C.c[k] = C.c[k] - tj * ak;  // a row that did not bid writes no cost
            C.rec_scol[base + r] = C.cmap[k];
            C.rec_sval[base + r] = ak;
        }
        base += tot;
    }
}

inline unsigned blocks_for(int64_t cnt, int threads) {
    return (unsigned)((cnt + threads - 1) / threads > 0 ? (cnt + threads - 1) / threads : 1);
}

}  // namespace

void launch_s5d(const Ctx &C, int32_t *rcand, uint8_t *relig, int32_t *cmin, int32_t *tasks, int32_t *ntask,
                double *cs_a, cudaStream_t s) {
    if (C.n <= 0 || C.m <= 0) return;
    const int32_t task_grid = std::min<int32_t>(C.m, 2 * 152);
    const int32_t nlong = C.A.cls_start[7] - C.A.cls_start[6];
    const bool chunked = nlong > 0 && C.A.nchunks > 0;
    const unsigned long_warps = blocks_for((int64_t)nlong * 32, kBlock);
    (k_s5d_detect<<<blocks_for(C.n, kBlock), kBlock, 0, s>>>(C, rcand), note_launch());
    (k_s5d_check<<<blocks_for(C.m, kBlock), kBlock, 0, s>>>(C, rcand, relig, cmin, tasks, ntask), note_launch());
    (k_s5d_check_long<<<task_grid, kTaskThreads, 0, s>>>(C, rcand, relig, cmin, tasks, ntask), note_launch());
    if (chunked) {
        (k_s5d_chunk_sums<<<C.A.nchunks, kTaskThreads, 0, s>>>(C, rcand, cs_a), note_launch());
        (k_s5d_chunk_elig<<<long_warps, kBlock, 0, s>>>(C, rcand, cs_a, relig), note_launch());
        (k_s5d_chunk_bid<<<C.A.nchunks, kTaskThreads, 0, s>>>(C, rcand, relig, cmin), note_launch());
    }
    (k_s5d_apply<<<blocks_for(C.m, kBlock), kBlock, 0, s>>>(C, rcand, relig, cmin), note_launch());
    (k_s5d_apply_long<<<task_grid, kTaskThreads, 0, s>>>(C, rcand, relig, cmin, tasks, ntask), note_launch());
    if (chunked) {
        (k_s5d_chunk_sel<<<C.A.nchunks, kTaskThreads, 0, s>>>(C, rcand, relig, cmin), note_launch());
        (k_s5d_chunk_row<<<long_warps, kBlock, 0, s>>>(C, rcand, cs_a, relig), note_launch());
        (k_s5d_chunk_apply<<<C.A.nchunks, kTaskThreads, 0, s>>>(C, rcand, cs_a, relig), note_launch());
    }
}

}  // namespace lpp
