// k_doubleton.cu -- S5e, doubleton equations (Sec. 2.1, the doubleton-row
// explorer; opt-in).
//
// A kept equality row i with two entries, a x_j + b x_k = c, whose columns
// are both unfixed and unmerged, eliminates x_k, the column with fewer
// entries in the round-start matrix (the larger index on a tie):
// x_k = g - f x_j with f = a / b, g = c / b.  Then
//   x_j's bounds meet the range x_k's bounds give it,
//     [(g - u_k) / f, (g - l_k) / f]   (ends swapped for f < 0),
//     finalised as S3' finalises bounds: crossing by more than
//     d = feas_tol max(1, |l|, |u|) is infeasible (the smallest original
//     column index of the round is reported), bounds within d of each
//     other snap to their midpoint;
//   c_j <- c_j - (c_k / b) a, and x_k takes the value g for the objective
//     constant (as a fixed column does);
//   every other kept row r of x_k (coefficient a_rk) loses that entry and
//     its sides a_rk g, and x_j's coefficient in r gains -(a_rk f): added to
//     an existing entry (dropped when the sum is within par_tol of
//     cancelling), else inserted at its column position;
//   row i and column k leave the LP with a substitution record (the entry
//     a of x_j and the right-hand side c), from which the postsolve sets
//     x_k = (c - a x_j) / b.
// Doubletons of one round touch disjoint columns and rows: each candidate
// claims its two columns and every kept row of x_k (itself included) with
// atomicMin, and applies only when it holds all its claims.
//
// GPU layout: one thread per row finds the candidates and claims; the
// walks over x_k's column (claims, the check of the claims, the side
// shifts) run on the owning thread for columns of at most 32 entries and on
// the whole warp, in turn, for longer ones.  The work per row and per entry
// is in s5e_logic.cuh, shared with a host build of the same steps.  When a
// round applies any doubleton, the CSR is rewritten into the other buffer
// (each changed row's new length by binary searches, a scan, one thread per
// entry placing it), the CSC is rebuilt from it by the ingest transpose, and
// S6 and the compaction then work on the rewritten matrices.
#include <algorithm>

#include "s5e_logic.cuh"

namespace lpp {

namespace {

inline unsigned blocks_for(int64_t cnt, int threads) {
    return (unsigned)((cnt + threads - 1) / threads > 0 ? (cnt + threads - 1) / threads : 1);
}

// Calls f(tag, k) for every k in [b, e) of every thread with `own`: by the
// thread itself for at most 32 entries, else by the whole warp in turn.
// Every lane of the warp must call it.
template <class F>
__device__ __forceinline__ void warp_walk(bool own, int32_t b, int32_t e, int32_t tag, F &&f) {
    const int lane = threadIdx.x & 31;
    if (own && e - b <= 32)
        for (int32_t k = b; k < e; k++) f(tag, k);
    unsigned todo = __ballot_sync(0xffffffffu, own && e - b > 32);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1u;
        const int32_t sb = __shfl_sync(0xffffffffu, b, src), se = __shfl_sync(0xffffffffu, e, src);
        const int32_t st = __shfl_sync(0xffffffffu, tag, src);
        for (int32_t k = sb + lane; k < se; k += 32) f(st, k);
    }
}

// Whether pred(tag, k) holds for some k in [b, e), for every thread with
// `own` (false for the others); walked as warp_walk does.
template <class P>
__device__ __forceinline__ bool warp_any(bool own, int32_t b, int32_t e, int32_t tag, P &&pred) {
    const int lane = threadIdx.x & 31;
    bool hit = false;
    if (own && e - b <= 32)
        for (int32_t k = b; k < e && !hit; k++) hit = pred(tag, k);
    unsigned todo = __ballot_sync(0xffffffffu, own && e - b > 32);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1u;
        const int32_t sb = __shfl_sync(0xffffffffu, b, src), se = __shfl_sync(0xffffffffu, e, src);
        const int32_t st = __shfl_sync(0xffffffffu, tag, src);
        bool h = false;
        for (int32_t k = sb + lane; k < se; k += 32) h |= pred(st, k);
        const bool any = __any_sync(0xffffffffu, h);
        if (lane == src) hit = any;
    }
    return hit;
}

// one thread per row: candidates, their column claims, and (by the walk of
// x_k's column) their row claims
__global__ void __launch_bounds__(kBlock) k_s5e_detect(Ctx C, S5eBufs D) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const S5eWalk w = i < C.m ? s5e_detect_row(C, D, i) : S5eWalk{false, 0, 0};
    warp_walk(w.own, w.b, w.e, i, [&](int32_t src, int32_t k) { s5e_claim_entry(C, D, src, k); });
}

// one thread per row: a candidate that holds both column claims, its own
// row's and those of every kept row of x_k is selected (dsel)
__global__ void __launch_bounds__(kBlock) k_s5e_select(Ctx C, S5eBufs D) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const S5eWalk w = i < C.m ? s5e_select_row(C, D, i) : S5eWalk{false, 0, 0};
    const bool lost =
        warp_any(w.own, w.b, w.e, i, [&](int32_t src, int32_t k) { return s5e_lost_entry(C, D, src, k); });
    if (i < C.m) D.dsel[i] = (uint8_t)(w.own && !lost);
}

// one thread per selected row: the bound transfer (or the verdict), the
// cost, the records; then the walk of x_k's column shifts the sides of its
// other kept rows and notes their change.  A row of x_k other than i is
// claimed by i alone, so no other thread writes it or its kind, and no
// selected row is one of them.
__global__ void __launch_bounds__(kBlock) k_s5e_apply(Ctx C, S5eBufs D) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    S5eApplied r{S5eWalk{false, 0, 0}, 0, -1};
    if (i < C.m && D.dsel[i]) r = s5e_apply_row(C, D, i);
    __syncwarp();  // the owners' dj, df, dg before the warp reads them
    warp_walk(r.w.own, r.w.b, r.w.e, i, [&](int32_t src, int32_t k) { s5e_shift_entry(C, D, src, k); });
    const int32_t applied = r.w.own ? 1 : 0;
    block_append(applied != 0, r.jj, &D.cnt[1], D.jlist);
    block_add(applied, &C.st->rows_removed);
    block_add(applied, &C.st->cols_fixed);
    block_add(r.changed, &C.st->bounds_changed);
    block_add(applied, &D.cnt[0]);
}

// one thread per row: the rewritten length and a changed row's note
__global__ void __launch_bounds__(kBlock) k_s5e_rowlen(Ctx C, S5eBufs D, int32_t *rlen) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < C.m) rlen[i] = s5e_rowlen_row(C, D, i);
}

// one thread per entry of the current CSR: its place in the rewritten CSR
__global__ void __launch_bounds__(kBlock) k_s5e_scatter(Ctx C, S5eBufs D, const int32_t *rp2, int32_t *ci2,
                                                       double *rv2, int32_t *row_of, int32_t nnz) {
    const int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nnz && !s5e_place_entry(C, D, rp2, ci2, rv2, row_of, e)) atomicOr(&C.st->err, 2);
}

// one thread per applied doubleton: the rows of x_j in the rewritten CSC
// (its own and those it gained) are evaluated next round (its bounds changed)
__global__ void __launch_bounds__(kBlock) k_s5e_mark(Ctx C, S5eBufs D, int32_t cnt) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    bool own = t < cnt;
    int32_t b = 0, e = 0;
    if (own) {
        const int32_t jj = D.jlist[t];
        b = C.T.ptr[jj];
        e = C.T.ptr[jj + 1];
    }
    warp_walk(own, b, e, 0, [&](int32_t, int32_t k) { C.rdnext[C.T.idx[k]] = 1; });
}

}  // namespace

void launch_s5e(const Ctx &C, const S5eBufs &D, cudaStream_t s) {
    if (C.m <= 0 || C.n <= 0) return;
    const unsigned g = blocks_for(C.m, kBlock);
    (k_s5e_detect<<<g, kBlock, 0, s>>>(C, D), note_launch());
    (k_s5e_select<<<g, kBlock, 0, s>>>(C, D), note_launch());
    (k_s5e_apply<<<g, kBlock, 0, s>>>(C, D), note_launch());
}

void launch_s5e_rowlen(const Ctx &C, const S5eBufs &D, int32_t *rlen, cudaStream_t s) {
    if (C.m > 0) (k_s5e_rowlen<<<blocks_for(C.m, kBlock), kBlock, 0, s>>>(C, D, rlen), note_launch());
}

void launch_s5e_scatter(const Ctx &C, const S5eBufs &D, const int32_t *rp2, int32_t *ci2, double *rv2,
                        int32_t *row_of, int64_t nnz, cudaStream_t s) {
    if (nnz > 0 && C.m > 0)
        (k_s5e_scatter<<<blocks_for(nnz, kBlock), kBlock, 0, s>>>(C, D, rp2, ci2, rv2, row_of, (int32_t)nnz),
         note_launch());
}

void launch_s5e_mark(const Ctx &C, const S5eBufs &D, int32_t cnt, cudaStream_t s) {
    if (cnt > 0) (k_s5e_mark<<<blocks_for(cnt, kBlock), kBlock, 0, s>>>(C, D, cnt), note_launch());
}

}  // namespace lpp
