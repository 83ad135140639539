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
// the whole warp, in turn, for longer ones.  When a round applies any
// doubleton, the CSR is rewritten into the other buffer (each changed row's
// new length by binary searches, a scan, one thread per entry placing it),
// the CSC is rebuilt from it by the ingest transpose, and S6 and the
// compaction then work on the rewritten matrices.
#include <algorithm>

#include "lpp_launch.h"
#include "s5e_rewrite.cuh"

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

// the other column of doubleton row i (entries at p, p + 1) than kk
__device__ __forceinline__ int32_t other_col(const Ctx &C, int32_t p, int32_t kk) {
    return C.A.idx[p] == kk ? C.A.idx[p + 1] : C.A.idx[p];
}

// one thread per row: candidates, their column claims, and (by the walk of
// x_k's column) their row claims; resets the row's note of a change
__global__ void __launch_bounds__(kBlock) k_s5e_detect(Ctx C, S5eBufs D) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    bool own = false;
    int32_t b = 0, e = 0;
    if (i < C.m) {
        int32_t kk = -1;
        const int32_t p = C.A.ptr[i];
        D.dmj[i] = -1;
        if (C.rkind[i] == RK_KEPT && C.A.ptr[i + 1] - p == 2) {
            const double Lv = C.L[i];
            const int32_t c0 = C.A.idx[p], c1 = C.A.idx[p + 1];
            if (is_fin(Lv) && Lv == C.U[i] && C.ckind[c0] == CK_KEPT && C.ckind[c1] == CK_KEPT) {
                const int32_t l0 = C.T.ptr[c0 + 1] - C.T.ptr[c0], l1 = C.T.ptr[c1 + 1] - C.T.ptr[c1];
                kk = l1 <= l0 ? c1 : c0;
                atomicMin(&D.cmin[c0], i);
                atomicMin(&D.cmin[c1], i);
                own = true;
                b = C.T.ptr[kk];
                e = C.T.ptr[kk + 1];
            }
        }
        D.dk[i] = kk;
    }
    warp_walk(own, b, e, i, [&](int32_t src, int32_t k) {
        const int32_t rr = C.T.idx[k];
        if (rr == src || C.rkind[rr] == RK_KEPT) atomicMin(&D.rmin[rr], src);
    });
}

// one thread per row: a candidate that holds both column claims, its own
// row's and those of every kept row of x_k is selected (dsel)
__global__ void __launch_bounds__(kBlock) k_s5e_select(Ctx C, S5eBufs D) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    bool own = false;
    int32_t b = 0, e = 0;
    if (i < C.m) {
        const int32_t kk = D.dk[i];
        if (kk >= 0) {
            const int32_t jj = other_col(C, C.A.ptr[i], kk);
            own = D.cmin[jj] == i && D.cmin[kk] == i && D.rmin[i] == i;
            b = C.T.ptr[kk];
            e = C.T.ptr[kk + 1];
        }
    }
    const bool lost = warp_any(own, b, e, i, [&](int32_t src, int32_t k) {
        const int32_t rr = C.T.idx[k];
        return rr != src && C.rkind[rr] == RK_KEPT && D.rmin[rr] != src;
    });
    if (i < C.m) D.dsel[i] = (uint8_t)(own && !lost);
}

// one thread per selected row: the bound transfer (or the verdict), the
// cost, the records; then the walk of x_k's column shifts the sides of its
// other kept rows and notes their change (x_j, -(a_rk f)).  A row of x_k
// other than i is claimed by i alone, so no other thread writes it or its
// kind, and no selected row is one of them.
__global__ void __launch_bounds__(kBlock) k_s5e_apply(Ctx C, S5eBufs D) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    bool sel = i < C.m && D.dsel[i];
    int32_t b = 0, e = 0, applied = 0, changed = 0, jj = -1;
    if (sel) {
        const int32_t kk = D.dk[i], p = C.A.ptr[i];
        const bool j_first = C.A.idx[p] != kk;
        jj = j_first ? C.A.idx[p] : C.A.idx[p + 1];
        const double a = j_first ? C.A.val[p] : C.A.val[p + 1];
        const double bk = j_first ? C.A.val[p + 1] : C.A.val[p];
        const double cv = C.L[i];
        const double f = a / bk, g = cv / bk;
        const double2 luj = C.lu[jj], luk = C.lu[kk];
        double lo, hi;
        if (f > 0.0) {
            lo = is_fin(luk.y) ? (g - luk.y) / f : ninf_();
            hi = is_fin(luk.x) ? (g - luk.x) / f : pinf();
        } else {
            lo = is_fin(luk.x) ? (g - luk.x) / f : ninf_();
            hi = is_fin(luk.y) ? (g - luk.y) / f : pinf();
        }
        double nl = lo > luj.x ? lo : luj.x;
        double nu = hi < luj.y ? hi : luj.y;
        const int32_t lp = lp_of_row(C, i);
        if (is_fin(nl) && is_fin(nu)) {
            const double d = C.feas_tol * fmax(1.0, fmax(fabs(nl), fabs(nu)));
            if (nl - nu > d) {
                atomicMin(&C.verdict[lp * V_SLOTS + V_S5E_COL], C.cmap[jj]);
                sel = false;
            } else if (nl != nu && fabs(nl - nu) <= d) {  // as S3' finalises: a symmetric snap
                nl = nu = 0.5 * (nl + nu);
            }
        }
        if (sel) {
            changed = nl != luj.x || nu != luj.y;
            C.lu[jj] = make_double2(nl, nu);
            const double t = C.c[kk] / bk;
            C.c[jj] = C.c[jj] - t * a;
            C.rkind[i] = RK_DOUBLETON;
            C.ckind[kk] = CK_DOUBLETON;
            C.fixv[kk] = g;
            const int32_t oi = C.rmap[i], ok = C.cmap[kk], oj = C.cmap[jj], rd = lp_round(C, lp);
            C.rec_rk[oi] = RK_DOUBLETON;
            C.rec_rr[oi] = rd;
            C.rec_ra[oi] = ok;
            C.rec_rv[oi] = bk;
            const unsigned long long pos = atomicAdd(C.sub_used, 1ULL);
            C.rec_sb[oi] = (long long)pos;
            C.rec_sl[oi] = 1;
            C.rec_srhs[oi] = cv;
            C.rec_scol[pos] = oj;
            C.rec_sval[pos] = a;
            C.rec_ck[ok] = CK_DOUBLETON;
            C.rec_cr[ok] = rd;
            C.rec_cv[ok] = g;
            C.lp_changed[lp] = 1;
            if (C.plen) C.plen[oj] = -1;  // x_j's entries change: its S5c key is recomputed
            D.dj[i] = jj;
            D.df[i] = f;
            D.dg[i] = g;
            b = C.T.ptr[kk];
            e = C.T.ptr[kk + 1];
            applied = 1;
        }
    }
    __syncwarp();  // the owners' dj, df, dg before the warp reads them
    warp_walk(sel, b, e, i, [&](int32_t src, int32_t k) {
        const int32_t rr = C.T.idx[k];
        if (rr == src || C.rkind[rr] != RK_KEPT) return;
        const double ark = C.T.val[k];
        const double f = D.df[src], g = D.dg[src];
        const double Lv = C.L[rr], Uv = C.U[rr];
        if (is_fin(Lv)) C.L[rr] = Lv - ark * g;
        if (is_fin(Uv)) C.U[rr] = Uv - ark * g;
        D.dmj[rr] = D.dj[src];
        D.dmk[rr] = D.dk[src];
        D.dmd[rr] = -(ark * f);
        C.rdnext[rr] = 1;
    });
    block_append(applied != 0, jj, &D.cnt[1], D.jlist);
    block_add(applied, &C.st->rows_removed);
    block_add(applied, &C.st->cols_fixed);
    block_add(changed, &C.st->bounds_changed);
    block_add(applied, &D.cnt[0]);
}

// one thread per row: the rewritten length (x_k out; x_j's entry merged,
// dropped when it cancels, or inserted) and, for a changed row, the
// positions of x_k and of x_j (or where x_j goes), the flags and the value
__global__ void __launch_bounds__(kBlock) k_s5e_rowlen(Ctx C, S5eBufs D, int32_t *rlen) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C.m) return;
    const int32_t p = C.A.ptr[i], len = C.A.ptr[i + 1] - p, jj = D.dmj[i];
    int32_t nl = len;
    if (jj >= 0) {
        const S5eNote t = s5e_note(C.A.idx + p, C.A.val + p, len, jj, D.dmk[i], D.dmd[i], C.par_tol);
        nl = t.len_new;
        D.dpk[i] = t.pk;
        D.dpj[i] = t.pj;
        D.dfl[i] = (uint8_t)((t.found ? 1 : 0) | (t.cancel ? 2 : 0));
        D.dnv[i] = t.v;
    }
    rlen[i] = nl;
}

// one thread per entry of the current CSR: its place in the rewritten CSR
// (rp2 the scanned new lengths).  In a changed row, with pk the position of
// x_k and pj that of x_j (or where it goes), an entry at position q moves to
//   rp2[i] + q - [q > pk] + [x_j inserted and q >= pj]
//                         - [x_j cancelled and q > pj];
// the thread of x_k's entry writes an inserted x_j at rp2[i] + pj - [pk < pj].
__global__ void __launch_bounds__(kBlock) k_s5e_scatter(Ctx C, S5eBufs D, const int32_t *rp2, int32_t *ci2,
                                                       double *rv2, int32_t *row_of, int32_t nnz) {
    const int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    // the row of e: the last i with ptr[i] <= e
    int32_t lo = 0, hi = C.m;
    while (hi - lo > 1) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (C.A.ptr[mid] <= e) lo = mid;
        else hi = mid;
    }
    const int32_t i = lo, q = e - C.A.ptr[i], base = rp2[i];
    int32_t col = C.A.idx[e];
    double v = C.A.val[e];
    int32_t dest = base + q;
    const int32_t jj = D.dmj[i];
    if (jj >= 0) {
        S5eNote t;
        t.pk = D.dpk[i];
        t.pj = D.dpj[i];
        t.found = D.dfl[i] & 1;
        t.cancel = D.dfl[i] & 2;
        if (q == t.pk) {
            if (!t.found) {
                const int32_t at = base + s5e_insert_at(t);
                ci2[at] = jj;
                rv2[at] = D.dnv[i];
                row_of[at] = i;
            }
            return;
        }
        if (t.found && q == t.pj) {
            if (t.cancel) return;
            v = D.dnv[i];
        }
        dest = base + s5e_dest(t, q);
    }
    ci2[dest] = col;
    rv2[dest] = v;
    row_of[dest] = i;
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
