// s5e_logic.cuh -- the per-row and per-entry work of S5e (doubleton
// equations, Sec. 2.1), host- and device-callable.
//
// The device kernels (k_doubleton.cu) call these from one thread per row,
// with the walks over x_k's column spread over a warp; a host build runs the
// same functions one row after another.  Both orders give the same result:
// the claims are minima, the check of the claims only reads, and the rows
// that apply write disjoint rows and columns (each holds all its claims).
#pragma once
#include <cmath>
#include <cstdint>
#include <limits>

#include "lpp_launch.h"
#include "s5e_rewrite.cuh"

namespace lpp {

__host__ __device__ inline void s5e_amin(int32_t *p, int32_t v) {
#ifdef __CUDA_ARCH__
    atomicMin(p, v);
#else
    if (v < *p) *p = v;
#endif
}

__host__ __device__ inline unsigned long long s5e_fetch_add(unsigned long long *p, unsigned long long v) {
#ifdef __CUDA_ARCH__
    return atomicAdd(p, v);
#else
    const unsigned long long o = *p;
    *p = o + v;
    return o;
#endif
}

__host__ __device__ inline bool s5e_fin(double x) {
#ifdef __CUDA_ARCH__
    return is_fin(x);
#else
    return std::isfinite(x);
#endif
}

__host__ __device__ inline double s5e_inf() {
#ifdef __CUDA_ARCH__
    return pinf();
#else
    return std::numeric_limits<double>::infinity();
#endif
}

__host__ __device__ inline int32_t s5e_lp_row(const Ctx &C, int32_t i) { return C.lp_row ? C.lp_row[i] : 0; }
__host__ __device__ inline int32_t s5e_lp_round(const Ctx &C, int32_t lp) {
    return C.lp_round0 ? C.round - C.lp_round0[lp] + 1 : C.round;
}

// a row's walk over x_k's column: [b, e) of the CSC when `own`
struct S5eWalk {
    bool own;
    int32_t b, e;
};

// Row i: candidate test (kept, two entries, L = U finite, both columns
// kept), the eliminated column (fewer entries, the second on a tie) in dk,
// the two column claims; resets the row's note of a change.
__host__ __device__ inline S5eWalk s5e_detect_row(const Ctx &C, const S5eBufs &D, int32_t i) {
    S5eWalk w{false, 0, 0};
    int32_t kk = -1;
    const int32_t p = C.A.ptr[i];
    D.dmj[i] = -1;
    if (C.rkind[i] == RK_KEPT && C.A.ptr[i + 1] - p == 2) {
        const double Lv = C.L[i];
        const int32_t c0 = C.A.idx[p], c1 = C.A.idx[p + 1];
        if (s5e_fin(Lv) && Lv == C.U[i] && C.ckind[c0] == CK_KEPT && C.ckind[c1] == CK_KEPT) {
            const int32_t l0 = C.T.ptr[c0 + 1] - C.T.ptr[c0], l1 = C.T.ptr[c1 + 1] - C.T.ptr[c1];
            kk = l1 <= l0 ? c1 : c0;
            s5e_amin(&D.cmin[c0], i);
            s5e_amin(&D.cmin[c1], i);
            w = S5eWalk{true, C.T.ptr[kk], C.T.ptr[kk + 1]};
        }
    }
    D.dk[i] = kk;
    return w;
}

// entry k of candidate src's x_k column: src claims its row if kept (or src itself)
__host__ __device__ inline void s5e_claim_entry(const Ctx &C, const S5eBufs &D, int32_t src, int32_t k) {
    const int32_t rr = C.T.idx[k];
    if (rr == src || C.rkind[rr] == RK_KEPT) s5e_amin(&D.rmin[rr], src);
}

// Row i: a candidate holding both column claims and its own row's; the walk
// then looks for a kept row of x_k claimed by another candidate
__host__ __device__ inline S5eWalk s5e_select_row(const Ctx &C, const S5eBufs &D, int32_t i) {
    const int32_t kk = D.dk[i];
    if (kk < 0) return S5eWalk{false, 0, 0};
    const int32_t p = C.A.ptr[i];
    const int32_t jj = C.A.idx[p] == kk ? C.A.idx[p + 1] : C.A.idx[p];
    const bool own = D.cmin[jj] == i && D.cmin[kk] == i && D.rmin[i] == i;
    return S5eWalk{own, C.T.ptr[kk], C.T.ptr[kk + 1]};
}

__host__ __device__ inline bool s5e_lost_entry(const Ctx &C, const S5eBufs &D, int32_t src, int32_t k) {
    const int32_t rr = C.T.idx[k];
    return rr != src && C.rkind[rr] == RK_KEPT && D.rmin[rr] != src;
}

struct S5eApplied {
    S5eWalk w;  // the side-shift walk (own: the doubleton applied)
    int32_t changed;  // x_j's bounds changed
    int32_t jj;
};

// Selected row i: the bound transfer onto x_j (finalised as S3' finalises;
// an empty one is a verdict on x_j and the row does not apply), x_j's cost,
// the kinds, x_k's value g, the records and the substitution store; dj, df,
// dg keep x_j, f, g for the walk.
__host__ __device__ inline S5eApplied s5e_apply_row(const Ctx &C, const S5eBufs &D, int32_t i) {
    S5eApplied r{S5eWalk{false, 0, 0}, 0, -1};
    const int32_t kk = D.dk[i], p = C.A.ptr[i];
    const bool j_first = C.A.idx[p] != kk;
    const int32_t jj = j_first ? C.A.idx[p] : C.A.idx[p + 1];
    const double a = j_first ? C.A.val[p] : C.A.val[p + 1];
    const double bk = j_first ? C.A.val[p + 1] : C.A.val[p];
    const double cv = C.L[i];
    const double f = a / bk, g = cv / bk;
    const double2 luj = C.lu[jj], luk = C.lu[kk];
    const double bhi = f > 0.0 ? luk.y : luk.x, blo = f > 0.0 ? luk.x : luk.y;
    const double lo = s5e_fin(bhi) ? (g - bhi) / f : -s5e_inf();
    const double hi = s5e_fin(blo) ? (g - blo) / f : s5e_inf();
    double nl = lo > luj.x ? lo : luj.x;
    double nu = hi < luj.y ? hi : luj.y;
    const int32_t lp = s5e_lp_row(C, i);
    if (s5e_fin(nl) && s5e_fin(nu)) {
        const double d = C.feas_tol * fmax(1.0, fmax(fabs(nl), fabs(nu)));
        if (nl - nu > d) {
            s5e_amin(&C.verdict[lp * V_SLOTS + V_S5E_COL], C.cmap[jj]);
            return r;
        }
        if (nl != nu && fabs(nl - nu) <= d) nl = nu = 0.5 * (nl + nu);
    }
    r.changed = nl != luj.x || nu != luj.y;
    r.jj = jj;
    C.lu[jj] = make_double2(nl, nu);
    const double t = C.c[kk] / bk;
    C.c[jj] = C.c[jj] - t * a;
    C.rkind[i] = RK_DOUBLETON;
    C.ckind[kk] = CK_DOUBLETON;
    C.fixv[kk] = g;
    const int32_t oi = C.rmap[i], ok = C.cmap[kk], oj = C.cmap[jj], rd = s5e_lp_round(C, lp);
    C.rec_rk[oi] = RK_DOUBLETON;
    C.rec_rr[oi] = rd;
    C.rec_ra[oi] = ok;
    C.rec_rv[oi] = bk;
    const unsigned long long pos = s5e_fetch_add(C.sub_used, 1ULL);
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
    r.w = S5eWalk{true, C.T.ptr[kk], C.T.ptr[kk + 1]};
    return r;
}

// entry k of applied row src's x_k column: a kept row other than src loses
// a_rk g on each finite side and notes (x_j, x_k, -(a_rk f)) for the rewrite
__host__ __device__ inline void s5e_shift_entry(const Ctx &C, const S5eBufs &D, int32_t src, int32_t k) {
    const int32_t rr = C.T.idx[k];
    if (rr == src || C.rkind[rr] != RK_KEPT) return;
    const double ark = C.T.val[k];
    const double f = D.df[src], g = D.dg[src];
    const double Lv = C.L[rr], Uv = C.U[rr];
    if (s5e_fin(Lv)) C.L[rr] = Lv - ark * g;
    if (s5e_fin(Uv)) C.U[rr] = Uv - ark * g;
    D.dmj[rr] = D.dj[src];
    D.dmk[rr] = D.dk[src];
    D.dmd[rr] = -(ark * f);
    C.rdnext[rr] = 1;
}

// Row i's length after the rewrite; a changed row also keeps its note
// (positions of x_k and x_j, flags, x_j's new coefficient)
__host__ __device__ inline int32_t s5e_rowlen_row(const Ctx &C, const S5eBufs &D, int32_t i) {
    const int32_t p = C.A.ptr[i], len = C.A.ptr[i + 1] - p, jj = D.dmj[i];
    if (jj < 0) return len;
    const S5eNote t = s5e_note(C.A.idx + p, C.A.val + p, len, jj, D.dmk[i], D.dmd[i], C.par_tol);
    D.dpk[i] = t.pk;
    D.dpj[i] = t.pj;
    D.dfl[i] = (uint8_t)((t.found ? 1 : 0) | (t.cancel ? 2 : 0));
    D.dnv[i] = t.v;
    return t.len_new;
}

// Entry e of the current CSR into the rewritten one (rp2: the scanned new
// lengths); the entry of x_k in a changed row writes an inserted x_j.  A
// place outside the row's new range is not written and returns false (the
// lengths and the notes disagree: an internal error the caller reports).
__host__ __device__ inline bool s5e_place_entry(const Ctx &C, const S5eBufs &D, const int32_t *rp2, int32_t *ci2,
                                                double *rv2, int32_t *row_of, int32_t e) {
    // the row of e: the last i with ptr[i] <= e
    int32_t lo = 0, hi = C.m;
    while (hi - lo > 1) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (C.A.ptr[mid] <= e) lo = mid;
        else hi = mid;
    }
    const int32_t i = lo, q = e - C.A.ptr[i], base = rp2[i];
    const int32_t col = C.A.idx[e];
    double v = C.A.val[e];
    int32_t dest = base + q;
    const int32_t jj = D.dmj[i];
    if (jj >= 0) {
        S5eNote t;
        t.pk = D.dpk[i];
        t.pj = D.dpj[i];
        t.found = D.dfl[i] & 1;
        t.cancel = (D.dfl[i] & 2) != 0;
        if (q == t.pk) {
            if (!t.found) {
                const int32_t at = base + s5e_insert_at(t);
                if (at < base || at >= rp2[i + 1]) return false;
                ci2[at] = jj;
                rv2[at] = D.dnv[i];
                row_of[at] = i;
            }
            return true;
        }
        if (t.found && q == t.pj) {
            if (t.cancel) return true;
            v = D.dnv[i];
        }
        dest = base + s5e_dest(t, q);
    }
    if (dest < base || dest >= rp2[i + 1]) return false;
    ci2[dest] = col;
    rv2[dest] = v;
    row_of[dest] = i;
    return true;
}

}  // namespace lpp
