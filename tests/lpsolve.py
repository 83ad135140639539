"""An independent LP solver (HiGHS through scipy) and a KKT check, for the
dual postsolve tests.

solve() returns a primal-dual optimum of an LP of the form of Eq. 1 in the
sign convention of the postsolve: y_i > 0 only at a finite lhs, y_i < 0 only
at a finite rhs, z = c - A^T y.  kkt() measures how far a triple (x, y, z)
is from optimality for an LP: primal residuals, dual sign errors,
complementarity and the gap between the primal and the dual objective.
"""
import numpy as np

HUGE = 1e20


def _inf(v):
    v = np.asarray(v, np.float64)
    return np.where(v >= HUGE, np.inf, np.where(v <= -HUGE, -np.inf, v))


def _csr(lp):
    import scipy.sparse as sp
    return sp.csr_matrix((np.asarray(lp.val, np.float64), np.asarray(lp.col_idx, np.int64),
                          np.asarray(lp.row_ptr, np.int64)), shape=(lp_m(lp), lp_n(lp)))


def lp_m(lp):
    return len(lp.lhs)


def lp_n(lp):
    return len(lp.c)


def solve(lp):
    """(status, x, y, objective without offset); status 0 = optimal."""
    import scipy.sparse as sp
    from scipy.optimize import linprog
    m, n = lp_m(lp), lp_n(lp)
    L, U, l, u = _inf(lp.lhs), _inf(lp.rhs), _inf(lp.lb), _inf(lp.ub)
    c = np.asarray(lp.c, np.float64)
    if n == 0:
        return 0, np.zeros(0), np.zeros(m), 0.0
    A = _csr(lp)
    eq = np.isfinite(L) & np.isfinite(U) & (L == U)
    up = np.isfinite(U) & ~eq
    lo = np.isfinite(L) & ~eq
    iu, il, ie = np.flatnonzero(up), np.flatnonzero(lo), np.flatnonzero(eq)
    Aub = sp.vstack([A[iu], -A[il]]).tocsr()
    bub = np.concatenate([U[iu], -L[il]])
    kw = {}
    if Aub.shape[0]:
        kw.update(A_ub=Aub, b_ub=bub)
    if len(ie):
        kw.update(A_eq=A[ie], b_eq=L[ie])
    r = linprog(c, bounds=np.column_stack([l, u]), method="highs", **kw)
    if r.status != 0:
        return r.status, None, None, None
    y = np.zeros(m)
    if Aub.shape[0]:
        mu = r.ineqlin.marginals
        y[iu] += mu[:len(iu)]
        y[il] -= mu[len(iu):]
    if len(ie):
        y[ie] += r.eqlin.marginals
    return 0, r.x, y, float(r.fun)


def kkt(lp, x, y, z):
    """Scaled optimality residuals of (x, y, z) on lp; all small at an optimum."""
    L, U, l, u = _inf(lp.lhs), _inf(lp.rhs), _inf(lp.lb), _inf(lp.ub)
    c = np.asarray(lp.c, np.float64)
    A = _csr(lp)
    ax = A @ x if lp_m(lp) else np.zeros(0)
    scale = 1.0 + max(np.abs(c).max(initial=0.0), np.abs(y).max(initial=0.0))
    out = {}
    out["primal"] = max(np.max(np.maximum(L - ax, 0) / (1 + np.abs(np.where(np.isfinite(L), L, 0))), initial=0.0),
                        np.max(np.maximum(ax - U, 0) / (1 + np.abs(np.where(np.isfinite(U), U, 0))), initial=0.0),
                        np.max(np.maximum(l - x, 0) / (1 + np.abs(np.where(np.isfinite(l), l, 0))), initial=0.0),
                        np.max(np.maximum(x - u, 0) / (1 + np.abs(np.where(np.isfinite(u), u, 0))), initial=0.0))
    zc = c - (A.T @ y if lp_m(lp) else 0.0)
    out["z_def"] = np.max(np.abs(zc - z), initial=0.0) / scale
    # a dual with no finite side to pay it is a sign error
    out["sign"] = max(np.max(np.where(~np.isfinite(L), np.maximum(y, 0), 0), initial=0.0),
                      np.max(np.where(~np.isfinite(U), np.maximum(-y, 0), 0), initial=0.0),
                      np.max(np.where(~np.isfinite(l), np.maximum(z, 0), 0), initial=0.0),
                      np.max(np.where(~np.isfinite(u), np.maximum(-z, 0), 0), initial=0.0)) / scale
    with np.errstate(invalid="ignore"):
        gr = np.where(y > 0, ax - L, np.where(y < 0, U - ax, 0.0))
        gc = np.where(z > 0, x - l, np.where(z < 0, u - x, 0.0))
    gr = np.where(np.isfinite(gr), gr, 0.0)
    gc = np.where(np.isfinite(gc), gc, 0.0)
    out["compl"] = max(np.max(np.abs(y * gr), initial=0.0), np.max(np.abs(z * gc), initial=0.0)) / scale
    pobj = float(c @ x)
    dobj = float(np.sum(np.where(y > 0, y * np.where(np.isfinite(L), L, 0), y * np.where(np.isfinite(U), U, 0)))
                 + np.sum(np.where(z > 0, z * np.where(np.isfinite(l), l, 0), z * np.where(np.isfinite(u), u, 0))))
    out["gap"] = abs(pobj - dobj) / (1.0 + abs(pobj))
    out["pobj"], out["dobj"] = pobj, dobj
    return out
