"""Brute-force helpers for the oracle pins (tiny LPs only).

Vertex enumeration: every choice of n constraints of G x <= h that is
nonsingular gives a candidate point; the feasible ones are the vertices of
the polytope.  For a bounded LP the optimum over the polytope is attained at
a vertex, so the minimum of c.x over the vertices is the LP optimum.
"""
from itertools import combinations

import numpy as np


def inequalities(row_ptr, col_idx, val, lhs, rhs, lb, ub, n):
    """G x <= h for lhs <= A x <= rhs and lb <= x <= ub (infinite sides dropped)."""
    G, h = [], []
    m = len(row_ptr) - 1
    for i in range(m):
        a = np.zeros(n)
        a[col_idx[row_ptr[i]:row_ptr[i + 1]]] = val[row_ptr[i]:row_ptr[i + 1]]
        if np.isfinite(rhs[i]):
            G.append(a); h.append(rhs[i])
        if np.isfinite(lhs[i]):
            G.append(-a); h.append(-lhs[i])
    for j in range(n):
        e = np.zeros(n); e[j] = 1.0
        if np.isfinite(ub[j]):
            G.append(e); h.append(ub[j])
        if np.isfinite(lb[j]):
            G.append(-e); h.append(-lb[j])
    return np.array(G, dtype=float).reshape(len(G), n), np.array(h, dtype=float)


def vertices(G, h, n, tol=1e-8):
    if n == 0:
        return np.zeros((1, 0)) if np.all(h >= -tol) else np.zeros((0, 0))
    k = len(G)
    if k < n:
        return np.zeros((0, n))
    idx = np.array(list(combinations(range(k), n)))
    A = G[idx]
    b = h[idx]
    det = np.linalg.det(A)
    ok = np.abs(det) > 1e-9
    if not ok.any():
        return np.zeros((0, n))
    x = np.linalg.solve(A[ok], b[ok][..., None])[..., 0]
    feas = np.all(x @ G.T <= h + tol * (1 + np.abs(h)), axis=1)
    x = x[feas]
    if len(x) == 0:
        return x
    # dedupe
    keyed = np.round(x, 6)
    _, first = np.unique(keyed, axis=0, return_index=True)
    return x[np.sort(first)]


def lp_vertices(lp):
    G, h = inequalities(lp.row_ptr, lp.col_idx, lp.val, lp.lhs, lp.rhs, lp.lb, lp.ub, lp.n)
    return vertices(G, h, lp.n)


def reduced_vertices_lifted(res, n_orig, fixed_values):
    """Vertices of the reduced LP, lifted to the original space."""
    G, h = inequalities(res.row_ptr, res.col_idx, res.val, res.lhs, res.rhs, res.lb, res.ub, res.n_red)
    v = vertices(G, h, res.n_red)
    out = np.zeros((len(v), n_orig))
    for j, val in fixed_values.items():
        out[:, j] = val
    if res.n_red:
        out[:, res.col_map] = v
    return out


def same_point_sets(P, Q, tol=1e-7):
    if len(P) != len(Q):
        return False
    if len(P) == 0:
        return True
    d = np.abs(P[:, None, :] - Q[None, :, :]).max(axis=2)
    return bool(np.all(d.min(axis=1) <= tol) and np.all(d.min(axis=0) <= tol))
