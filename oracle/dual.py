"""Dual postsolve of the oracle's records, plain numpy and Python loops.

TEST INFRASTRUCTURE ONLY: imported by tests/ (and nothing in the library
path).  It shares no code with the library's postsolve.

The paper's postsolver (Sec. 2.1, postsolver paragraph; Sec. 3.3) maps a
primal-dual solution of the reduced LP back to one of the input LP, popping
the reductions latest first.  Its dual side is not written out in the paper;
the reading restated here, for the reductions of the default path
(Sec. 3.1 activities and implied bounds, Sec. 2.1 removal of rows and fixing
of columns, Sec. 3.2 parallel rows) and for dual fixing, is:

  * Sign convention (Eq. 1, minimise): row duals y and reduced costs
    z = c - A^T y, with y_i > 0 only at a finite lhs, y_i < 0 only at a
    finite rhs, z_j > 0 only at a finite lower bound, z_j < 0 only at a
    finite upper bound.
  * A kept row takes the reduced dual through the row map; a removed row
    (empty, redundant, singleton, merged) starts at 0.
  * An implied bound (S3) or a singleton-row bound is a valid inequality of
    the input LP only through the row that implied it.  When the final
    reduced costs put a nonzero z_j on a side that such a row set (z_j < 0
    on an upper bound, z_j > 0 on a lower bound), the row takes it over:
    y_r += z_j / a_rj, and every column of that row has its reduced cost
    updated; z_j becomes 0.  Sides are taken latest round first (the
    postsolve stack order), then by column.  At an exact optimum the
    implying row is tight and its other columns sit at the bounds that
    implied the value, so the new reduced costs keep their signs.
  * Parallel rows (S5): every row merged into a leader, directly or through
    a chain of merges, is lambda times the chain's root row a_R.  The
    family's duals act on a_R x as one number Y = sum_g y_g Lambda_g; it is
    given whole to the member whose own side of the orientation Y selects is
    tightest at x (lhs of members with Lambda > 0 and rhs of those with
    Lambda < 0 when Y > 0, the other sides when Y < 0; the smallest relative
    residual, then the smallest row), as y_g = Y / Lambda_g.  Reduced costs
    do not change.
  * Every other removed column (fixed, empty, dual-fixed) takes
    z_j = c_j - a_j^T y at the end, like the kept ones.
  * Parallel columns (S5c): a column j merged into k (A_:j = lam A_:k,
    c_j = lam c_k) gets z_j = lam z_k from the same definition, and the
    primal postsolve puts x_k and x_j at the bounds of the merged column's
    side when it sits at one, so no step of its own is needed.
  * Column singletons (S5d): the substitution moved c_j(t) / a_ij times the
    row into the other columns' costs (c_j(t): column j's cost when it went,
    changed only by earlier substitutions).  So, before the transfers, the
    substitution rows take, earliest round first (then by column),
    y_i += (c_j - sum_r a_rj y_r) / a_ij over column j's input entries:
    the eliminated (free) column keeps no reduced cost, and every other
    column's z = c - A^T y equals its reduced-LP reduced cost.  Its own
    bound sides are not transferred.

Doubleton equations have no dual side restated here: the function refuses
their records.
"""
from __future__ import annotations

import numpy as np

from . import COL_DOUBLETON, COL_SUBST, ROW_DOUBLETON, ROW_PARALLEL, ROW_SUBST, postsolve_primal


def _inf(v, huge=1e20):
    v = np.asarray(v, np.float64)
    return np.where(v >= huge, np.inf, np.where(v <= -huge, -np.inf, v))


def reduced_costs(lp, y):
    """z = c - A^T y, entry by entry."""
    z = np.array(lp.c, np.float64, copy=True)
    for i in range(lp.m):
        for k in range(int(lp.row_ptr[i]), int(lp.row_ptr[i + 1])):
            z[int(lp.col_idx[k])] -= float(lp.val[k]) * y[i]
    return z


def postsolve_dual(lp, res, x_red, y_red, huge=1e20):
    """(x, y, z) of the input LP from a reduced primal-dual pair (x_red, y_red)."""
    if (res.col_kind == COL_DOUBLETON).any() or (res.row_kind == ROW_DOUBLETON).any():
        raise ValueError("no dual postsolve for doubletons")
    m, n = lp.m, lp.n
    x = postsolve_primal(res, x_red)
    y = np.zeros(m)
    y[np.asarray(res.row_map, np.int64)] = np.asarray(y_red, np.float64)

    # column singletons (S5d), earliest round first, then by column: the
    # substitution row takes the dual that leaves the eliminated column no
    # reduced cost
    colrows = {}
    for i in range(m):
        for k in range(int(lp.row_ptr[i]), int(lp.row_ptr[i + 1])):
            colrows.setdefault(int(lp.col_idx[k]), []).append((i, float(lp.val[k])))
    subs = sorted((int(res.row_round[i]), int(res.row_aux[i]), i) for i in range(m) if res.row_kind[i] == ROW_SUBST)
    for _, j, i in subs:
        zj = float(lp.c[j])
        for r, a in colrows.get(j, []):
            zj -= a * y[r]
        y[i] += zj / float(res.row_val[i])
    z = reduced_costs(lp, y)

    # bound sides set by a row, latest round first, then column, lower first
    events = []
    for j in range(n):
        if res.col_kind[j] == COL_SUBST:
            continue  # its substitution row carries its reduced cost
        if res.col_lsrc[j] >= 0:
            events.append((-int(res.col_lrnd[j]), j, 0, int(res.col_lsrc[j])))
        if res.col_usrc[j] >= 0:
            events.append((-int(res.col_urnd[j]), j, 1, int(res.col_usrc[j])))
    events.sort()
    for _, j, upper, r in events:
        if (upper and not z[j] < 0.0) or (not upper and not z[j] > 0.0):
            continue
        beg, end = int(lp.row_ptr[r]), int(lp.row_ptr[r + 1])
        a_rj = None
        for k in range(beg, end):
            if int(lp.col_idx[k]) == j:
                a_rj = float(lp.val[k])
        if a_rj is None:
            raise ValueError(f"record of column {j} names row {r}, which has no entry in it")
        d = z[j] / a_rj
        y[r] += d
        for k in range(beg, end):
            z[int(lp.col_idx[k])] -= float(lp.val[k]) * d
        z[j] = 0.0

    # parallel-row families: root and cumulative factor of every row
    L, U = _inf(lp.lhs, huge), _inf(lp.rhs, huge)
    root = np.arange(m)
    lam = np.ones(m)
    for i in range(m):
        g, f = i, 1.0
        while res.row_kind[g] == ROW_PARALLEL:
            f *= float(res.row_val[g])
            g = int(res.row_aux[g])
        root[i], lam[i] = g, f
    members = {}
    for i in range(m):
        if root[i] != i:
            members.setdefault(int(root[i]), [int(root[i])]).append(i)
    for rt, mem in members.items():
        mem = sorted(mem)
        Y = sum(y[g] * lam[g] for g in mem)
        for g in mem:
            y[g] = 0.0
        if Y == 0.0:
            continue
        best, best_res = -1, np.inf
        for g in mem:
            lower_side = (lam[g] > 0) == (Y > 0)
            side = L[g] if lower_side else U[g]
            if not np.isfinite(side):
                continue
            act = sum(float(lp.val[k]) * x[int(lp.col_idx[k])] for k in range(int(lp.row_ptr[g]), int(lp.row_ptr[g + 1])))
            rres = abs(act - side) / max(1.0, abs(side))
            if rres < best_res:
                best, best_res = g, rres
        if best < 0:
            raise ValueError(f"parallel family of row {rt} has no finite side for its dual")
        y[best] = Y / lam[best]

    return x, y, reduced_costs(lp, y)
