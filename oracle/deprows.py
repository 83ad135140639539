"""Linearly dependent equality rows, dense numpy (the oracle's side).

TEST INFRASTRUCTURE ONLY: imported by tests/ (and nothing in the library
path).  It shares no code with the library.

Sec. 5 proposes a hybrid design for this explorer: the equality rows go to
the CPU, which finds their linear dependencies by pivoting Gaussian
elimination (each pivot chosen numerically from the values the eliminations
before it produced), and the result goes back for the rest of presolve.  The
reading restated here, applied once after the presolve loop:

  * The equality rows (finite lhs == rhs) of the reduced LP are peeled
    first: a row holding a column that no other equality row still holds
    is in no linear dependency (that column's multiple would have to
    vanish), so it leaves, and its columns' counts drop; this repeats until
    every row left shares all its columns.  The rows left are taken in row
    order.  Each is reduced against the pivot rows found so far, in the
    order they were found: for a pivot row p with pivot column q and the
    current row w with w_q != 0, f = w_q / p_q, w := w - f p (element by
    element), w_q := 0, b := b - f b_p.
  * What is left is zero when max |w| <= dep_tol * max |row as given|: the
    row is a combination of earlier equality rows and is removed (record
    kind ROW_DEPENDENT).  Its rhs must then be zero too, within
    dep_tol * max(1, |b as given|, every |f b_p| used): else the equalities
    contradict each other and the LP is infeasible (the first such row).
    dep_tol is the presolve's feasibility tolerance (feas_tol).
  * Otherwise the row becomes a pivot row; its pivot column is the one of
    largest |w| (the first such column).
  * The step then runs S6 on the LP that is left (empty columns fixed at the
    bound their cost prefers; with dual fixing, every column that no kept
    row locks in that direction), with S6's records, side shifts and
    objective constant; its records carry round = rounds + 1.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import COL_EMPTY, COL_KEPT, INFEASIBLE, OK, ROW_KEPT, UNBOUNDED, WHERE_COL, WHERE_ROW

ROW_DEPENDENT = 7


def core_rows(red):
    """The equality rows left after peeling (in row order) and the number
    peeled."""
    m, n = len(red.lhs), len(red.c)
    eq = [i for i in range(m) if np.isfinite(red.lhs[i]) and red.lhs[i] == red.rhs[i]]
    cnt = np.zeros(n, np.int64)
    for i in eq:
        for k in range(int(red.row_ptr[i]), int(red.row_ptr[i + 1])):
            cnt[red.col_idx[k]] += 1
    alive = {i: True for i in eq}
    changed = True
    while changed:
        changed = False
        for i in eq:
            if not alive[i]:
                continue
            cols = red.col_idx[int(red.row_ptr[i]):int(red.row_ptr[i + 1])]
            if len(cols) and np.any(cnt[cols] == 1):
                alive[i] = False
                cnt[cols] -= 1
                changed = True
    core = [i for i in eq if alive[i]]
    return core, len(eq) - len(core)


def dependent_rows(red, dep_tol=1e-9):
    """(reduced indices of the dependent equality rows, the first
    inconsistent one or -1, the number of pivot rows among the rows left
    after peeling)."""
    n = len(red.c)
    pivots = []  # (column, dense row, rhs)
    dep, bad = [], -1
    for i in core_rows(red)[0]:
        w = np.zeros(n)
        k0, k1 = int(red.row_ptr[i]), int(red.row_ptr[i + 1])
        w[red.col_idx[k0:k1]] = red.val[k0:k1]
        scale = float(np.max(np.abs(w))) if k1 > k0 else 0.0
        b = float(red.rhs[i])
        sb = abs(b)
        for q, p, pb in pivots:
            if w[q] != 0.0:
                f = w[q] / p[q]
                w = w - f * p
                w[q] = 0.0
                b = b - f * pb
                sb = max(sb, abs(f * pb))
        mx = float(np.max(np.abs(w))) if n else 0.0
        if mx <= dep_tol * scale:
            dep.append(i)
            if bad < 0 and abs(b) > dep_tol * max(1.0, sb):
                bad = i
        else:
            pivots.append((int(np.argmax(np.abs(w))), w, b))
    return dep, bad, len(pivots)


def apply(lp, res, opts):
    """The oracle's result `res` of `lp` with the dependent-row step applied
    (a new Result; `res` is left as it was)."""
    if res.status != OK:
        return res
    dep, bad, _ = dependent_rows(res, opts.feas_tol)
    r = res.rounds + 1
    row_kind, row_round = res.row_kind.copy(), res.row_round.copy()
    col_kind, col_round, col_val = res.col_kind.copy(), res.col_round.copy(), res.col_val.copy()
    col_lb, col_ub = res.col_lb.copy(), res.col_ub.copy()
    out = dict(row_kind=row_kind, row_round=row_round, col_kind=col_kind, col_round=col_round, col_val=col_val,
               col_lb=col_lb, col_ub=col_ub)
    if bad >= 0:
        return dataclasses.replace(res, status=INFEASIBLE, where=WHERE_ROW, index=int(res.row_map[bad]), round=r,
                                   **out)
    m, n = len(res.lhs), len(res.c)
    keep = np.ones(m, bool)
    keep[dep] = False
    for i in dep:
        row_kind[res.row_map[i]] = ROW_DEPENDENT
        row_round[res.row_map[i]] = r
    # S6 on what is left: counts and locks of the kept rows
    cnt = np.zeros(n, np.int64)
    dlock = np.zeros(n, np.int64)
    ulock = np.zeros(n, np.int64)
    for i in range(m):
        if not keep[i]:
            continue
        for k in range(int(res.row_ptr[i]), int(res.row_ptr[i + 1])):
            j, a = int(res.col_idx[k]), float(res.val[k])
            cnt[j] += 1
            if a > 0:
                dlock[j] += np.isfinite(res.lhs[i])
                ulock[j] += np.isfinite(res.rhs[i])
            else:
                dlock[j] += np.isfinite(res.rhs[i])
                ulock[j] += np.isfinite(res.lhs[i])
    fixv = np.full(n, np.nan)
    if opts.dual_reductions:
        for j in range(n):
            if not opts.dual_fixing and cnt[j] != 0:
                continue
            c, lo, hi = float(res.c[j]), float(res.lb[j]), float(res.ub[j])
            if c > 0:
                fix, v = dlock[j] == 0, lo
            elif c < 0:
                fix, v = ulock[j] == 0, hi
            elif dlock[j] == 0 and np.isfinite(lo):
                fix, v = True, lo
            elif ulock[j] == 0 and np.isfinite(hi):
                fix, v = True, hi
            else:
                fix, v = dlock[j] == 0 and ulock[j] == 0, 0.0
            if not fix:
                continue
            o = int(res.col_map[j])
            if not np.isfinite(v):
                return dataclasses.replace(res, status=UNBOUNDED, where=WHERE_COL, index=o, round=r, **out)
            fixv[j] = v
            col_kind[o], col_round[o], col_val[o] = COL_EMPTY, r, v
            col_lb[o] = col_ub[o] = v
    gone = np.isfinite(fixv)
    # the reduced LP without the dependent rows and the fixed columns
    offset = res.obj_offset
    for j in range(n):
        if gone[j]:
            offset += float(res.c[j]) * fixv[j]
    newc = -np.ones(n, np.int64)
    newc[~gone] = np.arange(int((~gone).sum()))
    rp, ci, vv, L, U, rmap = [0], [], [], [], [], []
    for i in range(m):
        if not keep[i]:
            continue
        sh = 0.0
        for k in range(int(res.row_ptr[i]), int(res.row_ptr[i + 1])):
            j = int(res.col_idx[k])
            if gone[j]:
                sh += float(res.val[k]) * fixv[j]
            else:
                ci.append(int(newc[j]))
                vv.append(float(res.val[k]))
        rp.append(len(ci))
        L.append(res.lhs[i] - sh if np.isfinite(res.lhs[i]) else res.lhs[i])
        U.append(res.rhs[i] - sh if np.isfinite(res.rhs[i]) else res.rhs[i])
        rmap.append(int(res.row_map[i]))
    return dataclasses.replace(
        res, m_red=len(rmap), n_red=int((~gone).sum()), nnz_red=len(ci),
        row_ptr=np.array(rp, np.int32), col_idx=np.array(ci, np.int32), val=np.array(vv, np.float64),
        c=res.c[~gone].copy(), lhs=np.array(L, np.float64), rhs=np.array(U, np.float64),
        lb=res.lb[~gone].copy(), ub=res.ub[~gone].copy(), row_map=np.array(rmap, np.int32),
        col_map=res.col_map[~gone].copy(), obj_offset=offset, **out)


def presolve(lp, opts=None):
    """oracle.presolve followed by the dependent-row step."""
    from . import default_opts, presolve as _presolve
    o = opts if opts is not None else default_opts()
    return apply(lp, _presolve(lp, o), o)
