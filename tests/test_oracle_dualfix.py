"""Pins of the oracle's dual fixing (S6 with `dual_fixing`), without a GPU.

A column that no kept row locks in the direction its cost prefers is fixed
at that bound: moving it there keeps every row feasible and does not raise
the objective, so an optimal solution survives.  Pinned against hand-worked
locks, the optimal value of the LP (vertex enumeration, scipy) and a
postsolved point that is feasible and optimal.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from lpbrute import inequalities, lp_vertices, vertices
from lpmake import INF, make
from paper_2609_16182_gb300 import synth


def opts(**kw):
    return oracle.default_opts(dual_fixing=1, **kw)


def test_hand_worked_locks():
    # x0 (cost 2) in rows with a > 0 and no lhs: nothing locks it downwards -> lb = -1
    # x1 (cost -1) in row 0 (a = 1, rhs finite) locks it upwards -> kept
    # x2 (cost -3) in row 1 with a = -1 and no lhs: no up lock -> ub = 4
    lp = make([{0: 1.0, 1: 1.0}, {0: 2.0, 1: 1.0, 2: -1.0}], [-INF, -INF], [3.0, 5.0],
              [-1.0, 0.0, 0.0], [2.0, 10.0, 4.0], c=[2.0, -1.0, -3.0])
    res = oracle.presolve(lp, opts(max_rounds=1))
    assert res.col_kind[0] == oracle.COL_EMPTY and res.col_val[0] == -1.0
    assert res.col_kind[1] == oracle.COL_KEPT
    assert res.col_kind[2] == oracle.COL_EMPTY and res.col_val[2] == 4.0
    res0 = oracle.presolve(lp, oracle.default_opts(max_rounds=1))
    assert not np.any(res0.col_kind == oracle.COL_EMPTY)  # off by default: none is empty


def test_unbounded_when_the_preferred_bound_is_infinite():
    lp = make([{0: 1.0, 1: 1.0}], [-INF], [3.0], [-INF, 0.0], [2.0, 1.0], c=[1.0, 0.0])
    res = oracle.presolve(lp, opts())
    assert res.status == oracle.UNBOUNDED and res.index == 0


def one_sided(lp):
    """Every inequality row with a finite rhs loses its lhs: more columns
    without a lock downwards."""
    lhs = lp.lhs.copy()
    eq = np.isfinite(lp.lhs) & (lp.lhs == lp.rhs)
    lhs[~eq & np.isfinite(lp.rhs)] = -INF
    return dataclasses.replace(lp, lhs=lhs)


@pytest.mark.parametrize("variant", ["plain", "one_sided"])
@pytest.mark.parametrize("seed", range(60))
def test_optimum_kept_and_postsolve_optimal(seed, variant):
    lp = synth.micro(seed + 1300)
    if variant == "one_sided":
        lp = one_sided(lp)
    res = oracle.presolve(lp, opts())
    V = lp_vertices(lp)
    if len(V) == 0:
        assert res.status == oracle.INFEASIBLE
        return
    assert res.status == oracle.OK
    opt = float(np.min(V @ lp.c))
    if res.n_red:
        G, h = inequalities(res.row_ptr, res.col_idx, res.val, res.lhs, res.rhs, res.lb, res.ub, res.n_red)
        W = vertices(G, h, res.n_red)
        assert len(W) > 0
        xr = W[int(np.argmin(W @ res.c))]
        red_opt = float(xr @ res.c) + res.obj_offset
    else:
        xr = np.zeros(0)
        red_opt = res.obj_offset
    assert red_opt == pytest.approx(opt, rel=1e-9, abs=1e-9)
    x = oracle.postsolve_primal(res, xr)
    Gi, hi = inequalities(lp.row_ptr, lp.col_idx, lp.val, lp.lhs, lp.rhs, lp.lb, lp.ub, lp.n)
    assert np.all(Gi @ x <= hi + 1e-8 * (1 + np.abs(hi)))
    assert float(lp.c @ x) == pytest.approx(opt, rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("seed", range(4))
def test_reduced_optimum_matches_original_200_rows(seed):
    pytest.importorskip("scipy")
    from test_oracle_invariants import _linprog
    lp = synth.tiny(seed)
    res = oracle.presolve(lp, opts())
    st0, x0, f0 = _linprog(lp.c, lp.row_ptr, lp.col_idx, lp.val, lp.lhs, lp.rhs, lp.lb, lp.ub, lp.n)
    if res.status != oracle.OK:
        assert st0 != 0
        return
    st1, x1, f1 = _linprog(res.c, res.row_ptr, res.col_idx, res.val, res.lhs, res.rhs, res.lb, res.ub, res.n_red)
    assert st0 == 0 and st1 == 0
    assert f1 + res.obj_offset == pytest.approx(f0, rel=1e-7, abs=1e-7)
    x = oracle.postsolve_primal(res, x1)
    A = np.zeros((lp.m, lp.n))
    for i in range(lp.m):
        A[i, lp.col_idx[lp.row_ptr[i]:lp.row_ptr[i + 1]]] = lp.val[lp.row_ptr[i]:lp.row_ptr[i + 1]]
    ax = A @ x
    tol = 1e-6 * (1 + np.abs(ax))
    assert np.all(ax >= lp.lhs - tol) and np.all(ax <= lp.rhs + tol)
    assert np.all(x >= lp.lb - 1e-6) and np.all(x <= lp.ub + 1e-6)
    assert float(lp.c @ x) == pytest.approx(f0, rel=1e-7, abs=1e-7)
