"""Pins of the oracle's parallel-column step (S5c, opt-in), without a GPU.

The step merges column j into column k when A_:j = lam A_:k and c_j = lam
c_k: y = x_k + lam x_j replaces x_k.  Pinned here against what does not
depend on the oracle: the planted copies of synth.parcols and their exact
factors, the optimal value of the LP (unchanged by a merge), and the
postsolve, whose split of y must give an original point that is feasible
and optimal.
"""
import numpy as np
import pytest

import oracle
from lpbrute import inequalities, lp_vertices, vertices
from paper_2609_16182_gb300 import synth


def test_planted_copies_are_merged_into_their_base_with_the_planted_factor():
    lp = synth.parcols(0)
    res = oracle.presolve(lp, oracle.default_opts(parallel_cols=1))
    assert res.status == oracle.OK
    for b, cpy, lam in zip(lp.planted["base"], lp.planted["copies"], lp.planted["lam"]):
        assert res.col_kind[cpy] == oracle.COL_PARALLEL
        assert res.col_aux[cpy] == b  # the base has the smaller index: it leads
        assert res.col_val[cpy] == lam  # lam = a_copy / a_base, exact for a power of two
        lk, uk, lj, uj = res.col_mrg[cpy]
        # bounds at merge time: the round's tightening only narrows them
        assert lp.lb[cpy] <= lj <= uj <= lp.ub[cpy]
        assert lp.lb[b] <= lk <= uk <= lp.ub[b]


def test_a_chain_of_merges_in_one_pass():
    # columns 1, 2, 3 are copies of column 0 (factors 2, -1/2, 4): one pass
    # merges all three into column 0 in column order, each record holding the
    # leader's bounds before it; the final bounds are the interval sums
    from lpmake import make
    base = {0: 1.0, 1: -3.0}
    lam = {1: 2.0, 2: -0.5, 3: 4.0}
    rows = [{0: base[0], 1: lam[1] * base[0], 2: lam[2] * base[0], 3: lam[3] * base[0], 4: 1.0},
            {0: base[1], 1: lam[1] * base[1], 2: lam[2] * base[1], 3: lam[3] * base[1], 4: -1.0}]
    lb = [-1.0, 0.0, -2.0, 0.5, -1.0]
    ub = [2.0, 1.0, 3.0, 1.0, 1.0]
    c = [1.0, 2.0, -0.5, 4.0, 0.0]
    # sides 1 inside each row's activity range: the rows stay (not redundant)
    # and imply no bound (1 is below every row's span minus its largest term's)
    lo_act = [sum(a * (lb[j] if a > 0 else ub[j]) for j, a in r.items()) for r in rows]
    hi_act = [sum(a * (ub[j] if a > 0 else lb[j]) for j, a in r.items()) for r in rows]
    lp = make(rows, [x + 1.0 for x in lo_act], [x - 1.0 for x in hi_act], lb, ub, c=c)
    res = oracle.presolve(lp, oracle.default_opts(parallel_cols=1, max_rounds=1))
    assert list(res.col_kind[:4]) == [0, 3, 3, 3]
    ly, uy = lb[0], ub[0]
    for j in (1, 2, 3):
        assert res.col_aux[j] == 0 and res.col_pass[j] == 0 and res.col_val[j] == lam[j]
        assert list(res.col_mrg[j]) == [ly, uy, lb[j], ub[j]]
        ly, uy = (ly + lam[j] * lb[j], uy + lam[j] * ub[j]) if lam[j] > 0 else (ly + lam[j] * ub[j],
                                                                                uy + lam[j] * lb[j])
    k = int(np.flatnonzero(res.col_map == 0)[0])
    assert (res.lb[k], res.ub[k]) == (ly, uy) == (-1.0 + 0.0 - 1.5 + 2.0, 2.0 + 2.0 + 1.0 + 4.0)


def test_off_by_default():
    lp = synth.parcols(1)
    res = oracle.presolve(lp)
    assert not np.any(res.col_kind == oracle.COL_PARALLEL)


def test_merged_bounds_are_the_closed_form():
    # y = x_0 + lam x_1 with lam = -2: [l0 - 2 u1, u0 - 2 l1].  The row sides
    # cut neither activity range short enough to tighten a bound (checked by
    # hand on both sides of both rows), so the merge sees the original bounds.
    from lpmake import make
    lp = make([{0: 1.0, 1: -2.0, 2: 1.0}, {0: 3.0, 1: -6.0, 2: -1.0}], [-8.0, -22.0], [2.9, 4.9],
              [-1.0, 0.5, -2.0], [2.0, 3.0, 2.0], c=[1.0, -2.0, 0.5])
    res = oracle.presolve(lp, oracle.default_opts(parallel_cols=1, max_rounds=1))
    assert res.col_kind[1] == oracle.COL_PARALLEL and res.col_aux[1] == 0 and res.col_val[1] == -2.0
    k = int(np.flatnonzero(res.col_map == 0)[0])
    assert (res.lb[k], res.ub[k]) == (-1.0 - 2.0 * 3.0, 2.0 - 2.0 * 0.5)


def test_costs_must_be_in_the_same_ratio():
    # the closed-form LP with c1 = -2.5 instead of -2 = lam c0: the coefficients are parallel, the
    # costs are not, so nothing merges
    from lpmake import make
    lp = make([{0: 1.0, 1: -2.0, 2: 1.0}, {0: 3.0, 1: -6.0, 2: -1.0}], [-8.0, -22.0], [2.9, 4.9],
              [-1.0, 0.5, -2.0], [2.0, 3.0, 2.0], c=[1.0, -2.5, 0.5])
    res = oracle.presolve(lp, oracle.default_opts(parallel_cols=1, max_rounds=1))
    assert not np.any(res.col_kind == oracle.COL_PARALLEL)


@pytest.mark.parametrize("seed", range(40))
def test_optimum_kept_and_postsolve_optimal(seed):
    lp = synth.parcols(seed + 500, m=4, n_base=4, pairs=2, per_col=3, slack=1.0)
    res = oracle.presolve(lp, oracle.default_opts(parallel_cols=1))
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
        k = int(np.argmin(W @ res.c))
        xr = W[k]
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
    lp = synth.parcols(seed)
    res = oracle.presolve(lp, oracle.default_opts(parallel_cols=1))
    assert res.status == oracle.OK
    assert np.count_nonzero(res.col_kind == oracle.COL_PARALLEL) >= len(lp.planted["copies"])
    st0, x0, f0 = _linprog(lp.c, lp.row_ptr, lp.col_idx, lp.val, lp.lhs, lp.rhs, lp.lb, lp.ub, lp.n)
    st1, x1, f1 = _linprog(res.c, res.row_ptr, res.col_idx, res.val, res.lhs, res.rhs, res.lb, res.ub,
                           res.n_red)
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
