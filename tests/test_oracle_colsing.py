"""Pins of the oracle's column-singleton step (S5d, opt-in), without a GPU.

A column j in a single equality row i (a_ij x_j + sum_k a_ik x_k = b) that is
free, or whose bounds the row implies, is eliminated through the row:
c_k <- c_k - (c_j / a_ij) a_ik, the objective gains c_j b / a_ij, and the
postsolve sets x_j = (b - sum_k a_ik x_k) / a_ij.  Pinned against what does
not depend on the oracle: hand-worked costs and offsets, the optimal value
of the LP (unchanged by the elimination) and a postsolved point that is
feasible and optimal (vertex enumeration, scipy's LP solver).
"""
import numpy as np
import pytest

import oracle
from lpbrute import inequalities, lp_vertices, vertices
from lpmake import INF, make
from paper_2609_16182_gb300 import synth


def opts(**kw):
    return oracle.default_opts(col_singletons=1, **kw)


def test_hand_worked_substitution():
    # row 0: 2 x0 + x1 - x2 = 4 with x2 free and only in row 0; row 1: x0 + x1 <= 3
    # x2 = 2 x0 + x1 - 4: costs 1 + 3*2 = 7 and 2 + 3*1 = 5, constant 3 * 4 / (-1) = -12
    lp = make([{0: 2.0, 1: 1.0, 2: -1.0}, {0: 1.0, 1: 1.0}], [4.0, -INF], [4.0, 3.0],
              [0.0, 0.0, -INF], [2.0, 2.0, INF], c=[1.0, 2.0, 3.0])
    res = oracle.presolve(lp, opts(max_rounds=1))
    assert res.row_kind[0] == oracle.ROW_SUBST and res.row_aux[0] == 2 and res.row_val[0] == -1.0
    assert res.col_kind[2] == oracle.COL_SUBST and res.col_val[2] == -4.0
    assert list(res.col_map) == [0, 1] and list(res.c) == [7.0, 5.0] and res.obj_offset == -12.0
    b, n = res.sub_beg[0], res.sub_len[0]
    assert n == 2 and list(res.sub_col[b:b + n]) == [0, 1] and list(res.sub_val[b:b + n]) == [2.0, 1.0]
    assert res.sub_rhs[0] == 4.0
    x = oracle.postsolve_primal(res, np.array([1.5, 0.5]))
    assert list(x) == [1.5, 0.5, 2 * 1.5 + 0.5 - 4]


@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("lo,hi,eliminated", [(-100.0, 100.0, True), (-1.0, 1.0, False), (-INF, 3.0, True),
                                              (-INF, 1.0, False), (-3.0, 5.0, False), (-5.0, 3.0, True)])
def test_implied_free(lo, hi, eliminated, sign):
    # x2 = 2 x0 + x1 - 4 with x0, x1 in [0, 2]: the row implies x2 in [-4, 2], whichever sign the
    # row is written with (x2's coefficient -1, or +1 for the negated row)
    lp = make([{0: 2.0 * sign, 1: 1.0 * sign, 2: -1.0 * sign}, {0: 1.0, 1: 1.0}], [4.0 * sign, -INF],
              [4.0 * sign, 3.0], [0.0, 0.0, lo], [2.0, 2.0, hi], c=[1.0, 2.0, 3.0])
    res = oracle.presolve(lp, opts(max_rounds=1))
    assert (res.col_kind[2] == oracle.COL_SUBST) == eliminated


def test_inequality_rows_at_the_side_the_cost_selects():
    # row 0: x0 + x1 + x2 <= 4 with x2 free and only there.  c2 = -1 pushes x2 (a = 1) up: the row
    # is tight at 4 in an optimum, x2 = 4 - x0 - x1: costs 1 + 1 and 2 + 1, constant -4
    lp = make([{0: 1.0, 1: 1.0, 2: 1.0}, {0: 1.0, 1: 1.0}], [-INF, -INF], [4.0, 3.0],
              [0.0, 0.0, -INF], [2.0, 2.0, INF], c=[1.0, 2.0, -1.0])
    res = oracle.presolve(lp, opts(max_rounds=1))
    assert res.row_kind[0] == oracle.ROW_SUBST and res.sub_rhs[0] == 4.0
    assert list(res.c) == [2.0, 3.0] and res.obj_offset == -4.0
    # c2 = +1 pushes x2 down, to the side -inf: not a candidate
    lp2 = make([{0: 1.0, 1: 1.0, 2: 1.0}, {0: 1.0, 1: 1.0}], [-INF, -INF], [4.0, 3.0],
               [0.0, 0.0, -INF], [2.0, 2.0, INF], c=[1.0, 2.0, 1.0])
    res2 = oracle.presolve(lp2, opts(max_rounds=1))
    assert res2.row_kind[0] != oracle.ROW_SUBST
    # cost 0: the finite side (rhs 4 here, the lhs being -inf)
    lp3 = make([{0: 1.0, 1: 1.0, 2: 1.0}, {0: 1.0, 1: 1.0}], [-INF, -INF], [4.0, 3.0],
               [0.0, 0.0, -INF], [2.0, 2.0, INF], c=[1.0, 2.0, 0.0])
    res3 = oracle.presolve(lp3, opts(max_rounds=1))
    assert res3.row_kind[0] == oracle.ROW_SUBST and res3.sub_rhs[0] == 4.0 and list(res3.c) == [1.0, 2.0]


@pytest.mark.parametrize("seed", range(60))
def test_any_row_optimum_kept_and_postsolve_optimal(seed):
    test_optimum_kept_and_postsolve_optimal(seed, rows="any")


def test_one_substitution_per_column_and_round():
    # rows 0 and 1 are equalities that share x0, each with a free singleton (x2, x3):
    # round 1 applies row 0 only, round 2 row 1
    lp = make([{0: 1.0, 1: 1.0, 2: 1.0}, {0: 1.0, 3: 2.0}, {0: 1.0, 1: -1.0}], [1.0, 2.0, -INF],
              [1.0, 2.0, 1.0], [0.0, 0.0, -INF, -INF], [1.0, 1.0, INF, INF], c=[1.0, 1.0, 0.5, -0.25])
    res = oracle.presolve(lp, opts())
    assert res.row_kind[0] == oracle.ROW_SUBST and res.row_round[0] == 1
    assert res.row_kind[1] == oracle.ROW_SUBST and res.row_round[1] == 2


def test_zero_cost_singletons_do_not_wait():
    # the same two rows with zero-cost singletons change no cost: both in round 1
    lp = make([{0: 1.0, 1: 1.0, 2: 1.0}, {0: 1.0, 3: 2.0}, {0: 1.0, 1: -1.0}], [1.0, 2.0, -INF],
              [1.0, 2.0, 1.0], [0.0, 0.0, -INF, -INF], [1.0, 1.0, INF, INF], c=[1.0, 1.0, 0.0, 0.0])
    res = oracle.presolve(lp, opts())
    assert list(res.row_kind[:2]) == [oracle.ROW_SUBST] * 2 and list(res.row_round[:2]) == [1, 1]
    # x0, x1 kept their cost 1 (no update), so S6 later fixes both at lb = 0
    assert list(res.col_kind[:2]) == [oracle.COL_EMPTY] * 2 and list(res.col_val[:2]) == [0.0, 0.0]
    assert res.obj_offset == 0.0


def test_off_by_default():
    lp = synth.plant_col_singletons(synth.tiny(1), 1)
    res = oracle.presolve(lp)
    assert not np.any(res.row_kind == oracle.ROW_SUBST)


@pytest.mark.parametrize("seed", range(60))
def test_optimum_kept_and_postsolve_optimal(seed, rows="eq"):
    lp = synth.plant_col_singletons(synth.micro(seed + 900), seed, rows=rows)
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
    lp = synth.plant_col_singletons(synth.tiny(seed), seed, rows="any" if seed % 2 else "eq")
    res = oracle.presolve(lp, opts())
    assert res.status == oracle.OK
    assert np.count_nonzero(res.row_kind == oracle.ROW_SUBST) > 0
    st0, x0, f0 = _linprog(lp.c, lp.row_ptr, lp.col_idx, lp.val, lp.lhs, lp.rhs, lp.lb, lp.ub, lp.n)
    st1, x1, f1 = _linprog(res.c, res.row_ptr, res.col_idx, res.val, res.lhs, res.rhs, res.lb, res.ub,
                           res.n_red)
    assert st0 == st1
    if st0 != 0:  # a free singleton can make the LP unbounded: both agree
        return
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
