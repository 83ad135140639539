"""Pins of the oracle's doubleton-equation step (S5e, opt-in), without a GPU.

A kept equality a x_j + b x_k = c with two live columns eliminates x_k (the
column with fewer entries): x_k = g - f x_j with f = a / b, g = c / b.  The
other rows of x_k lose that entry and their sides a_rk g, and x_j's
coefficient there gains -(a_rk f); x_j's bounds meet those x_k's bounds give
it; c_j <- c_j - (c_k / b) a with the constant c_k g.  Pinned against
hand-worked rows, the optimal value of the LP (vertex enumeration, scipy) and
a postsolved point that is feasible and optimal.
"""
import numpy as np
import pytest

import oracle
from lpbrute import inequalities, lp_vertices, vertices
from lpmake import INF, make
from paper_2609_16182_gb300 import synth


def opts(**kw):
    return oracle.default_opts(doubletons=1, **kw)


def row_of(res, orig_row):
    i = int(np.flatnonzero(res.row_map == orig_row)[0])
    b, e = res.row_ptr[i], res.row_ptr[i + 1]
    return dict(zip(res.col_map[res.col_idx[b:e]].tolist(), res.val[b:e].tolist())), res.lhs[i], res.rhs[i]


def test_hand_worked_elimination():
    # row 0: x0 + 2 x1 = 4, x1 has fewer entries: x1 = 2 - x0 / 2 (f = 1/2, g = 2)
    # row 1: 3 x0 + 4 x1 + x2 <= 10 -> (3 - 4/2) x0 + x2 <= 10 - 4*2, i.e. x0 + x2 <= 2
    # row 2: x0 - x2 >= -5, untouched.  x1 in [0, 1.5] gives x0 in [1, 4]; x0 was in [0, 3]
    # costs 1, 2, 3: c0 = 1 - (2 / 2) * 1 = 0, constant 2 * 2 = 4
    lp = make([{0: 1.0, 1: 2.0}, {0: 3.0, 1: 4.0, 2: 1.0}, {0: 1.0, 2: -1.0}], [4.0, -INF, -5.0], [4.0, 10.0, INF],
              [0.0, 0.0, -1.0], [3.0, 1.5, 1.0], c=[1.0, 2.0, 3.0])
    res = oracle.presolve(lp, opts(max_rounds=1, dual_reductions=0))
    assert res.row_kind[0] == oracle.ROW_DOUBLETON and res.row_aux[0] == 1 and res.row_val[0] == 2.0
    assert res.col_kind[1] == oracle.COL_DOUBLETON and res.col_val[1] == 2.0
    entries, lhs, rhs = row_of(res, 1)
    assert entries == {0: 1.0, 2: 1.0} and rhs == 2.0 and lhs == -INF
    k0 = int(np.flatnonzero(res.col_map == 0)[0])
    assert (res.lb[k0], res.ub[k0]) == (1.0, 3.0) and res.c[k0] == 0.0 and res.obj_offset == 4.0
    b = res.sub_beg[0]
    assert res.sub_len[0] == 1 and res.sub_col[b] == 0 and res.sub_val[b] == 1.0 and res.sub_rhs[0] == 4.0
    x = oracle.postsolve_primal(res, np.array([2.0, 0.0]))
    assert list(x) == [2.0, 1.0, 0.0]


def test_both_sides_of_a_changed_row_shift():
    # the hand-worked LP with row 1 two-sided, -20 <= 3 x0 + 4 x1 + x2 <= 10: both sides lose 4 g = 8
    lp = make([{0: 1.0, 1: 2.0}, {0: 3.0, 1: 4.0, 2: 1.0}, {0: 1.0, 2: -1.0}], [4.0, -20.0, -5.0], [4.0, 10.0, INF],
              [0.0, 0.0, -1.0], [3.0, 1.5, 1.0], c=[1.0, 2.0, 3.0])
    res = oracle.presolve(lp, opts(max_rounds=1, dual_reductions=0))
    entries, lhs, rhs = row_of(res, 1)
    assert entries == {0: 1.0, 2: 1.0} and (lhs, rhs) == (-28.0, 2.0)


def test_doubletons_sharing_a_changed_row_wait_a_round():
    # rows 0 and 1 eliminate x1 and x3 (the shorter columns); row 2 holds both, so both claim it:
    # row 0 applies in round 1, row 1 in round 2
    lp = make([{0: 1.0, 1: 1.0}, {2: 1.0, 3: 1.0}, {1: 1.0, 3: 1.0, 4: 1.0}, {0: 1.0, 2: 1.0}, {0: 1.0, 2: -1.0}],
              [1.0, 1.0, -INF, -INF, -0.5], [1.0, 1.0, 2.0, 1.5, INF],
              [0.0] * 5, [1.0] * 5, c=[1.0] * 5)
    res = oracle.presolve(lp, opts(dual_reductions=0))
    assert res.status == oracle.OK
    assert list(res.row_kind[:2]) == [oracle.ROW_DOUBLETON] * 2 and list(res.row_round[:2]) == [1, 2]


def test_cancellation_drops_the_entry():
    # row 1: 2 x0 + 4 x1 + x2 <= 10 -> (2 - 2) x0 + x2 <= 2: x0 leaves row 1
    lp = make([{0: 1.0, 1: 2.0}, {0: 2.0, 1: 4.0, 2: 1.0}, {0: 1.0, 2: -1.0}], [4.0, -INF, -5.0], [4.0, 10.0, INF],
              [0.0, 0.0, -1.0], [3.0, 1.5, 1.0], c=[1.0, 2.0, 3.0])
    res = oracle.presolve(lp, opts(max_rounds=1, dual_reductions=0))
    assert res.row_kind[0] == oracle.ROW_DOUBLETON
    assert res.row_kind[1] != oracle.ROW_KEPT or 0 not in row_of(res, 1)[0]


def test_doubletons_sharing_a_column_wait_a_round():
    # rows 0 and 1 are doubletons on x0 (x1 and x2 are eliminated, fewer entries): they claim x0 both,
    # so row 0 applies in round 1 and row 1 in round 2
    lp = make([{0: 1.0, 1: 1.0}, {0: 2.0, 2: 1.0}, {0: 1.0, 3: 1.0}, {0: 1.0, 3: -1.0}],
              [1.0, 3.0, -INF, -INF], [1.0, 3.0, 5.0, 5.0],
              [0.0, 0.0, 0.0, 0.0], [1.0, 1.0, 2.0, 2.0], c=[1.0, 1.0, 1.0, 1.0])
    res = oracle.presolve(lp, opts(dual_reductions=0))
    assert list(res.row_kind[:2]) == [oracle.ROW_DOUBLETON] * 2
    assert list(res.row_round[:2]) == [1, 2]
    assert list(res.col_kind[1:3]) == [oracle.COL_DOUBLETON] * 2


def test_an_empty_bound_transfer_is_found_by_s2_first():
    # x0 + x1 = 10 with x1 in [0, 1] would force x0 into [9, 10], but x0 <= 2.  A two-entry row's
    # activity range is exactly the condition for the transferred range to meet x_j's bounds, so
    # S2's activity test reports the row (round 1) before S5e runs
    lp = make([{0: 1.0, 1: 1.0}, {0: 1.0, 2: 1.0}, {0: 1.0, 2: -1.0}], [10.0, -INF, -INF], [10.0, 50.0, 50.0],
              [0.0, 0.0, 0.0], [2.0, 1.0, 1.0], c=[1.0, 1.0, 1.0])
    res = oracle.presolve(lp, opts())
    assert (res.status, res.where, res.index, res.round) == (oracle.INFEASIBLE, oracle.WHERE_ROW, 0, 1)


def test_empty_bound_transfer_after_tightening():
    # x0 in [8.999995, 100]; row 0 (x0 + x1 = 10, x1 in [0, 1]) implies l0 >= 9, a gain below
    # bound_tol * 9, which S3 rejects; row 1 tightens u0 to 8.999998 in the same round.  S5e maps
    # x1's range onto x0, [9, 10], which misses [8.999995, 8.999998] by 2e-6 > feas_tol * 9:
    # infeasible at column 0 in round 1.  Without S5e, S2 finds row 0 in round 2.
    lp = make([{0: 1.0, 1: 1.0}, {0: 1.0, 2: 1.0}], [10.0, -INF], [10.0, 8.999998],
              [8.999995, 0.0, 0.0], [100.0, 1.0, 1.0], c=[1.0, 1.0, 1.0])
    res = oracle.presolve(lp, opts())
    assert (res.status, res.where, res.index, res.round) == (oracle.INFEASIBLE, oracle.WHERE_COL, 0, 1)
    res = oracle.presolve(lp, oracle.default_opts())
    assert (res.status, res.where, res.index, res.round) == (oracle.INFEASIBLE, oracle.WHERE_ROW, 0, 2)


def test_transferred_bounds_within_tolerance_snap():
    # x0 + x1 = 10, x1 in [0, 1] moves [9, 10] onto x0 in [9 - 4e-6, 9 + 5e-9] (S3 rejects row 0's
    # l0 >= 9, a gain below bound_tol * 9): [9, 9 + 5e-9], 5e-9 apart, within feas_tol * 9.  As in
    # S3', the bounds snap to their midpoint although they do not cross; x0 is fixed in round 2
    lp = make([{0: 1.0, 1: 1.0}], [10.0], [10.0], [9.0 - 4e-6, 0.0], [9.0 + 5e-9, 1.0], c=[1.0, 1.0])
    mid = 0.5 * (9.0 + (9.0 + 5e-9))
    res = oracle.presolve(lp, opts(max_rounds=1, dual_reductions=0))
    assert res.row_kind[0] == oracle.ROW_DOUBLETON and (res.lb[0], res.ub[0]) == (mid, mid)  # snapped in S5e
    res = oracle.presolve(lp, opts(dual_reductions=0))
    assert res.status == oracle.OK and res.row_kind[0] == oracle.ROW_DOUBLETON
    assert list(res.col_kind) == [oracle.COL_FIXED, oracle.COL_DOUBLETON] and list(res.col_round) == [2, 1]
    assert res.col_val[0] == mid


def test_two_empty_transfers_report_the_smaller_column():
    # the construction above twice: row 0 moves x3's range onto x2, row 1 x1's onto x0; both
    # miss.  The verdict names the smaller original column (0), not the first row's (2)
    lp = make([{2: 1.0, 3: 1.0}, {0: 1.0, 1: 1.0}, {2: 1.0, 4: 1.0}, {0: 1.0, 5: 1.0}],
              [10.0, 10.0, -INF, -INF], [10.0, 10.0, 8.999998, 8.999998],
              [8.999995, 0.0, 8.999995, 0.0, 0.0, 0.0], [100.0, 1.0, 100.0, 1.0, 1.0, 1.0], c=[1.0] * 6)
    res = oracle.presolve(lp, opts())
    assert (res.status, res.where, res.index, res.round) == (oracle.INFEASIBLE, oracle.WHERE_COL, 0, 1)


def test_steps_before_s5e_take_precedence():
    # x0 + x1 = 2 with x1 a free, zero-cost column singleton: S5d (when on) eliminates x1 through
    # row 0 first, so S5e finds no candidate; without S5d, S5e eliminates x1 (the shorter column)
    lp = make([{0: 1.0, 1: 1.0}, {0: 1.0, 2: 1.0}], [2.0, -INF], [2.0, 3.0],
              [0.0, -INF, 0.0], [5.0, INF, 5.0], c=[1.0, 0.0, 1.0])
    res = oracle.presolve(lp, opts(max_rounds=1, dual_reductions=0))
    assert (res.row_kind[0], res.col_kind[1]) == (oracle.ROW_DOUBLETON, oracle.COL_DOUBLETON)
    res = oracle.presolve(lp, opts(col_singletons=1, max_rounds=1, dual_reductions=0))
    assert (res.row_kind[0], res.col_kind[1]) == (oracle.ROW_SUBST, oracle.COL_SUBST)
    # x1 = 2 x0 column-wise (rows 0 and 1, costs 1 and 2): S5c merges x1 into x0 before S5e,
    # and row 0 then holds a merged column, which S5e does not take
    lp = make([{0: 1.0, 1: 2.0}, {0: 1.0, 1: 2.0, 2: 1.0}], [3.0, -INF], [3.0, 9.0],
              [0.0, 0.0, 0.0], [4.0, 4.0, 4.0], c=[1.0, 2.0, 1.0])
    res = oracle.presolve(lp, opts(max_rounds=1, dual_reductions=0))
    assert (res.row_kind[0], res.col_kind[1]) == (oracle.ROW_DOUBLETON, oracle.COL_DOUBLETON)
    res = oracle.presolve(lp, opts(parallel_cols=1, max_rounds=1, dual_reductions=0))
    assert (res.row_kind[0], res.col_kind[1]) == (oracle.ROW_KEPT, oracle.COL_PARALLEL)


def test_off_by_default():
    lp = synth.lprelax(1, m=600, n=1200, target_nnz=9_600, n_dense=1, dense_len=200)
    assert not np.any(oracle.presolve(lp).row_kind == oracle.ROW_DOUBLETON)


@pytest.mark.parametrize("seed", range(60))
def test_optimum_kept_and_postsolve_optimal(seed):
    base = synth.micro(seed + 1700)
    Vb = lp_vertices(base)
    # through the mean of the LP's vertices (feasible) when it has some: the LP stays feasible
    lp = synth.plant_doubletons(base, seed, point=Vb.mean(axis=0) if len(Vb) else None)
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


@pytest.mark.parametrize("seed", range(3))
def test_reduced_optimum_matches_original_lprelax(seed):
    pytest.importorskip("scipy")
    from test_oracle_invariants import _linprog
    lp = synth.lprelax(seed, m=1_500, n=3_000, target_nnz=24_000, n_dense=1, dense_len=600)
    res = oracle.presolve(lp, opts())
    assert res.status == oracle.OK
    assert np.count_nonzero(res.row_kind == oracle.ROW_DOUBLETON) > 0
    st0, x0, f0 = _linprog(lp.c, lp.row_ptr, lp.col_idx, lp.val, lp.lhs, lp.rhs, lp.lb, lp.ub, lp.n)
    st1, x1, f1 = _linprog(res.c, res.row_ptr, res.col_idx, res.val, res.lhs, res.rhs, res.lb, res.ub, res.n_red)
    assert st0 == st1
    if st0 != 0:
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
