"""Hand-worked LPs, one per reduction rule, pinning the oracle (CPU only).

Every expected value below is worked out by hand from the rule it tests; the
rules are the readings of Sec. 2.1 / 3.1 / 3.2 recorded in the design notes.
"""
import json
import os

import numpy as np
import pytest

import oracle
from lpmake import INF, from_json, make

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def run(lp, **kw):
    return oracle.presolve(lp, oracle.default_opts(**kw))


def test_worked_example_sec31():
    """Sec. 3.1: x1 + 2 x2 <= 4, x >= 0 implies x1 <= 4, x2 <= 2."""
    g = json.load(open(os.path.join(GOLDEN, "worked_example_sec31.json")))
    lp = from_json(g["lp"])
    r = run(lp)
    assert r.status == oracle.OK
    np.testing.assert_array_equal(r.col_ub, g["expect"]["ub"])
    np.testing.assert_array_equal(r.col_lb, g["expect"]["lb"])
    assert r.m_red == 1 and r.n_red == 2
    assert r.rounds == 2  # round 2 finds nothing new


def test_empty_row_removed_or_infeasible():
    lp = make([{}, {0: 1.0, 1: 1.0}], lhs=[-1, -INF], rhs=[2, 5], lb=[0, 0], ub=[10, 10])
    r = run(lp)
    assert r.row_kind[0] == oracle.ROW_EMPTY and r.row_round[0] == 1
    lp = make([{0: 1.0, 1: 1.0}, {}], lhs=[-INF, 1], rhs=[5, 2], lb=[0, 0], ub=[10, 10])
    r = run(lp)
    assert r.status == oracle.INFEASIBLE and r.where == 1 and r.index == 1 and r.round == 1


def test_redundant_row_then_empty_columns():
    # x1 + x2 <= 10 with 0 <= x <= 1: max activity 2 <= 10 -> redundant.
    # Both columns are then empty: c1 = 1 > 0 -> lb = 0, c2 = -1 < 0 -> ub = 1.
    lp = make([{0: 1.0, 1: 1.0}], lhs=[-INF], rhs=[10], lb=[0, 0], ub=[1, 1], c=[1.0, -1.0])
    r = run(lp)
    assert r.status == oracle.OK
    assert r.row_kind[0] == oracle.ROW_REDUNDANT
    assert list(r.col_kind) == [oracle.COL_EMPTY, oracle.COL_EMPTY]
    assert list(r.col_val) == [0.0, 1.0]
    assert r.obj_offset == -1.0
    assert r.m_red == 0 and r.n_red == 0


def test_singleton_rows_become_bounds():
    # 2 x1 <= 3 -> x1 <= 1.5 ; -2 x2 >= -3 -> x2 <= 1.5 ; 4 x3 in [-2, 2] -> x3 in [-0.5, 0.5]
    lp = make([{0: 2.0}, {1: -2.0}, {2: 4.0}, {0: 1.0, 1: 1.0, 2: 1.0}],
              lhs=[-INF, -3, -2, -INF], rhs=[3, INF, 2, 25], lb=[0, 0, -10], ub=[10, 10, 10])
    r = run(lp, dual_reductions=0)
    assert list(r.row_kind[:3]) == [oracle.ROW_SINGLETON] * 3
    assert list(r.row_aux[:3]) == [0, 1, 2]
    assert list(r.row_val[:3]) == [2.0, -2.0, 4.0]
    assert r.col_ub[0] == 1.5 and r.col_ub[1] == 1.5
    assert r.col_lb[0] == 0.0 and r.col_lb[1] == 0.0  # -2 x2 >= -3 bounds x2 above only
    assert r.col_lb[2] == -0.5 and r.col_ub[2] == 0.5
    # round 1: the last row has max activity 30 > 25; round 2: 1.5 + 1.5 + 0.5
    # = 3.5 <= 25 and lhs = -inf -> redundant
    assert r.row_kind[3] == oracle.ROW_REDUNDANT and r.row_round[3] == 2


def test_infeasible_activity():
    # x1 + x2 >= 5 with 0 <= x <= 1: max activity 2 < 5
    lp = make([{0: 1.0, 1: 1.0}], lhs=[5], rhs=[INF], lb=[0, 0], ub=[1, 1])
    r = run(lp)
    assert r.status == oracle.INFEASIBLE and r.where == 1 and r.index == 0


def test_infeasible_min_activity_is_a_row_verdict():
    # x1 + x2 <= -1 with x >= 0: min activity 0 > -1, found by S2 at the row (S3 alone would find
    # column 0's bounds crossing)
    lp = make([{0: 1.0, 1: 1.0}], lhs=[-INF], rhs=[-1], lb=[0, 0], ub=[1, 1])
    r = run(lp)
    assert (r.status, r.where, r.index, r.round) == (oracle.INFEASIBLE, 1, 0, 1)


def test_residual_activity_of_lower_bounds():
    # x1 + x2 <= 10 with x1 >= 2, x2 >= 3: u1 <= 10 - 3 = 7 and u2 <= 10 - 2 = 8
    lp = make([{0: 1.0, 1: 1.0}], lhs=[-INF], rhs=[10], lb=[2, 3], ub=[100, 100])
    r = run(lp, max_rounds=1)
    assert (r.ub[0], r.ub[1]) == (7.0, 8.0)


def test_the_one_infinite_term_gets_the_bound():
    # x1 + x2 <= 5 with x1 in (-inf, 100], x2 in [1, 3]: x1 is the row's one infinite term of the min
    # activity, so it alone gets u1 <= 5 - 1 = 4; x2's residual is infinite (no bound from this row)
    lp = make([{0: 1.0, 1: 1.0}], lhs=[-INF], rhs=[5], lb=[-INF, 1], ub=[100, 3])
    r = run(lp, max_rounds=1)
    assert (r.ub[0], r.ub[1], r.lb[0]) == (4.0, 3.0, -INF)


def test_crossing_bounds_infeasible_column():
    # singletons x1 >= 5 and x1 <= 3 give l = 5 > u = 3
    lp = make([{0: 1.0}, {0: 1.0}], lhs=[5, -INF], rhs=[INF, 3], lb=[0], ub=[10])
    r = run(lp)
    assert r.status == oracle.INFEASIBLE and r.where == 2 and r.index == 0 and r.round == 1
    lp = make([{0: 1.0, 1: 1.0}], lhs=[-INF], rhs=[100], lb=[2, 0], ub=[1, 1])  # lb > ub on input
    r = run(lp)
    assert r.status == oracle.INFEASIBLE and r.where == 2 and r.index == 0


def test_fix_shift_and_offset():
    # x1 + x2 + x3 = 4, x1 fixed at 1, x2, x3 in [0, 10], c = (2, 0, 0).
    # Round 1: min activity 1, candidates x2 <= 3, x3 <= 3 accepted; x1 fixed,
    # row shifted to x2 + x3 = 3; offset 2*1 = 2.
    lp = make([{0: 1.0, 1: 1.0, 2: 1.0}], lhs=[4], rhs=[4], lb=[1, 0, 0], ub=[1, 10, 10], c=[2.0, 0, 0])
    r = run(lp)
    assert r.status == oracle.OK
    assert r.col_kind[0] == oracle.COL_FIXED and r.col_val[0] == 1.0 and r.col_round[0] == 1
    assert r.obj_offset == 2.0
    assert r.m_red == 1 and r.n_red == 2
    assert list(r.lhs) == [3.0] and list(r.rhs) == [3.0]
    assert list(r.ub) == [3.0, 3.0] and list(r.lb) == [0.0, 0.0]
    assert list(r.col_map) == [1, 2] and list(r.row_map) == [0]
    assert r.rounds == 2


def test_empty_column_rules():
    # column 0 in no row, c=0, free -> 0 ; column 2 in no row, c=-1, ub=+inf -> unbounded
    lp = make([{1: 1.0, 3: 1.0}], lhs=[-INF], rhs=[1], lb=[-INF, 0, 0, 0], ub=[INF, 5, 5, 5],
              c=[0.0, 1.0, 0.0, 1.0])
    r = run(lp)
    assert r.col_kind[0] == oracle.COL_EMPTY and r.col_val[0] == 0.0
    assert r.col_kind[2] == oracle.COL_EMPTY and r.col_val[2] == 0.0  # c=0: finite lb first
    lp = make([{1: 1.0}], lhs=[-INF], rhs=[1], lb=[0, 0, 0], ub=[5, 5, INF], c=[0.0, 1.0, -1.0])
    r = run(lp)
    assert r.status == oracle.UNBOUNDED and r.where == 2 and r.index == 2
    r = run(lp, dual_reductions=0)
    assert r.status == oracle.OK and r.col_kind[2] == oracle.COL_KEPT


def test_parallel_rows_merge_into_equality_leader():
    # row0: x1 + 2x2 <= 6 ; row1: -2x1 - 4x2 = -8 (equality -> leader);
    # follower row0 has lambda = 1 / -2 = -0.5; its sides divided by lambda
    # give lo = 6 / -0.5 = -12, hi = +inf; leader stays -8 = -8.
    lp = make([{0: 1.0, 1: 2.0}, {0: -2.0, 1: -4.0}, {0: 1.0, 1: 1.0, 2: 1.0}],
              lhs=[-INF, -8, -INF], rhs=[6, -8, 50], lb=[-INF, -INF, 0], ub=[INF, INF, 1])
    r = run(lp)
    assert r.row_kind[0] == oracle.ROW_PARALLEL and r.row_aux[0] == 1 and r.row_val[0] == -0.5
    assert r.row_kind[1] == oracle.ROW_KEPT
    k = list(r.row_map).index(1)
    assert r.lhs[k] == -8.0 and r.rhs[k] == -8.0


def test_parallel_rows_inequality_leader_and_infeasible_pair():
    # x1 + x2 <= 1 and 2x1 + 2x2 >= 4 (free variables): leader row0,
    # lambda = 2, lo = 4/2 = 2 > 1 -> infeasible at the leader
    lp = make([{0: 1.0, 1: 1.0}, {0: 2.0, 1: 2.0}], lhs=[-INF, 4], rhs=[1, INF], lb=[-INF, -INF],
              ub=[INF, INF])
    r = run(lp)
    assert r.status == oracle.INFEASIBLE and r.where == 1 and r.index == 0
    # consistent version: sides merge to [2, 3]
    lp = make([{0: 1.0, 1: 1.0}, {0: 2.0, 1: 2.0}], lhs=[-INF, 4], rhs=[3, INF], lb=[-INF, -INF],
              ub=[INF, INF])
    r = run(lp)
    assert r.status == oracle.OK and r.row_kind[1] == oracle.ROW_PARALLEL and r.row_val[1] == 2.0
    assert list(r.lhs) == [2.0] and list(r.rhs) == [3.0]


def test_parallel_rows_negative_factor_swaps_the_sides():
    # leader x1 + x2 <= 3, follower -2 x1 - 2 x2 <= -2 (lambda = -2): the follower says x1 + x2 >= 1,
    # so the leader's sides become [1, 3]
    lp = make([{0: 1.0, 1: 1.0}, {0: -2.0, 1: -2.0}], lhs=[-INF, -INF], rhs=[3, -2], lb=[-INF, -INF],
              ub=[INF, INF])
    r = run(lp)
    assert r.row_kind[1] == oracle.ROW_PARALLEL and r.row_val[1] == -2.0
    assert list(r.lhs) == [1.0] and list(r.rhs) == [3.0]


def test_parallel_needs_same_pattern_and_ratio():
    # same pattern, ratio differs in the second coefficient -> not parallel
    lp = make([{0: 1.0, 1: 2.0}, {0: 2.0, 1: 4.000001}], lhs=[-INF, -INF], rhs=[1, 1],
              lb=[-INF, -INF], ub=[INF, INF])
    r = run(lp)
    assert list(r.row_kind) == [0, 0]
    lp = make([{0: 1.0, 1: 2.0}, {0: 2.0, 2: 4.0}], lhs=[-INF, -INF], rhs=[1, 1],
              lb=[-INF, -INF, -INF], ub=[INF, INF, INF])
    r = run(lp)
    assert list(r.row_kind) == [0, 0]


def test_huge_threshold_means_infinite():
    lp = make([{0: 1.0, 1: -1.0}], lhs=[-1e20], rhs=[1e21], lb=[-1e20, 0], ub=[1, 1e20])
    amin, amax, nmin, nmax = oracle.activities(lp)
    # min: a=1 uses lb0=-inf (count), a=-1 uses ub1=+inf (count)
    assert nmin[0] == 2 and nmax[0] == 0 and amax[0] == 1.0 - 0.0
    r = run(lp)
    assert r.row_kind[0] == oracle.ROW_REDUNDANT  # both sides infinite


def test_snap_close_bounds():
    lp = make([{0: 1.0, 1: 1.0}], lhs=[-INF], rhs=[100], lb=[1.0, 0], ub=[1.0 + 1e-12, 1], c=[1.0, 0])
    r = run(lp)
    assert r.col_kind[0] == oracle.COL_FIXED
    assert r.col_val[0] == 0.5 * (1.0 + (1.0 + 1e-12))


def test_acceptance_threshold_and_cap():
    # candidate u1 = 2 - 1 = 1 vs u1 = 1 + 1e-7: improvement 1e-7 < 1e-6 -> rejected
    lp = make([{0: 1.0, 1: 1.0}, {0: 1.0, 1: 1.0, 2: 1.0}], lhs=[-INF, -INF], rhs=[2, 1000],
              lb=[0, 1, 0], ub=[1 + 1e-7, 5, 5])
    r = run(lp)
    assert r.col_ub[0] == 1 + 1e-7
    # x1 + 1e-11 x2 <= 1, x1 in [0, 5], x2 >= 0: candidate x2 <= 1e11 > 1e10 -> dropped
    lp = make([{0: 1.0, 1: 1e-11}, {0: 1.0, 2: 1.0}], lhs=[-INF, -INF], rhs=[1, 1000],
              lb=[0, 0, 0], ub=[5, INF, 5])
    r = run(lp)
    assert r.col_ub[1] == INF
    assert r.col_ub[0] == 1.0  # x1 <= 1 - 1e-11*0 is accepted


def test_invalid_inputs_rejected():
    good = dict(lhs=[-INF], rhs=[1], lb=[0, 0], ub=[1, 1])
    lp = make([{0: 1.0, 1: 1.0}], **good)
    lp.col_idx[:] = [1, 0]
    with pytest.raises(ValueError):
        run(lp)
    lp = make([{0: 1.0, 1: 0.0}], **good)
    with pytest.raises(ValueError):
        run(lp)
    lp = make([{0: 1.0, 1: 1.0}], lhs=[-INF], rhs=[1], lb=[INF, 0], ub=[1, 1])
    with pytest.raises(ValueError):
        run(lp)


def test_round_cap():
    # a propagation chain needs several rounds; max_rounds=1 stops after one
    lp = make([{0: 1.0, 1: -1.0}, {1: 1.0, 2: -1.0}, {2: 1.0, 3: -1.0}, {0: 1.0, 1: 1.0, 2: 1.0, 3: 1.0}],
              lhs=[-INF] * 4, rhs=[0, 0, 0, 100], lb=[0, 0, 0, 0], ub=[10, 20, 30, 1])
    r1 = run(lp, max_rounds=1)
    assert r1.rounds == 1
    r = run(lp)
    assert r.rounds > 1
    assert r.col_ub[0] == 1.0 and r.col_ub[1] == 1.0 and r.col_ub[2] == 1.0
