"""Hand-worked pins of the parallel-row step's repeated leader pass (Sec. 3.2,
parallel rows: hashing, then a leader per group; the pass repeats on the rows
it left unmatched, at most par_max_iter times per group and round).

All LPs here have free columns, so that no activity is finite and parallel
rows are the only reduction: every expected record and side below is worked
out by hand from the leader rule and the merge rule.
  * leader: the first equality row of the live rows of the group (row order),
    else the first live row; it leaves the group whether or not it finds a
    follower;
  * a live row j follows leader i when a_j = lam a_i with lam = a_j1 / a_i1;
  * merge: lam > 0 gives [L_j / lam, U_j / lam], lam < 0 gives
    [U_j / lam, L_j / lam]; the leader keeps the largest lower and the smallest
    upper side over itself and all its followers.
No GPU needed."""
import numpy as np

import oracle
from lpmake import INF, make

FREE3 = dict(lb=[-INF] * 3, ub=[INF] * 3)


def run(lp, **kw):
    return oracle.presolve(lp, oracle.default_opts(**kw))


def sides_of(r, orig_row):
    k = list(r.row_map).index(orig_row)
    return r.lhs[k], r.rhs[k]


def three_classes(eq_last=False):
    """One key group (pattern {0,1,2}, all signs equal) holding three parallel
    classes: a, b, c and 2a, -3b, c/2 (rows 3, 4, 5)."""
    rows = [{0: 1, 1: 2, 2: 3}, {0: 1, 1: 1, 2: 1}, {0: 2, 1: 1, 2: 5},
            {0: 2, 1: 4, 2: 6}, {0: -3, 1: -3, 2: -3}, {0: 1, 1: 0.5, 2: 2.5}]
    lhs = [-INF, -INF, 0, -INF, -30, 1]
    rhs = [12, 20, INF, 20, 3, 4]
    if eq_last:  # c/2 = 3: an equality in the third class
        lhs[5], rhs[5] = 3, 3
    return make(rows, lhs, rhs, **FREE3)


def test_three_classes_need_three_passes():
    # pass 1: leader row 0, follower row 3 (lam 2, sides [-inf, 10]);
    # pass 2: leader row 1, follower row 4 (lam -3: [3 / -3, -30 / -3] = [-1, 10]);
    # pass 3: leader row 2, follower row 5 (lam 0.5: [2, 8])
    r = run(three_classes())
    assert r.status == oracle.OK
    assert list(r.row_kind) == [oracle.ROW_KEPT] * 3 + [oracle.ROW_PARALLEL] * 3
    assert list(r.row_aux[3:]) == [0, 1, 2]
    assert list(r.row_val[3:]) == [2.0, -3.0, 0.5]
    assert list(r.row_round[3:]) == [1, 1, 1]
    assert sides_of(r, 0) == (-INF, 10.0)
    assert sides_of(r, 1) == (-1.0, 10.0)
    assert sides_of(r, 2) == (2.0, 8.0)
    assert r.rounds == 2  # round 2 finds nothing


def test_pass_cap_leaves_the_later_classes():
    # par_max_iter = 2: passes 1 and 2 as above; row 5 stays unmatched.  In
    # later rounds the group {0, 1, 2, 5} is led by row 0, then row 1, again,
    # and the cap stops before row 2 leads: row 5 is never merged.
    r = run(three_classes(), par_max_iter=2)
    assert list(r.row_kind[:5]) == [oracle.ROW_KEPT] * 3 + [oracle.ROW_PARALLEL] * 2
    assert r.row_kind[5] == oracle.ROW_KEPT
    assert sides_of(r, 2) == (0.0, INF) and sides_of(r, 5) == (1.0, 4.0)
    # par_max_iter = 1: only row 3
    r = run(three_classes(), par_max_iter=1)
    assert list(r.row_kind) == [oracle.ROW_KEPT] * 3 + [oracle.ROW_PARALLEL] + [oracle.ROW_KEPT] * 2
    assert sides_of(r, 0) == (-INF, 10.0) and sides_of(r, 1) == (-INF, 20.0)
    # a cap of three passes is enough
    r3 = run(three_classes(), par_max_iter=3)
    assert list(r3.row_kind) == list(run(three_classes()).row_kind)


def test_rows_left_at_the_cap_are_counted():
    # no cap reached: nothing left
    r = run(three_classes())
    assert (r.s5_left, r.s5_capped_groups) == (0, 0)
    # cap 3: the third pass matches the last pair, the group is empty at the cap
    r = run(three_classes(), par_max_iter=3)
    assert (r.s5_left, r.s5_capped_groups) == (0, 0)
    # cap 2: rows 2 and 5 are live after the passes of round 1 and again of round 2
    r = run(three_classes(), par_max_iter=2)
    assert (r.s5_left, r.s5_capped_groups) == (4, 2)
    # cap 1: rows 1, 2, 4, 5 in round 1, the same four in round 2
    r = run(three_classes(), par_max_iter=1)
    assert (r.s5_left, r.s5_capped_groups) == (8, 2)


def test_equality_leads_first_in_every_pass():
    # row 5 is an equality: pass 1 is led by row 5 (the first equality), whose
    # follower is row 2 (lam = 2 / 1 = 2: [0 / 2, inf] = [0, inf]; the leader
    # keeps [3, 3]); pass 2 by row 0 (follower row 3), pass 3 by row 1 (row 4)
    r = run(three_classes(eq_last=True))
    assert r.status == oracle.OK
    kinds = [oracle.ROW_PARALLEL if i in (2, 3, 4) else oracle.ROW_KEPT for i in range(6)]
    assert list(r.row_kind) == kinds
    assert r.row_aux[2] == 5 and r.row_val[2] == 2.0
    assert r.row_aux[3] == 0 and r.row_aux[4] == 1
    assert sides_of(r, 5) == (3.0, 3.0)
    # with one pass only row 2 is merged: later rounds are led by row 5 again
    r = run(three_classes(eq_last=True), par_max_iter=1)
    assert [i for i in range(6) if r.row_kind[i] == oracle.ROW_PARALLEL] == [2]


def test_several_followers_merge_by_max_and_min():
    # leader row 0: x0 + x1 <= 10; followers, in row order:
    #   row 1: 2x0 + 2x1 in [2, 30]    -> lam 2:  [1, 15]
    #   row 2: -x0 - x1 in [-8, -3]    -> lam -1: [3, 8]
    #   row 3: 4x0 + 4x1 in [-4, 36]   -> lam 4:  [-1, 9]
    #   row 4: -0.5x0 - 0.5x1 >= -4.5  -> lam -0.5: [-inf, 9]
    # the leader's sides become [max(-inf, 1, 3, -1, -inf), min(10, 15, 8, 9, 9)] = [3, 8]
    lp = make([{0: 1, 1: 1}, {0: 2, 1: 2}, {0: -1, 1: -1}, {0: 4, 1: 4}, {0: -0.5, 1: -0.5}],
              [-INF, 2, -8, -4, -4.5], [10, 30, -3, 36, INF], [-INF] * 2, [INF] * 2)
    r = run(lp)
    assert list(r.row_kind) == [oracle.ROW_KEPT] + [oracle.ROW_PARALLEL] * 4
    assert list(r.row_aux[1:]) == [0, 0, 0, 0]
    assert list(r.row_val[1:]) == [2.0, -1.0, 4.0, -0.5]
    assert sides_of(r, 0) == (3.0, 8.0)
    # the same rows in another order: the merged sides do not depend on it
    perm = [0, 3, 4, 1, 2]
    lp2 = make([[{0: 1, 1: 1}, {0: 2, 1: 2}, {0: -1, 1: -1}, {0: 4, 1: 4}, {0: -0.5, 1: -0.5}][k] for k in perm],
               [[-INF, 2, -8, -4, -4.5][k] for k in perm], [[10, 30, -3, 36, INF][k] for k in perm],
               [-INF] * 2, [INF] * 2)
    assert sides_of(run(lp2), 0) == (3.0, 8.0)


def test_followers_that_cross_make_the_leader_infeasible():
    # leader x0 + x1 <= 10 with followers saying x0 + x1 >= 6 (2x0 + 2x1 >= 12)
    # and x0 + x1 <= 5 (-x0 - x1 >= -5): merged [6, 5] crosses by 1 > 1e-9 * 6
    lp = make([{0: 1, 1: 1}, {0: 2, 1: 2}, {0: -1, 1: -1}], [-INF, 12, -5], [10, INF, INF], [-INF] * 2,
              [INF] * 2)
    r = run(lp)
    assert r.status == oracle.INFEASIBLE and r.where == 1 and r.index == 0 and r.round == 1


def test_non_parallel_rows_of_one_key_stay():
    # same pattern and signs, no two rows parallel: every pass finds nothing,
    # each leader leaves the group, nothing is removed
    lp = make([{0: 1, 1: 2}, {0: 1, 1: 3}, {0: 1, 1: 4}, {0: 2, 1: 9}], [-INF] * 4, [1, 2, 3, 4], [-INF] * 2,
              [INF] * 2)
    r = run(lp)
    assert np.all(r.row_kind == oracle.ROW_KEPT) and r.rounds == 1


def later_pass_only_lp():
    """Rows p = x + y + 2z, q = y + 3z, q' = 5x + 2y + 6z and the singleton
    row x = 2 (x in [0, 10], y and z free).  Round 1 fixes x (S2, S3', S4);
    p and q' share a key but are not parallel.  Round 2 sees p = y + 2z,
    q = y + 3z, q' = 2y + 6z (sides shifted by the fixed x): one key group,
    pass 1 led by p finds nothing, pass 2 led by q takes q' (lambda 2).  That
    merge is the round's only reduction."""
    return make([{0: 1, 1: 1, 2: 2}, {1: 1, 2: 3}, {0: 5, 1: 2, 2: 6}, {0: 1}],
                [-INF, -INF, -20, 2], [12, 7, INF, 2], [0, -INF, -INF], [10, INF, INF])


def test_a_later_pass_alone_reduces_a_round():
    r = run(later_pass_only_lp())
    assert r.status == oracle.OK
    assert list(r.row_kind) == [oracle.ROW_KEPT, oracle.ROW_KEPT, oracle.ROW_PARALLEL, oracle.ROW_SINGLETON]
    assert r.row_aux[2] == 1 and r.row_val[2] == 2.0 and r.row_round[2] == 2
    assert r.col_kind[0] == oracle.COL_FIXED and r.col_val[0] == 2.0
    # q' after the shift: 2y + 6z >= -20 - 5 * 2 = -30, divided by 2: q gets [-15, 7]
    assert sides_of(r, 1) == (-15.0, 7.0)
    assert sides_of(r, 0) == (-INF, 10.0)  # 12 - 1 * 2
    assert list(r.round_rows_removed) == [1, 1, 0]
    assert r.m_red == 2 and r.rounds == 3


# ------------------------------------- rows parallel only on the reduced matrix
def test_rows_made_parallel_by_a_fixed_column_merge_in_round_two():
    """A = x1 + x2 <= 6 and B = x0 + 2 x1 + 2 x2 <= 13 with x0 fixed at 0: B
    loses x0 in round 1 (S4 fixes it, the compaction drops it and renumbers
    x1, x2), so round 2 finds B = 2 A with B's side 13 - 0 = 13 -> 6.5; A keeps
    min(6, 6.5) = 6.  Worked by hand: no bound moves (x_j <= 6, 6.5 > 5)."""
    lp = make([{1: 1.0, 2: 1.0}, {0: 1.0, 1: 2.0, 2: 2.0}], lhs=[-INF, -INF], rhs=[6, 13],
              lb=[0, 0, 0], ub=[0, 5, 5], c=[1, 1, 1])
    r = run(lp)
    assert list(r.col_kind) == [oracle.COL_FIXED, 0, 0] and list(r.col_round) == [1, 0, 0]
    assert r.row_kind[1] == oracle.ROW_PARALLEL and r.row_round[1] == 2
    assert r.row_aux[1] == 0 and r.row_val[1] == 2.0
    assert r.row_kind[0] == 0 and sides_of(r, 0) == (-INF, 6.0)


def test_late_parallel_recipe_every_planted_pair_merges_in_round_two():
    """synth.late_parallel by construction: each non-decoy pair (A_t, B_t)
    merges in round 2 (the lower row index leads, lam or 1/lam exactly: both
    are powers of two or +-1), each decoy pair stays; no column bound moves,
    only the fixed columns go."""
    from paper_2609_16182_gb300 import synth
    for seed in range(2):
        lp = synth.late_parallel(seed, pairs=120)
        P = lp.planted
        r = run(lp)
        assert r.status == 0
        assert list(np.flatnonzero(r.col_kind != 0)) == list(range(120))
        for t, (a, b) in enumerate(zip(P["a_row"], P["b_row"])):
            if P["decoy"][t]:
                assert r.row_kind[a] == 0 and r.row_kind[b] == 0
                continue
            lam = P["lam"][t]
            lead, fol, lv = (a, b, lam) if a < b else (b, a, 1.0 / lam)
            assert (r.row_kind[fol], r.row_aux[fol], r.row_round[fol]) == (oracle.ROW_PARALLEL, lead, 2)
            assert r.row_val[fol] == lv and r.row_kind[lead] == 0
