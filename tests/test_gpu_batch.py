"""Batched presolve (lpp_presolve_batch): ragged LPs in one arena.

Each member must get exactly the result it gets alone (lpp_presolve) --
records, maps, reduced structure bit for bit, values within the parity
tolerance -- and match the oracle; an infeasible member must not disturb
the others; host and device inputs give the same results.
"""
import numpy as np
import pytest

import oracle
from parity import compare, _close
from paper_2609_16182_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2609_16182_gb300 import lpp  # noqa: E402


def same_result(a, b):
    assert (a.status, a.where, a.index, a.round, a.rounds) == (b.status, b.where, b.index, b.round, b.rounds)
    if a.status != 0:
        return
    for f in ("row_kind", "row_round", "row_aux", "row_val", "col_kind", "col_round", "ninf_min", "ninf_max"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)
    for f in ("col_val", "col_lb", "col_ub", "act_min", "act_max"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)  # same arithmetic per row
    ra, rb = a.reduced(), b.reduced()
    for f in ("row_ptr", "col_idx", "val", "c", "lhs", "rhs", "lb", "ub", "row_map", "col_map", "csc_ptr", "csc_idx",
              "csc_val"):
        np.testing.assert_array_equal(getattr(ra, f), getattr(rb, f), err_msg=f)
    _close([ra.obj_offset], [rb.obj_offset], what="offset")


def to_device(lp):
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in lp.arrays().items()}
    return synth.LP(m=lp.m, n=lp.n, obj_offset=lp.obj_offset, **dev)


def test_batch_members_equal_their_solo_runs_and_the_oracle():
    lps = synth.batch_mix(5, count=48, m_lo=50, m_hi=1500)
    lps += [synth.tiny(s) for s in range(4)]
    res = lpp.presolve_batch(lps)
    for lp, r in zip(lps, res):
        same_result(r, lpp.presolve(lp))
        o = oracle.presolve(lp)
        if o.audit_below_1e3 == 0:
            compare(r, o, lp, arena_stats=True)


def test_infeasible_member_leaves_the_others_alone():
    from lpmake import INF, make
    bad = make([{0: 1.0, 1: 1.0}], lhs=[5], rhs=[INF], lb=[0, 0], ub=[1, 1])
    lps = [synth.mix(1), bad, synth.mix(2)]
    res = lpp.presolve_batch(lps)
    assert res[1].status == lpp.INFEASIBLE and res[1].where == lpp.WHERE_ROW and res[1].index == 0
    for k in (0, 2):
        same_result(res[k], lpp.presolve(lps[k]))


def test_device_batch_equals_host_batch():
    lps = synth.batch_mix(9, count=16, m_lo=50, m_hi=800)
    a = lpp.presolve_batch(lps)
    b = lpp.presolve_batch([to_device(lp) for lp in lps])
    for x, y in zip(a, b):
        same_result(x, y)


def test_batch_with_long_rows_and_empty_members():
    from lpmake import make
    lps = [synth.skewed(4, m=8000, n=12000, target_nnz=90_000, row_cap=9000),
           make([], [], [], [], [], None, n=0),
           synth.mix(7),
           make([{}, {}], [-1, 0], [1, 0], [], [], None, n=0)]
    res = lpp.presolve_batch(lps)
    for lp, r in zip(lps, res):
        same_result(r, lpp.presolve(lp))


# ---------------------------------------------------------- persistent kernel
# lpp_presolve_batch runs every round of each LP in one persistent kernel (a
# thread block per LP) when every row and column has at most 4096 entries
# and no step it does not carry is on; batch_persistent = 0 forces the
# per-round launches over the arena.  Both must give every LP its solo result.

def same_counters(a, b):
    np.testing.assert_array_equal(a.round_nnz, b.round_nnz, err_msg="nnz per round")
    np.testing.assert_array_equal(a.round_rows_removed, b.round_rows_removed, err_msg="rows removed per round")
    np.testing.assert_array_equal(a.round_cols_fixed, b.round_cols_fixed, err_msg="columns removed per round")
    np.testing.assert_array_equal(a.round_bounds_changed, b.round_bounds_changed, err_msg="bounds changed per round")
    assert a.s5_left == b.s5_left


@pytest.mark.parametrize("kw", [{}, {"dual_fixing": 1}, {"par_max_iter": 2}, {"max_rounds": 1}])
def test_persistent_batch_equals_solo_and_per_round_batch(kw):
    lps = synth.batch_mix(11, count=64, m_lo=50, m_hi=2000)
    lps += [synth.tiny(s) for s in range(6)] + [synth.mix(3)]
    fused = lpp.presolve_batch(lps, **kw)
    arena = lpp.presolve_batch(lps, batch_persistent=0, **kw)
    assert fused[0].info.launches < arena[0].info.launches  # the persistent kernel ran
    for lp, f, a in zip(lps, fused, arena):
        solo = lpp.presolve(lp, **kw)
        same_result(f, solo)
        same_result(a, solo)
        if f.status == 0:
            same_counters(f, solo)  # the persistent kernel counts per LP
        o = oracle.presolve(lp, oracle.default_opts(**kw))
        if o.audit_below_1 == 0:
            compare(f, o, lp)


def test_persistent_batch_parallel_rows_over_many_passes_and_verdicts():
    from lpmake import INF, make
    # key groups needing many leader passes, a later pass alone reducing a
    # round, an infeasible member and an unbounded one
    many = make([{0: 1.0, 1: float(k + 2)} for k in range(12)] + [{0: 2.0, 1: float(2 * (k + 2))} for k in range(12)],
                [-INF] * 24, [float(10 + k) for k in range(24)], [-INF, -INF], [INF, INF])
    later = make([{0: 1, 1: 1, 2: 2}, {1: 1, 2: 3}, {0: 5, 1: 2, 2: 6}, {0: 1}],
                 [-INF, -INF, -20, 2], [12, 7, INF, 2], [0, -INF, -INF], [10, INF, INF])
    bad = make([{0: 1.0, 1: 1.0}], lhs=[5], rhs=[INF], lb=[0, 0], ub=[1, 1])
    unb = make([{0: 1.0}], lhs=[-INF], rhs=[1], lb=[0, 0], ub=[5, INF], c=[0.0, -1.0])
    lps = [many, later, bad, unb, synth.mix(4)]
    for cap in (1, 3, 16):
        res = lpp.presolve_batch(lps, par_max_iter=cap)
        for lp, r in zip(lps, res):
            solo = lpp.presolve(lp, par_max_iter=cap)
            same_result(r, solo)
            if r.status == 0:
                same_counters(r, solo)
            compare(r, oracle.presolve(lp, oracle.default_opts(par_max_iter=cap)), lp)
    assert res[2].status == lpp.INFEASIBLE and res[3].status == lpp.UNBOUNDED


def test_persistent_batch_with_empty_and_degenerate_members():
    from lpmake import INF, make
    lps = [make([], [], [], [], [], None, n=0),                      # nothing
           make([], [], [], [0, -1], [1, 2], [1.0, -1.0]),           # columns only
           make([{}, {}], [-1, 0], [1, 0], [], [], None, n=0),       # rows only, empty
           make([{0: 1.0, 1: 2.0}], [3], [3], [1, 1], [1, 1], [1.0, 1.0]),  # every column fixed on input
           synth.tiny(5), synth.mix(6)]
    fused = lpp.presolve_batch(lps)
    arena = lpp.presolve_batch(lps, batch_persistent=0)
    assert fused[0].info.launches < arena[0].info.launches
    for lp, f, a in zip(lps, fused, arena):
        solo = lpp.presolve(lp)
        same_result(f, solo)
        same_result(a, solo)
        compare(f, oracle.presolve(lp), lp)


def test_batch_results_free_each_or_all():
    """BatchResults: results made on first access (the same object again),
    slices and negative indices, a result closed on its own, then every other
    handle freed by one lpp_free_results call."""
    lps = synth.batch_mix(31, count=6, m_lo=50, m_hi=300)
    res = lpp.presolve_batch(lps)
    assert len(res) == 6 and res[1] is res[1] and len(res[2:5]) == 3 and res[-1] is res[5]
    for r, lp in zip(res, lps):
        same_result(r, lpp.presolve(lp))
    res[0].close()
    assert not res._recs[0] and res._recs[1]
    r3 = res[3]
    res.close()
    assert all(not res._recs[k] for k in range(len(res)))
    assert r3._rec is None  # handed out before the close: now empty
    with pytest.raises(ValueError):
        res[2]
