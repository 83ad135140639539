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
