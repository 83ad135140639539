"""Serving (lpp_server_*): continuous batching of presolve rounds.

LPs submitted while others are resident join the arena at a round boundary;
each result must equal the LP presolved alone (records, maps and reduced LP
bit for bit, the objective constant within the parity tolerance) and match
the oracle within the parity bar.
"""
import time

import numpy as np
import pytest

import oracle
from parity import _close, compare
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
    for f in ("row_kind", "row_round", "row_aux", "row_val", "col_kind", "col_round", "ninf_min", "ninf_max",
              "col_val", "col_lb", "col_ub", "act_min", "act_max"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)
    ra, rb = a.reduced(), b.reduced()
    for f in ("row_ptr", "col_idx", "val", "c", "lhs", "rhs", "lb", "ub", "row_map", "col_map", "csc_ptr", "csc_idx",
              "csc_val"):
        np.testing.assert_array_equal(getattr(ra, f), getattr(rb, f), err_msg=f)
    _close([ra.obj_offset], [rb.obj_offset], what="offset")


def test_served_results_equal_solo_results_with_staggered_arrivals():
    # a burst longer than the queue an idle server still serves one at a time
    # (64) fills the arena; the later arrivals join running rounds
    lps = [synth.tiny(100 + s) for s in range(72)]
    lps += [synth.mix(s, m=int(m), n=int(1.5 * m)) for s, m in zip(range(12), [200, 800, 3000, 60, 500] * 3)]
    lps.insert(75, synth.skewed(2, m=20_000, n=30_000, target_nnz=200_000, row_cap=6000))
    solo = [lpp.presolve(lp) for lp in lps]
    with lpp.Server(2 << 30) as srv:
        tickets = []
        for k, lp in enumerate(lps):
            tickets.append(srv.submit(lp))
            if k >= 72 and k % 4 == 3:
                time.sleep(0.002)  # later arrivals join running rounds
        res = [srv.take(t, 60_000) for t in tickets]
        st = srv.stats()
    assert st["submitted"] == len(lps) and st["finished"] == len(lps)
    assert st["max_concurrent"] >= 2
    for a, b, lp in zip(res, solo, lps):
        same_result(a, b)
        # the per-round counters of a served LP describe the shared arena
        compare(a, oracle.presolve(lp), lp, arena_stats=True)


def test_server_device_inputs_infeasible_member_and_timeout():
    from lpmake import INF, make
    bad = make([{0: 1.0, 1: 1.0}], lhs=[5], rhs=[INF], lb=[0, 0], ub=[1, 1])
    good = synth.mix(21)
    dev = synth.LP(m=good.m, n=good.n, **{k: torch.from_numpy(np.ascontiguousarray(v)).cuda()
                                          for k, v in good.arrays().items()})
    with lpp.Server(1 << 30) as srv:
        tb = srv.submit(bad)
        tg = srv.submit(dev)
        rb = srv.take(tb, 60_000)
        rg = srv.take(tg, 60_000)
        with pytest.raises(lpp.LppError) as e:
            srv.take(987654, 10)
        assert e.value.status == lpp.ERR_TIMEOUT
    assert rb.status == lpp.INFEASIBLE and rb.where == lpp.WHERE_ROW and rb.index == 0
    same_result(rg, lpp.presolve(good))
    compare(rb, oracle.presolve(bad), bad, arena_stats=True)
    compare(rg, oracle.presolve(good), good, arena_stats=True)


def test_server_rejects_what_cannot_fit():
    with lpp.Server(8 << 20) as srv:
        big = synth.mix(1, m=40_000, n=60_000)  # more rows than 8 MiB of arena holds
        with pytest.raises(lpp.LppError) as e:
            srv.submit(big)
        assert e.value.status == lpp.ERR_BUDGET


def test_a_request_to_an_idle_server_runs_at_once_and_equals_solo():
    lp = synth.skewed(5, m=20_000, n=30_000, target_nnz=200_000, row_cap=6000)
    solo = lpp.presolve(lp)
    with lpp.Server(2 << 30) as srv:
        r = srv.take(srv.submit(lp), 60_000)
        st = srv.stats()
    assert st["solo"] == 1 and st["ticks"] == 0
    same_result(r, solo)
    compare(r, oracle.presolve(lp), lp)
