"""GPU parity of dual fixing by locks (S6 with `dual_fixing`) against the oracle.

Small LPs (plain and with one-sided rows), the 200-row mix, a 60k-row skewed
LP with long columns (locks OR-ed over chunks), an LP-relaxation-like LP,
all three opt-in steps together, a batch, and the server (which allows this
option: it adds no records).
"""
import dataclasses

import numpy as np
import pytest

import oracle
from lpmake import INF, make
from parity import compare
from paper_2609_16182_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2609_16182_gb300 import lpp  # noqa: E402
from test_gpu_serve import same_result  # noqa: E402


def both(lp, **kw):
    kw.setdefault("dual_fixing", 1)
    g = lpp.presolve(lp, **kw)
    o = oracle.presolve(lp, oracle.default_opts(**kw))
    return g, o


def one_sided(lp):
    lhs = lp.lhs.copy()
    eq = np.isfinite(lp.lhs) & (lp.lhs == lp.rhs)
    lhs[~eq & np.isfinite(lp.rhs)] = -INF
    return dataclasses.replace(lp, lhs=lhs)


@pytest.mark.parametrize("variant", ["plain", "one_sided"])
@pytest.mark.parametrize("seed", range(40))
def test_micro(seed, variant):
    lp = synth.micro(seed + 1300)
    if variant == "one_sided":
        lp = one_sided(lp)
    g, o = both(lp)
    compare(g, o, lp)


def test_hand_worked_locks():
    lp = make([{0: 1.0, 1: 1.0}, {0: 2.0, 1: 1.0, 2: -1.0}], [-INF, -INF], [3.0, 5.0],
              [-1.0, 0.0, 0.0], [2.0, 10.0, 4.0], c=[2.0, -1.0, -3.0])
    g, o = both(lp, max_rounds=1)
    compare(g, o, lp)
    assert list(g.col_kind) == [lpp.COL_EMPTY, lpp.COL_KEPT, lpp.COL_EMPTY] and list(g.col_val[[0, 2]]) == [-1.0, 4.0]


@pytest.mark.parametrize("seed", range(4))
def test_tiny(seed):
    lp = synth.tiny(seed)
    g, o = both(lp)
    if o.audit_below_1e3:
        pytest.skip("instance has a decision within 1000x of its error bound")
    compare(g, o, lp)


@pytest.mark.parametrize("seed", range(2))
def test_skewed_mid_size(seed):
    lp = synth.skewed(seed, m=60_000, n=90_000, target_nnz=600_000, row_cap=20_000)
    g, o = both(lp)
    compare(g, o, lp)
    assert np.count_nonzero(g.col_kind == lpp.COL_EMPTY) > np.count_nonzero(lpp.presolve(lp).col_kind == lpp.COL_EMPTY)


def test_lprelax():
    lp = synth.lprelax(1, m=6_000, n=12_000, target_nnz=96_000, n_dense=2, dense_len=2_500)
    g, o = both(lp)
    compare(g, o, lp)


@pytest.mark.parametrize("seed", range(3))
def test_all_opt_in_steps(seed):
    lp = synth.plant_col_singletons(synth.parcols(seed), seed)
    g, o = both(lp, parallel_cols=1, col_singletons=1)
    compare(g, o, lp)


def test_batch_and_server():
    lps = [synth.tiny(s) for s in range(3)] + [one_sided(synth.micro(s + 1300)) for s in range(5)]
    res = lpp.presolve_batch(lps, dual_fixing=1)
    solo = [lpp.presolve(lp, dual_fixing=1) for lp in lps]
    for lp, r in zip(lps, res):
        compare(r, oracle.presolve(lp, oracle.default_opts(dual_fixing=1)), lp, arena_stats=True)
    with lpp.Server(1 << 30, dual_fixing=1) as srv:
        tickets = [srv.submit(lp) for lp in lps]
        served = [srv.take(t, 60_000) for t in tickets]
    for a, b in zip(served, solo):
        same_result(a, b)
