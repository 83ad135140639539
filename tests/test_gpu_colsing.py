"""GPU parity of the opt-in column-singleton step (S5d) against the oracle.

Planted singleton columns (free or boxed) in equality rows of small LPs
(vertex-enumerable), of the 200-row mix and of a 60k-row skewed LP whose
candidate rows reach thousands of entries (the block tasks); the
one-substitution-per-column rule over two rounds; the step together with
parallel columns; a batch; and the postsolve.
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


def both(lp, **kw):
    kw.setdefault("col_singletons", 1)
    g = lpp.presolve(lp, **kw)
    o = oracle.presolve(lp, oracle.default_opts(**kw))
    return g, o


@pytest.mark.parametrize("rows", ["eq", "any"])
@pytest.mark.parametrize("seed", range(60))
def test_micro_planted(seed, rows):
    # rows="any": singletons in inequality rows too (substituted at the side their cost selects)
    lp = synth.plant_col_singletons(synth.micro(seed + 900), seed, rows=rows)
    g, o = both(lp)
    compare(g, o, lp)


@pytest.mark.parametrize("rows", ["eq", "any"])
@pytest.mark.parametrize("seed", range(6))
def test_tiny_planted(seed, rows):
    lp = synth.plant_col_singletons(synth.tiny(seed), seed, rows=rows)
    g, o = both(lp)
    if o.audit_below_1e3:
        pytest.skip("instance has a decision within 1000x of its error bound")
    compare(g, o, lp)
    assert np.count_nonzero(g.row_kind == lpp.ROW_SUBST) > 0


@pytest.mark.parametrize("seed", [0, 1, 3])
def test_skewed_planted_long_rows(seed):
    # zero-cost singletons (the LP stays bounded): rows of 65..4096 entries run
    # as block tasks, longer ones by chunks (seeds 1 and 3 substitute rows of
    # 4605 and 7534 entries)
    lp = synth.plant_col_singletons(synth.skewed(seed, m=60_000, n=90_000, target_nnz=600_000, row_cap=20_000), seed,
                                    frac=0.3, free_frac=1.0, cost_scale=0.0)
    g, o = both(lp)
    compare(g, o, lp)
    lens = np.diff(lp.row_ptr)[g.row_kind == lpp.ROW_SUBST]
    assert np.any(lens > 64)
    if seed in (1, 3):
        assert np.any(lens > 4096)


@pytest.mark.parametrize("seed", range(2))
def test_skewed_boxed_costly_singletons(seed):
    # finite bounds everywhere (bounded LP) and singletons with costs: the
    # substituted rows bid for their columns, long rows included (by chunks)
    base = synth.skewed(seed, m=60_000, n=90_000, target_nnz=600_000, row_cap=20_000)
    base = dataclasses.replace(base, lb=np.maximum(base.lb, -1e3), ub=np.minimum(base.ub, 1e3))
    lp = synth.plant_col_singletons(base, seed, frac=0.3, free_frac=1.0, cost_scale=1.0)
    g, o = both(lp)
    compare(g, o, lp)
    assert np.count_nonzero(g.row_kind == lpp.ROW_SUBST) > 1000


def test_inequality_row_sides():
    for c2, subst in ((-1.0, True), (1.0, False), (0.0, True)):
        lp = make([{0: 1.0, 1: 1.0, 2: 1.0}, {0: 1.0, 1: 1.0}], [-INF, -INF], [4.0, 3.0],
                  [0.0, 0.0, -INF], [2.0, 2.0, INF], c=[1.0, 2.0, c2])
        g, o = both(lp, max_rounds=1)
        compare(g, o, lp)
        assert (g.row_kind[0] == lpp.ROW_SUBST) == subst


def test_one_substitution_per_column_and_round():
    lp = make([{0: 1.0, 1: 1.0, 2: 1.0}, {0: 1.0, 3: 2.0}, {0: 1.0, 1: -1.0}], [1.0, 2.0, -INF],
              [1.0, 2.0, 1.0], [0.0, 0.0, -INF, -INF], [1.0, 1.0, INF, INF], c=[1.0, 1.0, 0.5, -0.25])
    g, o = both(lp)
    compare(g, o, lp)
    assert list(g.row_round[:2]) == [1, 2] and list(g.row_kind[:2]) == [lpp.ROW_SUBST] * 2


@pytest.mark.parametrize("seed", range(3))
def test_with_parallel_columns(seed):
    lp = synth.plant_col_singletons(synth.parcols(seed), seed)
    g, o = both(lp, parallel_cols=1)
    compare(g, o, lp)


def test_off_by_default_batch_and_server():
    lps = [synth.plant_col_singletons(synth.tiny(s), s) for s in range(3)]
    g = lpp.presolve(lps[0])
    assert not np.any(g.row_kind == lpp.ROW_SUBST)
    res = lpp.presolve_batch(lps, col_singletons=1)
    for lp, r in zip(lps, res):
        o = oracle.presolve(lp, oracle.default_opts(col_singletons=1))
        compare(r, o, lp, arena_stats=True)
    with pytest.raises(lpp.LppError):
        lpp.Server(64 << 20, col_singletons=1)


@pytest.mark.parametrize("seed", range(3))
def test_postsolve_matches_oracle(seed):
    lp = synth.plant_col_singletons(synth.tiny(seed), seed)
    g, o = both(lp, parallel_cols=1)
    rng = np.random.default_rng(seed)
    red = g.reduced()
    lo = np.where(np.isfinite(red.lb), red.lb, -5.0)
    hi = np.where(np.isfinite(red.ub), red.ub, 5.0)
    xr = lo + (hi - lo) * rng.random(red.n)
    # b can come out of side shifts (sums): the eliminated values agree to the sum tolerance
    np.testing.assert_allclose(g.postsolve_primal(xr), oracle.postsolve_primal(o, xr), rtol=1e-9, atol=1e-9)
