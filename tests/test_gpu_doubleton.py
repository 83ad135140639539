"""GPU parity of the doubleton-equation step (S5e, `doubletons`) against the
oracle: hand-worked rows, cancellation and insertion, an empty bound
transfer, planted micro and 200-row LPs, long x_k columns of the
LP-relaxation generator (warp walks), every opt-in step together, a batch,
and the postsolve."""
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
    kw.setdefault("doubletons", 1)
    return lpp.presolve(lp, **kw), oracle.presolve(lp, oracle.default_opts(**kw))


def test_hand_worked():
    lp = make([{0: 1.0, 1: 2.0}, {0: 3.0, 1: 4.0, 2: 1.0}, {0: 1.0, 2: -1.0}], [4.0, -INF, -5.0], [4.0, 10.0, INF],
              [0.0, 0.0, -1.0], [3.0, 1.5, 1.0], c=[1.0, 2.0, 3.0])
    for mr in (1, 20):
        g, o = both(lp, max_rounds=mr, dual_reductions=0)
        compare(g, o, lp)


def test_cancellation_and_insertion():
    # row 1 holds x0 and x1: x0's coefficient cancels; row 2 holds x1 only: x0 is inserted
    lp = make([{0: 1.0, 1: 1.0}, {0: 1.0, 1: 1.0, 2: 1.0}, {1: 2.0, 3: 1.0}], [2.0, -INF, -INF], [2.0, 5.0, 6.0],
              [0.0, 0.0, 0.0, 0.0], [3.0, 3.0, 3.0, 3.0], c=[1.0, 1.0, 1.0, 1.0])
    g, o = both(lp, dual_reductions=0)
    compare(g, o, lp)


def test_infeasible_transfer():
    lp = make([{2: 1.0, 3: 1.0}, {0: 1.0, 1: 1.0}, {2: 1.0, 4: 1.0}, {0: 1.0, 5: 1.0}],
              [10.0, 10.0, -INF, -INF], [10.0, 10.0, 8.999998, 8.999998],
              [8.999995, 0.0, 8.999995, 0.0, 0.0, 0.0], [100.0, 1.0, 100.0, 1.0, 1.0, 1.0], c=[1.0] * 6)
    g, o = both(lp)
    compare(g, o, lp)


@pytest.mark.parametrize("through_x0", [True, False])
@pytest.mark.parametrize("seed", range(40))
def test_micro_planted(seed, through_x0):
    # planted through the LP's feasible point (the LP stays feasible), or through a point of the
    # columns' box (often infeasible: the verdict's location and round are compared)
    base = synth.micro(seed + 2100)
    lp = synth.plant_doubletons(base, seed, point=base.planted["x0"] if through_x0 else None)
    g, o = both(lp)
    compare(g, o, lp)


@pytest.mark.parametrize("seed", range(4))
def test_tiny_planted(seed):
    lp = synth.plant_doubletons(synth.tiny(seed), seed)
    g, o = both(lp)
    if o.audit_below_1e3:
        pytest.skip("instance has a decision within 1000x of its error bound")
    compare(g, o, lp)
    assert np.count_nonzero(g.row_kind == lpp.ROW_DOUBLETON) > 0


@pytest.mark.parametrize("seed", range(2))
def test_lprelax_long_columns(seed):
    # 4% doubleton equations and dense columns: x_k walks of hundreds of rows (warp walks)
    lp = synth.lprelax(seed, m=6_000, n=12_000, target_nnz=96_000, n_dense=2, dense_len=2_500)
    g, o = both(lp)
    compare(g, o, lp)


@pytest.mark.parametrize("seed", range(3))
def test_all_opt_in_steps(seed):
    lp = synth.plant_doubletons(synth.plant_col_singletons(synth.parcols(seed), seed), seed)
    g, o = both(lp, parallel_cols=1, col_singletons=1, dual_fixing=1)
    compare(g, o, lp)


def test_batch_matches_solo():
    lps = [synth.plant_doubletons(synth.tiny(s), s) for s in range(3)]
    res = lpp.presolve_batch(lps, doubletons=1)
    for lp, r in zip(lps, res):
        compare(r, oracle.presolve(lp, oracle.default_opts(doubletons=1)), lp, arena_stats=True)


@pytest.mark.parametrize("seed", range(3))
def test_postsolve_matches_oracle(seed):
    lp = synth.plant_doubletons(synth.tiny(seed), seed)
    g, o = both(lp)
    red = g.reduced()
    rng = np.random.default_rng(seed)
    lo = np.where(np.isfinite(red.lb), red.lb, -5.0)
    hi = np.where(np.isfinite(red.ub), red.ub, 5.0)
    xr = lo + (hi - lo) * rng.random(red.n)
    np.testing.assert_allclose(g.postsolve_primal(xr), oracle.postsolve_primal(o, xr), rtol=1e-9, atol=1e-9)
