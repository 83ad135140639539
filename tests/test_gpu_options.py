"""GPU parity under non-default options, and S5 with many leader passes.

The default-option paths are covered by test_gpu_parity.py; here the
tolerances, the dual rule, the pass cap of the parallel-row iteration and
the round cap change, on the 200-row mix and on a small LP-relaxation-like
instance.  A hand-built LP whose parallel rows need ten leader passes
exercises the later S5 passes (their chunks of 2, 4, 8 passes), the cap
carrying the iteration over into the next round, and the skip of S5 once
every group is resolved.
"""
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
    g = lpp.presolve(lp, **kw)
    o = oracle.presolve(lp, oracle.default_opts(**kw))
    return g, o


OPTS = [dict(dual_reductions=0), dict(par_max_iter=1), dict(par_max_iter=2), dict(bound_tol=1e-3),
        dict(bound_tol=0.0), dict(max_implied=1e3), dict(feas_tol=1e-6), dict(max_rounds=3)]


def _id(kw):
    return ",".join(f"{k}={v}" for k, v in kw.items())


@pytest.mark.parametrize("kw", OPTS, ids=_id)
@pytest.mark.parametrize("seed", [0, 1, 3])
def test_options_tiny(seed, kw):
    lp = synth.tiny(seed)
    g, o = both(lp, **kw)
    if o.audit_below_1e3:
        pytest.skip("instance has a decision within 1000x of its error bound under these options")
    compare(g, o, lp)


@pytest.mark.parametrize("kw", OPTS, ids=_id)
def test_options_lprelax(kw):
    lp = synth.lprelax(1, m=6_000, n=12_000, target_nnz=96_000, n_dense=2, dense_len=2_500)
    g, o = both(lp, **kw)
    if o.audit_below_1e3:
        pytest.skip("instance has a decision within 1000x of its error bound under these options")
    compare(g, o, lp)


def many_pass_lp(groups=10, seed=0):
    """`groups` rows on columns 0..2 with distinct coefficient ratios, then a
    copy of each scaled by 2: all share one parallel-row key, and the leader
    iteration needs one pass per base row.  The rows are not redundant and
    imply no bound; a few unrelated rows fill out the LP."""
    rng = np.random.default_rng(seed)
    base = [dict(zip(range(3), rng.uniform(1.0, 5.0, 3))) for _ in range(groups)]
    rows = list(base) + [{j: 2.0 * a for j, a in r.items()} for r in base]
    rhs = [5.0 + 0.1 * k for k in range(groups)] + [2.0 * (5.0 + 0.1 * k) + 0.5 for k in range(groups)]
    for k in range(4):  # unrelated rows on other columns
        rows.append({3 + k: 1.0, 4 + k: -2.0})
        rhs.append(3.0)
    n = 8
    lhs = [-INF] * len(rows)
    return make(rows, lhs, rhs, [0.0] * n, [1.0] * n, c=np.linspace(-1.0, 1.0, n))


@pytest.mark.parametrize("cap", [1, 2, 4, 16])
def test_parallel_rows_needing_many_passes(cap):
    lp = many_pass_lp()
    g, o = both(lp, par_max_iter=cap)
    compare(g, o, lp)
    if cap >= 10:  # one round resolves every group: each copy went into its base row
        assert np.count_nonzero(g.row_kind == lpp.ROW_PARALLEL) == 10


@pytest.mark.parametrize("cap", [2, 16])
def test_round_reduced_only_by_a_later_parallel_pass(cap):
    # x = 2 is fixed in round 1; in round 2 the rows y + 2z, y + 3z, 2y + 6z
    # form one key group whose first pass finds nothing and whose second
    # pass merges 2y + 6z into y + 3z: the round's only reduction, which must
    # still compact the matrix
    lp = make([{0: 1, 1: 1, 2: 2}, {1: 1, 2: 3}, {0: 5, 1: 2, 2: 6}, {0: 1}],
              [-INF, -INF, -20, 2], [12, 7, INF, 2], [0, -INF, -INF], [10, INF, INF])
    g, o = both(lp, par_max_iter=cap)
    assert o.row_kind[2] == lpp.ROW_PARALLEL and o.row_round[2] == 2
    compare(g, o, lp)
