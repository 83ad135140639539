"""GPU parity of the opt-in parallel-column step (S5c) against the oracle.

Planted copies (synth.parcols, factors +-1/2, 2, 4), the 200-row mix and a
small LP-relaxation-like instance with the step switched on; a group of
columns that needs many leader passes (one merge per leader and pass), with
the pass cap cutting it short; long columns (more than 4096 entries); a
batch; and the postsolve of merged columns.
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
    kw.setdefault("parallel_cols", 1)
    g = lpp.presolve(lp, **kw)
    o = oracle.presolve(lp, oracle.default_opts(**kw))
    return g, o


@pytest.mark.parametrize("seed", range(6))
def test_planted_copies(seed):
    lp = synth.parcols(seed)
    g, o = both(lp)
    compare(g, o, lp)
    assert np.count_nonzero(g.col_kind == lpp.COL_PARALLEL) >= len(lp.planted["copies"])


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_tiny_mix(seed):
    lp = synth.tiny(seed)
    g, o = both(lp)
    if o.audit_below_1e3:
        pytest.skip("instance has a decision within 1000x of its error bound")
    compare(g, o, lp)


def test_lprelax():
    lp = synth.lprelax(1, m=6_000, n=12_000, target_nnz=96_000, n_dense=2, dense_len=2_500)
    g, o = both(lp)
    if o.audit_below_1e3:
        pytest.skip("instance has a decision within 1000x of its error bound")
    compare(g, o, lp)


def copies_lp(k=12, long_len=0, seed=0):
    """Column 0 and k scaled copies of it (factors 2^e, alternating sign) on
    rows 0..2 (rows 0..long_len-1 when long_len > 0), plus filler columns.
    All copies share one key: the leader takes one per pass."""
    rng = np.random.default_rng(seed)
    rows_n = max(3, long_len)
    # a positive base column: every row's activity is smallest at the same
    # point (each x_j at the bound its coefficient's sign picks), so the LP
    # is feasible whatever the right-hand sides between min and max activity
    base = rng.uniform(1.0, 3.0, rows_n)
    n = 1 + k + 2
    cols = [base] + [base * ((-1) ** q) * 2.0 ** (q % 5 - 2) for q in range(k)]
    c = [1.0] + [((-1) ** q) * 2.0 ** (q % 5 - 2) for q in range(k)] + [0.5, -0.5]
    rows = []
    for i in range(rows_n):
        r = {j: float(cols[j][i]) for j in range(1 + k)}
        r[1 + k + (i % 2)] = 1.0
        rows.append(r)
    lb = [0.0] * (1 + k) + [-1.0, -1.0]
    ub = [1.0] * (1 + k) + [1.0, 1.0]
    # rhs between the row's min and max activity: no row is redundant, so
    # the columns stay and a capped leader iteration continues next round
    rhs = []
    for r in rows:
        a = np.array(list(r.values()))
        hi, lo = a[a > 0].sum(), a[a < 0].sum()
        rhs.append(0.7 * lo + 0.3 * hi - 1.0)
    return make(rows, [-INF] * rows_n, rhs, lb, ub, c=c)


@pytest.mark.parametrize("cap", [1, 3, 16])
def test_many_passes_and_the_cap(cap):
    lp = copies_lp(k=12)
    g, o = both(lp, par_max_iter=cap)
    compare(g, o, lp)
    merged = np.count_nonzero(g.col_kind == lpp.COL_PARALLEL)
    assert merged == np.count_nonzero(o.col_kind == oracle.COL_PARALLEL)
    if cap == 16:  # one merge per pass: all twelve copies within one round
        assert merged == 12 and np.all(g.col_pass[g.col_kind == lpp.COL_PARALLEL] < 12)


def test_long_columns():
    lp = copies_lp(k=3, long_len=5_000)
    g, o = both(lp)
    compare(g, o, lp)
    assert np.count_nonzero(g.col_kind == lpp.COL_PARALLEL) == 3


def test_off_by_default_and_batch():
    lps = [synth.parcols(s) for s in range(3)]
    g = lpp.presolve(lps[0])
    assert not np.any(g.col_kind == lpp.COL_PARALLEL)
    res = lpp.presolve_batch(lps, parallel_cols=1)
    for lp, r in zip(lps, res):
        o = oracle.presolve(lp, oracle.default_opts(parallel_cols=1))
        compare(r, o, lp, arena_stats=True)


def test_server_rejects_the_option():
    with pytest.raises(lpp.LppError):
        lpp.Server(64 << 20, parallel_cols=1)


@pytest.mark.parametrize("seed", range(3))
def test_postsolve_matches_oracle(seed):
    lp = synth.parcols(seed)
    g, o = both(lp)
    rng = np.random.default_rng(seed)
    red = g.reduced()
    lo = np.where(np.isfinite(red.lb), red.lb, -5.0)
    hi = np.where(np.isfinite(red.ub), red.ub, 5.0)
    xr = lo + (hi - lo) * rng.random(red.n)
    xg = g.postsolve_primal(xr)
    xo = oracle.postsolve_primal(o, xr)
    np.testing.assert_allclose(xg, xo, rtol=1e-12, atol=1e-12)
    # every split puts x_j inside its bounds at the merge and keeps y
    for j in np.flatnonzero(g.col_kind == lpp.COL_PARALLEL):
        lk, uk, lj, uj = g.col_mrg[j]
        assert lj - 1e-9 <= xg[j] <= uj + 1e-9
