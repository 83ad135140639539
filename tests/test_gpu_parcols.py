"""GPU parity of the opt-in parallel-column step (S5c) against the oracle.

Planted copies (synth.parcols, factors +-1/2, 2, 4), the 200-row mix, a
small LP-relaxation-like instance and a 60k-row skewed LP with 1% of its
columns copied, all with the step switched on; a group of
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


@pytest.mark.parametrize("seed", range(2))
def test_skewed_with_planted_copies(seed):
    # 1% of the columns copied and scaled; rows up to 20k entries (chunked),
    # heavy columns, and the skewed LP's own parallel columns (singletons
    # sharing a row, zero costs)
    lp = synth.plant_parallel_cols(synth.skewed(seed, m=60_000, n=90_000, target_nnz=600_000, row_cap=20_000),
                                   seed)
    g, o = both(lp)
    compare(g, o, lp)
    assert np.count_nonzero(g.col_kind == lpp.COL_PARALLEL) > 0.5 * len(lp.planted["par_copies"])


def copies_lp(classes=4, k=3, long_len=0, seed=0):
    """`classes` positive base columns on the same rows (rows 0..2, or
    0..long_len-1), different in their ratios, and k scaled copies of each
    (factors 2^e, alternating sign), interleaved in column order, plus two
    filler columns.  All share one key: pass p's leader is base p, which takes
    the copies of its class.  No row is redundant, so a capped iteration
    continues next round."""
    rng = np.random.default_rng(seed)
    rows_n = max(3, long_len)
    # positive bases: every row's activity is smallest at the same point
    # (each x_j at the bound its coefficient's sign picks), so the LP is
    # feasible for any right-hand side between min and max activity
    bases = [rng.uniform(1.0, 3.0, rows_n) for _ in range(classes)]
    cols, c = list(bases), list(rng.uniform(0.5, 1.5, classes))
    for q in range(k):
        for b in range(classes):
            f = ((-1) ** (q + b)) * 2.0 ** ((q + 2 * b) % 5 - 2)
            cols.append(bases[b] * f)
            c.append(c[b] * f)
    nc = len(cols)
    c += [0.5, -0.5]
    rows = []
    for i in range(rows_n):
        r = {j: float(cols[j][i]) for j in range(nc)}
        r[nc + (i % 2)] = 1.0
        rows.append(r)
    lb = [0.0] * nc + [-1.0, -1.0]
    ub = [1.0] * nc + [1.0, 1.0]
    rhs = []
    for r in rows:
        a = np.array(list(r.values()))
        hi, lo = a[a > 0].sum(), a[a < 0].sum()
        rhs.append(0.7 * lo + 0.3 * hi - 1.0)
    return make(rows, [-INF] * rows_n, rhs, lb, ub, c=c)


@pytest.mark.parametrize("cap", [1, 2, 16])
def test_many_passes_and_the_cap(cap):
    lp = copies_lp(classes=4, k=3)
    g, o = both(lp, par_max_iter=cap)
    compare(g, o, lp)
    merged = g.col_kind == lpp.COL_PARALLEL
    assert np.count_nonzero(merged) == np.count_nonzero(o.col_kind == oracle.COL_PARALLEL)
    if cap == 16:  # one class per pass, all in round 1
        assert np.count_nonzero(merged) == 12 and sorted(set(g.col_pass[merged])) == [0, 1, 2, 3]


def test_long_columns():
    lp = copies_lp(classes=2, k=2, long_len=5_000)
    g, o = both(lp)
    compare(g, o, lp)
    assert np.count_nonzero(g.col_kind == lpp.COL_PARALLEL) == 4


def tolerance_edge_lp(tol, seed=0):
    """A base column and copies whose costs are off by relative factors
    around the tolerance (inside and outside, both signs), on three rows; the
    entries are exact multiples.  Which copies merge, and in which pass, is
    decided by the cost test alone."""
    rng = np.random.default_rng(seed)
    base = rng.uniform(1.0, 3.0, 3)
    c0 = rng.uniform(0.5, 1.5)
    deltas = [f * tol for f in (0.0, 0.3, -0.3, 0.7, -0.7, 0.95, -0.95, 1.05, -1.05, 1.5, -1.5, 3.0, -3.0)]
    cols, c = [base], [c0]
    for q, d in enumerate(deltas):
        lam = ((-1) ** q) * 2.0 ** (q % 5 - 2)
        cols.append(base * lam)
        c.append(c0 * lam * (1.0 + d))
    nc = len(cols)
    rows = [{j: float(cols[j][i]) for j in range(nc)} | {nc + (i % 2): 1.0} for i in range(3)]
    lb, ub = [0.0] * nc + [-1.0, -1.0], [1.0] * nc + [1.0, 1.0]
    rhs = []
    for r in rows:
        a = np.array(list(r.values()))
        rhs.append(0.7 * a[a < 0].sum() + 0.3 * a[a > 0].sum() - 1.0)
    return make(rows, [-INF] * 3, rhs, lb, ub, c=c + [0.5, -0.5])


@pytest.mark.parametrize("tol", [1e-12, 1e-9, 1e-5])
def test_cost_tolerance_edges(tol):
    # the GPU skips the cost test for pairs whose cost ratios are far apart
    # (a window of about twice the tolerance, off from 1e-6 on): near the
    # tolerance the oracle's exact test decides alone
    for seed in range(4):
        lp = tolerance_edge_lp(tol, seed)
        g, o = both(lp, par_tol=tol)
        compare(g, o, lp)
        assert np.count_nonzero(o.col_kind == oracle.COL_PARALLEL) >= 1


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
