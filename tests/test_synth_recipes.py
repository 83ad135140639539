"""The seeded generators against the recipes they state (the inputs of every
test and of the benchmark): valid CSR, the planted point x0 feasible, the
planted counts and shares, determinism.  Scaled-down sizes; no GPU."""
import dataclasses

import numpy as np

from paper_2609_16182_gb300 import synth


def valid_csr(lp):
    rp, ci, v = lp.row_ptr, lp.col_idx, lp.val
    assert rp[0] == 0 and rp[-1] == lp.nnz == len(ci) == len(v) and np.all(np.diff(rp) >= 0)
    assert ci.dtype == np.int32 and rp.dtype == np.int32
    assert np.all((ci >= 0) & (ci < lp.n)) and np.all(np.isfinite(v)) and np.all(v != 0)
    rows = np.repeat(np.arange(lp.m), np.diff(rp))
    same = rows[1:] == rows[:-1]
    assert np.all(ci[1:][same] > ci[:-1][same]), "columns increasing inside every row"
    assert np.all(lp.lb <= lp.ub) and not np.any(np.isnan(lp.c))
    assert not np.any(np.isnan(lp.lhs) | np.isnan(lp.rhs)) and np.all(lp.lhs <= lp.rhs)


def x0_feasible(lp, tol=1e-9):
    x0 = lp.planted["x0"]
    assert np.all(x0 >= lp.lb) and np.all(x0 <= lp.ub)
    rows = np.repeat(np.arange(lp.m), np.diff(lp.row_ptr))
    ax = np.bincount(rows, weights=lp.val * x0[lp.col_idx], minlength=lp.m)
    scale = 1.0 + np.bincount(rows, weights=np.abs(lp.val * x0[lp.col_idx]), minlength=lp.m)
    assert np.all(ax >= lp.lhs - tol * scale) and np.all(ax <= lp.rhs + tol * scale)


def same(a, b):
    for k in ("row_ptr", "col_idx", "val", "c", "lhs", "rhs", "lb", "ub"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))


def test_tiny_recipe():
    for seed in range(4):
        lp = synth.tiny(seed)
        valid_csr(lp)
        x0_feasible(lp)
        p = lp.planted
        assert (lp.m, lp.n) == (200, 300) and 1000 < lp.nnz < 2000
        assert (p["empty"], p["singleton"], p["fixed"], p["redundant"], p["parallel"]) == (10, 15, 20, 10, 8)
        lens = np.diff(lp.row_ptr)
        assert np.count_nonzero(lens == 0) >= 10 and np.count_nonzero(lens == 1) >= 15
        assert np.count_nonzero(lp.lb == lp.ub) >= 20
        for (i, k), lam in zip(p["pairs"], p["lambdas"]):  # scaled copies: row k = lam * row i
            a = slice(lp.row_ptr[i], lp.row_ptr[i + 1])
            b = slice(lp.row_ptr[k], lp.row_ptr[k + 1])
            assert np.array_equal(lp.col_idx[a], lp.col_idx[b])
            np.testing.assert_allclose(lp.val[b], lam * lp.val[a], rtol=1e-15)
            assert 0.5 <= abs(lam) <= 4
    same(synth.tiny(1), synth.tiny(1))


def test_skewed_recipe():
    lp = synth.skewed(0, m=200_000, n=300_000, target_nnz=2_000_000, row_cap=50_000)
    valid_csr(lp)
    x0_feasible(lp)
    lens = np.diff(lp.row_ptr)
    assert np.median(lens) <= 3 and lens.max() > 100 * np.median(lens)  # a few very long rows
    assert 0.9 * 2_000_000 <= lp.nnz <= 1.1 * 2_000_000
    assert np.count_nonzero(lens == 1) >= 0.05 * lp.m
    eq = np.isfinite(lp.lhs) & (lp.lhs == lp.rhs)
    assert 0.25 <= np.mean(eq) <= 0.35
    assert 0.15 <= np.mean(np.isinf(lp.lb)) <= 0.25 and 0.15 <= np.mean(np.isinf(lp.ub)) <= 0.25
    assert np.all(np.bincount(lp.col_idx, minlength=lp.n) >= 1)  # every column has an entry
    logs = np.log(np.abs(lp.val))
    assert abs(np.mean(logs)) < 0.05 and abs(np.std(logs) - 1.0) < 0.05  # lognormal(0, 1) magnitudes
    assert lp.planted["redundant"] == 6000


def test_lprelax_recipe():
    lp = synth.lprelax(0, m=50_000, n=100_000, target_nnz=800_000, n_dense=10, dense_len=20_000)
    valid_csr(lp)
    x0_feasible(lp)
    cl = np.bincount(lp.col_idx, minlength=lp.n)
    assert np.count_nonzero(cl >= 20_000) == 10
    lens = np.diff(lp.row_ptr)
    dbl = (lens == 2) & np.isfinite(lp.lhs) & (lp.lhs == lp.rhs)
    assert np.count_nonzero(dbl) >= 0.04 * lp.m
    p = lp.planted
    assert (p["parallel"], p["doubleton"], p["dominated"]) == (2500, 2000, 2000)


def test_micro_and_plants():
    for seed in range(20):
        lp = synth.micro(seed)
        valid_csr(lp)
        assert lp.n <= 6 and np.all(np.isfinite(lp.lb)) and np.all(np.isfinite(lp.ub))
        x0_feasible(lp)
        d = synth.plant_doubletons(lp, seed, point=lp.planted["x0"])
        valid_csr(d)
        assert d.m == lp.m + 2
        assert np.all(np.diff(d.row_ptr)[-2:] == 2) and np.all(d.lhs[-2:] == d.rhs[-2:])
        x0_feasible(dataclasses.replace(d, planted={"x0": lp.planted["x0"]}))
    base = synth.parcols(0)
    valid_csr(base)
    q = synth.plant_col_singletons(base, 0)
    valid_csr(q)
    assert q.n > base.n and np.all(np.bincount(q.col_idx, minlength=q.n)[base.n:] == 1)
