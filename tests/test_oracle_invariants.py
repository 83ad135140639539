"""Invariants that pin the oracle to the mathematics (CPU only).

* S1: the min/max activity of a row is the min/max of a linear function over
  a box, brute-forced over the box corners.
* Every primal reduction keeps the feasible set: the vertex set of the
  original LP equals the vertex set of the reduced LP lifted with the fixed
  values (brute-force vertex enumeration, n <= 6).
* Postsolve maps an optimal reduced solution to a feasible, optimal original
  one (vertex enumeration on tiny LPs, scipy's HiGHS on the 200-row mix).
* The fixpoint is a fixpoint: presolving the reduced LP again finds nothing.
* Planted structures are found (a lower bound), scaled copies with their
  planted factor.
"""
from itertools import product

import numpy as np
import pytest

import oracle
from lpbrute import lp_vertices, reduced_vertices_lifted, same_point_sets, inequalities, vertices
from paper_2609_16182_gb300 import synth


def test_activity_equals_box_corner_extremes():
    rng = np.random.default_rng(7)
    for _ in range(60):
        ln = int(rng.integers(1, 11))
        n = ln + 2
        cols = np.sort(rng.choice(n, ln, replace=False))
        a = rng.uniform(-5, 5, ln)
        a[np.abs(a) < 0.1] = 1.0
        lb = rng.uniform(-4, 1, n)
        ub = lb + rng.uniform(0, 4, n)
        inf_l = rng.random(n) < 0.2
        inf_u = rng.random(n) < 0.2
        lb[inf_l] = -np.inf
        ub[inf_u] = np.inf
        lp = synth.LP(m=1, n=n, row_ptr=np.array([0, ln], np.int32), col_idx=cols.astype(np.int32), val=a,
                      c=np.zeros(n), lhs=np.array([-np.inf]), rhs=np.array([np.inf]), lb=lb, ub=ub)
        amin, amax, nmin, nmax = oracle.activities(lp)

        def corners(M):
            lo = np.where(np.isfinite(lb[cols]), lb[cols], -M)
            hi = np.where(np.isfinite(ub[cols]), ub[cols], M)
            vals = [float(np.dot(a, np.where(np.array(bits), hi, lo))) for bits in product([0, 1], repeat=ln)]
            return min(vals), max(vals)

        # an infinite contributor moves the extreme linearly in M: the slope
        # counts them (each |a|), the intercept is the finite part
        M1, M2 = 1e6, 2e6
        (mn1, mx1), (mn2, mx2) = corners(M1), corners(M2)
        slope_min = (mn1 - mn2) / (M2 - M1)
        slope_max = (mx2 - mx1) / (M2 - M1)
        inf_min_set = [k for k in range(ln) if (a[k] > 0 and not np.isfinite(lb[cols[k]]))
                       or (a[k] < 0 and not np.isfinite(ub[cols[k]]))]
        assert nmin[0] == len(inf_min_set)
        assert slope_min == pytest.approx(sum(abs(a[k]) for k in inf_min_set), rel=1e-9, abs=1e-9)
        assert amin[0] == pytest.approx(mn1 + M1 * slope_min, rel=1e-9, abs=1e-6)
        assert amax[0] == pytest.approx(mx1 - M1 * slope_max, rel=1e-9, abs=1e-6)
        if nmin[0] == 0:
            assert amin[0] == pytest.approx(mn1, rel=1e-12, abs=1e-12)
        if nmax[0] == 0:
            assert amax[0] == pytest.approx(mx1, rel=1e-12, abs=1e-12)


def _fixed_values(res):
    return {int(j): float(res.col_val[j]) for j in np.flatnonzero(res.col_kind != oracle.COL_KEPT)}


@pytest.mark.parametrize("seed", range(120))
def test_primal_reductions_keep_the_vertex_set(seed):
    lp = synth.micro(seed, m=5, n=6)
    res = oracle.presolve(lp, oracle.default_opts(dual_reductions=0))
    V = lp_vertices(lp)
    if res.status == oracle.INFEASIBLE:
        assert len(V) == 0
        return
    assert res.status == oracle.OK
    W = reduced_vertices_lifted(res, lp.n, _fixed_values(res))
    assert same_point_sets(V, W, tol=1e-7), (seed, len(V), len(W))


@pytest.mark.parametrize("seed", range(120))
def test_postsolve_maps_reduced_optimum_to_original_optimum(seed):
    lp = synth.micro(seed + 1000, m=5, n=6)
    res = oracle.presolve(lp)
    V = lp_vertices(lp)
    if len(V) == 0:
        assert res.status == oracle.INFEASIBLE
        return
    assert res.status == oracle.OK
    opt = float(np.min(V @ lp.c))
    G, h = inequalities(res.row_ptr, res.col_idx, res.val, res.lhs, res.rhs, res.lb, res.ub, res.n_red)
    W = vertices(G, h, res.n_red)
    assert len(W) > 0
    k = int(np.argmin(W @ res.c)) if res.n_red else 0
    red_opt = (float(W[k] @ res.c) if res.n_red else 0.0) + res.obj_offset
    assert red_opt == pytest.approx(opt, rel=1e-9, abs=1e-9)
    x = oracle.postsolve_primal(res, W[k] if res.n_red else np.zeros(0))
    # feasible for the original
    Gi, hi = inequalities(lp.row_ptr, lp.col_idx, lp.val, lp.lhs, lp.rhs, lp.lb, lp.ub, lp.n)
    assert np.all(Gi @ x <= hi + 1e-8 * (1 + np.abs(hi)))
    assert float(lp.c @ x) == pytest.approx(opt, rel=1e-9, abs=1e-9)


def _linprog(c, row_ptr, col_idx, val, lhs, rhs, lb, ub, n):
    from scipy.optimize import linprog
    from scipy.sparse import csr_matrix
    m = len(row_ptr) - 1
    if n == 0:
        return 0, np.zeros(0), 0.0
    A = csr_matrix((val, col_idx, row_ptr), shape=(m, n))
    ub_rows = np.isfinite(rhs)
    lb_rows = np.isfinite(lhs)
    eq = ub_rows & lb_rows & (lhs == rhs)
    A_ub = [A[ub_rows & ~eq], -A[lb_rows & ~eq]]
    b_ub = np.concatenate([rhs[ub_rows & ~eq], -lhs[lb_rows & ~eq]])
    from scipy.sparse import vstack
    A_ub = vstack(A_ub) if b_ub.size else None
    r = linprog(c, A_ub=A_ub, b_ub=b_ub if b_ub.size else None,
                A_eq=A[eq] if eq.any() else None, b_eq=lhs[eq] if eq.any() else None,
                bounds=list(zip(np.where(np.isfinite(lb), lb, None), np.where(np.isfinite(ub), ub, None))),
                method="highs")
    return r.status, r.x, r.fun


@pytest.mark.parametrize("seed", range(8))
def test_reduced_optimum_matches_original_tiny(seed):
    pytest.importorskip("scipy")
    lp = synth.tiny(seed)
    res = oracle.presolve(lp)
    assert res.status == oracle.OK
    st0, x0, f0 = _linprog(lp.c, lp.row_ptr, lp.col_idx, lp.val, lp.lhs, lp.rhs, lp.lb, lp.ub, lp.n)
    st1, x1, f1 = _linprog(res.c, res.row_ptr, res.col_idx, res.val, res.lhs, res.rhs, res.lb, res.ub,
                           res.n_red)
    assert st0 == 0 and st1 == 0
    assert f1 + res.obj_offset == pytest.approx(f0, rel=1e-7, abs=1e-7)
    x = oracle.postsolve_primal(res, x1)
    A = np.zeros((lp.m, lp.n))
    for i in range(lp.m):
        A[i, lp.col_idx[lp.row_ptr[i]:lp.row_ptr[i + 1]]] = lp.val[lp.row_ptr[i]:lp.row_ptr[i + 1]]
    ax = A @ x
    tol = 1e-6 * (1 + np.abs(ax))
    assert np.all(ax >= lp.lhs - tol) and np.all(ax <= lp.rhs + tol)
    assert np.all(x >= lp.lb - 1e-6) and np.all(x <= lp.ub + 1e-6)
    assert float(lp.c @ x) == pytest.approx(f0, rel=1e-7, abs=1e-7)


@pytest.mark.parametrize("seed", range(6))
def test_fixpoint_is_idempotent(seed):
    lp = synth.tiny(seed)
    res = oracle.presolve(lp)
    assert res.status == oracle.OK and res.rounds < 20
    red = synth.LP(m=res.m_red, n=res.n_red, row_ptr=res.row_ptr, col_idx=res.col_idx, val=res.val,
                   c=res.c, lhs=res.lhs, rhs=res.rhs, lb=res.lb, ub=res.ub)
    again = oracle.presolve(red)
    assert again.status == oracle.OK and again.rounds == 1
    assert again.m_red == res.m_red and again.n_red == res.n_red and again.nnz_red == res.nnz_red
    np.testing.assert_array_equal(again.lb, res.lb)
    np.testing.assert_array_equal(again.ub, res.ub)
    np.testing.assert_array_equal(again.lhs, res.lhs)
    np.testing.assert_array_equal(again.rhs, res.rhs)


@pytest.mark.parametrize("seed", range(32))
def test_planted_structures_are_found(seed):
    lp = synth.tiny(seed)
    res = oracle.presolve(lp)
    assert res.status == oracle.OK
    kinds = np.bincount(res.row_kind, minlength=5)
    assert kinds[oracle.ROW_EMPTY] >= 10
    assert kinds[oracle.ROW_SINGLETON] + kinds[oracle.ROW_REDUNDANT] >= 15 + 10
    assert np.count_nonzero(res.col_kind == oracle.COL_FIXED) >= 20
    # every planted pair (source, scaled copy) whose rows both reach S5 of
    # round 1 is merged there, with the planted factor (or its inverse)
    merged = 0
    for (src, cp), lam in zip(lp.planted["pairs"], lp.planted["lambdas"]):
        if any(res.row_kind[r] != oracle.ROW_PARALLEL and res.row_round[r] == 1 for r in (src, cp)):
            continue  # one of them left by an S2 rule first
        if res.row_kind[cp] == oracle.ROW_PARALLEL and res.row_aux[cp] == src:
            assert res.row_val[cp] == pytest.approx(lam, rel=1e-15)
        else:
            assert res.row_kind[src] == oracle.ROW_PARALLEL and res.row_aux[src] == cp
            assert res.row_val[src] == pytest.approx(1.0 / lam, rel=1e-15)
        merged += 1
    assert merged >= 4


def test_parallel_factor_is_the_planted_one():
    hits = 0
    for seed in range(16):
        lp = synth.tiny(seed)
        res = oracle.presolve(lp)
        # rebuild (row -> first coefficient) of the input to check lambda exactly
        first = {i: lp.val[lp.row_ptr[i]] for i in range(lp.m) if lp.row_ptr[i + 1] > lp.row_ptr[i]}
        for j in np.flatnonzero(res.row_kind == oracle.ROW_PARALLEL):
            i = res.row_aux[j]
            lam = res.row_val[j]
            if res.row_round[j] == 1:
                assert lam == first[j] / first[i]
                a_i = lp.val[lp.row_ptr[i]:lp.row_ptr[i + 1]]
                a_j = lp.val[lp.row_ptr[j]:lp.row_ptr[j + 1]]
                np.testing.assert_allclose(a_j, lam * a_i, rtol=1e-12)
                hits += 1
    assert hits >= 16 * 6


def test_tie_audit_on_tiny():
    """The generated LPs keep every decision far from its threshold: no
    decision lies within 10x its worst-case error bound, and most seeds are
    clear by 1000x (the seeds the GPU parity tests use)."""
    clear = 0
    for seed in range(8):
        res = oracle.presolve(synth.tiny(seed))
        assert res.audit_decisions > 0
        assert res.audit_min_ratio > 10.0, (seed, res.audit_min_ratio)
        clear += res.audit_below_1e3 == 0
    assert clear >= 6
