"""All opt-in steps of the oracle at once (parallel columns, column
singletons, doubleton equations, dual fixing) on small LPs with every
structure planted: the records of the different steps chain within and
across rounds, and the postsolve undoes them in one latest-first order.
Pinned against vertex enumeration: the reduced LP keeps the optimal value
and the postsolved point is feasible and optimal."""
import numpy as np
import pytest

import oracle
from lpbrute import inequalities, lp_vertices, vertices
from paper_2609_16182_gb300 import synth

ALL = dict(parallel_cols=1, col_singletons=1, doubletons=1, dual_fixing=1)


def planted(seed):
    # small enough for vertex enumeration: 4 base columns + 2 copies + about 1 singleton
    lp = synth.micro(seed + 2100, m=4, n=4)
    lp = synth.plant_parallel_cols(lp, seed, frac=0.5)
    lp = synth.plant_col_singletons(lp, seed, frac=0.5, free_frac=0.0, box=20.0)
    V = lp_vertices(lp)
    return synth.plant_doubletons(lp, seed, count=2, point=V.mean(axis=0) if len(V) else None)


@pytest.mark.parametrize("seed", range(40))
def test_all_steps_optimum_kept_and_postsolve_optimal(seed):
    lp = planted(seed)
    res = oracle.presolve(lp, oracle.default_opts(**ALL))
    V = lp_vertices(lp)
    if len(V) == 0:
        assert res.status == oracle.INFEASIBLE
        return
    assert res.status == oracle.OK
    opt = float(np.min(V @ lp.c))
    if res.n_red:
        G, h = inequalities(res.row_ptr, res.col_idx, res.val, res.lhs, res.rhs, res.lb, res.ub, res.n_red)
        W = vertices(G, h, res.n_red)
        assert len(W) > 0
        xr = W[int(np.argmin(W @ res.c))]
        red_opt = float(xr @ res.c) + res.obj_offset
    else:
        xr = np.zeros(0)
        red_opt = res.obj_offset
    assert red_opt == pytest.approx(opt, rel=1e-9, abs=1e-9)
    x = oracle.postsolve_primal(res, xr)
    Gi, hi = inequalities(lp.row_ptr, lp.col_idx, lp.val, lp.lhs, lp.rhs, lp.lb, lp.ub, lp.n)
    assert np.all(Gi @ x <= hi + 1e-8 * (1 + np.abs(hi)))
    assert float(lp.c @ x) == pytest.approx(opt, rel=1e-9, abs=1e-9)


def test_the_planted_structures_are_used():
    kinds = np.zeros(7, int)
    for seed in range(40):
        res = oracle.presolve(planted(seed), oracle.default_opts(**ALL))
        if res.status == oracle.OK:
            kinds += np.bincount(res.row_kind, minlength=7)[:7]
            kinds[3] += np.count_nonzero(res.col_kind == oracle.COL_PARALLEL)
    # row kinds 5 (substitution) and 6 (doubleton), and merged columns (counted in slot 3)
    assert kinds[5] > 0 and kinds[6] > 0 and kinds[3] >= 10
