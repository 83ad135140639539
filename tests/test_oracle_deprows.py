"""Pins of the oracle's dependent-row step (oracle/deprows.py; Sec. 5: the
equality rows' linear dependencies found on the CPU by pivoting Gaussian
elimination, the result returned to the presolve).

What fixes the step's result, independently of how it eliminates:
* the number of rows it removes is (equality rows) - rank (numpy's SVD rank),
  and the rows peeled before the elimination plus its pivot rows are the rank;
* the equality rows it keeps are independent (full rank);
* every removed row lies in the span of the kept ones, its rhs too (a least
  squares solve);
* a planted contradiction makes the LP infeasible at the planted row;
* the LP it returns has the input LP's optimum (HiGHS on both).
Planted mistakes in the step fail these pins.
"""
import os
import types

import numpy as np
import pytest

import oracle
from oracle import deprows
from paper_2609_16182_gb300 import synth
import lpsolve

INF = np.inf


def _eq_matrix(red, rows=None):
    eq = [i for i in range(len(red.lhs)) if np.isfinite(red.lhs[i]) and red.lhs[i] == red.rhs[i]]
    if rows is not None:
        eq = [i for i in eq if i in rows]
    E = np.zeros((len(eq), len(red.c)))
    for a, i in enumerate(eq):
        k0, k1 = int(red.row_ptr[i]), int(red.row_ptr[i + 1])
        E[a, red.col_idx[k0:k1]] = red.val[k0:k1]
    return eq, E, np.array([red.rhs[i] for i in eq])


def _cases():
    out = [(f"tiny{s}+dep", synth.plant_dependent_rows(synth.tiny(s), s), {}) for s in range(3)]
    out += [(f"mix{s}+dep", synth.plant_dependent_rows(synth.mix(s), s, count=6, terms=2), {}) for s in range(1, 4)]
    out += [("mix5+dep dual fixing", synth.plant_dependent_rows(synth.mix(5), 5, count=5), {"dual_fixing": 1}),
            ("tiny3 (none planted)", synth.tiny(3), {}),
            ("lprelax+dep", synth.plant_dependent_rows(
                synth.lprelax(2, m=800, n=1600, target_nnz=9000, n_dense=1, dense_len=600), 2, count=8), {})]
    return out


CASES = _cases()


@pytest.mark.parametrize("name,lp,kw", CASES, ids=[c[0] for c in CASES])
def test_removed_rows_match_the_rank_and_lie_in_the_span(name, lp, kw):
    o = oracle.presolve(lp, oracle.default_opts(**kw))
    dep, bad, npiv = deprows.dependent_rows(o, 1e-9)
    assert bad < 0
    eq, E, b = _eq_matrix(o)
    rank = np.linalg.matrix_rank(E) if len(eq) else 0
    core, peeled = deprows.core_rows(o)
    assert len(dep) == len(eq) - rank and npiv + peeled == rank and peeled > 0
    kept = [i for i in eq if i not in set(dep)]
    _, K, bk = _eq_matrix(o, set(kept))
    assert np.linalg.matrix_rank(K) == len(kept)
    for i in dep:  # a_i = K^T t and b_i = bk . t for some t
        a = np.zeros(len(o.c))
        k0, k1 = int(o.row_ptr[i]), int(o.row_ptr[i + 1])
        a[o.col_idx[k0:k1]] = o.val[k0:k1]
        t, *_ = np.linalg.lstsq(K.T, a, rcond=None)
        assert np.max(np.abs(K.T @ t - a)) <= 1e-9 * max(1.0, np.max(np.abs(a)))
        assert abs(bk @ t - o.rhs[i]) <= 1e-8 * max(1.0, abs(o.rhs[i]))
    planted = set(lp.planted.get("dependent_rows", np.zeros(0, int)).tolist())
    if planted:  # appended last, so the planted rows the loop kept are the ones found
        assert {int(o.row_map[i]) for i in dep} == {i for i in planted if o.row_kind[i] == oracle.ROW_KEPT}
        assert len(dep) >= len(planted) // 2


def test_contradiction_is_infeasible_at_the_planted_row():
    lp = synth.plant_dependent_rows(synth.mix(2), 1, count=3, inconsistent=1)
    r = deprows.presolve(lp)
    assert r.status == oracle.INFEASIBLE and r.where == oracle.WHERE_ROW
    assert r.index == int(lp.planted["dependent_rows"][-1]) and r.round == oracle.presolve(lp).rounds + 1


def test_hand_case():
    """x + y = 2, y + z = 3, x + 2y + z = 5 (row 0 + row 1), x, y, z free (the
    loop finds nothing): row 2 goes (kind 7, round rounds + 1); with rhs 6
    instead the LP is infeasible at row 2."""
    from lpmake import make
    rows = [{0: 1.0, 1: 1.0}, {1: 1.0, 2: 1.0}, {0: 1.0, 1: 2.0, 2: 1.0}]
    free = ([-INF] * 3, [INF] * 3)
    lp = make(rows, [2, 3, 5], [2, 3, 5], *free, c=[1.0, 0.0, 1.0])
    base = oracle.presolve(lp)
    assert base.status == oracle.OK and base.m_red == 3
    r = deprows.presolve(lp)
    assert r.status == oracle.OK and list(r.row_kind) == [0, 0, deprows.ROW_DEPENDENT]
    assert r.row_round[2] == base.rounds + 1 and list(r.row_map) == [0, 1] and r.m_red == 2
    bad = make(rows, [2, 3, 6], [2, 3, 6], *free, c=[1.0, 0.0, 1.0])
    assert oracle.presolve(bad).status == oracle.OK
    rb = deprows.presolve(bad)
    assert rb.status == oracle.INFEASIBLE and rb.where == oracle.WHERE_ROW and rb.index == 2


class _Red:
    def __init__(self, o):
        for f in ("row_ptr", "col_idx", "val", "c", "lhs", "rhs", "lb", "ub"):
            setattr(self, f, getattr(o, f))


@pytest.mark.parametrize("name,lp,kw", CASES, ids=[c[0] for c in CASES])
def test_the_reduced_lp_keeps_the_optimum(name, lp, kw):
    r = deprows.presolve(lp, oracle.default_opts(**kw))
    assert r.status == oracle.OK
    st, _, _, f = lpsolve.solve(_Red(r))
    st0, _, _, f0 = lpsolve.solve(lp)
    assert st == 0 and st0 == 0
    assert abs(f + r.obj_offset - f0) <= 1e-8 * (1.0 + abs(f0)), (name, f + r.obj_offset, f0)


# -------------------------------------------------------------------- mutants
_MUTANTS = [
    ("elimination adds instead of subtracting", "                w = w - f * p\n", "                w = w + f * p\n"),
    ("rhs not carried along", "                b = b - f * pb\n", "                b = b\n"),
    ("factor inverted", "                f = w[q] / p[q]\n", "                f = p[q] / w[q]\n"),
    ("earlier pivots ignored", "        for q, p, pb in pivots:\n", "        for q, p, pb in pivots[-1:]:\n"),
    ("rhs never checked", "            if bad < 0 and abs(b) > dep_tol * max(1.0, sb):\n",
     "            if False:\n"),
    ("dependent rows left in the reduced LP", "    keep[dep] = False\n", "    keep[:] = True\n"),
    ("peeling rows that share every column", "            if len(cols) and np.any(cnt[cols] == 1):\n",
     "            if len(cols) and np.any(cnt[cols] <= 2):\n"),
]


def _mutant(old, new):
    src = open(deprows.__file__).read()
    assert src.count(old) == 1, old
    mod = types.ModuleType("oracle._deprows_mutant")
    mod.__package__ = "oracle"
    mod.__file__ = os.path.join(os.path.dirname(deprows.__file__), "_deprows_mutant.py")
    exec(compile(src.replace(old, new), mod.__file__, "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("what,old,new", _MUTANTS, ids=[m[0] for m in _MUTANTS])
def test_mutant_fails_a_pin(what, old, new):
    mod = _mutant(old, new)
    fails = 0
    lps = [c for c in CASES] + [("bad", synth.plant_dependent_rows(synth.mix(2), 1, count=3, inconsistent=1), {})]
    for name, lp, kw in lps:
        try:
            o = oracle.presolve(lp, oracle.default_opts(**kw))
            dep, bad, npiv = mod.dependent_rows(o, 1e-9)
            eq, E, _ = _eq_matrix(o)
            want_bad = name == "bad"
            if (bad >= 0) != want_bad:
                fails += 1
                continue
            if len(dep) != len(eq) - (np.linalg.matrix_rank(E) if len(eq) else 0):
                fails += 1
                continue
            if not want_bad:
                r = mod.presolve(lp, oracle.default_opts(**kw))
                if r.m_red != o.m_red - len(dep):
                    fails += 1
                    continue
                st, _, _, f = lpsolve.solve(_Red(r))
                _, _, _, f0 = lpsolve.solve(lp)
                if st != 0 or abs(f + r.obj_offset - f0) > 1e-8 * (1.0 + abs(f0)):
                    fails += 1
        except (ValueError, ZeroDivisionError, IndexError, FloatingPointError):
            fails += 1
    assert fails > 0, what
