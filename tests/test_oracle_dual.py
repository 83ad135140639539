"""Pins of the oracle's dual postsolve (oracle/dual.py) and of the bound-source
records it reads (Sec. 2.1 postsolver, Sec. 3.3: postsolve returns a
primal-dual solution of the input LP).

* Optimality: an independent solver (HiGHS) solves the reduced LP; the
  postsolved triple (x, y, z) must satisfy the KKT conditions of the INPUT LP
  (primal feasibility, dual signs, complementarity, zero duality gap) and
  reach the optimum HiGHS finds on the input LP directly.  Without the dual
  transfers the same triple fails by orders of magnitude (checked below), so
  the pin is not vacuous.
* Records from first principles: the row recorded for a bound side, with the
  bounds that held at the start of the recorded round, implies exactly that
  bound (its residual activity, Sec. 3.1) and no row of the column implies a
  tighter one.  (Which of two rows with equal values is named is decided on
  the oracle's own rounding; this recomputation rounds differently.)
* Mutants: every planted mistake in the dual postsolve fails the KKT pin.
"""
import os
import types

import numpy as np
import pytest

import oracle
from oracle import dual
from paper_2609_16182_gb300 import synth
import lpsolve

INF = np.inf


class _Red:
    def __init__(self, o):
        for f in ("row_ptr", "col_idx", "val", "c", "lhs", "rhs", "lb", "ub"):
            setattr(self, f, getattr(o, f))


def _cases():
    out = [(f"tiny{s}", synth.tiny(s), {}) for s in range(4)]
    out += [(f"mix{s}", synth.mix(s), {}) for s in range(1, 5)]
    out += [(f"micro{s}", synth.micro(s), {}) for s in range(6)]
    out += [(f"late{s}", synth.late_parallel(s, pairs=40), {}) for s in range(2)]
    out += [("skewed", synth.skewed(3, m=3000, n=4500, target_nnz=30000, row_cap=2000), {}),
            ("lprelax", synth.lprelax(1, m=3000, n=6000, target_nnz=40000, n_dense=2, dense_len=1000), {}),
            ("dualfix", synth.mix(5), {"dual_fixing": 1}),
            ("parcols0", synth.parcols(0), {"parallel_cols": 1}),
            ("parcols3 + planted", synth.plant_parallel_cols(synth.tiny(3), 3, frac=0.05), {"parallel_cols": 1}),
            ("colsing0", synth.plant_col_singletons(synth.tiny(0), 0), {"col_singletons": 1}),
            ("colsing2 free", synth.plant_col_singletons(synth.mix(3), 2, frac=0.5, free_frac=1.0), {"col_singletons": 1}),
            ("colsing + parcols + dual fixing", synth.plant_col_singletons(synth.parcols(1), 1),
             {"col_singletons": 1, "parallel_cols": 1, "dual_fixing": 1})]
    from lpmake import make
    # row 1 implies x0, x1 <= 4 in round 1 and is then merged into row 0
    # (twice row 0): a transfer lands on a merged row
    out += [("follower_transfer", make([{0: 1.0, 1: 1.0}, {0: 2.0, 1: 2.0}], [-INF, -INF], [10.0, 8.0], [0, 0],
                                       [10, 10], c=[-2.0, -1.0]), {})]
    return out


_CACHE = {}


def _solved():
    if not _CACHE:
        for name, lp, kw in _cases():
            o = oracle.presolve(lp, oracle.default_opts(**kw))
            assert o.status == 0, name
            st, xr, yr, _ = lpsolve.solve(_Red(o))
            st0, _, _, f0 = lpsolve.solve(lp)
            assert st == 0 and st0 == 0, name
            _CACHE[name] = (lp, o, xr, yr, f0 + float(getattr(lp, "obj_offset", 0.0)))
    return _CACHE


def _check(lp, o, xr, yr, f0, fn=dual.postsolve_dual, tol=1e-8):
    x, y, z = fn(lp, o, xr, yr)
    k = lpsolve.kkt(lp, x, y, z)
    bad = {a: b for a, b in k.items() if a in ("primal", "z_def", "sign", "compl", "gap") and not b <= tol}
    obj = k["pobj"] + float(getattr(lp, "obj_offset", 0.0))
    if abs(obj - f0) > tol * (1.0 + abs(f0)):
        bad["objective"] = obj - f0
    return bad, y


def test_dual_postsolve_is_optimal_for_the_input_lp():
    moved = fam = 0
    for name, (lp, o, xr, yr, f0) in _solved().items():
        bad, y = _check(lp, o, xr, yr, f0)
        assert not bad, (name, bad)
        moved += int(((y != 0) & (o.row_kind != oracle.ROW_KEPT)).sum())
        fam += int(((y != 0) & (o.row_kind == oracle.ROW_PARALLEL)).sum())
    assert moved > 100 and fam > 0  # transfers to removed rows and to merged rows happened


def test_without_the_transfers_the_pin_fails():
    fails = 0
    for name, (lp, o, xr, yr, f0) in _solved().items():
        y = np.zeros(lp.m)
        y[o.row_map] = yr
        z = dual.reduced_costs(lp, y)
        k = lpsolve.kkt(lp, oracle.postsolve_primal(o, xr), y, z)
        fails += k["compl"] > 1e-3 or k["sign"] > 1e-3
    assert fails >= 8


def test_hand_case_singleton_row_takes_the_dual():
    """min -x0 - x1 s.t. x0 + x1 <= 4 (row 0), x0 <= 1 (row 1, a singleton
    row), 0 <= x <= 10.  Presolve turns row 1 into the bound x0 <= 1; the
    reduced optimum (x0, x1) = (1, 3) has y0 = -1 and z_x0 = 0 at the
    reduced level, so nothing moves: row 1's dual is 0.  With costs (-2, -1)
    instead, z_x0 = -1 at x0's bound 1, which row 1 implied: y1 = -1,
    the input LP's dual (y0, y1) = (-1, -1), objective -2 - 3 = -5."""
    from lpmake import make
    lp = make([{0: 1.0, 1: 1.0}, {0: 1.0}], [-INF, -INF], [4.0, 1.0], [0, 0], [10, 10], c=[-2.0, -1.0])
    o = oracle.presolve(lp)
    assert o.row_kind[1] == oracle.ROW_SINGLETON and o.col_usrc[0] == 1 and o.col_urnd[0] == 1
    st, xr, yr, _ = lpsolve.solve(_Red(o))
    x, y, z = dual.postsolve_dual(lp, o, xr, yr)
    np.testing.assert_allclose(x, [1.0, 3.0], atol=1e-12)
    np.testing.assert_allclose(y, [-1.0, -1.0], atol=1e-12)
    np.testing.assert_allclose(z, [0.0, 0.0], atol=1e-12)


def test_hand_case_parallel_follower_holds_the_side():
    """Row 1 = 2 * row 0 with the tighter side: x0 + x1 <= 10 and
    2x0 + 2x1 <= 8, min -x0 - x1 over 0 <= x <= 10.  S5 merges row 1 into row
    0 (rhs 4); the reduced dual -1 of row 0 belongs to row 1, whose side is
    the tight one: y = (0, -1/2)."""
    from lpmake import make
    lp = make([{0: 1.0, 1: 1.0}, {0: 2.0, 1: 2.0}], [-INF, -INF], [10.0, 8.0], [0, 0], [10, 10], c=[-1.0, -1.0])
    o = oracle.presolve(lp)
    assert o.row_kind[1] == oracle.ROW_PARALLEL and o.row_aux[1] == 0
    st, xr, yr, _ = lpsolve.solve(_Red(o))
    x, y, z = dual.postsolve_dual(lp, o, xr, yr)
    np.testing.assert_allclose(y, [0.0, -0.5], atol=1e-12)
    assert lpsolve.kkt(lp, x, y, z)["compl"] < 1e-12


# ----------------------------------------------------- records from first principles
def _bounds_at_round_start(lp, t, kw):
    """Column bounds as they stood at the start of round t (t >= 1)."""
    l, u = lpsolve._inf(lp.lb), lpsolve._inf(lp.ub)
    if t == 1:
        return l, u
    o = oracle.presolve(lp, oracle.default_opts(max_rounds=t - 1, **kw))
    return o.col_lb.copy(), o.col_ub.copy()


def _implied(lp, r, j, B, upper, sides):
    """The bound on x_j that row r (with sides `sides`) implies under bounds B
    = (l, u): the row's residual activity over its other columns."""
    l, u = B
    L, U = sides
    a = None
    rmin = rmax = 0.0
    for k in range(int(lp.row_ptr[r]), int(lp.row_ptr[r + 1])):
        c, v = int(lp.col_idx[k]), float(lp.val[k])
        if c == j:
            a = v
            continue
        lo, hi = (v * l[c], v * u[c]) if v > 0 else (v * u[c], v * l[c])
        rmin += lo
        rmax += hi
    if a is None:
        return None
    # a x_j <= U - rmin and a x_j >= L - rmax
    if upper:
        return (U - rmin) / a if a > 0 else (L - rmax) / a
    return (L - rmax) / a if a > 0 else (U - rmin) / a


def _sides_at(lp, o, r, t):
    """Row r's sides at round t: its own, tightened by the rows merged into it
    (directly or through merges into those) in rounds before t."""
    L, U = float(lpsolve._inf(lp.lhs)[r]), float(lpsolve._inf(lp.rhs)[r])
    for f in np.flatnonzero(o.row_kind == oracle.ROW_PARALLEL):
        g, lam, ok = int(f), 1.0, True
        while o.row_kind[g] == oracle.ROW_PARALLEL and g != r:
            ok &= int(o.row_round[g]) < t
            lam *= float(o.row_val[g])
            g = int(o.row_aux[g])
        if g != r or not ok or int(f) == r:
            continue
        fl, fu = float(lpsolve._inf(lp.lhs)[f]), float(lpsolve._inf(lp.rhs)[f])
        lo, hi = (fl / lam, fu / lam) if lam > 0 else (fu / lam, fl / lam)
        L, U = max(L, lo), min(U, hi)
    return L, U


@pytest.mark.parametrize("name", ["tiny0", "mix1", "mix3", "skewed", "lprelax"])
def test_records_name_the_row_that_implies_the_bound(name):
    cases = {c[0]: c for c in _cases()}
    _, lp, kw = cases[name]
    o = oracle.presolve(lp, oracle.default_opts(**kw))
    rows_of = {}
    for i in range(lp.m):
        for k in range(int(lp.row_ptr[i]), int(lp.row_ptr[i + 1])):
            rows_of.setdefault(int(lp.col_idx[k]), []).append(i)
    starts, ends, checked = {}, {}, 0
    for upper, src, rnd in ((False, o.col_lsrc, o.col_lrnd), (True, o.col_usrc, o.col_urnd)):
        for j in np.flatnonzero(src >= 0):
            r, t = int(src[j]), int(rnd[j])
            assert 1 <= t <= o.rounds
            if t not in starts:
                starts[t] = _bounds_at_round_start(lp, t, kw)
                e = oracle.presolve(lp, oracle.default_opts(max_rounds=t, **kw))
                ends[t] = (e.col_lb.copy(), e.col_ub.copy(), e.col_kind.copy())
            lb_t, ub_t, ck_t = ends[t]
            if ck_t[j] == oracle.COL_EMPTY:
                continue  # fixed by its cost (S6) in the same round: the value is not the bound
            B = starts[t]
            got = ub_t[j] if upper else lb_t[j]
            v = _implied(lp, r, j, B, upper, _sides_at(lp, o, r, t))
            assert v is not None, (j, r)
            tol = 1e-9 * max(1.0, abs(got)) + (2e-9 * max(1.0, abs(got)) if ck_t[j] == oracle.COL_FIXED else 0.0)
            assert abs(v - got) <= tol, (name, j, upper, r, t, v, got)
            # no row of the column implies a tighter value
            for i in rows_of.get(int(j), []):
                if int(o.row_round[i]) < t and o.row_kind[i] != oracle.ROW_KEPT:
                    continue  # gone before round t
                w = _implied(lp, i, j, B, upper, _sides_at(lp, o, i, t))
                if w is None or not np.isfinite(w) or abs(w) > 1e10:
                    continue
                tighter = (w < v - 1e-9 * max(1.0, abs(v))) if upper else (w > v + 1e-9 * max(1.0, abs(v)))
                assert not tighter, (name, j, upper, r, i, v, w)
            checked += 1
    assert checked >= 20


# -------------------------------------------------------------------- mutants
_MUTANTS = [
    ("transfer sign", "        y[r] += d\n", "        y[r] -= d\n"),
    ("no transfers", "        if (upper and not z[j] < 0.0) or (not upper and not z[j] > 0.0):\n",
     "        if True:\n"),
    ("transfer of either sign", "        if (upper and not z[j] < 0.0) or (not upper and not z[j] > 0.0):\n",
     "        if z[j] == 0.0:\n"),
    ("transfer scaled the wrong way", "        d = z[j] / a_rj\n", "        d = z[j] * a_rj\n"),
    ("family orientation", "            lower_side = (lam[g] > 0) == (Y > 0)\n",
     "            lower_side = (lam[g] > 0) != (Y > 0)\n"),
    ("family dual not rescaled", "        y[best] = Y / lam[best]\n", "        y[best] = Y\n"),
    ("families skipped", "    for rt, mem in members.items():\n", "    for rt, mem in []:\n"),
    ("loosest member", "            if rres < best_res:\n", "            if best < 0 or rres > best_res:\n"),
    ("family dual summed unscaled", "        Y = sum(y[g] * lam[g] for g in mem)\n",
     "        Y = sum(y[g] for g in mem)\n"),
    ("substitution rows keep no dual", "        y[i] += zj / float(res.row_val[i])\n", "        pass\n"),
    ("substitution dual from the cost alone", "            zj -= a * y[r]\n", "            pass\n"),
]


def _mutant(old, new):
    src = open(dual.__file__).read()
    assert src.count(old) == 1, old
    mod = types.ModuleType("oracle._dual_mutant")
    mod.__package__ = "oracle"
    mod.__file__ = os.path.join(os.path.dirname(dual.__file__), "_dual_mutant.py")
    exec(compile(src.replace(old, new), mod.__file__, "exec"), mod.__dict__)
    return mod.postsolve_dual


@pytest.mark.parametrize("what,old,new", _MUTANTS, ids=[m[0] for m in _MUTANTS])
def test_mutant_fails_the_pin(what, old, new):
    fn = _mutant(old, new)
    caught = False
    for name, (lp, o, xr, yr, f0) in _solved().items():
        try:
            bad, _ = _check(lp, o, xr, yr, f0, fn=fn)
        except (ValueError, ZeroDivisionError, IndexError):
            bad = True
        if bad:
            caught = True
            break
    assert caught, what
