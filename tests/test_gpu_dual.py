"""Dual records and the primal-dual postsolve through the C ABI
(opts.dual_records, lpp_result_bound_sources, lpp_postsolve_dual; Sec. 2.1
postsolver, Sec. 3.3).

* Bound sources against the oracle's: the same row and round for every
  column side, except where the two sides' activity sums (summed in another
  order) make a different row win a near tie; there both rows must imply
  the final bound, re-derived from first principles.  No side is left
  without its row (-2).
* The primal-dual postsolve of a HiGHS optimum of the GPU's reduced LP is a
  KKT point of the input LP with the optimum HiGHS finds on the input LP.
* Batched runs give every member its solo records; refusals are errors.
"""
import numpy as np
import pytest

import oracle
from paper_2609_16182_gb300 import synth
import lpsolve
from test_oracle_dual import _bounds_at_round_start, _implied, _sides_at

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2609_16182_gb300 import lpp  # noqa: E402


def _cases():
    from lpmake import make
    INF = np.inf
    out = [(f"tiny{s}", synth.tiny(s), {}) for s in range(3)]
    out += [(f"mix{s}", synth.mix(s), {}) for s in range(1, 4)]
    out += [("late", synth.late_parallel(1, pairs=40), {}),
            ("skewed", synth.skewed(3, m=3000, n=4500, target_nnz=30000, row_cap=2000), {}),
            ("skewed_long", synth.skewed(4, m=8000, n=12000, target_nnz=90_000, row_cap=9000), {}),
            ("lprelax", synth.lprelax(1, m=3000, n=6000, target_nnz=40000, n_dense=2, dense_len=2500), {}),
            ("dualfix", synth.mix(5), {"dual_fixing": 1}),
            ("parcols", synth.parcols(0), {"parallel_cols": 1}),
            ("colsing", synth.plant_col_singletons(synth.tiny(0), 0), {"col_singletons": 1}),
            ("colsing + parcols + dual fixing", synth.plant_col_singletons(synth.parcols(1), 1),
             {"col_singletons": 1, "parallel_cols": 1, "dual_fixing": 1}),
            ("follower_transfer", make([{0: 1.0, 1: 1.0}, {0: 2.0, 1: 2.0}], [-INF, -INF], [10.0, 8.0], [0, 0],
                                       [10, 10], c=[-2.0, -1.0]), {})]
    return out


CASES = _cases()


def _src_check(name, lp, got, o, kw):
    """got: the library's bound sources; o: the oracle's result."""
    starts = {}
    mism = 0
    for side, upper in (("l", False), ("u", True)):
        gs, gr = got[side + "src"], got[side + "rnd"]
        os_, or_ = getattr(o, f"col_{side}src"), getattr(o, f"col_{side}rnd")
        assert (gs >= -1).all(), (name, "a side without its source row")
        np.testing.assert_array_equal(gs >= 0, os_ >= 0, err_msg=f"{name}: sides with a source ({side})")
        np.testing.assert_array_equal(gr, or_, err_msg=f"{name}: rounds ({side})")
        for j in np.flatnonzero(gs != os_):
            mism += 1
            t = int(gr[j])
            if t not in starts:
                starts[t] = _bounds_at_round_start(lp, t, kw)
            vg = _implied(lp, int(gs[j]), int(j), starts[t], upper, _sides_at(lp, o, int(gs[j]), t))
            vo = _implied(lp, int(os_[j]), int(j), starts[t], upper, _sides_at(lp, o, int(os_[j]), t))
            assert vg is not None and abs(vg - vo) <= 1e-9 * max(1.0, abs(vo)), (name, j, side, gs[j], os_[j], vg, vo)
    return mism


@pytest.mark.parametrize("name,lp,kw", CASES, ids=[c[0] for c in CASES])
def test_bound_sources_match_the_oracle(name, lp, kw):
    r = lpp.presolve(lp, dual_records=1, **kw)
    o = oracle.presolve(lp, oracle.default_opts(**kw))
    assert r.status == o.status == 0
    got = r.bound_sources()
    mism = _src_check(name, lp, got, o, kw)
    assert mism <= max(2, (got["lsrc"] >= 0).sum() // 100), (name, mism)
    # the same presolve without the records: the same reduced LP
    plain = lpp.presolve(lp, **kw)
    a, b = r.reduced(), plain.reduced()
    for f in ("row_ptr", "col_idx", "val", "lhs", "rhs", "lb", "ub", "row_map", "col_map"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)


class _Red:
    def __init__(self, red):
        for f in ("row_ptr", "col_idx", "val", "c", "lhs", "rhs", "lb", "ub"):
            setattr(self, f, getattr(red, f))


@pytest.mark.parametrize("name,lp,kw", CASES, ids=[c[0] for c in CASES])
def test_dual_postsolve_is_optimal_for_the_input_lp(name, lp, kw):
    r = lpp.presolve(lp, dual_records=1, **kw)
    red = r.reduced()
    np.testing.assert_array_equal(red.row_map, np.flatnonzero(r.row_kind == lpp.ROW_KEPT))
    st, xr, yr, fr = lpsolve.solve(_Red(red))
    st0, _, _, f0 = lpsolve.solve(lp)
    assert st == 0 and st0 == 0
    x, y, z = r.postsolve_dual(lp, xr, yr)
    np.testing.assert_array_equal(x, r.postsolve_primal(xr))
    k = lpsolve.kkt(lp, x, y, z)
    assert max(k["primal"], k["z_def"], k["sign"], k["compl"], k["gap"]) < 1e-8, (name, k)
    obj = k["pobj"] + float(getattr(lp, "obj_offset", 0.0))
    assert abs(obj - f0) <= 1e-8 * (1.0 + abs(f0)), (name, obj, f0)


def test_batch_members_get_their_solo_records():
    lps = [c[1] for c in CASES if c[2] == {}]
    res = lpp.presolve_batch(lps, dual_records=1)
    assert res[0].info.launches > 0
    for lp, b in zip(lps, res):
        s = lpp.presolve(lp, dual_records=1)
        gb, gs = b.bound_sources(), s.bound_sources()
        for f in gb:
            np.testing.assert_array_equal(gb[f], gs[f], err_msg=f)


def test_refusals():
    lp = synth.mix(2)
    r = lpp.presolve(lp)
    with pytest.raises(lpp.LppError):
        r.bound_sources()
    with pytest.raises(lpp.LppError):
        r.postsolve_dual(lp, np.zeros(r.info.n_red), np.zeros(r.info.m_red))
    db = synth.plant_doubletons(synth.tiny(5), 5, count=6)
    p = lpp.presolve(db, dual_records=1, doubletons=1)
    assert (p.col_kind == lpp.COL_DOUBLETON).any()
    with pytest.raises(lpp.LppError):
        p.postsolve_dual(db, np.zeros(p.info.n_red), np.zeros(p.info.m_red))
    d = lpp.presolve(lp, dual_records=1)
    with pytest.raises(lpp.LppError):  # another LP's sizes
        d.postsolve_dual(synth.micro(0), np.zeros(d.info.n_red), np.zeros(d.info.m_red))
    with pytest.raises(lpp.LppError):
        lpp.Server(hbm_budget=1 << 30, dual_records=1)


def test_full_size_records_are_valid_at_sampled_columns():
    """The benchmark LP (skewed, 2M rows, 3M columns, 20M nonzeros; 740
    columns longer than a warp's share) with the records on: every side has
    its row, the reduced LP equals the run without records, and at 200
    sampled sides set in round 1 the named row implies the bound they have
    after round 1 (input bounds, the row's own sides)."""
    lp = synth.skewed(0)
    r = lpp.presolve(lp, dual_records=1)
    plain = lpp.presolve(lp)
    a, b = r.reduced(csc=False), plain.reduced(csc=False)
    for f in ("row_ptr", "col_idx", "lb", "ub", "row_map", "col_map"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)
    src = r.bound_sources()
    assert (src["lsrc"] >= -1).all() and (src["usrc"] >= -1).all()
    one = lpp.presolve(lp, max_rounds=1)
    l, u = lpsolve._inf(lp.lb), lpsolve._inf(lp.ub)
    L, U = lpsolve._inf(lp.lhs), lpsolve._inf(lp.rhs)
    rng = np.random.default_rng(0)
    checked = 0
    for side, upper, fin in (("l", False, one.col_lb), ("u", True, one.col_ub)):
        cand = np.flatnonzero((src[side + "rnd"] == 1) & (one.col_kind == lpp.COL_KEPT))
        for j in rng.choice(cand, size=min(100, len(cand)), replace=False):
            rr = int(src[side + "src"][j])
            k0, k1 = int(lp.row_ptr[rr]), int(lp.row_ptr[rr + 1])
            cols, vals = lp.col_idx[k0:k1], lp.val[k0:k1]
            me = cols == j
            assert me.sum() == 1, (j, rr)
            a_j = float(vals[me][0])
            oc, ov = cols[~me], vals[~me]
            rmin = float(np.sum(np.where(ov > 0, ov * l[oc], ov * u[oc])))
            rmax = float(np.sum(np.where(ov > 0, ov * u[oc], ov * l[oc])))
            if upper:
                v = (U[rr] - rmin) / a_j if a_j > 0 else (L[rr] - rmax) / a_j
            else:
                v = (L[rr] - rmax) / a_j if a_j > 0 else (U[rr] - rmin) / a_j
            got = fin[j]  # the side's last change came in round 1: its bound after round 1
            side_v = U[rr] if (upper == (a_j > 0)) else L[rr]
            scale = (abs(side_v) + float(np.sum(np.abs(ov) * np.where(np.isfinite(l[oc]), np.abs(l[oc]), 0)))
                     + float(np.sum(np.abs(ov) * np.where(np.isfinite(u[oc]), np.abs(u[oc]), 0)))) / abs(a_j)
            assert abs(v - got) <= 1e-9 * max(1.0, abs(got)) + 1e-12 * scale, (j, side, rr, v, got)
            checked += 1
    assert checked >= 100


def test_edge_cases():
    """An LP the rounds reduce to nothing (empty reduced pair), and an
    infeasible LP (refused: no primal-dual solution to map)."""
    from lpmake import INF, make
    lp = make([{0: 1.0, 1: 2.0}], [3], [3], [1, 1], [1, 1], [1.0, 1.0])
    r = lpp.presolve(lp, dual_records=1)
    assert r.info.m_red == 0 and r.info.n_red == 0
    x, y, z = r.postsolve_dual(lp, np.zeros(0), np.zeros(0))
    np.testing.assert_array_equal(x, [1.0, 1.0])
    k = lpsolve.kkt(lp, x, y, z)
    assert max(k["primal"], k["sign"], k["compl"]) < 1e-12
    bad = make([{0: 1.0, 1: 1.0}], lhs=[5], rhs=[INF], lb=[0, 0], ub=[1, 1])
    rb = lpp.presolve(bad, dual_records=1)
    assert rb.status == lpp.INFEASIBLE
    with pytest.raises(lpp.LppError):
        rb.postsolve_dual(bad, np.zeros(rb.info.n_red), np.zeros(rb.info.m_red))
