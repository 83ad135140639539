"""The dependent-row step through the C ABI (opts.dep_rows; Sec. 5: the
equality rows' dependencies found on the CPU, the rows removed on the
device by one more compaction).

* Against the oracle's step (oracle/deprows.py) on the same LPs: records
  (kind 7 in round rounds + 1), the reduced LP, maps and the last round's
  activities within the parity bar.
* A planted contradiction is LPP_INFEASIBLE at its row in round rounds + 1.
* Without dependencies the result is the plain run's; with dual records on,
  the primal-dual postsolve of a HiGHS optimum still meets the input LP's
  KKT conditions.
* A batch and a server refuse the option.
"""
import numpy as np
import pytest

import oracle
from oracle import deprows
from paper_2609_16182_gb300 import synth
from parity import compare
import lpsolve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2609_16182_gb300 import lpp  # noqa: E402


def _cases():
    out = [(f"tiny{s}+dep", synth.plant_dependent_rows(synth.tiny(s), s), {}) for s in range(3)]
    out += [(f"mix{s}+dep", synth.plant_dependent_rows(synth.mix(s), s, count=6, terms=2), {}) for s in range(1, 4)]
    out += [("mix5+dep dual fixing", synth.plant_dependent_rows(synth.mix(5), 5, count=5), {"dual_fixing": 1}),
            ("lprelax+dep", synth.plant_dependent_rows(
                synth.lprelax(2, m=800, n=1600, target_nnz=9000, n_dense=1, dense_len=600), 2, count=8), {}),
            ("skewed+dep", synth.plant_dependent_rows(
                synth.skewed(3, m=3000, n=4500, target_nnz=30000, row_cap=2000), 3, count=10), {})]
    return out


CASES = _cases()


@pytest.mark.parametrize("name,lp,kw", CASES, ids=[c[0] for c in CASES])
def test_matches_the_oracle(name, lp, kw):
    r = lpp.presolve(lp, dep_rows=1, **kw)
    o = deprows.presolve(lp, oracle.default_opts(**kw))
    compare(r, o, lp)
    dep = int(np.count_nonzero(o.row_kind == deprows.ROW_DEPENDENT))
    assert dep > 0 and r.info.dep_rows == dep and r.info.dep_stopped == 0
    red = r.reduced()
    assert red.m == o.m_red and red.n == o.n_red
    np.testing.assert_array_equal(red.row_map, o.row_map)
    np.testing.assert_array_equal(red.col_map, o.col_map)
    np.testing.assert_array_equal(red.row_ptr, o.row_ptr)
    np.testing.assert_array_equal(red.col_idx, o.col_idx)


def test_contradiction_is_infeasible():
    lp = synth.plant_dependent_rows(synth.mix(2), 1, count=3, inconsistent=1)
    r = lpp.presolve(lp, dep_rows=1)
    plain = lpp.presolve(lp)
    assert plain.status == lpp.OK
    assert r.status == lpp.INFEASIBLE and r.where == lpp.WHERE_ROW
    assert r.index == int(lp.planted["dependent_rows"][-1]) and r.round == plain.rounds + 1


def test_without_dependencies_the_plain_result():
    lp = synth.tiny(3)
    r, p = lpp.presolve(lp, dep_rows=1), lpp.presolve(lp)
    assert r.info.dep_rows == 0 and r.info.dep_pivots + r.info.dep_peeled > 0
    a, b = r.reduced(), p.reduced()
    for f in ("row_ptr", "col_idx", "val", "lhs", "rhs", "lb", "ub", "row_map", "col_map", "csc_ptr", "csc_idx"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)


class _Red:
    def __init__(self, red):
        for f in ("row_ptr", "col_idx", "val", "c", "lhs", "rhs", "lb", "ub"):
            setattr(self, f, getattr(red, f))


@pytest.mark.parametrize("name,lp,kw", CASES[:4] + CASES[-2:], ids=[c[0] for c in CASES[:4] + CASES[-2:]])
def test_primal_dual_postsolve_with_the_step(name, lp, kw):
    r = lpp.presolve(lp, dep_rows=1, dual_records=1, **kw)
    st, xr, yr, _ = lpsolve.solve(_Red(r.reduced()))
    st0, _, _, f0 = lpsolve.solve(lp)
    assert st == 0 and st0 == 0
    x, y, z = r.postsolve_dual(lp, xr, yr)
    k = lpsolve.kkt(lp, x, y, z)
    assert max(k["primal"], k["z_def"], k["sign"], k["compl"], k["gap"]) < 1e-8, (name, k)
    assert abs(k["pobj"] + float(getattr(lp, "obj_offset", 0.0)) - f0) <= 1e-8 * (1.0 + abs(f0))
    assert np.all(y[r.row_kind == lpp.ROW_DEPENDENT] == 0.0)


def test_refused_by_batch_and_server():
    with pytest.raises(lpp.LppError):
        lpp.presolve_batch([synth.tiny(0), synth.tiny(1)], dep_rows=1)
    with pytest.raises(lpp.LppError):
        lpp.Server(hbm_budget=1 << 30, dep_rows=1)


def test_benchmark_lp_with_planted_dependencies():
    """The benchmark LP (2M rows, 20M nonzeros) with 20 planted dependent
    equality rows: the step finds the planted rows the loop kept (four), and
    the reduced LP is the plain one less the rows it removed."""
    lp = synth.plant_dependent_rows(synth.skewed(0), 0, count=20)
    r = lpp.presolve(lp, dep_rows=1)
    p = lpp.presolve(lp)
    assert r.status == lpp.OK
    dep = np.flatnonzero(r.row_kind == lpp.ROW_DEPENDENT)
    kept_planted = [i for i in lp.planted["dependent_rows"] if p.row_kind[i] == lpp.ROW_KEPT]
    if r.info.dep_stopped == 0:
        assert set(kept_planted) <= set(dep.tolist())
    assert len(dep) == r.info.dep_rows
    a, b = r.reduced(csc=False), p.reduced(csc=False)
    assert a.m == b.m - len(dep)
    np.testing.assert_array_equal(a.row_map, np.setdiff1d(b.row_map, dep))


def test_edge_cases():
    """No equality rows, an empty LP, rows only, and every row removed by the
    rounds: the step finds nothing and the result is the plain run's."""
    from lpmake import make
    INF = np.inf
    lps = [make([{0: 1.0, 1: 1.0}, {1: 2.0, 2: 1.0}], [-INF, 1.0], [4.0, INF], [0, 0, 0], [5, 5, 5],
                c=[1.0, -1.0, 0.5]),                                    # inequalities only
           make([], [], [], [], [], None, n=0),                         # nothing
           make([{}, {}], [-1, 0], [1, 0], [], [], None, n=0),          # rows only, empty
           make([{0: 1.0, 1: 2.0}], [3], [3], [1, 1], [1, 1], [1.0, 1.0])]  # all fixed on input
    for lp in lps:
        r, p = lpp.presolve(lp, dep_rows=1), lpp.presolve(lp)
        assert (r.status, r.info.dep_rows) == (p.status, 0)
        a, b = r.reduced(), p.reduced()
        for f in ("row_ptr", "col_idx", "val", "lhs", "rhs", "row_map", "col_map"):
            np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)
