"""The library's dual postsolve (postsolve.h postsolve_dual, the code behind
lpp_postsolve_dual) built for the host and run on the oracle's records and a
reduced optimum from HiGHS: the same duals and reduced costs as the oracle's
dual postsolve (oracle/dual.py), bit for bit, and a KKT point of the input
LP, with and without parallel-column merges and column-singleton
substitutions.  Refusal: records of doubletons (no dual postsolve).  No GPU needed."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import dual
from paper_2609_16182_gb300 import synth
import lpsolve

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not found")
    out = str(tmp_path_factory.mktemp("dual") / "libpostsolve_host.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-o", out,
                    os.path.join(ROOT, "tests", "host", "postsolve_host.cpp")], check=True)
    L = C.CDLL(out)
    L.postsolve_dual_host.restype = C.c_int32
    return L


def run(L, lp, o, x, y_red):
    a = lambda v, t: np.ascontiguousarray(v, dtype=t)  # noqa: E731
    row_map = a(np.flatnonzero(o.row_kind == oracle.ROW_KEPT), np.int32)
    assert np.array_equal(row_map, o.row_map)  # the reduced rows are the kept rows in order
    arrs = [a(lp.row_ptr, np.int32), a(lp.col_idx, np.int32), a(lp.val, float), a(lp.c, float), a(lp.lhs, float),
            a(lp.rhs, float)]
    recs = [row_map, a(o.row_kind, np.int32), a(o.row_round, np.int32), a(o.row_aux, np.int32), a(o.row_val, float),
            a(o.col_kind, np.int32),
            a(o.col_lsrc, np.int32), a(o.col_lrnd, np.int32), a(o.col_usrc, np.int32), a(o.col_urnd, np.int32),
            a(x, float), a(y_red, float)]
    y, z = np.full(lp.m, np.nan), np.full(lp.n, np.nan)
    P = C.c_void_p
    rc = L.postsolve_dual_host(C.c_int64(lp.m), C.c_int64(lp.n), C.c_int64(len(row_map)),
                               *[P(v.ctypes.data) for v in arrs], C.c_double(1e20),
                               *[P(v.ctypes.data) for v in recs], P(y.ctypes.data), P(z.ctypes.data))
    return rc, y, z


class _Red:
    def __init__(self, o):
        for f in ("row_ptr", "col_idx", "val", "c", "lhs", "rhs", "lb", "ub"):
            setattr(self, f, getattr(o, f))


CASES = [("tiny", lambda s: synth.tiny(s), {}), ("mix", lambda s: synth.mix(s), {}),
         ("late_parallel", lambda s: synth.late_parallel(s, pairs=40), {}),
         ("dual_fixing", lambda s: synth.mix(s), {"dual_fixing": 1}),
         ("skewed", lambda s: synth.skewed(s, m=3000, n=4500, target_nnz=30000, row_cap=2000), {}),
         ("parallel_cols", lambda s: synth.parcols(s), {"parallel_cols": 1}),
         ("col_singletons", lambda s: synth.plant_col_singletons(synth.tiny(s), s), {"col_singletons": 1}),
         ("all but doubletons", lambda s: synth.plant_col_singletons(synth.parcols(s), s),
          {"col_singletons": 1, "parallel_cols": 1, "dual_fixing": 1})]


@pytest.mark.parametrize("name, make_lp, kw", CASES, ids=[c[0] for c in CASES])
def test_matches_the_oracle_and_is_optimal(lib, name, make_lp, kw):
    done = 0
    for seed in range(3):
        lp = make_lp(seed)
        o = oracle.presolve(lp, oracle.default_opts(**kw))
        if o.status != oracle.OK:
            continue
        st, xr, yr, _ = lpsolve.solve(_Red(o))
        if st != 0:
            continue
        x0, y0, z0 = dual.postsolve_dual(lp, o, xr, yr)
        rc, y, z = run(lib, lp, o, x0, yr)
        assert rc == 0
        np.testing.assert_array_equal(y, y0)
        np.testing.assert_array_equal(z, z0)
        k = lpsolve.kkt(lp, x0, y, z)
        assert max(k["primal"], k["sign"], k["compl"], k["gap"]) < 1e-8, k
        done += 1
    assert done >= 2


def test_refuses_records_without_a_dual_postsolve(lib):
    lp = synth.plant_doubletons(synth.tiny(5), 5, count=6)
    o = oracle.presolve(lp, oracle.default_opts(doubletons=1))
    assert (o.col_kind == oracle.COL_DOUBLETON).any()
    rc, _, _ = run(lib, lp, o, np.zeros(lp.n), np.zeros(o.m_red))
    assert rc == -1
