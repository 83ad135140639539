"""The library's dependent-row elimination (deprows.h, run by lpp_presolve
with dep_rows = 1) built for the host and run on the oracle's reduced LPs:
the same dependent rows, the same contradiction and the same number of
pivot rows as the oracle's dense elimination (oracle/deprows.py); the fill
cap stops it early with what it found valid.  No GPU needed."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import deprows
from paper_2609_16182_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not found")
    out = str(tmp_path_factory.mktemp("dep") / "libdeprows_host.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-o", out,
                    os.path.join(ROOT, "tests", "host", "deprows_host.cpp")], check=True)
    L = C.CDLL(out)
    L.deprows_host.restype = C.c_int64
    return L


def run(L, red, tol=1e-9, max_fill=1 << 40):
    a = lambda v, t: np.ascontiguousarray(v, dtype=t)  # noqa: E731
    m, n = len(red.lhs), len(red.c)
    arrs = [a(red.row_ptr, np.int32), a(red.col_idx, np.int32), a(red.val, float), a(red.lhs, float),
            a(red.rhs, float)]
    dep = np.zeros(max(m, 1), np.int32)
    bad, piv, stopped = C.c_int32(0), C.c_int64(0), C.c_int32(0)
    P = C.c_void_p
    cnt = L.deprows_host(C.c_int64(m), C.c_int64(n), *[P(v.ctypes.data) for v in arrs], C.c_double(tol),
                         C.c_int64(max_fill), P(dep.ctypes.data), C.byref(bad), C.byref(piv), C.byref(stopped))
    return dep[:cnt].tolist(), bad.value, piv.value, stopped.value


CASES = [(f"tiny{s}+dep", lambda s=s: synth.plant_dependent_rows(synth.tiny(s), s)) for s in range(3)]
CASES += [(f"mix{s}+dep", lambda s=s: synth.plant_dependent_rows(synth.mix(s), s, count=6, terms=2))
          for s in range(1, 4)]
CASES += [("contradiction", lambda: synth.plant_dependent_rows(synth.mix(2), 1, count=3, inconsistent=1)),
          ("lprelax+dep", lambda: synth.plant_dependent_rows(
              synth.lprelax(2, m=800, n=1600, target_nnz=9000, n_dense=1, dense_len=600), 2, count=8)),
          ("skewed", lambda: synth.plant_dependent_rows(
              synth.skewed(3, m=3000, n=4500, target_nnz=30000, row_cap=2000), 3, count=10))]


@pytest.mark.parametrize("name,make_lp", CASES, ids=[c[0] for c in CASES])
def test_matches_the_oracle(lib, name, make_lp):
    o = oracle.presolve(make_lp())
    assert o.status == oracle.OK
    dep, bad, piv = deprows.dependent_rows(o, 1e-9)
    got = run(lib, o)
    assert got == (dep, bad, piv, 0)
    if name != "contradiction":
        assert bad < 0 and len(dep) > 0


def test_fill_cap_stops_early_with_valid_rows(lib):
    o = oracle.presolve(synth.plant_dependent_rows(synth.mix(1), 1, count=6, terms=2))
    dep, _, _ = deprows.dependent_rows(o, 1e-9)
    full = run(lib, o)
    capped = run(lib, o, max_fill=50)
    assert capped[3] == 1 and set(capped[0]) <= set(full[0]) and capped[2] < full[2]
    assert full[0] == dep
