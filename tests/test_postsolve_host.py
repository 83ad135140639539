"""The library's primal postsolve (postsolve.h, the code behind
lpp_postsolve_primal) built for the host and run on the oracle's records,
against the oracle's own postsolve: fixed values, merges, column-singleton
substitutions and doubletons undone in the same order give the same point,
bit for bit.  Records of doubletons come from the oracle only (the device
step is not enabled), so this is where the library's handling of them is
checked.  No GPU needed."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2609_16182_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not found")
    out = str(tmp_path_factory.mktemp("post") / "libpostsolve_host.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-o", out,
                    os.path.join(ROOT, "tests", "host", "postsolve_host.cpp")], check=True)
    L = C.CDLL(out)
    L.postsolve_host.restype = C.c_int32
    return L


def run(L, o, x_red):
    a = lambda x, t: np.ascontiguousarray(x, dtype=t)  # noqa: E731
    arrs = [a(o.col_kind, np.int32), a(o.col_round, np.int32), a(o.col_aux, np.int32), a(o.col_map, np.int32),
            a(o.col_val, float), a(np.asarray(o.col_mrg).reshape(-1), float), a(o.row_kind, np.int32),
            a(o.row_round, np.int32), a(o.row_aux, np.int32), a(o.row_val, float), a(o.sub_beg, np.int64),
            a(o.sub_len, np.int32), a(o.sub_col, np.int32), a(o.sub_rhs, float), a(o.sub_val, float)]
    xr = a(x_red, float)
    n = len(o.col_kind)
    x = np.full(n, np.nan)
    P = C.c_void_p
    rc = L.postsolve_host(C.c_int64(n), C.c_int64(len(o.row_kind)), C.c_int64(len(o.col_map)),
                          *[P(v.ctypes.data) for v in arrs], C.c_int64(len(o.sub_col)), P(xr.ctypes.data),
                          P(x.ctypes.data))
    assert rc == 0
    return x


def reduced_point(o, rng):
    lo = np.where(np.isfinite(o.lb), o.lb, -5.0)
    hi = np.where(np.isfinite(o.ub), o.ub, 5.0)
    return lo + (hi - lo) * rng.random(len(lo))


CASES = [
    ("plain", lambda s: synth.tiny(s), {}),
    ("merges", lambda s: synth.parcols(s), dict(parallel_cols=1)),
    ("substitutions", lambda s: synth.plant_col_singletons(synth.tiny(s), s), dict(col_singletons=1)),
    ("doubletons", lambda s: synth.plant_doubletons(synth.tiny(s), s, count=6), dict(doubletons=1)),
    ("all", lambda s: synth.plant_doubletons(synth.plant_col_singletons(synth.parcols(s), s), s, count=6),
     dict(parallel_cols=1, col_singletons=1, doubletons=1, dual_fixing=1)),
]


@pytest.mark.parametrize("name, make_lp, kw", CASES, ids=[c[0] for c in CASES])
def test_matches_the_oracle(lib, name, make_lp, kw):
    kinds = set()
    for seed in range(6):
        lp = make_lp(seed)
        o = oracle.presolve(lp, oracle.default_opts(**kw))
        if o.status != oracle.OK:
            continue
        kinds |= set(np.unique(o.row_kind).tolist()) | set(np.unique(o.col_kind).tolist())
        rng = np.random.default_rng(seed)
        for _ in range(3):
            xr = reduced_point(o, rng)
            np.testing.assert_array_equal(run(lib, o, xr), oracle.postsolve_primal(o, xr))
    want = {"merges": oracle.COL_PARALLEL, "substitutions": oracle.ROW_SUBST, "doubletons": oracle.ROW_DOUBLETON}
    if name in want:
        assert want[name] in kinds  # the records of the case were exercised


def test_corrupt_records_are_reported(lib):
    for seed in range(10):
        lp = synth.plant_doubletons(synth.tiny(seed), seed, count=6)
        o = oracle.presolve(lp, oracle.default_opts(doubletons=1))
        if o.status == oracle.OK and np.any(o.row_kind == oracle.ROW_DOUBLETON):
            break
    i = int(np.flatnonzero(o.row_kind == oracle.ROW_DOUBLETON)[0])
    o.sub_beg[i] = len(o.sub_col) + 5
    with pytest.raises(AssertionError):
        run(lib, o, reduced_point(o, np.random.default_rng(0)))
