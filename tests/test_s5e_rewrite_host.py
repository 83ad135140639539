"""The S5e row rewrite's index arithmetic (doubleton equations, Sec. 2.1),
compiled for the host and run on random rows, against a plain rebuild: x_k
out, x_j's coefficient merged (dropped when it cancels within par_tol) or
inserted in column order.  Every placement stays inside the new row and
every slot is written once (no GPU needed)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PAR_TOL = 1e-12


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("s5e") / "libs5e_host.so")
    src = os.path.join(ROOT, "tests", "host", "s5e_rewrite_host.cu")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-fmad=false", "-shared", "-Xcompiler", "-fPIC",
                    "-Xcompiler", "-ffp-contract=off", "-o", out, src], check=True)
    L = C.CDLL(out)
    P = C.c_void_p
    L.s5e_rewrite_row.argtypes = [P, P, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double, P, P, P]
    L.s5e_rewrite_row.restype = C.c_int32
    return L


def plain(idx, val, jj, kk, d):
    cols, vals, placed = [], [], False
    for c, v in zip(idx.tolist(), val.tolist()):
        if c == kk:
            continue
        if not placed and c > jj:
            cols.append(jj), vals.append(d)
            placed = True
        if c == jj:
            placed = True
            s = v + d
            if abs(s) <= PAR_TOL * max(abs(v), abs(d)):
                continue
            cols.append(jj), vals.append(s)
            continue
        cols.append(c), vals.append(v)
    if not placed:
        cols.append(jj), vals.append(d)
    return cols, vals


def run(L, idx, val, jj, kk, d):
    n = len(idx)
    oi = np.full(n + 1, -7, np.int32)
    ov = np.full(n + 1, np.nan)
    w = np.zeros(n + 1, np.int32)
    ln = L.s5e_rewrite_row(idx.ctypes.data, val.ctypes.data, n, jj, kk, d, PAR_TOL, oi.ctypes.data,
                           ov.ctypes.data, w.ctypes.data)
    assert ln >= 0, ("a placement left the row", ln)
    assert np.all(w[:ln] == 1) and np.all(w[ln:] == 0)
    return oi[:ln].tolist(), ov[:ln].tolist()


@pytest.mark.parametrize("seed", range(40))
def test_random_rows(lib, seed):
    rng = np.random.default_rng(seed)
    for _ in range(200):
        n = int(rng.integers(1, 40))
        idx = np.sort(rng.choice(60, size=n, replace=False)).astype(np.int32)
        val = rng.uniform(-3, 3, n)
        kk = int(idx[rng.integers(n)])
        case = rng.integers(3)
        others = [c for c in idx.tolist() if c != kk]
        if case == 0 or not others:  # x_j absent: inserted
            jj = int(rng.choice([c for c in range(61) if c not in idx.tolist()]))
            d = float(rng.uniform(-2, 2))
        else:
            jj = int(rng.choice(others))
            v = float(val[np.flatnonzero(idx == jj)[0]])
            d = -v if case == 1 else float(rng.uniform(-2, 2))  # case 1: exact cancellation
        cols, vals = run(lib, idx, val, jj, kk, d)
        pc, pv = plain(idx, val, jj, kk, d)
        assert cols == pc and vals == pv
        assert all(a < b for a, b in zip(cols, cols[1:]))


def test_edges(lib):
    idx = np.array([3, 5], np.int32)
    val = np.array([1.0, 2.0])
    # x_k first / last, x_j before both, between, after both, present
    for kk in (3, 5):
        for jj in (0, 4, 9, 3 if kk == 5 else 5):
            for d in (0.5, -1.0, -2.0):
                assert run(lib, idx, val, jj, kk, d) == tuple(map(list, plain(idx, val, jj, kk, d)))
    # a one-entry row (x_k alone): x_j takes its place
    one = np.array([4], np.int32)
    assert run(lib, one, np.array([1.5]), 2, 4, 0.25) == ([2], [0.25])
    # cancellation within par_tol of a nonzero sum, and just outside it
    v = 1.0 + 2.0 ** -40
    assert run(lib, idx, np.array([v, 2.0]), 3, 5, -1.0) == ([], [])
    assert run(lib, idx, np.array([1.0 + 2.0 ** -30, 2.0]), 3, 5, -1.0)[0] == [3]
