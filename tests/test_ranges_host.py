"""The server's record-space allocator (first fit over sorted, merged free
ranges), built for the host and driven by random take / give sequences
against a cell-by-cell model (no GPU needed)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not found")
    out = str(tmp_path_factory.mktemp("ranges") / "libranges_host.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out,
                    os.path.join(ROOT, "tests", "host", "ranges_host.cpp")], check=True)
    L = C.CDLL(out)
    L.ranges_new.restype = C.c_void_p
    L.ranges_new.argtypes = [C.c_int32]
    L.ranges_free.argtypes = [C.c_void_p]
    L.ranges_take.argtypes = [C.c_void_p, C.c_int32]
    L.ranges_take.restype = C.c_int32
    L.ranges_give.argtypes = [C.c_void_p, C.c_int32, C.c_int32]
    L.ranges_list.argtypes = [C.c_void_p, C.c_void_p, C.c_int32]
    L.ranges_list.restype = C.c_int32
    return L


def first_fit(used, length):
    run = 0
    for i, u in enumerate(used):
        run = 0 if u else run + 1
        if run == length:
            return i - length + 1
    return -1


def free_runs(used):
    runs, start = [], None
    for i, u in enumerate(list(used) + [True]):
        if not u and start is None:
            start = i
        if u and start is not None:
            runs.append((start, i - start))
            start = None
    return runs


@pytest.mark.parametrize("seed", range(20))
def test_random_sequences(lib, seed):
    rng = np.random.default_rng(seed)
    cap = int(rng.integers(1, 300))
    r = lib.ranges_new(cap)
    used = np.zeros(cap, bool)
    live = []
    buf = np.zeros(2 * (cap + 1), np.int32)
    try:
        for _ in range(400):
            if live and rng.random() < 0.45:
                s, ln = live.pop(int(rng.integers(len(live))))
                lib.ranges_give(r, s, ln)
                used[s:s + ln] = False
            else:
                ln = int(rng.integers(0, max(2, cap // 4)))
                s = lib.ranges_take(r, ln)
                if ln == 0:
                    assert s == 0
                    continue
                assert s == first_fit(used, ln)
                if s >= 0:
                    assert not used[s:s + ln].any()
                    used[s:s + ln] = True
                    live.append((s, ln))
            k = lib.ranges_list(r, buf.ctypes.data, cap + 1)
            got = [(int(buf[2 * i]), int(buf[2 * i + 1])) for i in range(k)]
            assert got == free_runs(used)  # sorted, merged, exactly the free cells
    finally:
        lib.ranges_free(r)


def test_full_and_exact_fit(lib):
    r = lib.ranges_new(10)
    try:
        assert lib.ranges_take(r, 11) == -1
        assert [lib.ranges_take(r, 5), lib.ranges_take(r, 5), lib.ranges_take(r, 1)] == [0, 5, -1]
        lib.ranges_give(r, 0, 5)
        assert lib.ranges_take(r, 5) == 0
    finally:
        lib.ranges_free(r)
