"""The host check of the S5e device logic catches plausible mistakes.

Each case plants one mistake in a copy of s5e_logic.cuh or s5e_rewrite.cuh
(the per-row and per-entry work the kernels call), builds the host harness
on it, and runs the comparison of tests/test_s5e_host.py on random round
states: it must fail.  The unaltered headers pass.  No GPU needed."""
import concurrent.futures as cf
import ctypes as C
import os
import shutil
import subprocess

import pytest

import test_s5e_host as base

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2609_16182_gb300", "csrc")
HEADERS = ["s5e_logic.cuh", "s5e_rewrite.cuh", "lpp_launch.h", "lpp_dev.cuh"]

# (name, header, text, replacement)
MUTANTS = [
    ("rewrite: a cancelled entry still counted", "s5e_rewrite.cuh",
     "t.len_new = len - 1 + (t.found ? (t.cancel ? -1 : 0) : 1);", "t.len_new = len - 1 + (t.found ? 0 : 1);"),
    ("rewrite: the entry at an inserted x_j's place not moved", "s5e_rewrite.cuh",
     "(!t.found && q >= t.pj ? 1 : 0)", "(!t.found && q > t.pj ? 1 : 0)"),
    ("rewrite: an inserted x_j placed one too far", "s5e_rewrite.cuh",
     "return t.pj - (t.pk < t.pj ? 1 : 0);", "return t.pj;"),
    ("candidates: ties eliminate the first column", "s5e_logic.cuh",
     "kk = l1 <= l0 ? c1 : c0;", "kk = l1 < l0 ? c1 : c0;"),
    ("selection: x_j's column claim ignored", "s5e_logic.cuh",
     "const bool own = D.cmin[jj] == i && D.cmin[kk] == i && D.rmin[i] == i;",
     "const bool own = D.cmin[kk] == i && D.rmin[i] == i;"),
    ("application: x_j's cost updated with the wrong sign", "s5e_logic.cuh",
     "C.c[jj] = C.c[jj] - t * a;", "C.c[jj] = C.c[jj] + t * a;"),
    ("application: coefficient change with the wrong sign", "s5e_logic.cuh",
     "D.dmd[rr] = -(ark * f);", "D.dmd[rr] = (ark * f);"),
    ("application: bounds within the tolerance left apart", "s5e_logic.cuh",
     "if (nl != nu && fabs(nl - nu) <= d) nl = nu = 0.5 * (nl + nu);",
     "if (nl > nu && fabs(nl - nu) <= d) nl = nu = 0.5 * (nl + nu);"),
    ("application: an empty transfer still applied", "s5e_logic.cuh",
     "s5e_amin(&C.verdict[lp * V_SLOTS + V_S5E_COL], C.cmap[jj]);\n            return r;",
     "s5e_amin(&C.verdict[lp * V_SLOTS + V_S5E_COL], C.cmap[jj]);"),
    ("application: only the finite lhs shifted", "s5e_logic.cuh",
     "if (s5e_fin(Uv)) C.U[rr] = Uv - ark * g;", "(void)Uv;"),
    ("placement: a cancelled entry written", "s5e_logic.cuh",
     "if (t.cancel) return true;", "if (0) return true;"),
]


def build(tmp, mutated=None):
    d = os.path.join(tmp, "paper_2609_16182_gb300", "csrc")
    os.makedirs(d)
    os.makedirs(os.path.join(tmp, "tests", "host"))
    for h in HEADERS:
        text = open(os.path.join(CSRC, h)).read()
        if mutated and mutated[0] == h:
            assert text.count(mutated[1]) == 1, f"mutation site not unique or gone: {mutated[1]!r}"
            text = text.replace(mutated[1], mutated[2])
        with open(os.path.join(d, h), "w") as f:
            f.write(text)
    shutil.copy(os.path.join(ROOT, "tests", "host", "s5e_host.cu"), os.path.join(tmp, "tests", "host"))
    out = os.path.join(tmp, "libs5e_round.so")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    subprocess.run([nvcc, "-O2", "-std=c++17", "-fmad=false", "-shared", "-Xcompiler", "-fPIC", "-Xcompiler",
                    "-ffp-contract=off", "-o", out, os.path.join(tmp, "tests", "host", "s5e_host.cu")],
                   check=True, capture_output=True)
    return out


def caught(lib_path, seeds=40):
    L = C.CDLL(lib_path)
    L.s5e_host_round.restype = C.c_int32
    for seed in range(seeds):
        try:
            base.check(L, base.random_state(seed))
        except AssertionError:
            return True
    return False


@pytest.fixture(scope="module")
def libs(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    jobs = [("control", None)] + [(m[0], m[1:]) for m in MUTANTS]
    # the directories are made here, before the threads: the factory is not thread-safe
    dirs = [str(tmp_path_factory.mktemp("s5e_mut")) for _ in jobs]

    def one(job_dir):
        (name, mutated), d = job_dir
        return name, build(d, mutated)

    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        return dict(ex.map(one, zip(jobs, dirs)))


def test_control_passes(libs):
    assert not caught(libs["control"])


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_mutant_is_caught(libs, name):
    assert caught(libs[name]), name
