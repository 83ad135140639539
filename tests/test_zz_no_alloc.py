"""lpp_row_activity_noalloc: the allocation-free activity entry point.

It is for callers that cannot allocate device memory when they need row
activities (a solver whose memory budget is fixed up front).  The test calls
it through the C ABI on device-resident LPs, twice in a row on different LPs
(the shared scratch array keeps the first call's contents), and checks each
result against lpp_presolve's activities of round 1 (same input bounds),
within the parity tolerance: counts of infinite terms exactly, finite parts
to 1e-9 * max(1, |value|, sum of |a_ij * bound|).
This file sorts last so that a stop at the first failure has run the rest.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2609_16182_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2609_16182_gb300 import _build, lpp  # noqa: E402


def reference(lp):
    """lpp_presolve with one round: its reported activities are round 1's."""
    r = lpp.presolve(lp, max_rounds=1)
    assert r.rounds == 1
    return r


def abs_scale(lp):
    rows = np.repeat(np.arange(lp.m), np.diff(lp.row_ptr))
    lb = np.where(np.abs(lp.lb) >= 1e20, 0.0, lp.lb)
    ub = np.where(np.abs(lp.ub) >= 1e20, 0.0, lp.ub)
    b = np.maximum(np.abs(lb[lp.col_idx]), np.abs(ub[lp.col_idx]))
    return np.bincount(rows, weights=np.abs(lp.val) * b, minlength=lp.m)


def call_noalloc(L, lp):
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in lp.arrays().items()}
    amin = torch.empty(lp.m, dtype=torch.float64, device="cuda")
    amax = torch.empty(lp.m, dtype=torch.float64, device="cuda")
    nmin = torch.empty(lp.m, dtype=torch.int32, device="cuda")
    nmax = torch.empty(lp.m, dtype=torch.int32, device="cuda")
    st = L.lpp_row_activity_noalloc(lp.m, lp.n, lp.nnz, dev["row_ptr"].data_ptr(), dev["col_idx"].data_ptr(),
                                    dev["val"].data_ptr(), dev["lb"].data_ptr(), dev["ub"].data_ptr(), 1e20,
                                    amin.data_ptr(), amax.data_ptr(), nmin.data_ptr(), nmax.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert st == 0, lpp.last_error()
    torch.cuda.synchronize()
    return amin.cpu().numpy(), amax.cpu().numpy(), nmin.cpu().numpy(), nmax.cpu().numpy()


def check(lp, got, ref):
    amin, amax, nmin, nmax = got
    np.testing.assert_array_equal(nmin, ref.ninf_min)
    np.testing.assert_array_equal(nmax, ref.ninf_max)
    s = np.maximum(1.0, np.maximum(np.abs(ref.act_min), abs_scale(lp)))
    assert np.all(np.abs(amin - ref.act_min) <= 1e-9 * s)
    s = np.maximum(1.0, np.maximum(np.abs(ref.act_max), abs_scale(lp)))
    assert np.all(np.abs(amax - ref.act_max) <= 1e-9 * s)


def test_noalloc_activities_match_presolve_on_two_calls_in_a_row():
    _build.build()
    L = lpp.load()
    # rows longer than 4096 entries (the scratch path) and short rows
    a = synth.skewed(11, m=40_000, n=60_000, target_nnz=400_000, row_cap=30_000)
    b = synth.skewed(12, m=30_000, n=45_000, target_nnz=300_000, row_cap=20_000)
    assert np.diff(a.row_ptr).max() > 4096 and np.diff(b.row_ptr).max() > 4096
    ra, rb = reference(a), reference(b)
    check(a, call_noalloc(L, a), ra)
    check(b, call_noalloc(L, b), rb)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = lpp.load()
    st = L.lpp_row_activity_noalloc(1, 1, 268_435_457, None, None, None, None, None, 1e20, None, None, None, None,
                                    None)
    assert st == lpp.ERR_INVALID
    assert "scratch" in lpp.last_error()
