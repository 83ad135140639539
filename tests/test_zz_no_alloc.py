"""lpp_row_activity_noalloc: the allocation-free activity entry point.

It is for callers that cannot allocate device memory when they need row
activities: a solver that reserved its whole memory budget up front and
treats a later allocation as a failure, or a pipeline whose device memory
plan is fixed while it runs.  The tests call it through the C ABI on
device-resident LPs and check:

* several calls in a row (the shared scratch array keeps the previous call's
  contents), the first of them on an LP with at most 4096 entries, so that
  the window kernels run for the first time only in a later call, each
  against the oracle's activities (``oracle.activities``) and against
  ``lpp_presolve``'s activities of round 1, within the parity tolerance:
  counts of infinite terms exactly, finite parts to
  1e-9 * max(1, |value|, sum of |a_ij * bound|);
* a hand-built CSR whose long rows sit on the window edges: two long rows
  sharing one 4096-entry window (both of its slots used), a long row
  starting exactly on a window boundary, a long row ending exactly on one,
  and empty rows at window edges;
* that a call after the first allocates nothing: the device's free memory
  and the caching allocator's counters are unchanged across it;
* the size limit of the scratch array.

This file sorts last so that a stop at the first failure has run the rest.
"""
import numpy as np
import pytest

import oracle
from paper_2609_16182_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2609_16182_gb300 import _build, lpp  # noqa: E402

WINDOW = 4096


def abs_scale(lp):
    rows = np.repeat(np.arange(lp.m), np.diff(lp.row_ptr))
    lb = np.where(np.abs(lp.lb) >= 1e20, 0.0, lp.lb)
    ub = np.where(np.abs(lp.ub) >= 1e20, 0.0, lp.ub)
    b = np.maximum(np.abs(lb[lp.col_idx]), np.abs(ub[lp.col_idx]))
    return np.bincount(rows, weights=np.abs(lp.val) * b, minlength=lp.m)


class Dev:
    """The LP's arrays and the four outputs, on the device."""

    def __init__(self, lp):
        self.lp = lp
        self.a = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in lp.arrays().items()}
        self.amin = torch.empty(max(lp.m, 1), dtype=torch.float64, device="cuda")
        self.amax = torch.empty(max(lp.m, 1), dtype=torch.float64, device="cuda")
        self.nmin = torch.empty(max(lp.m, 1), dtype=torch.int32, device="cuda")
        self.nmax = torch.empty(max(lp.m, 1), dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()

    def call(self, L):
        a, lp = self.a, self.lp
        st = L.lpp_row_activity_noalloc(lp.m, lp.n, lp.nnz, a["row_ptr"].data_ptr(), a["col_idx"].data_ptr(),
                                        a["val"].data_ptr(), a["lb"].data_ptr(), a["ub"].data_ptr(), 1e20,
                                        self.amin.data_ptr(), self.amax.data_ptr(), self.nmin.data_ptr(),
                                        self.nmax.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert st == 0, lpp.last_error()
        torch.cuda.synchronize()
        m = lp.m
        return (self.amin.cpu().numpy()[:m], self.amax.cpu().numpy()[:m], self.nmin.cpu().numpy()[:m],
                self.nmax.cpu().numpy()[:m])


def check(lp, got, ref_min, ref_max, ref_nmin, ref_nmax):
    amin, amax, nmin, nmax = got
    np.testing.assert_array_equal(nmin, ref_nmin)
    np.testing.assert_array_equal(nmax, ref_nmax)
    S = abs_scale(lp)
    bad = np.abs(amin - ref_min) > 1e-9 * np.maximum(1.0, np.maximum(np.abs(ref_min), S))
    assert not bad.any(), np.flatnonzero(bad)[:10]
    bad = np.abs(amax - ref_max) > 1e-9 * np.maximum(1.0, np.maximum(np.abs(ref_max), S))
    assert not bad.any(), np.flatnonzero(bad)[:10]


def check_oracle(lp, got):
    check(lp, got, *oracle.activities(lp))


def check_presolve(lp, got):
    r = lpp.presolve(lp, max_rounds=1)  # its reported activities are round 1's, on the input bounds
    assert r.rounds == 1
    check(lp, got, r.act_min, r.act_max, r.ninf_min, r.ninf_max)
    r.close()


def test_noalloc_matches_oracle_and_presolve_on_calls_in_a_row():
    _build.build()
    L = lpp.load()
    # first call: no row beyond 4096 entries, nnz <= 4096 (the window kernels do not run)
    s = synth.tiny(3)
    assert s.nnz <= WINDOW
    a = synth.skewed(11, m=40_000, n=60_000, target_nnz=400_000, row_cap=30_000)
    b = synth.skewed(12, m=30_000, n=45_000, target_nnz=300_000, row_cap=20_000)
    assert np.diff(a.row_ptr).max() > WINDOW and np.diff(b.row_ptr).max() > WINDOW
    for lp in (s, a, b, a):
        got = Dev(lp).call(L)
        check_oracle(lp, got)
        check_presolve(lp, got)


def edge_csr(seed=0):
    """Rows placed on the window edges (entry positions are what matter):
    row 0: 100 entries; row 1: empty; row 2: ends exactly at entry 4096
    (a window boundary) with 3996 entries (short); rows 3-4: empty, at the
    boundary; row 5: 5000 entries starting exactly at 4096 (a long row on a
    window boundary); row 6: 6000 entries, starting inside window 2 after row
    5 ended there, so window 2 holds two long rows (slots 0 and 1); row 7:
    empty; row 8: ends exactly on a window boundary, long; row 9: 10 entries;
    row 10: empty (last row)."""
    rng = np.random.default_rng(seed)
    n = 9000
    lens = [100, 0, 3996, 0, 0, 5000, 6000, 0, 0, 10, 0]
    end6 = 4096 + 5000 + 6000
    lens[8] = (end6 // WINDOW + 2) * WINDOW - end6  # row 8 ends on a boundary, more than 4096 entries
    assert lens[8] > WINDOW
    ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    assert ptr[3] == WINDOW and ptr[6] == WINDOW + 5000 and ptr[9] % WINDOW == 0
    w5, w6 = ptr[5] // WINDOW, ptr[6] // WINDOW
    assert (ptr[6] - 1) // WINDOW == w6 and ptr[6] % WINDOW != 0  # rows 5 and 6 share window w6
    cols = np.concatenate([np.sort(rng.choice(n, k, replace=False)) for k in lens]).astype(np.int32)
    nnz = int(ptr[-1])
    val = rng.lognormal(0.0, 1.0, nnz) * np.where(rng.random(nnz) < 0.5, -1.0, 1.0)
    lb = -rng.uniform(0.0, 10.0, n)
    ub = rng.uniform(1.0, 100.0, n)
    lb[rng.random(n) < 0.1] = -np.inf
    ub[rng.random(n) < 0.1] = np.inf
    m = len(lens)
    lp = synth.LP(m=m, n=n, row_ptr=ptr, col_idx=cols, val=val, c=np.zeros(n), lhs=np.full(m, -np.inf),
                  rhs=np.full(m, np.inf), lb=lb, ub=ub)
    return lp, w5


def brute(lp):
    """The activities written out row by row with math.fsum (correctly rounded sums)."""
    import math
    out = ([], [], [], [])
    for i in range(lp.m):
        b, e = lp.row_ptr[i], lp.row_ptr[i + 1]
        v, j = lp.val[b:e], lp.col_idx[b:e]
        bmin = np.where(v > 0, lp.lb[j], lp.ub[j])
        bmax = np.where(v > 0, lp.ub[j], lp.lb[j])
        fmin, fmax = np.isfinite(bmin), np.isfinite(bmax)
        out[0].append(math.fsum(v[fmin] * bmin[fmin]))
        out[1].append(math.fsum(v[fmax] * bmax[fmax]))
        out[2].append(int((~fmin).sum()))
        out[3].append(int((~fmax).sum()))
    return np.array(out[0]), np.array(out[1]), np.array(out[2], np.int32), np.array(out[3], np.int32)


def test_noalloc_window_edges():
    L = lpp.load()
    lp, _ = edge_csr()
    got = Dev(lp).call(L)
    check(lp, got, *brute(lp))
    check_oracle(lp, got)
    # the same rows shifted by one entry: row 5 then starts one past the boundary
    lp2, _ = edge_csr(1)
    lens = np.diff(lp2.row_ptr)
    lens[0] += 1
    lens[9] -= 1
    ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    rng = np.random.default_rng(5)
    cols = np.concatenate([np.sort(rng.choice(lp2.n, k, replace=False)) for k in lens]).astype(np.int32)
    lp3 = synth.LP(m=lp2.m, n=lp2.n, row_ptr=ptr, col_idx=cols, val=lp2.val, c=lp2.c, lhs=lp2.lhs, rhs=lp2.rhs,
                   lb=lp2.lb, ub=lp2.ub)
    got = Dev(lp3).call(L)
    check(lp3, got, *brute(lp3))
    check_oracle(lp3, got)


def test_noalloc_call_allocates_nothing():
    L = lpp.load()
    small = Dev(synth.tiny(4))
    small.call(L)  # any set-up happens here, before the measured call
    big = Dev(synth.skewed(13, m=30_000, n=45_000, target_nnz=300_000, row_cap=20_000))
    assert np.diff(big.lp.row_ptr).max() > WINDOW
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    st = L.lpp_row_activity_noalloc(big.lp.m, big.lp.n, big.lp.nnz, big.a["row_ptr"].data_ptr(),
                                    big.a["col_idx"].data_ptr(), big.a["val"].data_ptr(), big.a["lb"].data_ptr(),
                                    big.a["ub"].data_ptr(), 1e20, big.amin.data_ptr(), big.amax.data_ptr(),
                                    big.nmin.data_ptr(), big.nmax.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert st == 0, lpp.last_error()
    assert free1 == free0, (free0, free1)
    for k in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(k, 0) == stats0.get(k, 0), k
    got = (big.amin.cpu().numpy(), big.amax.cpu().numpy(), big.nmin.cpu().numpy(), big.nmax.cpu().numpy())
    check_oracle(big.lp, got)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = lpp.load()
    st = L.lpp_row_activity_noalloc(1, 1, 268_435_457, None, None, None, None, None, 1e20, None, None, None, None,
                                    None)
    assert st == lpp.ERR_INVALID
    assert "scratch" in lpp.last_error()
