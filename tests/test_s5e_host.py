"""The library's S5e step (doubleton equations, Sec. 2.1) built for the host
from the same source the kernels use (s5e_logic.cuh), run on random round
states against a plain statement of the step written here: candidates
(kept equality rows of two entries, both columns kept; x_k the column with
fewer entries, the second on a tie), claims (the first candidate per
column, and per kept row of x_k), the bound transfer onto x_j finalised as
S3' finalises, x_j's cost, the side shifts and the rewritten rows (x_k out,
x_j merged, cancelled within par_tol, or inserted).  Everything is compared
bit for bit: the two compute each value with the same IEEE operations.
No GPU needed."""
import ctypes as C
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INF = math.inf
NONE = 0x7FFFFFFF
V_SLOTS, V_S5E_COL = 5, 3
FEAS_TOL, PAR_TOL = 1e-9, 1e-12


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("s5e") / "libs5e_round.so")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-fmad=false", "-shared", "-Xcompiler", "-fPIC",
                    "-Xcompiler", "-ffp-contract=off", "-o", out,
                    os.path.join(ROOT, "tests", "host", "s5e_host.cu")], check=True)
    L = C.CDLL(out)
    L.s5e_host_round.restype = C.c_int32
    return L


# ------------------------------------------------------------ random states
def random_state(seed, m=80, n=60):
    rng = np.random.default_rng(seed)
    lb = rng.uniform(-5, 0, n)
    ub = lb + rng.uniform(0.5, 10, n)
    lb[rng.random(n) < 0.12] = -INF
    ub[rng.random(n) < 0.12] = INF
    x0 = np.where(np.isfinite(lb), lb, np.where(np.isfinite(ub), ub - 1.0, 0.0))
    box = np.isfinite(lb) & np.isfinite(ub)
    x0[box] = lb[box] + (ub[box] - lb[box]) * rng.random(n)[box]
    rows, L, U = [], [], []
    for i in range(m):
        ln = 2 if rng.random() < 0.5 else int(rng.integers(1, 7))
        cols = np.sort(rng.choice(n, size=ln, replace=False))
        vals = rng.uniform(0.5, 3.0, ln) * rng.choice([-1.0, 1.0], ln)
        rows.append([cols.tolist(), vals.tolist()])
        act = float(np.dot(vals, x0[cols]))
        if ln == 2 and rng.random() < 0.8:
            side = act if rng.random() < 0.9 else act + 40.0 * vals[0]  # some transfers miss
            L.append(side), U.append(side)
        else:
            lo = act - rng.uniform(0, 3) if rng.random() < 0.7 else -INF
            hi = act + rng.uniform(0, 3) if rng.random() < 0.7 else INF
            L.append(lo), U.append(hi)
    # plant cancellations: a row holding x_j and x_k whose x_j coefficient is
    # a_rk (a / b) for a two-entry equality row a x_j + b x_k (x_k the column
    # with fewer entries, as the step picks it)
    clen = np.bincount([c_ for r in rows for c_ in r[0]], minlength=n)
    for i in range(m):
        if len(rows[i][0]) != 2 or L[i] != U[i] or rng.random() < 0.3:
            continue
        (c0, c1), (v0, v1) = rows[i]
        (j, a), (k, b) = ((c0, v0), (c1, v1)) if clen[c1] <= clen[c0] else ((c1, v1), (c0, v0))
        for r in range(m):
            cols, vals = rows[r]
            if r != i and j in cols and k in cols and rng.random() < 0.5:
                vals[cols.index(j)] = vals[cols.index(k)] * (a / b)
    # plant transfers that end within the tolerance of x_j's upper bound (the snap)
    for i in range(m):
        if len(rows[i][0]) != 2 or L[i] != U[i] or rng.random() < 0.7:
            continue
        (c0, c1), (v0, v1) = rows[i]
        (j, a), (k, b) = ((c0, v0), (c1, v1)) if clen[c1] <= clen[c0] else ((c1, v1), (c0, v0))
        f, g = a / b, L[i] / b
        bhi = ub[k] if f > 0 else lb[k]
        if math.isfinite(bhi):
            lo = (g - bhi) / f
            if lo > lb[j]:
                ub[j] = lo + 0.5e-9 * max(1.0, abs(lo))
    rp = np.zeros(m + 1, np.int32)
    rp[1:] = np.cumsum([len(r[0]) for r in rows])
    ci = np.array([c for r in rows for c in r[0]], np.int32)
    rv = np.array([v for r in rows for v in r[1]], float)
    rkind = np.where(rng.random(m) < 0.1, rng.integers(1, 6, m), 0).astype(np.uint8)
    ckind = np.where(rng.random(n) < 0.08, rng.integers(1, 5, n), 0).astype(np.uint8)
    c = rng.normal(size=n)
    rmap = np.sort(rng.choice(m + 30, size=m, replace=False)).astype(np.int32)
    cmap = np.sort(rng.choice(n + 30, size=n, replace=False)).astype(np.int32)
    return dict(m=m, n=n, rp=rp, ci=ci, rv=rv, L=np.array(L), U=np.array(U), lb=lb, ub=ub, c=c,
                rkind=rkind, ckind=ckind, rmap=rmap, cmap=cmap, m_orig=m + 30, n_orig=n + 30)


def csc(st):
    m, n = st["m"], st["n"]
    rows = np.repeat(np.arange(m), np.diff(st["rp"]))
    order = np.lexsort((rows, st["ci"]))
    cp = np.zeros(n + 1, np.int32)
    cp[1:] = np.cumsum(np.bincount(st["ci"], minlength=n))
    return cp, rows[order].astype(np.int32), st["rv"][order].copy()


# ------------------------------------------------- the step, stated plainly
def reference(st, rnd):
    m, n = st["m"], st["n"]
    rp, ci, rv = st["rp"].tolist(), st["ci"].tolist(), st["rv"].tolist()
    cp, ri, cv = (a.tolist() for a in csc(st))
    rkind, ckind = st["rkind"].astype(int).tolist(), st["ckind"].astype(int).tolist()
    L, U, lb, ub, c = (st[k].tolist() for k in ("L", "U", "lb", "ub", "c"))
    rmap, cmap = st["rmap"].tolist(), st["cmap"].tolist()
    out = dict(fixv={}, rec_row={}, rec_col={}, store={}, rdnext=set(), verdict=None, applied=0, changed=0,
               cancelled=0, merged=0, inserted=0, snapped=0)
    cand, cmin, rmin = {}, [NONE] * n, [NONE] * m
    for i in range(m):
        if rkind[i] != 0 or rp[i + 1] - rp[i] != 2 or not math.isfinite(L[i]) or L[i] != U[i]:
            continue
        c0, c1 = ci[rp[i]], ci[rp[i] + 1]
        if ckind[c0] != 0 or ckind[c1] != 0:
            continue
        kk = c1 if cp[c1 + 1] - cp[c1] <= cp[c0 + 1] - cp[c0] else c0
        cand[i] = kk
        cmin[c0], cmin[c1] = min(cmin[c0], i), min(cmin[c1], i)
        for q in range(cp[kk], cp[kk + 1]):
            if ri[q] == i or rkind[ri[q]] == 0:
                rmin[ri[q]] = min(rmin[ri[q]], i)
    sel = []
    for i, kk in sorted(cand.items()):
        p = rp[i]
        jj = ci[p + 1] if ci[p] == kk else ci[p]
        if cmin[jj] == i and cmin[kk] == i and rmin[i] == i and all(
                ri[q] == i or rkind[ri[q]] != 0 or rmin[ri[q]] == i for q in range(cp[kk], cp[kk + 1])):
            sel.append(i)
    notes = {}
    for i in sel:
        kk, p = cand[i], rp[i]
        jj = ci[p + 1] if ci[p] == kk else ci[p]
        a = rv[p] if ci[p] == jj else rv[p + 1]
        b = rv[p] if ci[p] == kk else rv[p + 1]
        cc = L[i]
        f, g = a / b, cc / b
        if f > 0:
            lo = (g - ub[kk]) / f if math.isfinite(ub[kk]) else -INF
            hi = (g - lb[kk]) / f if math.isfinite(lb[kk]) else INF
        else:
            lo = (g - lb[kk]) / f if math.isfinite(lb[kk]) else -INF
            hi = (g - ub[kk]) / f if math.isfinite(ub[kk]) else INF
        nl = lo if lo > lb[jj] else lb[jj]
        nu = hi if hi < ub[jj] else ub[jj]
        if math.isfinite(nl) and math.isfinite(nu):
            d = FEAS_TOL * max(1.0, max(abs(nl), abs(nu)))
            if nl - nu > d:
                out["verdict"] = cmap[jj] if out["verdict"] is None else min(out["verdict"], cmap[jj])
                continue
            if nl != nu and abs(nl - nu) <= d:
                nl = nu = 0.5 * (nl + nu)
                out["snapped"] += 1
        out["changed"] += nl != lb[jj] or nu != ub[jj]
        lb[jj], ub[jj] = nl, nu
        t = c[kk] / b
        c[jj] = c[jj] - t * a
        rkind[i], ckind[kk] = 6, 5
        out["fixv"][kk] = g
        out["rec_row"][rmap[i]] = (6, rnd, cmap[kk], b)
        out["rec_col"][cmap[kk]] = (5, rnd, g)
        out["store"][rmap[i]] = (cc, cmap[jj], a)
        out["applied"] += 1
        for q in range(cp[kk], cp[kk + 1]):
            rr, ark = ri[q], cv[q]
            if rr == i or rkind[rr] != 0:
                continue
            if math.isfinite(L[rr]):
                L[rr] = L[rr] - ark * g
            if math.isfinite(U[rr]):
                U[rr] = U[rr] - ark * g
            notes[rr] = (jj, kk, -(ark * f))
            out["rdnext"].add(rr)
    # the rewritten rows
    nrp, nci, nrv = [0], [], []
    for i in range(m):
        cols, vals = ci[rp[i]:rp[i + 1]], rv[rp[i]:rp[i + 1]]
        if i in notes:
            jj, kk, dd = notes[i]
            row = {cc_: vv for cc_, vv in zip(cols, vals) if cc_ != kk}
            if jj in row:
                s = row[jj] + dd
                if abs(s) <= PAR_TOL * max(abs(row[jj]), abs(dd)):
                    del row[jj]
                    out["cancelled"] += 1
                else:
                    row[jj] = s
                    out["merged"] += 1
            else:
                row[jj] = dd
                out["inserted"] += 1
            cols, vals = sorted(row), [row[k_] for k_ in sorted(row)]
        nci += cols
        nrv += vals
        nrp.append(len(nci))
    out.update(rkind=rkind, ckind=ckind, L=L, U=U, lb=lb, ub=ub, c=c, rp=nrp, ci=nci, rv=nrv)
    return out


# -------------------------------------------------------------- the library
def run_host(L_, st, rnd):
    m, n, mo, no = st["m"], st["n"], st["m_orig"], st["n_orig"]
    nnz = int(st["rp"][m])
    cp, ri, cv = csc(st)
    a = {k: np.ascontiguousarray(st[k]).copy() for k in ("rkind", "ckind", "L", "U", "lb", "ub", "c")}
    rec = dict(rk=np.zeros(mo, np.int32), rr=np.zeros(mo, np.int32), ra=np.full(mo, -1, np.int32),
               rv=np.zeros(mo), ck=np.zeros(no, np.int32), cr=np.zeros(no, np.int32), cv=np.zeros(no),
               sb=np.full(mo, -1, np.int64), sl=np.zeros(mo, np.int32), srhs=np.zeros(mo),
               scol=np.full(nnz + 1, -1, np.int32), sval=np.zeros(nnz + 1))
    fixv, rdnext = np.zeros(n), np.zeros(m, np.uint8)
    verdict = np.full(V_SLOTS, NONE, np.int32)
    counts = np.zeros(2, np.int32)
    rp2, ci2, rv2 = np.zeros(m + 1, np.int32), np.full(nnz + 1, -1, np.int32), np.full(nnz + 1, np.nan)
    P = lambda x: C.c_void_p(x.ctypes.data)  # noqa: E731
    nnz2 = L_.s5e_host_round(
        C.c_int32(m), C.c_int32(n), C.c_int32(rnd), P(st["rp"]), P(st["ci"]), P(st["rv"]), P(cp), P(ri), P(cv),
        P(a["rkind"]), P(a["ckind"]), P(a["L"]), P(a["U"]), P(a["lb"]), P(a["ub"]), P(a["c"]), P(st["rmap"]),
        P(st["cmap"]), C.c_double(FEAS_TOL), C.c_double(PAR_TOL), P(rec["rk"]), P(rec["rr"]), P(rec["ra"]),
        P(rec["rv"]), P(rec["ck"]), P(rec["cr"]), P(rec["cv"]), P(rec["sb"]), P(rec["sl"]), P(rec["srhs"]),
        P(rec["scol"]), P(rec["sval"]), P(fixv), P(rdnext), P(verdict), P(counts), P(rp2), P(ci2), P(rv2))
    assert nnz2 >= 0, ("rewrite check failed", nnz2)
    return a, rec, fixv, rdnext, verdict, counts, rp2, ci2[:nnz2], rv2[:nnz2]


def check(L_, st, rnd=3):
    ref = reference(st, rnd)
    a, rec, fixv, rdnext, verdict, counts, rp2, ci2, rv2 = run_host(L_, st, rnd)
    assert int(verdict[V_S5E_COL]) == (NONE if ref["verdict"] is None else ref["verdict"])
    assert list(counts) == [ref["applied"], ref["changed"]]
    assert a["rkind"].tolist() == ref["rkind"] and a["ckind"].tolist() == ref["ckind"]
    for k in ("L", "U", "lb", "ub", "c"):
        np.testing.assert_array_equal(a[k], np.array(ref[k]), err_msg=k)
    assert rp2.tolist() == ref["rp"] and ci2.tolist() == ref["ci"]
    np.testing.assert_array_equal(rv2, np.array(ref["rv"], float))
    assert set(np.flatnonzero(rdnext).tolist()) == ref["rdnext"]
    for kk, g in ref["fixv"].items():
        assert fixv[kk] == g
    rows = set(np.flatnonzero(rec["rk"]).tolist())
    assert rows == set(ref["rec_row"])
    for o, (k, r, aux, val) in ref["rec_row"].items():
        assert (rec["rk"][o], rec["rr"][o], rec["ra"][o], rec["rv"][o]) == (k, r, aux, val)
        cc, oj, av = ref["store"][o]
        sb = int(rec["sb"][o])
        assert rec["sl"][o] == 1 and rec["srhs"][o] == cc and (rec["scol"][sb], rec["sval"][sb]) == (oj, av)
    assert set(np.flatnonzero(rec["ck"]).tolist()) == set(ref["rec_col"])
    for o, (k, r, g) in ref["rec_col"].items():
        assert (rec["ck"][o], rec["cr"][o], rec["cv"][o]) == (k, r, g)
    return ref


def test_random_round_states(lib):
    tally = dict(applied=0, cancelled=0, merged=0, inserted=0, snapped=0, verdicts=0)
    for seed in range(120):
        ref = check(lib, random_state(seed))
        for k in ("applied", "cancelled", "merged", "inserted", "snapped"):
            tally[k] += ref[k]
        tally["verdicts"] += ref["verdict"] is not None
    # the states exercise every branch
    assert tally["applied"] > 500 and tally["verdicts"] > 10, tally
    assert tally["cancelled"] > 20 and tally["merged"] > 20 and tally["inserted"] > 500, tally
    assert tally["snapped"] > 20, tally


def test_long_columns_and_ties(lib):
    # x_k columns of hundreds of rows (the device walks them with a whole warp)
    for seed in range(6):
        st = random_state(1000 + seed, m=600, n=40)
        check(lib, st)


def test_no_candidates(lib):
    st = random_state(7, m=30, n=30)
    st["rkind"][:] = 1  # every row already removed: nothing applies, the matrix is copied
    ref = check(lib, st)
    assert ref["applied"] == 0 and ref["rp"] == st["rp"].tolist()
