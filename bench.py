"""Benchmark: LP presolve to fixpoint on the 2M-row skewed LP (GB300).

One step = one full presolve (S1..S8 rounds until nothing changes) of the
skewed LP (m = 2M, n = 3M, ~20M nonzeros, row lengths 1 + Zipf(2) capped at
500k, column weights Zipf(1.8)), inputs resident in HBM, through the C ABI
(lpp_presolve).  `value` is nonzeros processed per second: the sum over the
rounds of the nonzeros present at each round's start, divided by the step
time.  `e2e` repeats the step from pinned host buffers with the host->device
copy of the input and the device->host copy of the reduced LP inside the
timed region.

Launch: python bench.py [--gpus N --steps K --warmup W] (N > 1 under
torch.distributed.run: one independent replica per GPU, weak scaling).
--impl reference times the CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "presolve ms & nnz/s per round vs HBM roofline; batched LPs/s, p50/p99 latency"
WORKLOAD = ("skewed LP: m=2,000,000 rows, n=3,000,000 cols, ~20M nnz FP64 CSR, row lengths 1+Zipf(2) capped at "
            "500k, column weights Zipf(1.8), lognormal values, 30% equality rows, 20% infinite bounds, "
            "5% singleton and 3% redundant rows planted; full fixpoint loop")


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int, period_ms: int = 50):
        self.gpu = gpu
        self.period_ms = period_ms
        self.rows = []  # (arrival time, fields)
        self.t0 = None  # the timed region, set by the caller
        self.t1 = None
        self._p = None
        self._t = None

    def _run(self):
        try:
            self._p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                        "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                       stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            return
        for line in self._p.stdout:
            if line.strip():
                self.rows.append((time.monotonic(), [x.strip() for x in line.strip().split(",")]))

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        time.sleep(0.2)  # the sampler is running before the timed region starts
        return self

    def __exit__(self, *a):
        if self._p is not None:
            self._p.terminate()
            try:
                self._p.wait(timeout=5)
            except Exception:
                self._p.kill()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        rows = [r for t, r in self.rows if self.t0 is None or (self.t0 <= t <= (self.t1 or t))]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def reduce_over_ranks(ms_total: float, nnz_proc: int, device, world_size: int):
    """Whole-job throughput of independent replicas: the slowest rank's time
    and the nonzeros of all ranks (weak scaling, no data-path collective)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_total], device=device, dtype=torch.float64)
    tot = torch.tensor([float(nnz_proc)], device=device, dtype=torch.float64)
    if world_size > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    return ms_max, float(tot.item()) / (ms_max / 1e3)


def round_sizes(m0, n0, rows_removed, cols_fixed):
    """Rows and columns present at the start of each round, from the per-round
    removal counters (every removed row or column leaves in that round's
    compaction)."""
    m, n = [m0], [n0]
    for a, b in zip(rows_removed[:-1], cols_fixed[:-1]):
        m.append(m[-1] - a)
        n.append(n[-1] - b)
    return m, n


def prop_bytes(nnz, m, n):
    """Algorithmic bytes of the activity and tightening steps of one round:
    S1 reads the CSR (12 per entry), row_ptr (4 per row), the bounds (16 per
    column) and writes activities and counts (24 per row); S3 reads the CSC
    (12 per entry), col_ptr (4 per column), the activities and sides (40 per
    row) and reads and writes the bounds (32 per column)."""
    return 24 * nnz + 68 * m + 52 * n


def round_bytes(nnz, nnz_next, m, n, compacted):
    """Algorithmic bytes of one whole round: S1 + S3 as prop_bytes; the row
    classes, fixings and empty columns 60 per row + 40 per column; parallel
    rows 12 per surviving entry + 120 per row (keys and their sort passes);
    compaction, in rounds that removed something, reads 24 per entry, writes
    24 per surviving entry and rewrites the maps (8 per row and column)."""
    b = prop_bytes(nnz, m, n) + 60 * m + 40 * n + 12 * nnz_next + 120 * m
    if compacted:
        b += 24 * nnz + 24 * nnz_next + 8 * (m + n)
    return b


def describe_rounds(info, first, peak_gbs):
    """Per-round sizes, times, nnz/s and the HBM fraction of each whole round
    (its algorithmic bytes / its time / the peak)."""
    round_ms, round_nnz, round_rows, round_cols, round_bounds = first
    m_r, n_r = round_sizes(info.m, info.n, round_rows, round_cols)
    exact = info.status != 0 or (m_r[-1] - round_rows[-1] == info.m_red and n_r[-1] - round_cols[-1] == info.n_red)
    nxt = list(round_nnz[1:]) + [info.nnz_red]
    rb = [round_bytes(z, z2, a, b, ra > 0 or cb > 0)
          for z, z2, a, b, ra, cb in zip(round_nnz, nxt, m_r, n_r, round_rows, round_cols)]
    return {"rounds": len(round_ms), "presolve_ms": info.presolve_ms, "round_ms": round_ms, "round_nnz": round_nnz,
            "round_m": m_r, "round_n": n_r, "round_sizes_exact": bool(exact),
            "nnz_per_s_per_round": [n_ / (t / 1e3) for n_, t in zip(round_nnz, round_ms)],
            "round_hbm_frac": [b / (t / 1e3) / 1e9 / peak_gbs for b, t in zip(rb, round_ms)],
            "round_rows_removed": round_rows, "round_cols_fixed": round_cols, "round_bounds_changed": round_bounds,
            "reduced": {"m": info.m_red, "n": info.n_red, "nnz": info.nnz_red,
                        "nnz_ratio": info.nnz_red / max(1, info.nnz)},
            "s5_rows_left_at_cap": int(info.s5_left)}


def prop_roofline(kern, rounds, peak_gbs, peak_src, traffic):
    """Roofline of the fused activity kernel family: its algorithmic bytes
    (prop_bytes of each round's nnz, m, n) over its CUDA-event time, against
    the measured HBM copy bandwidth; the FP64 view beside it."""
    pk = kern.get("prop", {"ms": 0.0, "bytes": 0.0, "launches": 1, "fp64_ops": 0.0})
    secs = pk["ms"] / 1e3
    alg = sum(prop_bytes(z, a, b) for z, a, b in zip(rounds["round_nnz"], rounds["round_m"], rounds["round_n"]))
    launches = max(1, pk["launches"])
    achieved = alg / secs / 1e9 if secs > 0 else 0.0
    # FP64 view: 2 DFMA per SM per clock x 152 SMs x 2.07 GHz x 2 flops = 1.26 TFLOP/s
    fp64_peak = 2 * 152 * 2.070e9 * 2 / 1e12
    fp64 = pk["fp64_ops"] * 2 / secs / 1e12 if secs > 0 else 0.0
    return {"bound": "hbm", "kernel": "k_prop_groups + long-row chunks (S1+S2+S3 fused)",
            "achieved": achieved, "peak": peak_gbs, "unit": "GB/s", "frac": achieved / peak_gbs,
            "peak_source": f"{peak_src} hbm_gbs (copy bandwidth)",
            "bytes_per_launch": alg / launches,
            "bytes_basis": "per round 24 nnz + 68 m + 52 n (S1 + S3 algorithmic bytes), one launch per round",
            "traffic": traffic, "launches": pk["launches"], "avg_ms": pk["ms"] / launches,
            "fp64_view": {"achieved_TFLOPs": fp64, "peak_TFLOPs": fp64_peak, "frac": fp64 / fp64_peak,
                          "work": "2 FMA per evaluated nonzero (activities) + 2 FMA per entry side S3 tests; "
                                  "2 flops per FMA",
                          "peak_source": "2 DFMA/SM/clk (ncu peak_sustained) x 152 SMs x 2.07 GHz"},
            "kernel_families": {k: {"ms": v["ms"], "launches": v["launches"],
                                    "GBps": v["bytes"] / (v["ms"] / 1e3) / 1e9 if v["ms"] > 0 else None}
                                for k, v in kern.items()}}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(seconds_budget: float = 20.0):
    """The oracle (single thread) on a bounded sample of the workload: the
    skewed generator at m = 200k (about a tenth of the nonzeros)."""
    import oracle
    from paper_2609_16182_gb300 import synth
    lp = synth.skewed(0, m=200_000, n=300_000, target_nnz=2_000_000, row_cap=50_000)
    t0 = time.perf_counter()
    res = oracle.presolve(lp)
    dt = time.perf_counter() - t0
    nnz_proc = int(res.round_nnz.sum())
    return {"value": nnz_proc / dt, "unit": "nnz/s", "cores": 1, "kind": "oracle",
            "sample": f"skewed LP m=200k n=300k nnz={lp.nnz} (one full presolve, {res.rounds} rounds, "
                      f"{dt:.2f} s on one host core)"}


def batched_leg(lpp, synth, torch, dev, stream, count=4096):
    """Ragged batch (m log-uniform in [50, 5000], n = 1.5 m, ~6 nonzeros per
    row, the 200-row planted mix scaled by m/200): one lpp_presolve_batch call
    against `count` lpp_presolve calls, device-resident inputs, same results."""
    lps = synth.batch_mix(0, count=count)
    d = [synth.LP(m=lp.m, n=lp.n, **{k: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
                                     for k, v in lp.arrays().items()}) for lp in lps]
    o = lpp.opts(stream=stream.cuda_stream)
    packed = lpp.pack_lps(d)  # the lpp_lp array a C caller would hold
    # warm-up at full size (memory pool); the first calls also let the
    # library time each launch geometry of its persistent kernel once
    for _ in range(8):
        lpp.presolve_batch(packed, o).close()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record(stream)
    for q in range(reps):
        res = lpp.presolve_batch(packed, o)
        if q < reps - 1:
            res.close()  # every handle of the batch in one call
    e1.record(stream)
    torch.cuda.synchronize(dev)
    batch_ms = e0.elapsed_time(e1) / reps
    kernel_ms = res[0].info.presolve_ms
    keys = [(r.status, r.info.m_red, r.info.n_red, r.info.nnz_red, r.rounds) for r in res]
    recs = [(r.row_kind.copy(), r.col_kind.copy()) for r in res]
    res.close()
    # the per-round launches over the arena, for comparison
    o_arena = lpp.opts(stream=stream.cuda_stream, batch_persistent=0)
    lpp.presolve_batch(packed, o_arena).close()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    res_a = lpp.presolve_batch(packed, o_arena)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    arena_ms = e0.elapsed_time(e1)
    same_arena = all(np.array_equal(r.row_kind, a) and np.array_equal(r.col_kind, b)
                     for r, (a, b) in zip(res_a, recs))
    res_a.close()
    e0.record(stream)
    plain = []
    for x in d:
        r = lpp.presolve(x, o)
        plain.append((r.status, r.info.m_red, r.info.n_red, r.info.nnz_red, r.rounds))
        r.close()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = e0.elapsed_time(e1)
    nnz_all = int(sum(lp.nnz for lp in lps))
    return {"lps": count, "nnz": nnz_all, "batched_ms": batch_ms,
            "batched_lps_per_s": count / (batch_ms / 1e3), "batched_nnz_per_s": nnz_all / (batch_ms / 1e3),
            "persistent_kernel_ms": kernel_ms, "host_reads_per_round": 0,
            "per_round_launches_ms": arena_ms, "per_round_launches_lps_per_s": count / (arena_ms / 1e3),
            "plain_ms": plain_ms,
            "plain_lps_per_s": count / (plain_ms / 1e3), "speedup": plain_ms / batch_ms,
            "identical_results": keys == plain and same_arena,
            "workload": "4096 LPs, m log-uniform in [50, 5000], n = 1.5 m, ~6 nnz/row, planted mix of the "
                        "200-row LP scaled by m/200; device inputs; one batched call (every round of each LP in one "
                        "persistent kernel) vs the same call with per-round launches vs 4096 plain calls"}


def opt_in_leg(lpp, torch, dev, stream, q, workload, option, fam, count, steps=10):
    """One opt-in presolve step on LP q, timed with the step on and off (CUDA
    events, `steps` presolves each after two warm-ups); outside the timed
    steps, one presolve with per-family events gives the step's own time
    (family `fam`) and count(result) its reductions."""
    d = synth_lp_to(q, torch, dev)
    out = {"workload": workload}
    for on in (1, 0):
        o = lpp.opts(stream=stream.cuda_stream, **{option: on})
        for _ in range(2):
            lpp.presolve(d, o).close()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        proc = 0
        e0.record(stream)
        for _ in range(steps):
            r = lpp.presolve(d, o)
            proc += int(r.info.nnz_processed)
            r.close()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        out["on" if on else "off"] = {"ms_per_step": ms, "nnz_per_s": proc / steps / (ms / 1e3)}
    rt = lpp.presolve(d, lpp.opts(stream=stream.cuda_stream, timing=1, **{option: 1}))
    k = rt.kernels.get(fam, {"ms": 0.0, "launches": 0})
    out.update(count(rt), rounds=rt.rounds, step_family=fam, step_ms=k["ms"],
               reduced_nnz=int(rt.info.nnz_red))
    rt.close()
    return out


def synth_lp_to(q, torch, dev):
    from paper_2609_16182_gb300 import synth
    return synth.LP(m=q.m, n=q.n, **{k: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
                                     for k, v in q.arrays().items()})


def parcols_leg(lpp, synth, torch, dev, stream, lp):
    """The benchmark LP with 1% of its columns copied and scaled (planted
    parallel columns), with the parallel-column step on and off."""
    q = synth.plant_parallel_cols(lp, 0, frac=0.01)
    return opt_in_leg(lpp, torch, dev, stream, q,
                      f"benchmark LP + {len(q.planted['par_copies'])} scaled column copies (n = {q.n}, nnz = {q.nnz})",
                      "parallel_cols", "s5c",
                      lambda r: {"merged": int(np.count_nonzero(r.col_kind == lpp.COL_PARALLEL))})


def colsing_leg(lpp, synth, torch, dev, stream, lp):
    """The benchmark LP with a free column singleton (cost 0, so that the LP
    stays bounded) in 30% of its equality rows, with the column-singleton
    step on and off."""
    q = synth.plant_col_singletons(lp, 0, frac=0.3, free_frac=1.0, cost_scale=0.0)

    def count(r):
        sub = r.row_kind == lpp.ROW_SUBST
        return {"substitutions": int(np.count_nonzero(sub)),
                "longest_row": int(np.diff(q.row_ptr)[sub].max()) if sub.any() else 0}

    return opt_in_leg(lpp, torch, dev, stream, q,
                      f"benchmark LP + {len(q.planted['cs_cols'])} free singleton columns in equality rows "
                      f"(n = {q.n}, nnz = {q.nnz})", "col_singletons", "s5d", count)


def dualfix_leg(lpp, torch, dev, stream, lp):
    """The benchmark LP itself with dual fixing by locks on and off (the
    locks are counted in the compaction family)."""
    return opt_in_leg(lpp, torch, dev, stream, lp, "benchmark LP", "dual_fixing", "compact_count",
                      lambda r: {"dual_fixed": int(np.count_nonzero(r.col_kind == lpp.COL_EMPTY))})


def dualrec_leg(lpp, torch, dev, stream, lp):
    """The benchmark LP with the bound-source records (dual_records) on and
    off; their kernels run in the colfin family.  Outside the timed steps,
    the host time of one primal-dual postsolve (lpp_postsolve_dual) of that
    LP from a reduced pair: x at the middle of each finite range (else at its
    finite end, else 0), y = 0, so every reduced cost c_j on a row-set side
    is carried back to its row."""

    def count(r):
        red = r.reduced(csc=False)
        lo, hi = red.lb, red.ub
        fl, fh = np.abs(lo) < 1e20, np.abs(hi) < 1e20
        lo0, hi0 = np.where(fl, lo, 0.0), np.where(fh, hi, 0.0)
        xr = np.where(fl & fh, 0.5 * (lo0 + hi0), lo0 + hi0)
        yr = np.zeros(r.info.m_red)
        src = r.bound_sources()
        t0 = time.perf_counter()
        _, y, _ = r.postsolve_dual(lp, xr, yr)
        dt = time.perf_counter() - t0
        return {"sides_with_source": int((src["lsrc"] >= 0).sum() + (src["usrc"] >= 0).sum()),
                "rows_given_a_dual": int(np.count_nonzero(y)), "postsolve_dual_host_ms": 1e3 * dt}

    return opt_in_leg(lpp, torch, dev, stream, lp, "benchmark LP", "dual_records", "colfin", count)


def deprows_leg(lpp, synth, torch, dev, stream, lp):
    """The benchmark LP with 20 planted dependent equality rows (each a
    combination of three of its equality rows), with the dependent-row step
    (dep_rows: the reduced LP's equality rows eliminated on the host, the
    rows found removed on the device) on and off."""
    q = synth.plant_dependent_rows(lp, 0, count=20)
    return opt_in_leg(lpp, torch, dev, stream, q, "benchmark LP + 20 planted dependent equality rows", "dep_rows",
                      "compact_count",
                      lambda r: {"dependent_rows": int(r.info.dep_rows), "pivot_rows": int(r.info.dep_pivots),
                                 "peeled_rows": int(r.info.dep_peeled),
                                 "stopped_at_fill_cap": int(r.info.dep_stopped)}, steps=5)


def doubleton_leg(lpp, synth, torch, dev, stream, q):
    """The LP-relaxation workload (500k rows, 1M columns, 7.8M nonzeros,
    4% doubleton equations, 10 dense columns) with the doubleton step on and
    off."""

    def count(r):
        return {"doubletons": int(np.count_nonzero(r.row_kind == lpp.ROW_DOUBLETON))}

    return opt_in_leg(lpp, torch, dev, stream, q,
                      f"LP relaxation (m = {q.m}, n = {q.n}, nnz = {q.nnz}), 4% doubleton equations",
                      "doubletons", "s5e", count)


def lprelax_leg(lpp, synth, torch, dev, stream, q, peak_gbs, peak_src, steps=20, warmup=3):
    """The LP-relaxation workload (m = 500k, n = 1M, 8M nonzeros, 10 dense
    columns of 200k entries, 5% scaled row copies, 4% doubleton equations, 2%
    loosened bounds) with the default steps: ms per presolve, nnz/s, per-round
    sizes and times, and the activity kernel's roofline."""
    d = synth_lp_to(q, torch, dev)
    o = lpp.opts(stream=stream.cuda_stream)
    for _ in range(warmup):
        lpp.presolve(d, o).close()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    proc, first = 0, None
    e0.record(stream)
    for _ in range(steps):
        r = lpp.presolve(d, o)
        proc += int(r.info.nnz_processed)
        if first is None:
            first = (r.info, ([float(x) for x in r.round_ms], [int(x) for x in r.round_nnz],
                              [int(x) for x in r.round_rows_removed], [int(x) for x in r.round_cols_fixed],
                              [int(x) for x in r.round_bounds_changed]))
        r.close()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    rounds_d = describe_rounds(first[0], first[1], peak_gbs)
    rt = lpp.presolve(d, lpp.opts(stream=stream.cuda_stream, timing=1))
    kern = rt.kernels
    rt.close()
    roof = prop_roofline(kern, rounds_d, peak_gbs, peak_src, None)
    roof.pop("kernel_families")
    return {"workload": f"LP relaxation (m = {q.m}, n = {q.n}, nnz = {q.nnz}): 10 dense columns of 200k, 5% "
                        "scaled row copies, 4% doubleton equations, 2% loosened bounds; default steps",
            "steps": steps, "ms_per_step": ms, "nnz_per_s": proc / steps / (ms / 1e3), **rounds_d,
            "roofline": roof,
            "kernel_families": {k: {"ms": v["ms"], "launches": v["launches"]} for k, v in kern.items()}}


def serving_leg(lpp, synth, torch, dev, pool_size=16, requests=2000, nnz_hi=1e7, budget=120 << 30, seed=0):
    """Poisson arrivals of skewed-like LPs (nnz log-uniform in [1e3, 1e7],
    m = nnz/10, n = 1.5 m; requests draw from a pool of `pool_size` distinct
    LPs, generated once before any timing), replayed in real time at 0.5x,
    0.8x and 1.2x the serial capacity: the continuous-batching server against
    a serial loop of lpp_presolve on the same arrivals.  Latency = completion
    - arrival."""
    import threading
    rng = np.random.default_rng(seed)
    nnz = np.exp(rng.uniform(np.log(1e3), np.log(nnz_hi), pool_size)).astype(int)
    pool = [synth.skewed_like(seed * 1_000_003 + k, int(z)) for k, z in enumerate(nnz)]
    dpool = [synth.LP(m=lp.m, n=lp.n, **{k: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
                                         for k, v in lp.arrays().items()}) for lp in pool]
    # serial service time of each pool LP
    for x in dpool[:4]:
        lpp.presolve(x).close()
    svc = []
    for x in dpool:
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        lpp.presolve(x).close()
        svc.append(time.perf_counter() - t0)
    mean_svc = float(np.mean(svc))
    out = {"pool": pool_size, "requests": requests, "budget_bytes": budget, "serial_capacity_lps": 1.0 / mean_svc,
           "pool_nnz_mean": float(np.mean([lp.nnz for lp in pool])), "pool_nnz_max": int(max(lp.nnz for lp in pool)),
           "workload": f"Poisson arrivals, {requests} requests per load, skewed-like LPs with nnz log-uniform in "
                       f"[1e3, {nnz_hi:.0e}] (pool of {pool_size}), {budget >> 30} GB budget", "rates": []}

    def pct(a, q):
        return float(np.percentile(np.asarray(a) * 1e3, q))

    srv = lpp.Server(budget)
    try:
        for f in (0.5, 0.8, 1.2):
            lam = f / mean_svc
            arr = np.cumsum(rng.exponential(1.0 / lam, requests))
            pick = rng.integers(0, pool_size, requests)
            # serial loop on the same arrivals
            t0 = time.perf_counter()
            lat_s, last = [], 0.0
            for k in range(requests):
                while time.perf_counter() - t0 < arr[k]:
                    pass
                lpp.presolve(dpool[pick[k]]).close()
                last = time.perf_counter() - t0
                lat_s.append(last - arr[k])
            serial_span = last
            # the server
            tickets = [None] * requests
            done_at = [0.0] * requests
            nsub = [0]
            t0 = time.perf_counter()

            def submitter():
                for k in range(requests):
                    dt = arr[k] - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
                    tickets[k] = srv.submit(dpool[pick[k]])
                    nsub[0] = k + 1

            th = threading.Thread(target=submitter)
            th.start()
            # wait on the oldest request not yet taken (in the library, without
            # the interpreter lock and without spinning), then sweep the others
            pending, nxt = [], 0
            while nxt < requests or pending:
                while nxt < nsub[0]:
                    pending.append(nxt)
                    nxt += 1
                if not pending:
                    time.sleep(0.00005)
                    continue
                still = []
                for q, k in enumerate(pending):
                    try:
                        r = srv.take(tickets[k], 1 if q == 0 else 0)
                    except lpp.LppError as e:
                        if e.status == lpp.ERR_TIMEOUT:
                            still.append(k)
                            continue
                        raise
                    done_at[k] = time.perf_counter() - t0
                    r.close()
                pending = still
            th.join()
            lat = [done_at[k] - arr[k] for k in range(requests)]
            span = max(done_at)
            out["rates"].append({"load": f, "arrival_lps": lam,
                                 "served_lps": requests / span, "served_p50_ms": pct(lat, 50),
                                 "served_p99_ms": pct(lat, 99), "serial_lps": requests / serial_span,
                                 "serial_p50_ms": pct(lat_s, 50), "serial_p99_ms": pct(lat_s, 99)})
        out["server_stats"] = srv.stats()
    finally:
        srv.close()
    return out


def run_reference(args):
    """--impl reference: the CPU oracle as the reference arm."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2609_16182_gb300 import synth
    lp = synth.skewed(0, m=200_000, n=300_000, target_nnz=2_000_000, row_cap=50_000)
    for _ in range(args.warmup):
        oracle.presolve(lp)
    times, procs = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res = oracle.presolve(lp)
        times.append(time.perf_counter() - t0)
        procs.append(int(res.round_nnz.sum()))
    tot = sum(times)
    value = sum(procs) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "m=200k n=300k bounded sample of the workload"},
            "cpu_baseline": {"value": value, "unit": "nnz/s", "cores": 1, "kind": "oracle",
                             "sample": f"skewed LP m=200k n=300k nnz={lp.nnz} per step"},
            "e2e": {"value": value, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_batch(args):
    """W + K calls of lpp_presolve_batch on the 4,096-LP workload (device
    inputs), for a profiler: no timing, no other leg."""
    import torch
    from paper_2609_16182_gb300 import lpp, synth
    dev = torch.device("cuda", 0)
    lpp.load()
    lps = synth.batch_mix(0, count=4096)
    d = [synth.LP(m=lp.m, n=lp.n, **{k: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
                                     for k, v in lp.arrays().items()}) for lp in lps]
    packed = lpp.pack_lps(d)
    o = lpp.opts(stream=torch.cuda.current_stream(dev).cuda_stream)
    kernel_ms = []
    for _ in range(args.warmup + args.steps):
        res = lpp.presolve_batch(packed, o)
        kernel_ms.append(res[0].info.presolve_ms)
        res.close()
    torch.cuda.synchronize(dev)
    print(json.dumps({"profile_batch": True, "calls": args.warmup + args.steps, "kernel_ms": kernel_ms}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-presolve leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-parcols", action="store_true", help="skip the parallel-columns leg")
    ap.add_argument("--no-colsing", action="store_true", help="skip the column-singletons leg")
    ap.add_argument("--no-dualfix", action="store_true", help="skip the dual-fixing leg")
    ap.add_argument("--no-dualrec", action="store_true", help="skip the dual-records leg")
    ap.add_argument("--no-deprows", action="store_true", help="skip the dependent-rows leg")
    ap.add_argument("--no-doubletons", action="store_true", help="skip the doubleton-equations leg")
    ap.add_argument("--no-lprelax", action="store_true", help="skip the LP-relaxation workload leg")
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the LP (profiling runs only)")
    ap.add_argument("--profile", action="store_true",
                    help="profiling run: W + K steps only (no timing pass, e2e or CPU baseline)")
    ap.add_argument("--parallel-cols", action="store_true",
                    help="with --profile: the LP with 1%% of its columns copied, parallel-column step on")
    ap.add_argument("--col-singletons", action="store_true",
                    help="with --profile: the LP with free singletons in 30%% of its equality rows, step on")
    ap.add_argument("--profile-batch", action="store_true",
                    help="profiling run: W + K batched presolves of the 4,096-LP workload only")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_batch:
        return profile_batch(args)

    import torch
    import torch.distributed as dist
    from paper_2609_16182_gb300 import lpp, synth

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lpp.load()

    s = args.scale
    lp = synth.skewed(rank, m=int(2_000_000 * s), n=int(3_000_000 * s), target_nnz=int(20_000_000 * s),
                      row_cap=int(500_000 * s) if s < 1 else 500_000)
    if (args.parallel_cols or args.col_singletons) and not args.profile:
        raise SystemExit("--parallel-cols / --col-singletons are profiling options (use with --profile)")
    if args.parallel_cols:
        lp = synth.plant_parallel_cols(lp, 0, frac=0.01)
    if args.col_singletons:
        lp = synth.plant_col_singletons(lp, 0, frac=0.3, free_frac=1.0, cost_scale=0.0)
    d_lp = synth.LP(m=lp.m, n=lp.n, **{k: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
                                        for k, v in lp.arrays().items()})
    stream = torch.cuda.current_stream(dev)
    o_dev = lpp.opts(stream=stream.cuda_stream, timing=0, parallel_cols=1 if args.parallel_cols else 0,
                     col_singletons=1 if args.col_singletons else 0)
    o_time = lpp.opts(stream=stream.cuda_stream, timing=1)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # warm-up
    for _ in range(args.warmup):
        r = lpp.presolve(d_lp, o_dev)
        r.close()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nnz_proc = 0
    launches = 0
    first = None
    with ClockSampler(local) as clk:
        barrier()
        clk.t0 = time.monotonic()
        ev0.record(stream)
        for _ in range(args.steps):
            r = lpp.presolve(d_lp, o_dev)
            nnz_proc += int(r.info.nnz_processed)
            launches += int(r.info.launches)
            if first is None:  # host-side copies: no device work
                first = (r.info, ([float(x) for x in r.round_ms], [int(x) for x in r.round_nnz],
                                  [int(x) for x in r.round_rows_removed], [int(x) for x in r.round_cols_fixed],
                                  [int(x) for x in r.round_bounds_changed]))
            r.close()  # the reduced LP is handed on and freed, as a caller would
        ev1.record(stream)
        barrier()
        clk.t1 = time.monotonic()
    ms_total = ev0.elapsed_time(ev1)
    if args.profile:
        print(json.dumps({"profile": True, "steps": args.steps, "ms_per_step": ms_total / max(1, args.steps),
                          "nnz": lp.nnz}), flush=True)
        return
    info, per_round = first
    ms_max, value = reduce_over_ranks(ms_total, nnz_proc, dev, ws)
    peak_gbs, peak_src = measured_peaks()
    rounds_d = describe_rounds(info, per_round, peak_gbs)

    # per-kernel times: one more step with CUDA events around every launch family
    rt = lpp.presolve(d_lp, o_time)
    kern = rt.kernels
    rt.close()
    traffic_file = os.path.join(ROOT, "profiles", "prop_traffic.json")
    traffic = None
    if os.path.exists(traffic_file):
        with open(traffic_file) as f:
            traffic = json.load(f).get("bytes_per_launch")
    roofline = prop_roofline(kern, rounds_d, peak_gbs, peak_src, traffic)

    # end to end: pinned host buffers, H2D + presolve + D2H of the reduced LP
    pinned = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in lp.arrays().items()}
    h_lp = synth.LP(m=lp.m, n=lp.n, **{k: v.numpy() for k, v in pinned.items()})
    h2d = sum(v.numel() * v.element_size() for v in pinned.values())
    e2e_steps = max(1, min(args.steps, 5))
    for _ in range(2):  # warm: the pinned host block of the reduced LP, the device pool
        r = lpp.presolve(h_lp, o_dev)
        r.reduced(copy=False, csc=False)
        r.close()
    barrier()
    t0 = time.perf_counter()
    d2h = 0
    e2e_proc = 0
    for _ in range(e2e_steps):
        r = lpp.presolve(h_lp, o_dev)
        # the reduced LP of Eq. 1 (CSR, c, sides, bounds) and its index maps, read
        # in the library's pinned host block
        red = r.reduced(copy=False, csc=False)
        d2h = sum(a.nbytes for a in (red.row_ptr, red.col_idx, red.val, red.c, red.lhs, red.rhs, red.lb, red.ub,
                                     red.row_map, red.col_map))
        e2e_proc += int(r.info.nnz_processed)
        r.close()
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": e2e_proc / e2e_s, "unit": "nnz/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * e2e_s / e2e_steps}

    batched = None
    if not args.no_batch:
        batched = batched_leg(lpp, synth, torch, dev, stream)
    serving = None
    if not args.no_serve:
        serving = serving_leg(lpp, synth, torch, dev)
    parcols = None
    if not args.no_parcols:
        parcols = parcols_leg(lpp, synth, torch, dev, stream, lp)
    colsing = None
    if not args.no_colsing:
        colsing = colsing_leg(lpp, synth, torch, dev, stream, lp)
    dualfix = None
    if not args.no_dualfix:
        dualfix = dualfix_leg(lpp, torch, dev, stream, lp)
    dualrec = None
    if not args.no_dualrec:
        dualrec = dualrec_leg(lpp, torch, dev, stream, lp)
    deprows = None
    if not args.no_deprows:
        deprows = deprows_leg(lpp, synth, torch, dev, stream, lp)
    lprelax = doubletons = None
    if not (args.no_lprelax and args.no_doubletons):
        q = synth.lprelax(0)
        if not args.no_lprelax:
            lprelax = lprelax_leg(lpp, synth, torch, dev, stream, q, peak_gbs, peak_src)
        if not args.no_doubletons:
            doubletons = doubleton_leg(lpp, synth, torch, dev, stream, q)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD if s == 1 else f"{WORKLOAD} (scaled by {s})",
                           "m": lp.m, "n": lp.n, "nnz": lp.nnz, **rounds_d,
                           "l2": "inputs larger than L2 (CSR alone ~245 MB > 129 MB)",
                           "parallelism": f"replicas x{ws}"},
                "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(),
                "batched": batched, "serving": serving, "parallel_cols": parcols, "col_singletons": colsing,
                "dual_fixing": dualfix, "dual_records": dualrec, "dependent_rows": deprows, "doubletons": doubletons,
                "lp_relaxation": lprelax}
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
