#!/usr/bin/env python
"""Benchmark: NGS-FAS Richards solver on the 3D drainage workload (256^3).

One bench step is one implicit BDF2 time step of the whole path (FP64
per-step preparation, an FP64 outer defect correction of the FP64 state
around FP32 FAS cycles with red-black NGS, the FP64 stop test, FP64 water
balance, history shift) on 256^3 cells of heterogeneous van Genuchten soil
draining from saturation.  --precision 1 times the float-float outer layer
instead; the line carries the other one's figures beside the headline.  Inputs (16.8 M cells, 134 MB per
FP64 array) are larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank solves its own
replica (the path has no exchange step here): weak scaling, value = the
cell-updates of all ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NGS cell-updates/s and time-steps/s at 256^3; p50/p99 solve latency, vs FP64 plain @1e-8"
UNIT = "cell-updates/s"
def workload_name(precision):
    outer = ("FP64 outer defect correction (FP64 lagged K, history, deciding defect, stop test and water "
             "balance; float-float steering defects)" if precision == 2 else
             "float-float outer defect correction on the FP64 state")
    return ("3D drainage 256^3, heterogeneous VG (lognormal Ks, sigma_lnK=1, corr 8 cells; alpha U[2,5], "
            f"n U[1.5,2.5]), psi0=0, free drainage bottom, BDF2 dt=300 s, mixed: FP32 inner cycles, {outer}, "
            "tol 1e-8")


DTYPE = {2: "f32 inner / f64 outer, f64 state", 1: "f32 inner / float-float (f32x2) outer, f64 state"}

# Algorithmic bytes per unit for the kernels that can dominate (per cell the
# launch covers; a half-sweep covers the cells of one colour).  The NGS
# figure is the mixed-mode inner update of the heterogeneous workload:
# delta read+write, Kc, r, psi0, alpha, n (7 x 4 B).
# DRAM bytes (read + write) per launch of the finest level's half-sweep of
# 256^3 (8,388,608 cells, colour-split parameters, 128-thread blocks, two
# planes), from an ncu capture of this kernel (dram__bytes_read.sum +
# dram__bytes_write.sum); the roofline's traffic.
TRAFFIC_PER_LAUNCH = {("sweep32", 8388608): 318.5e6}
# What binds that launch instead of DRAM, from the same capture: the share of
# issue slots active (smsp__issue_active) and of DRAM bandwidth in use.
BINDING_PER_LAUNCH = {("sweep32", 8388608): {"limit": "instruction issue", "issue_active": 0.81,
                                             "dram_throughput": 0.42, "thread_instructions_per_update": 345,
                                             "source": "ncu --set full (profiles/sweep32_drainage256_mixed.md)"}}

BYTES_PER_CELL = {
    "sweep32": 28.0,
    "residual32": 28.0,
    "sweep64": 48.0,
    "residual64": 56.0,
    "outer_residual": 52.0,
    "prep": 88.0,
    "restrict32": 9.0,
    "prolong32": 9.0,
    "tau32": 36.0,
    "apply_delta": 12.0,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-other-outer", action="store_true",
                    help="skip timing the other outer layer (float-float beside FP64, or the reverse)")
    ap.add_argument("--profile-steps", type=int, default=None,
                    help="steps with kernel timing (default: all timed steps)")
    ap.add_argument("--no-columns", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-gardner", action="store_true")
    ap.add_argument("--no-layered", action="store_true")
    ap.add_argument("--no-table3", action="store_true")
    ap.add_argument("--no-celia", action="store_true")
    ap.add_argument("--no-strip", action="store_true")
    ap.add_argument("--temporal-study", action="store_true",
                    help="add Section 4.1's temporal-convergence study (N=1024 vs N=2048, tau_ref=1e-4; ~4 min)")
    ap.add_argument("--gamma", type=int, default=2, help="1 = V-cycles, 2 = W-cycles")
    ap.add_argument("--precision", type=int, default=2, choices=[1, 2],
                    help="outer defect correction of the headline: 2 = FP64, 1 = float-float")
    ap.add_argument("--profile-json", default=None, help="write the per-kernel timing records here")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={CLOCK_Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not self.path:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def roofline(prof, steps, ms_pass):
    """Roofline of the dominant kernel (largest summed device time) from the
    event-timed pass of `steps` steps that took ms_pass in all."""
    by_name = {}
    for r in prof:
        by_name.setdefault(r["name"], []).append(r)
    totals = {k: sum(x["ms"] for x in v) for k, v in by_name.items()}
    dom = max(totals, key=totals.get)
    recs = by_name[dom]
    fine = [r for r in recs if r["level"] == 0] or sorted(recs, key=lambda r: -r["ms"])[:1]
    launches = sum(r["launches"] for r in fine)
    ms = sum(r["ms"] for r in fine)
    cells = sum(r["cells"] for r in fine)
    pk, src = peaks()
    shares = {k: round(v / max(sum(totals.values()), 1e-30), 4) for k, v in
              sorted(totals.items(), key=lambda kv: -kv[1])}
    out = {"kernel": dom, "level": fine[0]["level"], "launches": launches,
           "avg_launch_ms": ms / max(launches, 1), "share_of_kernel_time": shares[dom],
           "kernel_shares": shares,
           "timing": f"CUDA events around every launch on the solver's stream over {steps} steps right "
                     f"after the timed region ({ms_pass / steps:.1f} ms/step with the events)"}
    if dom in BYTES_PER_CELL:
        bytes_per_launch = BYTES_PER_CELL[dom] * cells / max(launches, 1)
        achieved = bytes_per_launch / (ms / max(launches, 1) * 1e-3) / 1e9
        out.update({"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / pk["hbm_gbs"], "peak_source": src + " hbm_gbs",
                    "algorithmic_bytes_per_launch": bytes_per_launch,
                    "traffic": TRAFFIC_PER_LAUNCH.get((dom, round(cells / max(launches, 1)))),
                    "binding": BINDING_PER_LAUNCH.get((dom, round(cells / max(launches, 1))))})
    else:
        out.update({"bound": "hbm", "achieved": None, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": None,
                    "traffic": None})
    return out


# ---------------------------------------------------------------------------
def columns_bench(stream, steps=10, rank=0, world=1):
    """Batched root-uptake columns: 4096 columns of U{64..1024} cells, per-column
    van Genuchten soil, Feddes sink, BDF1 dt = 600 s; every column advances
    `steps` steps in one call: a persistent launch per length class (block
    size autotuned first).
    Under torchrun each rank takes every world-th column (replicas.shard) and
    the ranks' summaries are merged: the slowest rank's time, summed work."""
    import numpy as np
    import torch
    from paper_2606_04292_gb300 import replicas
    from paper_2606_04292_gb300 import richards as R
    from paper_2606_04292_gb300 import workloads as W
    allp = W.columns()
    ids = replicas.shard(range(len(allp)), rank, world)
    probs = [allp[k] for k in ids]
    cols = R.Columns(probs, stream=stream.cuda_stream)
    dt = probs[0]["dt"]
    threads = cols.autotune(dt)
    cols.run(dt, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = cols.run(dt, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    stt = cols.stats()
    part = {"ids": ids, "ms": ms, "units": len(ids), "updates": float(np.sum(stt["updates"])),
            "unit_steps": len(ids) * steps, "ok": bool(np.all(stt["status"] == R.RICH_OK) and st == R.RICH_OK)}
    parts = replicas.gather(part)
    allpart = replicas.combine(parts)
    out = {"workload": "4096 columns U{64..1024} cells, VG per column, Feddes sink, BDF1 dt=600 s, mixed "
                       "(float-float outer)",
           "columns": len(allp), "cells": int(sum(p["n"][0] for p in allp)), "steps": steps, "threads": threads,
           "ranks": world, "status": R.STATUS_NAMES[st], "all_columns_ok": all(p["ok"] for p in parts),
           "column_steps_per_s": allpart["unit_steps"] / (allpart["ms"] * 1e-3),
           "cell_updates_per_s": allpart["updates"] / (allpart["ms"] * 1e-3), "ms": allpart["ms"]}
    psi = cols.state()
    # the CPU leg's sample: every COLUMN_CPU_EVERY-th column this rank took
    sample = {k: cols.column(psi, j).copy() for j, k in enumerate(ids) if k % COLUMN_CPU_EVERY == 0}
    cols.close()
    return out, sample


COLUMN_CPU_EVERY = 64     # the CPU leg runs every 64th column: 64 columns across the length mix


def columns_cpu(sample, steps):
    """The oracle on the sampled columns of the batched-column workload: the
    same 1 + steps BDF1 steps (the first untimed, as on the GPU), single
    thread; column-steps/s over the timed steps, and the largest distance of
    the GPU's mixed-precision states to the oracle's FP64 ones."""
    import numpy as np
    from oracle.oracle import Oracle
    from paper_2606_04292_gb300 import workloads as W
    probs = W.columns()
    total = 0.0
    cells = 0
    dmax = 0.0
    failed = 0
    for k, psi_gpu in sample.items():
        o = Oracle(probs[k])
        failed += o.step()[0] != 0
        t0 = time.perf_counter()
        for _ in range(steps):
            failed += o.step()[0] != 0
        total += time.perf_counter() - t0
        cells += len(psi_gpu)
        dmax = max(dmax, float(np.max(np.abs(o.state() - psi_gpu))))
    return {"cores": 1, "columns": len(sample), "steps": steps, "cells": cells, "failed_steps": int(failed),
            "column_steps_per_s": len(sample) * steps / total, "cell_steps_per_s": cells * steps / total,
            "max_abs_dpsi_gpu_vs_oracle": dmax,
            "sample": f"every {COLUMN_CPU_EVERY}th column ({len(sample)} columns, {cells} cells), {steps} timed steps"}


SERVING_MODES = {
    # label: (precision, batched)
    "batched_mixed_fp64_outer": (2, True),
    "streams_mixed_fp64_outer": (2, False),
    "streams_mixed_float_float_outer": (1, False),
    "streams_fp64_plain": (0, False),
}


def _serve(trace, ids, precision, batched):
    from paper_2606_04292_gb300 import replicas
    from paper_2606_04292_gb300 import serve
    srv = serve.Server(max_active=16 if batched else 8, opts={"precision": precision}, batched=batched)
    results, summary = srv.run([trace[k] for k in ids], realtime=True)
    part = {"ids": ids, "ms": summary["makespan_s"] * 1e3, "completed": summary["completed"],
            "rejected": summary.get("rejected", 0),
            "updates": summary["cell_updates_per_s"] * summary["makespan_s"],
            "latencies": [r["latency"] for r in results if r["status"] == "OK"]}
    m = replicas.combine(replicas.gather(part))
    mk = m["ms"] * 1e-3
    return {"completed": m["completed"], "makespan_s": mk, "solves_per_s": m["completed"] / mk,
            "cell_updates_per_s": m["updates"] / mk, "p50_latency_s": m["p50_latency_s"],
            "p99_latency_s": m["p99_latency_s"]}


SERVING_RATES = (25.0, 50.0, 100.0, 200.0)   # offered loads of the rate sweep, requests/s


def serving_bench(nreq=24, max_steps=20, rank=0, world=1):
    """Served streams of Poisson arrivals at 200/s (three soil laws, half with a
    sink, BDF2), at most `max_steps` steps each.  Two traces: a reduced size
    mix (2D 129^2/257^2, 3D 65^3), served by continuous batching
    (richards_batcher_step) and by per-request streams, in the FP64-outer and
    float-float mixed modes and FP64 plain; and the configured size mix (2D
    129^2-1025^2, 3D 65^3-257^3), mixed with the FP64 outer layer, batched and
    per-stream.  Offered load is the arrival rate; served load the solve rate;
    the reduced mix is also served at 25, 50, 100 and 200 requests/s.
    Under torchrun each rank serves every world-th request (replicas.shard);
    completions and latencies are merged over the ranks."""
    from paper_2606_04292_gb300 import replicas
    from paper_2606_04292_gb300 import workloads as W

    def trace_of(sizes2d, sizes3d):
        tr = W.serving_trace(rate=200.0, seconds=60.0, seed=6, sizes2d=sizes2d, sizes3d=sizes3d, max_requests=nreq)
        for p in tr:
            p["nsteps"] = min(p["nsteps"], max_steps)
        return tr

    out = {"offered_requests_per_s": 200.0, "ranks": world, "max_steps": max_steps}
    red = trace_of((129, 257), (65,))
    ids = replicas.shard(range(len(red)), rank, world)
    out["reduced_mix"] = {"workload": f"{len(red)} Poisson requests (200/s), 2D 129^2-257^2 and 3D 65^3, "
                                      f"<= {max_steps} BDF2 steps"}
    for label, (prec, batched) in SERVING_MODES.items():
        out["reduced_mix"][label] = _serve(red, ids, prec, batched)
    # offered against served load: the same requests at lower Poisson rates
    # (an exponential gap drawn at 200/s, times 200/r, is one drawn at r/s),
    # continuous batching with the FP64 outer layer
    sweep = []
    for rate in SERVING_RATES:
        r = _serve([dict(p, arrival=p["arrival"] * 200.0 / rate) for p in red], ids, 2, True)
        sweep.append({"offered_requests_per_s": rate, "served_solves_per_s": r["solves_per_s"],
                      "p50_latency_s": r["p50_latency_s"], "p99_latency_s": r["p99_latency_s"]})
    out["reduced_mix"]["rate_sweep_batched_mixed_fp64_outer"] = sweep
    full = trace_of((129, 257, 513, 1025), (65, 129, 257))
    ids = replicas.shard(range(len(full)), rank, world)
    out["configured_mix"] = {
        "workload": f"{len(full)} Poisson requests (200/s) of the configured size mix, 2D 129^2-1025^2 and 3D "
                    f"65^3-257^3, <= {max_steps} BDF2 steps (FP64 plain not run on this mix: its 257^3 requests "
                    "take ~0.6 s a step)",
        "sizes": sorted({f"{p['dim']}D {p['n'][0]}" for p in full})}
    for label in ("batched_mixed_fp64_outer", "streams_mixed_fp64_outer"):
        prec, batched = SERVING_MODES[label]
        out["configured_mix"][label] = _serve(full, ids, prec, batched)
    return out


SERVING_CPU_REQUESTS = 6   # the CPU leg times the first step of this many requests of the trace


def serving_cpu(nreq=24, max_steps=20):
    """The oracle on the served trace, bounded: the first step of each of the
    first SERVING_CPU_REQUESTS requests (single thread), its time as measured;
    the trace's serial solve rate at those per-step times is an estimate
    (every step of a request is taken to cost its first step)."""
    import numpy as np
    from oracle.oracle import Oracle
    from paper_2606_04292_gb300 import workloads as W
    trace = W.serving_trace(rate=200.0, seconds=60.0, seed=6, sizes2d=(129, 257), sizes3d=(65,),
                            max_requests=nreq)
    per_step, names, failed = [], [], 0
    for p in trace[:SERVING_CPU_REQUESTS]:
        o = Oracle(p)
        t0 = time.perf_counter()
        failed += o.step()[0] != 0
        per_step.append(time.perf_counter() - t0)
        names.append(f"{p['dim']}D {p['n'][0]}^{p['dim']}")
    steps = [min(p["nsteps"], max_steps) for p in trace[:SERVING_CPU_REQUESTS]]
    solve_s = float(np.sum(np.array(per_step) * np.array(steps)))
    return {"cores": 1, "requests": names, "s_per_step": per_step, "failed_steps": int(failed),
            "serial_solves_per_s_estimate": len(per_step) / solve_s,
            "sample": f"first step of the first {len(per_step)} of {len(trace)} requests"}


def gardner_bench(stream):
    """The paper's 2D Gardner infiltration test in full (Section 4.2: 128^2,
    tau = 0.1 day, 3 days = 30 steps), FP64 plain and mixed, wall time of the
    whole run beside the CPU oracle's and the paper's 2.216 s (its hardware
    unstated).  Returns the summary and the final states (the CPU-baseline
    leg times the oracle on the same run and compares)."""
    import torch
    from paper_2606_04292_gb300 import richards as R
    from paper_2606_04292_gb300 import workloads as W
    out = {"workload": "2D Gardner infiltration 128^2, tau 0.1 day x 30 steps, tol 1e-8",
           "paper_total_cpu_s": 2.216}
    states = {}
    for label, prec in (("fp64_plain", 0), ("mixed", 1)):
        prob = W.gardner_2d(precision=prec)
        gs = R.Solver(prob, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cyc = 0
        for _ in range(prob["nsteps"]):
            st, info = gs.step(check=False)
            cyc += info["cycles"]
        torch.cuda.synchronize()
        out[label] = {"total_s": time.perf_counter() - t0, "status_last": R.STATUS_NAMES[st],
                      "cycles_per_step": cyc / prob["nsteps"]}
        states[label] = gs.state()
        gs.close()
    return out, states


def gardner_cpu(states):
    """The oracle on the whole 2D Gardner run (single thread), and its distance
    to the GPU results."""
    import numpy as np
    from oracle.oracle import Oracle
    from paper_2606_04292_gb300 import workloads as W
    prob = W.gardner_2d()
    o = Oracle(prob)
    t0 = time.perf_counter()
    for _ in range(prob["nsteps"]):
        o.step()
    ref = o.state()
    return {"total_s": time.perf_counter() - t0, "cores": 1,
            "max_abs_dpsi_gpu_vs_oracle": {k: float(np.max(np.abs(v - ref))) for k, v in states.items()}}


def celia_bench(stream):
    """The 1-d infiltration column in full (128 cells over 40 cm, Haverkamp,
    BDF1 dt = 10 s for 36 steps, V(2,2), FP64), red-black and the paper's
    lexicographic order: wall time of the whole run and cycles per step; and
    the same run in mixed precision through the batched-column solver."""
    import torch
    from paper_2606_04292_gb300 import richards as R
    from paper_2606_04292_gb300 import workloads as W
    out = {"workload": "1D Haverkamp column 128 cells, BDF1 dt=10 s x 36 steps, V(2,2), FP64, tol 1e-8"}
    states = {}
    for label, ordering in (("red_black_fp64", 1), ("lexicographic_fp64", 0)):
        prob = W.celia_1d(ordering=ordering)
        gs = R.Solver(prob, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cyc, worst = 0, 0
        for _ in range(prob["nsteps"]):
            st, info = gs.step(check=False)
            cyc += info["cycles"]
            worst = max(worst, st)
        torch.cuda.synchronize()
        out[label] = {"total_s": time.perf_counter() - t0, "steps": prob["nsteps"],
                      "worst_status": R.STATUS_NAMES[worst], "cycles_per_step": cyc / prob["nsteps"]}
        states[label] = gs.state()
        gs.close()
    # the same column through the batched-column solver: the whole run in one
    # launch, FP32 inner cycles inside the float-float outer layer (the path
    # of Table 3's column); a first one-step run loads the column kernels
    import numpy as np
    prob = W.celia_1d(precision=1)
    try:
        warm = R.Columns([prob], stream=stream.cuda_stream)
        warm.run(prob["dt"], 1, 1)
        warm.close()
        cols = R.Columns([prob], stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = cols.run(prob["dt"], prob["nsteps"], 1)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        sts = cols.stats()
        out["columns_mixed_float_float_outer"] = {
            "total_s": wall, "steps": prob["nsteps"], "run_status": R.STATUS_NAMES.get(st, str(st)),
            "status": R.STATUS_NAMES.get(int(sts["status"][0]), str(int(sts["status"][0]))),
            "cycles_per_step": float(sts["cycles"][0]) / prob["nsteps"],
            "max_abs_dpsi_vs_red_black_fp64": float(np.max(np.abs(cols.state() - states["red_black_fp64"])))}
        cols.close()
    except R.RichardsError as e:
        out["columns_mixed_float_float_outer"] = {"error": str(e)}
    return out, states


def celia_cpu(states):
    """The oracle on the whole column run, both orderings (single thread),
    and the distance of the GPU states."""
    import numpy as np
    from oracle.oracle import Oracle
    from paper_2606_04292_gb300 import workloads as W
    res = {"cores": 1}
    for label, ordering in (("red_black_fp64", 1), ("lexicographic_fp64", 0)):
        o = Oracle(W.celia_1d(ordering=ordering))
        t0 = time.perf_counter()
        for _ in range(o.prob["nsteps"]):
            o.step()
        res[label + "_total_s"] = time.perf_counter() - t0
        res[label + "_max_abs_dpsi"] = float(np.max(np.abs(states[label] - o.state())))
    return res


STRIP_CPU_STEPS = 2


def strip_bench(stream, nsteps=100):
    """The 2-d infiltration workload in full (513^2 over 1 m^2, van Genuchten,
    Dirichlet strip on the top, BDF2 dt = 60 s for 100 steps, K lagged at
    psi^n): FP64 plain and the FP64-outer mixed mode, each with the
    configured V(2,2) cycles and with W(2,2) cycles on the three finest
    levels (V(2,2) stalls on about 15 steps of the run, where the wet bulb
    spreads along the no-flux surface beside the strip; the W-cycles converge
    every step); wall time, steps/s, cell-updates/s, steps that missed tol.
    Returns the summary and the states after STRIP_CPU_STEPS steps of the
    V(2,2) runs for the CPU leg."""
    import torch
    from paper_2606_04292_gb300 import richards as R
    from paper_2606_04292_gb300 import workloads as W
    out = {"workload": f"2D strip infiltration 513^2, VG, BDF2 (K lagged at psi^n) dt=60 s x {nsteps} steps, "
                       "V(2,2) as configured and W(2,2) on the 3 finest levels, tol 1e-8"}
    states = {}
    for label, prec, w in (("fp64_plain", 0, False), ("mixed_fp64_outer", 2, False),
                           ("fp64_plain_w", 0, True), ("mixed_fp64_outer_w", 2, True)):
        kw = dict(cycle_gamma=2, gamma_levels=3) if w else {}
        prob = W.strip_2d(n=513, nsteps=nsteps, precision=prec, **kw)
        gs = R.Solver(prob, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cyc, worst, upd, failed = 0, 0, 0, 0
        for k in range(nsteps):
            st, info = gs.step(check=False)
            cyc += info["cycles"]
            upd += info["cell_updates"]
            worst = max(worst, st)
            failed += st != 0
            if k + 1 == STRIP_CPU_STEPS and not w:
                states[label] = gs.state()
        torch.cuda.synchronize()
        tt = time.perf_counter() - t0
        out[label] = {"total_s": tt, "steps": nsteps, "time_steps_per_s": nsteps / tt,
                      "cell_updates_per_s": upd / tt, "cycles_per_step": cyc / nsteps,
                      "steps_missing_tol": failed, "worst_status": R.STATUS_NAMES[worst]}
        gs.close()
    return out, states


def strip_cpu(states):
    """The oracle on the first STRIP_CPU_STEPS steps of the 513^2 strip
    (single thread): seconds per step, and the distance of the GPU states."""
    import numpy as np
    from oracle.oracle import Oracle
    from paper_2606_04292_gb300 import workloads as W
    o = Oracle(W.strip_2d(n=513))
    t0 = time.perf_counter()
    for _ in range(STRIP_CPU_STEPS):
        o.step()
    per = (time.perf_counter() - t0) / STRIP_CPU_STEPS
    return {"cores": 1, "s_per_step": per, "sample": f"first {STRIP_CPU_STEPS} steps",
            **{k + "_max_abs_dpsi": float(np.max(np.abs(v - o.state()))) for k, v in states.items()}}


LAYERED_STEPS = 100       # two-layer field, FP64 plain: 1 h at tau = 0.01 h
LAYERED_FULL_STEPS = 4200  # the paper's whole two-layer run: 1.75 days = 42 h at tau = 0.01 h
LAYERED_CPU_STEPS = 3


def layered_bench(stream):
    """The paper's layered workloads: Section 4.1's composite column (128
    cells, 36 steps of 10 s, FP64) and Section 4.2's two-layer field (256^2,
    tau = 0.01 h, FMG(10,10), kappa = 0.1): the paper's whole run (1.75
    days, LAYERED_FULL_STEPS steps) mixed, beside the paper's total CPU time
    of 2320 s (its hardware unstated), and LAYERED_STEPS steps FP64 plain;
    wall time of each run.  Returns the summary and
    the states the CPU leg compares with."""
    import torch
    from paper_2606_04292_gb300 import richards as R
    from paper_2606_04292_gb300 import workloads as W
    out = {"workload": f"composite column 128 x 36 steps; two-layer 256^2 x {LAYERED_FULL_STEPS} steps (mixed) "
                       f"and x {LAYERED_STEPS} steps (FP64 plain), tol 1e-8",
           "paper_two_layer_total_cpu_s": 2320.0}
    states = {}
    runs = [("composite_column_fp64", W.celia_composite_1d(), None),
            ("two_layer_fp64_plain", W.two_layer_2d(nsteps=LAYERED_STEPS, precision=0), LAYERED_CPU_STEPS),
            ("two_layer_mixed", W.two_layer_2d(nsteps=LAYERED_FULL_STEPS, precision=1), LAYERED_CPU_STEPS)]
    for label, prob, keep in runs:
        gs = R.Solver(prob, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cyc, worst = 0, 0
        for k in range(prob["nsteps"]):
            st, info = gs.step(check=False)
            cyc += info["cycles"]
            worst = max(worst, st)
            if keep is not None and k + 1 == keep:
                states[label] = gs.state()
        torch.cuda.synchronize()
        out[label] = {"total_s": time.perf_counter() - t0, "steps": prob["nsteps"],
                      "worst_status": R.STATUS_NAMES[worst], "cycles_per_step": cyc / prob["nsteps"]}
        if keep is None:
            states[label] = gs.state()
        gs.close()
    return out, states


def layered_cpu(states):
    """The oracle on the composite column (whole run) and on the first
    LAYERED_CPU_STEPS steps of the two-layer field (single thread, seconds
    per step), with the distance of the GPU states at the same points."""
    import numpy as np
    from oracle.oracle import Oracle
    from paper_2606_04292_gb300 import workloads as W
    res = {"cores": 1}
    o = Oracle(W.celia_composite_1d())
    t0 = time.perf_counter()
    for _ in range(o.prob["nsteps"]):
        o.step()
    res["composite_column_total_s"] = time.perf_counter() - t0
    res["composite_column_max_abs_dpsi"] = float(np.max(np.abs(states["composite_column_fp64"] - o.state())))
    o = Oracle(W.two_layer_2d())
    t0 = time.perf_counter()
    for _ in range(LAYERED_CPU_STEPS):
        o.step()
    res["two_layer_s_per_step"] = (time.perf_counter() - t0) / LAYERED_CPU_STEPS
    res["two_layer_sample"] = f"first {LAYERED_CPU_STEPS} steps"
    for k in ("two_layer_fp64_plain", "two_layer_mixed"):
        res[k + "_max_abs_dpsi"] = float(np.max(np.abs(states[k] - o.state())))
    return res


TABLE3_CPU_STEPS = 20


def table3_cpu():
    """The oracle on the first TABLE3_CPU_STEPS steps of Table 3's column
    (single thread, red-black V(5,5)): seconds per step, and that rate over
    the whole run."""
    from oracle.oracle import Oracle
    from paper_2606_04292_gb300 import workloads as W
    o = Oracle(W.celia_1d(n=2048, dt=0.1, nu1=5, nu2=5, kappa=0.1))
    t0 = time.perf_counter()
    for _ in range(TABLE3_CPU_STEPS):
        o.step()
    per = (time.perf_counter() - t0) / TABLE3_CPU_STEPS
    return {"cores": 1, "s_per_step": per, "whole_run_at_that_rate_s": per * 3600,
            "sample": f"first {TABLE3_CPU_STEPS} steps"}


# ---------------------------------------------------------------------------
def host_info():
    """The host the CPU legs run on: logical core count and CPU model."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return {"host_cores": os.cpu_count(), "cpu_model": model or "unknown", "machine": platform.machine()}


def cpu_baseline(prob, psi, nsweeps_all=6, nsweeps_lex=2):
    """The CPU oracle, as it stands, on a bounded sample of the same workload
    at the given state of the 256^3 fine level: red-black NGS sweeps with each
    colour's cells shared among all host cores (OpenMP; the same updates as
    the serial sweep), and, beside it, the paper's single-threaded
    lexicographic sweep."""
    from oracle.oracle import Oracle
    o = Oracle(prob)
    o.set_state(psi)
    o.prepare(prob["dt"], 1)
    n = len(psi)
    cur = psi
    t0 = time.perf_counter()
    for _ in range(nsweeps_all):
        cur, used = o.sweep_threads(cur, 0)
    t_all = time.perf_counter() - t0
    cur = psi
    t0 = time.perf_counter()
    for _ in range(nsweeps_lex):
        cur = o.sweep(cur, ordering=0)
    t_lex = time.perf_counter() - t0
    k = prob["opts"]["newton_iters"]
    side = round(n ** (1 / 3))
    return dict({"value": nsweeps_all * n / t_all, "unit": UNIT, "cores": used, "kind": "oracle",
                 "sample": f"{nsweeps_all} red-black NGS sweeps (Newton k={k}) of the {side}^3 fine level at the "
                           f"benchmark state, C oracle with each colour's cells on {used} OpenMP threads, "
                           f"{t_all:.1f} s",
                 "single_thread_lexicographic": {
                     "value": nsweeps_lex * n / t_lex, "unit": UNIT, "cores": 1,
                     "sample": f"{nsweeps_lex} lexicographic NGS sweeps (the paper's order), same level and "
                               f"state, {t_lex:.1f} s"}}, **host_info())


def run_reference(args):
    """--impl reference: the CPU oracle timed on the host's cores, one
    fine-level red-black sweep of the same 256^3 workload per step (each
    colour's cells on all cores, OpenMP)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    from oracle.oracle import Oracle
    from paper_2606_04292_gb300 import workloads as W
    prob = W.drainage_3d(n=args.n, precision=args.precision)
    o = Oracle(prob)
    o.prepare(prob["dt"], 1)
    psi = np.array(prob["psi0"], dtype=np.float64)
    for _ in range(args.warmup):
        psi, used = o.sweep_threads(psi, 0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        psi, used = o.sweep_threads(psi, 0)
    dt = time.perf_counter() - t0
    n = len(psi)
    v = args.steps * n / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(args.precision),
                                            "sample": "one red-black NGS sweep of the fine level of the first "
                                                      "time step per step"},
            "cpu_baseline": dict({"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
                                  "sample": f"{args.steps} fine-level red-black NGS sweeps at {args.n}^3, "
                                            f"{used} OpenMP threads"}, **host_info()),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2606_04292_gb300 import replicas
    from paper_2606_04292_gb300 import richards as R
    from paper_2606_04292_gb300 import workloads as W

    prob = W.drainage_3d(n=args.n, cycle_gamma=args.gamma, precision=args.precision)
    N = W.ncells(prob)
    # a stream of its own: the inner cycles are captured into CUDA graphs,
    # which the legacy default stream does not allow
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    gs = R.Solver(prob, stream=stream.cuda_stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    infos = []
    for _ in range(args.warmup):
        st, info = gs.step()
    # launch shapes of the big FP32 grid levels, timed on this state (the
    # choice never changes the arithmetic)
    gs.prepare(prob["dt"], prob["scheme"])
    tuned = gs.autotune()
    barrier()
    # timed region: the context counts its launches on the host (no events)
    gs.profile(True, mode=3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        t_wall = time.perf_counter()
        e0.record(stream)
        for k in range(args.steps):
            st, info = gs.step(check=False)
            if st != R.RICH_OK:
                raise RuntimeError(f"step failed: {R.STATUS_NAMES[st]} {info}")
            infos.append(info)
        e1.record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall
    gs.profile(False)
    ms = e0.elapsed_time(e1)
    launches = sum(r["launches"] for r in gs.profile_read())
    # kernel durations: the next steps again, with CUDA events on the solver's
    # stream around every launch (the events lengthen a step, not a kernel)
    prof_steps = args.steps if args.profile_steps is None else args.profile_steps
    gs.profile(True, mode=1)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    p0.record(stream)
    for k in range(prof_steps):
        st, info = gs.step(check=False)
        if st != R.RICH_OK:
            raise RuntimeError(f"step failed: {R.STATUS_NAMES[st]} {info}")
    p1.record(stream)
    barrier()
    gs.profile(False)
    ms_prof = p0.elapsed_time(p1)
    prof = gs.profile_read()
    if args.profile_json and rank == 0:
        with open(args.profile_json, "w") as f:
            json.dump({"steps": prof_steps, "records": prof}, f, indent=1)
    updates = sum(i["cell_updates"] for i in infos)
    ms_max, updates_all = replicas.aggregate(ms, updates, device="cuda")
    value = replicas.throughput(ms_max, updates_all)
    steps_per_s = world * args.steps / (ms_max * 1e-3)

    # end to end through the C ABI: inputs from pinned host memory each step,
    # result read back each step
    e2e = None
    if not args.no_e2e:
        host_psi = torch.empty(N, dtype=torch.float64, pin_memory=True).numpy()
        host_prev = torch.empty(N, dtype=torch.float64, pin_memory=True).numpy()
        host_out = torch.empty(N, dtype=torch.float64, pin_memory=True).numpy()
        host_psi[:] = gs.state()
        host_prev[:] = host_psi
        ge = R.Solver(prob, stream=stream.cuda_stream)
        ge.set_state(host_psi, host_prev)
        ge.step()
        ge.prepare(prob["dt"], prob["scheme"])
        ge.autotune()
        barrier()
        ke = max(1, min(args.steps, 5))
        upd = cyc = 0
        t0 = time.perf_counter()
        for _ in range(ke):
            ge.set_state(host_psi, host_prev)
            st, info = ge.step(check=False)
            upd += info["cell_updates"]
            cyc += info["cycles"]
            lib = R.lib()
            R._check(lib.richards_get_state(ge.h, R._dp(host_out), 0), ge.h)
            host_prev, host_psi, host_out = host_psi, host_out, host_prev
        barrier()
        te = time.perf_counter() - t0
        e2e = {"value": upd / te * world, "unit": UNIT, "h2d_bytes_per_step": 16 * N, "d2h_bytes_per_step": 8 * N,
               "steps": ke, "time_steps_per_s": ke / te, "v_cycles_per_step": cyc / ke,
               "note": "each step hands psi^n (the last result) and psi^{n-1} in from pinned host memory and reads "
                       "psi back; a state equal bit for bit to the context's own keeps its FP64 theta cache"}
        ge.close()

    # the other outer layer on the same workload: float-float beside an FP64
    # headline (or FP64 beside a float-float one), device time of a few steps
    other = None
    if not args.no_other_outer and rank == 0:
        oprec = 1 if args.precision == 2 else 2
        go = R.Solver(W.with_opts(prob, precision=oprec), stream=stream.cuda_stream)
        for _ in range(args.warmup):
            go.step()
        go.prepare(prob["dt"], prob["scheme"])
        go.autotune()
        ko = max(1, min(args.steps, 5))
        oi = []
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        q0.record(stream)
        for _ in range(ko):
            st, info = go.step(check=False)
            oi.append(info)
        q1.record(stream)
        torch.cuda.synchronize()
        mo = q0.elapsed_time(q1)
        other = {"precision": oprec, "dtype": DTYPE[oprec], "steps": ko, "warmup": args.warmup,
                 "ms_per_step": mo / ko, "time_steps_per_s": ko / (mo * 1e-3),
                 "cell_updates_per_s": sum(i["cell_updates"] for i in oi) / (mo * 1e-3),
                 "v_cycles_per_step": statistics.mean(i["cycles"] for i in oi),
                 "outer_iters_per_step": statistics.mean(i["outer_iters"] for i in oi),
                 "status_last": R.STATUS_NAMES[st]}
        go.close()

    fp64 = None
    if not args.no_fp64 and rank == 0:
        # FP64 plain on the same workload from the same initial state; the
        # mixed result of the same number of steps is compared with it.
        nfp = 3
        gf = R.Solver(W.with_opts(prob, precision=0), stream=stream.cuda_stream)
        gm = R.Solver(prob, stream=stream.cuda_stream)
        gf.step()
        gm.step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        upd = 0
        for _ in range(nfp - 1):
            st, info = gf.step(check=False)
            upd += info["cell_updates"]
        torch.cuda.synchronize()
        tf = time.perf_counter() - t0
        t0 = time.perf_counter()
        for _ in range(nfp - 1):
            gm.step()
        torch.cuda.synchronize()
        tm = time.perf_counter() - t0
        a, b = gm.state(), gf.state()
        fp64 = {"time_steps_per_s": (nfp - 1) / tf, "cell_updates_per_s": upd / tf,
                "mixed_time_steps_per_s_same_steps": (nfp - 1) / tm,
                "mixed_speedup_in_steps_per_s": tf / tm,
                "mixed_vs_fp64_max_abs_dpsi_after_3_steps": float(np.max(np.abs(a - b))),
                "status_last": R.STATUS_NAMES[st]}
        gf.close()
        gm.close()

    # batched columns and served requests: every rank takes its share of the
    # units (no data-path collective; the summaries are gathered)
    columns = csample = None
    if not args.no_columns:
        columns, csample = columns_bench(stream, rank=rank, world=world)
    serving = None
    if not args.no_serving:
        serving = serving_bench(rank=rank, world=world)

    gardner = gstates = None
    if rank == 0 and not args.no_gardner:
        gardner, gstates = gardner_bench(stream)
    layered = lstates = None
    if rank == 0 and not args.no_layered:
        layered, lstates = layered_bench(stream)

    celia = cstates = None
    if rank == 0 and not args.no_celia:
        celia, cstates = celia_bench(stream)
    strip = sstates = None
    if rank == 0 and not args.no_strip:
        strip, sstates = strip_bench(stream)

    table3 = None
    if rank == 0 and not args.no_table3:
        from paper_2606_04292_gb300 import studies
        table3 = studies.table3_column()
        table3.pop("state")
        table3["paper_cpu_s_vcycle55"] = 20.0
        table3["workload"] = "Section 4.1 column, N=2048, tau 0.1 s to t=360 s (3600 BDF1 steps), V(5,5), tol 1e-8"

    temporal = None
    if rank == 0 and args.temporal_study:
        from paper_2606_04292_gb300 import studies
        t_study = time.perf_counter()
        temporal = studies.temporal_convergence()
        temporal["total_wall_s"] = time.perf_counter() - t_study

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(prob, gs.state())
        if gardner is not None:
            gardner["cpu_oracle"] = gardner_cpu(gstates)
        if layered is not None:
            layered["cpu_oracle"] = layered_cpu(lstates)
        if table3 is not None:
            table3["cpu_oracle"] = table3_cpu()
        if celia is not None:
            celia["cpu_oracle"] = celia_cpu(cstates)
        if strip is not None:
            strip["cpu_oracle"] = strip_cpu(sstates)
        if columns is not None:
            columns["cpu_oracle"] = columns_cpu(csample, columns["steps"])
        if serving is not None:
            serving["cpu_oracle"] = serving_cpu()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": workload_name(args.precision), "cells": N, "levels": gs.nlevels, "l2": "inputs larger than L2",
                       "launch_shapes": {f"level{l}": {"planes": t[0], "block_x": t[1], "resid_block_x": t[2]}
                                         for l, t in enumerate(tuned) if any(t)},
                       "cycle": f"{'W' if args.gamma == 2 else 'V'}({prob['opts']['nu1']},{prob['opts']['nu2']})",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "time_steps_per_s": steps_per_s,
            "v_cycles_per_step": statistics.mean(i["cycles"] for i in infos),
            "outer_iters_per_step": statistics.mean(i["outer_iters"] for i in infos),
            "resid_last": infos[-1]["resid"],
            "wall_s_timed": t_wall,
            "gpu_launches": launches,
            "roofline": roofline(prof, prof_steps, ms_prof) if prof else None,
            "clocks": clk.summary(),
            "e2e": e2e,
            "other_outer": other,
            "fp64_plain": fp64,
            "columns": columns,
            "serving": serving,
            "celia_column_c1": celia,
            "strip_513_c2": strip,
            "paper_gardner_2d": gardner,
            "paper_layered": layered,
            "paper_temporal_study": temporal,
            "paper_table3": table3,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    gs.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
