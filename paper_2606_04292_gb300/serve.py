"""Continuous-batching request loop for Richards solves on one GPU.

Requests (problem dicts with an ``arrival`` time in seconds) are admitted in
arrival order as soon as a slot is free and their device memory fits the
budget (``richards_device_bytes``).  Each admitted request gets its own
context on its own CUDA stream and keeps its state resident on the device for
all of its time steps.  Two ways to run them: continuous batching
(``batched=True``, ``richards_batcher_advance``: the inner cycles of all
resident requests run as shared launches over a device table of their
levels), or a native worker thread per request (``richards_batch_submit``)
whose kernels overlap with the others' on the device.  Finished requests
free their slot and memory at once, so later arrivals are admitted while
others are still running.  Latency = completion time minus arrival time.
"""
from __future__ import annotations

import collections
import ctypes as C
import time

import numpy as np

from . import richards as R


def request_bytes(prob, opts=None):
    o = dict(prob["opts"])
    if opts:
        o.update(opts)
    grid = R.richards_grid(prob["dim"], (C.c_int * 3)(*prob["n"]), (C.c_double * 3)(*prob["L"]))
    s = prob["soil"]
    fields = int(any(s.get(k) is not None for k in ("Ks_field", "p1_field", "p2_field")))
    return int(R.lib().richards_device_bytes(C.byref(grid), C.byref(R.make_opts(o)), fields,
                                             int(prob["sink"]["enabled"])))


class Server:
    """batched=False: every admitted request runs on its own stream and host
    worker thread (richards_batch_submit), their kernels overlapping on the
    device.  batched=True: continuous batching through
    richards_batcher_advance -- every admitted request advances on its own
    schedule (preparation, outer defects, inner cycles, end of step), the
    FP32 inner cycles of all requests in an inner solve run as shared
    launches, and a call returns when a request has done all its steps (or,
    while more requests may be admitted, after admit_ticks ticks); requests
    are admitted and retired between calls (every request in a mixed mode
    with the same cycle options)."""

    def __init__(self, budget_bytes=None, max_active=16, keep_states=False, opts=None, poll_s=2e-4,
                 batched=False, admit_ticks=8):
        import torch
        self.torch = torch
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            budget_bytes = int(0.8 * free)
        self.budget = int(budget_bytes)
        self.max_active = int(max_active)
        self.keep_states = keep_states
        self.opts = opts
        self.poll_s = poll_s
        self.batched = batched
        self.admit_ticks = int(admit_ticks)

    def run(self, requests, realtime=True):
        """Serve ``requests``; returns (results, summary)."""
        if self.batched:
            return self._run_batched(requests, realtime)
        lib = R.lib()
        reqs = sorted(enumerate(requests), key=lambda kv: kv[1].get("arrival", 0.0))
        pending = collections.deque(reqs)
        waiting = collections.deque()
        active = {}
        results = {}
        used = 0
        t0 = time.perf_counter()
        while pending or waiting or active:
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0][1].get("arrival", 0.0) <= now):
                waiting.append(pending.popleft())
            # admission: arrival order, slot and memory permitting
            while waiting and len(active) < self.max_active:
                rid, prob = waiting[0]
                need = request_bytes(prob, self.opts)
                if need > self.budget:
                    waiting.popleft()
                    results[rid] = dict(id=rid, status="rejected", bytes=need)
                    continue
                if used + need > self.budget:
                    break
                waiting.popleft()
                stream = self.torch.cuda.Stream()
                solver = R.Solver(prob, stream=stream.cuda_stream, opts=self.opts)
                h = (C.c_void_p * 1)(solver.h.value)
                st = lib.richards_batch_submit(h, 1, float(prob["dt"]), int(prob["nsteps"]), int(prob["scheme"]))
                if st != R.RICH_OK:
                    raise R.RichardsError(st, "richards_batch_submit failed")
                used += need
                arrival = prob.get("arrival", 0.0) if realtime else 0.0
                active[rid] = dict(solver=solver, stream=stream, handle=h, bytes=need, arrival=arrival,
                                   start=time.perf_counter() - t0, prob=prob)
            # completions
            for rid in list(active):
                a = active[rid]
                done = (C.c_int * 1)()
                status = (C.c_int * 1)()
                info = (R.richards_step_info * 1)()
                lib.richards_batch_poll(a["handle"], 1, done, status, info)
                if not done[0]:
                    continue
                end = time.perf_counter() - t0
                res = dict(id=rid, status=R.STATUS_NAMES[status[0]], arrival=a["arrival"], start=a["start"], end=end,
                           latency=end - a["arrival"], queue=a["start"] - a["arrival"], steps=a["prob"]["nsteps"],
                           cells=int(np.prod(a["prob"]["n"])), info=info[0].as_dict(), bytes=a["bytes"])
                if self.keep_states:
                    res["state"] = a["solver"].state()
                a["solver"].close()
                used -= a["bytes"]
                results[rid] = res
                del active[rid]
            if not (waiting and len(active) < self.max_active):
                time.sleep(self.poll_s)
        makespan = time.perf_counter() - t0
        done_ok = [r for r in results.values() if r.get("status") == "OK"]
        lat = np.array([r["latency"] for r in done_ok]) if done_ok else np.array([np.nan])
        summary = dict(requests=len(requests), completed=len(done_ok),
                       rejected=sum(1 for r in results.values() if r.get("status") == "rejected"),
                       makespan_s=makespan, solves_per_s=len(done_ok) / makespan,
                       cell_updates_per_s=sum(r["info"]["cell_updates"] for r in done_ok) / makespan,
                       p50_latency_s=float(np.percentile(lat, 50)), p99_latency_s=float(np.percentile(lat, 99)),
                       max_active=self.max_active, budget_bytes=self.budget)
        return [results[k] for k in sorted(results)], summary

    def _summary(self, requests, results, makespan):
        done_ok = [r for r in results.values() if r.get("status") == "OK"]
        lat = np.array([r["latency"] for r in done_ok]) if done_ok else np.array([np.nan])
        return dict(requests=len(requests), completed=len(done_ok),
                    rejected=sum(1 for r in results.values() if r.get("status") == "rejected"),
                    makespan_s=makespan, solves_per_s=len(done_ok) / makespan,
                    cell_updates_per_s=sum(r["info"]["cell_updates"] for r in done_ok) / makespan,
                    p50_latency_s=float(np.percentile(lat, 50)), p99_latency_s=float(np.percentile(lat, 99)),
                    max_active=self.max_active, budget_bytes=self.budget)

    def _run_batched(self, requests, realtime):
        reqs = sorted(enumerate(requests), key=lambda kv: kv[1].get("arrival", 0.0))
        pending = collections.deque(reqs)
        waiting = collections.deque()
        active = {}
        results = {}
        used = 0
        stream = self.torch.cuda.Stream()
        batcher = R.Batcher(max_contexts=self.max_active, stream=stream.cuda_stream)
        # each admitted request keeps a stream of its own for the work that is
        # its alone (preparation, outer defects, water balance), which then
        # overlaps between requests; the batched cycles run on `stream`
        free_streams = [self.torch.cuda.Stream() for _ in range(self.max_active)]
        t0 = time.perf_counter()
        try:
            while pending or waiting or active:
                now = time.perf_counter() - t0
                while pending and (not realtime or pending[0][1].get("arrival", 0.0) <= now):
                    waiting.append(pending.popleft())
                while waiting and len(active) < self.max_active:
                    rid, prob = waiting[0]
                    need = request_bytes(prob, self.opts)
                    if need > self.budget:
                        waiting.popleft()
                        results[rid] = dict(id=rid, status="rejected", bytes=need)
                        continue
                    if used + need > self.budget:
                        break
                    waiting.popleft()
                    own = free_streams.pop()
                    solver = R.Solver(prob, stream=own.cuda_stream, opts=self.opts)
                    used += need
                    arrival = prob.get("arrival", 0.0) if realtime else 0.0
                    active[rid] = dict(solver=solver, stream=own, bytes=need, arrival=arrival,
                                       start=time.perf_counter() - t0, prob=prob, done=0,
                                       acc=dict(cycles=0, outer_iters=0, cell_updates=0))
                if not active:
                    time.sleep(self.poll_s)
                    continue
                ids = list(active)
                # continuous batching: every request advances on its own
                # schedule until one of them is done (or, while requests may
                # still be admitted, for a few ticks)
                more = bool(pending or waiting)
                left, done, statuses, infos = batcher.advance(
                    [active[r]["solver"] for r in ids], [float(active[r]["prob"]["dt"]) for r in ids],
                    [int(active[r]["prob"]["scheme"]) for r in ids],
                    [active[r]["prob"]["nsteps"] - active[r]["done"] for r in ids],
                    max_ticks=self.admit_ticks if more else 0)
                end = time.perf_counter() - t0
                for rid, rest, d, st, info in zip(ids, left, done, statuses, infos):
                    a = active[rid]
                    if d == 0:
                        continue
                    a["done"] += d
                    for k in ("cycles", "outer_iters", "cell_updates"):
                        a["acc"][k] += info[k]
                    a["acc"]["resid"] = info["resid"]
                    if st != R.RICH_OK or rest == 0:
                        res = dict(id=rid, status=R.STATUS_NAMES[st], arrival=a["arrival"], start=a["start"],
                                   end=end, latency=end - a["arrival"], queue=a["start"] - a["arrival"],
                                   steps=a["done"], cells=int(np.prod(a["prob"]["n"])), info=dict(a["acc"]),
                                   bytes=a["bytes"])
                        if self.keep_states:
                            res["state"] = a["solver"].state()
                        a["solver"].close()
                        free_streams.append(a["stream"])
                        used -= a["bytes"]
                        results[rid] = res
                        del active[rid]
        finally:
            for a in active.values():
                a["solver"].close()
            batcher.close()
        makespan = time.perf_counter() - t0
        return [results[k] for k in sorted(results)], self._summary(requests, results, makespan)
