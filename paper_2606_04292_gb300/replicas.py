"""Runs on several GPUs of one node, one process per GPU.

The solver path has no exchange step at these sizes: every rank solves its
own field (weak scaling), and batched columns or served requests split by
unit.  Ranks therefore meet only to time and count: the job's time is the
slowest rank's, its work the sum over ranks.  These helpers take any
``torch.distributed`` process group (NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations


def shard(units, rank, world):
    """The units (columns, requests) rank ``rank`` of ``world`` takes: every
    world-th one, starting at its rank; disjoint across ranks, covering all."""
    if not 0 <= rank < world:
        raise ValueError("rank outside the world")
    return list(units)[rank::world]


def aggregate(ms, updates, device="cpu", group=None):
    """(max over ranks of ms, sum over ranks of updates); without an
    initialised process group, the inputs themselves."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return t.item(), u.item()


def throughput(ms_max, updates_all):
    """Whole-job units per second: all ranks' work over the slowest rank's time."""
    return updates_all / (ms_max * 1e-3)


def gather(obj, group=None):
    """Every rank's ``obj`` in rank order (a picklable summary); without an
    initialised process group, ``[obj]``."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        out = [None] * dist.get_world_size(group)
        dist.all_gather_object(out, obj, group=group)
        return out
    return [obj]


def percentile(xs, q):
    """The q-th percentile (0..100) of xs by linear interpolation; nan if empty."""
    import numpy as np
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else float("nan")


def combine(parts):
    """Merge the per-rank summaries of a sharded leg.  Each part holds ``ids``
    (the units the rank took) and ``ms`` (its device or wall time), and may
    hold counters (``units``, ``updates``, ``completed``, ``rejected``,
    ``unit_steps``) and a list of per-unit ``latencies``.  The job's time is
    the slowest rank's, its counters the sums; the ids must be disjoint."""
    ids = [i for p in parts for i in p["ids"]]
    if len(ids) != len(set(ids)):
        raise ValueError("a unit was taken by two ranks")
    out = {"ids": sorted(ids), "ranks": len(parts), "ms": max(p["ms"] for p in parts)}
    for key in ("units", "updates", "completed", "rejected", "unit_steps"):
        if any(key in p for p in parts):
            out[key] = sum(p.get(key, 0) for p in parts)
    if any("latencies" in p for p in parts):
        lat = [x for p in parts for x in p.get("latencies", [])]
        out["latencies"] = lat
        out["p50_latency_s"] = percentile(lat, 50)
        out["p99_latency_s"] = percentile(lat, 99)
    return out
