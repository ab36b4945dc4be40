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
