"""The multi-GPU path's host logic with two gloo ranks on the CPU.

Under torchrun every rank solves its own field and the ranks meet only to
time and count (no exchange step): the job's time is the slowest rank's and
its work the sum, and units of batched work split disjointly.  Here two
processes run those helpers over a gloo group (no GPU)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2606_04292_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 30.25][rank]                 # the slower rank sets the job's time
        updates = [1000, 3000][rank]
        ms_max, up = replicas.aggregate(ms, updates)
        units = replicas.shard(range(11), rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, units)
        out.put((rank, ms_max, up, replicas.throughput(ms_max, up), gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_by_the_slowest_and_count_all_work():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, up, thr, gathered in res:
        assert ms_max == 30.25 and up == 4000.0
        assert thr == pytest.approx(4000.0 / 30.25e-3)
        flat = sorted(u for part in gathered for u in part)
        assert flat == list(range(11))                       # disjoint and complete
        assert gathered[0] == [0, 2, 4, 6, 8, 10] and gathered[1] == [1, 3, 5, 7, 9]


def _units_main(rank, world, port, out):
    """Each rank takes its share of the batched-column and served-request
    units of the real workloads and reports what a sharded leg reports."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2606_04292_gb300 import workloads as W
        cols = W.columns(ncol=37, nmin=8, nmax=20)
        mine = replicas.shard(range(len(cols)), rank, world)
        cells = sum(cols[k]["n"][0] for k in mine)
        col_part = {"ids": mine, "ms": 10.0 + rank, "units": len(mine), "updates": cells * 3,
                    "unit_steps": len(mine) * 3}
        trace = W.serving_trace(rate=200.0, seconds=0.2, seed=6, sizes2d=(9,), sizes3d=(5,), max_requests=13)
        req = replicas.shard(range(len(trace)), rank, world)
        srv_part = {"ids": req, "ms": 5.0 * (rank + 1), "completed": len(req), "rejected": 0,
                    "latencies": [0.1 * (k + 1) for k in req]}
        out.put((rank, replicas.combine(replicas.gather(col_part)), replicas.combine(replicas.gather(srv_part)),
                 len(cols), sum(p["n"][0] for p in cols), len(trace)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_columns_and_requests():
    """Column and request ids split disjointly and completely over two ranks;
    per-rank counts sum to the whole workload's, the time is the slowest
    rank's, and the latency percentiles are over every request."""
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_units_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, col, srv, ncol, ncells, nreq in res:
        assert col["ids"] == list(range(ncol)) and col["ranks"] == 2
        assert col["units"] == ncol and col["updates"] == 3 * ncells and col["unit_steps"] == 3 * ncol
        assert col["ms"] == 11.0
        assert srv["ids"] == list(range(nreq)) and srv["completed"] == nreq and srv["ms"] == 10.0
        lat = sorted(0.1 * (k + 1) for k in range(nreq))
        assert srv["p50_latency_s"] == pytest.approx(float(np.percentile(lat, 50)))
        assert srv["p99_latency_s"] == pytest.approx(float(np.percentile(lat, 99)))
    assert res[0][1:] == res[1][1:]                 # every rank sees the same merged summary


def test_combine_rejects_overlapping_shards():
    with pytest.raises(ValueError):
        replicas.combine([{"ids": [0, 1], "ms": 1.0}, {"ids": [1, 2], "ms": 2.0}])


def test_single_process_aggregate_is_the_identity():
    assert replicas.aggregate(7.0, 42) == (7.0, 42.0)
    with pytest.raises(ValueError):
        replicas.shard(range(3), 2, 2)
