"""The multi-GPU path's host logic with two gloo ranks on the CPU.

Under torchrun every rank solves its own field and the ranks meet only to
time and count (no exchange step): the job's time is the slowest rank's and
its work the sum, and units of batched work split disjointly.  Here two
processes run those helpers over a gloo group (no GPU)."""
import os
import socket

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


def test_single_process_aggregate_is_the_identity():
    assert replicas.aggregate(7.0, 42) == (7.0, 42.0)
    with pytest.raises(ValueError):
        replicas.shard(range(3), 2, 2)
