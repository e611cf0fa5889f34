"""The N > 1 path of bench.py on CPU with the gloo backend (world size 2): every rank solves its
own independent units, the job's time is the maximum over ranks, and shares cover all units
exactly once. No GPU involved."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.reduce_max(10.0 + rank, torch.device("cpu"))  # rank 1 is slower
        lo, hi = bench.shard_range(1000, rank, world)
        shares = [None] * world
        dist.all_gather_object(shares, (lo, hi))
        q.put((rank, ms, shares))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_max_time_and_shards():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, shares in res:
        assert ms == 11.0
        covered = sorted(i for lo, hi in shares for i in range(lo, hi))
        assert covered == list(range(1000))


def test_single_process_helpers():
    import bench
    assert bench.reduce_max(3.5, torch.device("cpu")) == 3.5
    assert bench.shard_range(7, 0, 1) == (0, 7)
    assert [bench.shard_range(10, r, 3) for r in range(3)] == [(0, 3), (3, 6), (6, 10)]
