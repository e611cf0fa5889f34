"""The N > 1 path of bench.py on CPU with the gloo backend (world size 2): the ranks shard the lines
of one grid (lines along z; a rank takes whole y-rows), solve them with no collective on the data
path, and the job's time is the maximum over ranks. The sharded solve runs bench.py's own shard
and workload helpers with the oracle's Thomas standing in for the GPU kernel; the test checks that
every line of the global grid is solved by exactly one rank and that the assembled result equals
the unsharded solve of the same grid, for weak scaling (a taller grid, a fixed share per rank) and
strong scaling (one grid split). No GPU involved."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


N, NY = 16, 6  # small grid: n = 16 rows per line, 6 y-rows per rank (weak) or in all (strong)


def _lines(g):
    import synth
    return [synth.line_view(g[k].double(), 0).numpy() for k in ("a32", "b32", "c32", "d")]


def _worker(rank, world, port, scaling, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        y0, y1, ny_global = bench.rank_rows(NY, rank, world, scaling)
        g = bench.make_workload(N, "cpu", y1 - y0, y0, ny_global)
        x = oracle.thomas(*_lines(g))  # stands in for the kernel: the rank's own lines only
        ms = bench.reduce_max(10.0 + rank, torch.device("cpu"))  # rank 1 is slower
        parts = [None] * world
        dist.all_gather_object(parts, (y0, y1, x))
        q.put((rank, ms, parts, ny_global))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("scaling", ["weak", "strong"])
def test_gloo_two_ranks_shard_lines_of_one_grid(scaling):
    import bench
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, scaling, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, parts, ny_global in res:
        assert ms == 11.0  # the slowest rank's time
        assert ny_global == (2 * NY if scaling == "weak" else NY)
        rows = sorted(i for y0, y1, _ in parts for i in range(y0, y1))
        assert rows == list(range(ny_global))  # every y-row (n whole lines) solved exactly once
        got = np.concatenate([x for _, _, x in sorted(parts, key=lambda p: p[0])])
        full = bench.make_workload(N, "cpu", ny_global, 0, ny_global)
        assert got.shape == (N * ny_global, N)
        assert np.array_equal(got, oracle.thomas(*_lines(full)))


def test_single_process_helpers():
    import bench
    assert bench.reduce_max(3.5, torch.device("cpu")) == 3.5
    assert bench.shard_range(7, 0, 1) == (0, 7)
    assert [bench.shard_range(10, r, 3) for r in range(3)] == [(0, 3), (3, 6), (6, 10)]
    assert bench.rank_rows(1024, 0, 1, "weak") == (0, 1024, 1024)
    assert [bench.rank_rows(8, r, 2, "weak") for r in range(2)] == [(0, 8, 16), (8, 16, 16)]
    assert [bench.rank_rows(9, r, 2, "strong") for r in range(2)] == [(0, 4, 9), (4, 9, 9)]


def test_shard_draws_the_same_values_as_the_whole_grid():
    # a rank's block of a taller grid equals the same rows of that grid drawn whole
    import bench
    whole = bench.make_workload(N, "cpu", 2 * NY, 0, 2 * NY)
    part = bench.make_workload(N, "cpu", NY, NY, 2 * NY)
    for k in ("a32", "b32", "c32", "d"):
        assert torch.equal(part[k], whole[k][:, NY:, :])
