"""The split-line schedule (Algorithm 2 with even distribution of Stage B) on CPU ranks with the
gloo backend: every rank holds a slab of rows of every line, batches of lines go through Stage A,
the all-to-all to the ranks that own their Stage B, Stage B, the all-to-all back and Stage C. The
stages here are written from the oracle's Thomas in the paper's spike form (Algorithm 1), with a
dense Stage B, so that the test checks the schedule's bookkeeping (shares, record order, batches,
slots in flight) against the plain solve of the whole lines. No GPU involved."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O


class SpikeStages:
    """Stage A/B/C of one slab in the spike form, records of K = 6 and E = 2 doubles per line."""

    K, E, nrhs = 6, 2, 1
    device = torch.device("cpu")

    def __init__(self, n_local, n_lines, first, last):
        self.m, self.L, self.first, self.last = n_local, n_lines, first, last

    def scratch(self, count):
        return torch.zeros(3 * self.m * count, dtype=torch.float64)

    def work(self, W, count):
        return torch.zeros(1, dtype=torch.float64)

    def reduce(self, a, b, c, d, line0, count, red, scratch):
        sl = slice(line0, line0 + count)
        A, B, C, D = (t[:, sl].T.numpy().copy() for t in (a, b, c, d))  # [count][m]
        a_s, c_e = A[:, 0].copy(), C[:, -1].copy()
        A[:, 0] = 0.0
        C[:, -1] = 0.0
        xt = O.thomas(A, B, C, D)
        e0 = np.zeros_like(D)
        e0[:, 0] = 0.0 if self.first else a_s
        v = O.thomas(A, B, C, e0)
        e1 = np.zeros_like(D)
        e1[:, -1] = 0.0 if self.last else c_e
        w = O.thomas(A, B, C, e1)
        rec = np.stack([v[:, 0], w[:, 0], v[:, -1], w[:, -1], xt[:, 0], xt[:, -1]], axis=1)
        red[:count * 6] = torch.from_numpy(rec.reshape(-1))
        scratch[:3 * self.m * count] = torch.from_numpy(np.stack([xt, v, w]).reshape(-1))

    def pairs_solve(self, W, count, gathered, ends, work):
        g = gathered[:W * count * 6].numpy().reshape(W, count, 6)
        out = np.zeros((W, count, 2))
        for j in range(count):
            # unknowns: first(r) at 2r, last(r) at 2r + 1; each relation x_row + v x_last(r-1) +
            # w x_first(r+1) = xt_row (the spike form of the slab's end rows)
            Z = np.eye(2 * W)
            rhs = np.zeros(2 * W)
            for r in range(W):
                vf, wf, vl, wl, tf, tl = g[r, j]
                for row, (v, w, t) in ((2 * r, (vf, wf, tf)), (2 * r + 1, (vl, wl, tl))):
                    if r > 0:
                        Z[row, 2 * (r - 1) + 1] += v
                    if r < W - 1:
                        Z[row, 2 * (r + 1)] += w
                    rhs[row] = t
            y = np.linalg.solve(Z, rhs)
            for r in range(W):  # slab r's neighbour values: last of r-1, first of r+1
                out[r, j, 0] = y[2 * (r - 1) + 1] if r > 0 else 0.0
                out[r, j, 1] = y[2 * (r + 1)] if r < W - 1 else 0.0
        ends[:W * count * 2] = torch.from_numpy(out.reshape(-1))

    def finish(self, line0, count, ends, scratch, x):
        e = ends.numpy().reshape(count, 2)
        xt, v, w = scratch[:3 * self.m * count].numpy().reshape(3, count, self.m)
        sol = xt - v * e[:, :1] - w * e[:, 1:]
        x[:, line0:line0 + count] = torch.from_numpy(sol.T.copy())


class WideRecords(SpikeStages):
    """The same stages with two right-hand sides' worth of record size (K = 8, E = 4): the extra
    values are filler the stages write and check, so the schedule's record bookkeeping is tested
    for sizes other than the first."""

    K, E = 8, 4

    def reduce(self, a, b, c, d, line0, count, red, scratch):
        tmp = torch.zeros(count * 6, dtype=torch.float64)
        super().reduce(a, b, c, d, line0, count, tmp, scratch)
        rec = torch.cat([tmp.view(count, 6), torch.full((count, 2), 7.0, dtype=torch.float64)], dim=1)
        red[:count * 8] = rec.reshape(-1)

    def pairs_solve(self, W, count, gathered, ends, work):
        g = gathered[:W * count * 8].view(W, count, 8)
        assert bool((g[..., 6:] == 7.0).all())
        out = torch.zeros(W * count * 2, dtype=torch.float64)
        super().pairs_solve(W, count, g[..., :6].reshape(-1).clone(), out, work)
        e = torch.cat([out.view(W, count, 2), torch.full((W, count, 2), -3.0, dtype=torch.float64)], dim=2)
        ends[:W * count * 4] = e.reshape(-1)

    def finish(self, line0, count, ends, scratch, x):
        e = ends.view(count, 4)
        assert bool((e[:, 2:] == -3.0).all())
        super().finish(line0, count, e[:, :2].reshape(-1).clone(), scratch, x)


def _problem(n, L, seed=12):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1, 0, (n, L))
    c = rng.uniform(-1, 0, (n, L))
    b = 2 + np.abs(a) + np.abs(c) + rng.uniform(0, 1, (n, L))
    d = rng.uniform(-1, 1, (n, L))
    return a, b, c, d


def _rows(n, W, r):
    return n * r // W, n * (r + 1) // W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, L, batch, q, wide=False):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2509_03933_gb300.split_line import SplitLineSolver
        a, b, c, d = _problem(n, L)
        r0, r1 = _rows(n, world, rank)
        slab = [torch.from_numpy(t[r0:r1].copy()) for t in (a, b, c, d)]
        x = torch.zeros_like(slab[3])
        st = (WideRecords if wide else SpikeStages)(r1 - r0, L, rank == 0, rank == world - 1)
        SplitLineSolver(st, L, batch).solve(*slab, x)
        q.put((rank, r0, x.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n,L,batch,wide", [(2, 40, 50, 16, False), (3, 31, 37, 8, False),
                                                  (2, 8, 5, 64, False), (3, 12, 2, 1, False), (3, 20, 23, 5, True)])
def test_split_line_schedule_on_gloo_ranks(world, n, L, batch, wide):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, L, batch, q, wide)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    x = np.zeros((n, L))
    for rank, r0, xs in res:
        x[r0:r0 + xs.shape[0]] = xs
    a, b, c, d = _problem(n, L)
    ref = O.thomas(a.T, b.T, c.T, d.T).T
    assert O.rel_l2(x, ref) <= 1e-12


def test_even_shares_cover_every_line_once():
    from paper_2509_03933_gb300.split_line import shares
    for count in (0, 1, 5, 64, 1000):
        for W in (1, 2, 3, 8):
            sh = shares(count, W)
            assert sh[0][0] == 0 and sh[-1][1] == count
            assert all(sh[i][1] == sh[i + 1][0] for i in range(W - 1))
            assert max(h - l for l, h in sh) - min(h - l for l, h in sh) <= 1


def test_pipeline_model():
    from paper_2509_03933_gb300.split_line import pipeline_time, choose_batch
    # no exchange cost: the compute stream runs every A and C back to back
    assert pipeline_time(4, 1.0, 0.0, 1.0) == 8.0
    # exchange-bound: one A, then the exchanges back to back, then one C
    assert pipeline_time(3, 1.0, 5.0, 1.0) == 17.0
    # one batch: nothing overlaps
    assert pipeline_time(1, 2.0, 3.0, 4.0) == 9.0
    assert pipeline_time(0, 1.0, 1.0, 1.0) == 0.0
    # balanced stages: A_{k+1} and C_{k-1} hide X_k
    assert pipeline_time(5, 1.0, 2.0, 1.0) == 1.0 + 5 * 2.0 + 1.0
    # the estimator weighs per-batch costs that do not shrink with the batch (launch latency,
    # exchange latency) against the tail of an underfilled pipeline
    L = 1024
    times = {b: (0.02 + b * 1e-3, 0.05 + b * 4e-4, 0.01 + b * 5e-4) for b in (16, 64, 256, 1024)}
    best, est = choose_batch(L, times)
    assert best == min(est, key=est.get)
    assert est[1024] == pytest.approx(sum(times[1024]))  # one batch: the plain sum
    assert best != 1024 and best != 16
