#!/usr/bin/env python
"""Throughput of the batched tridiagonal solve on one GB300 per rank.

Workload: the general-coefficient 1024^3 grid (a, c ~ U(-1, 0), b = 2 + |a| + |c| + U(0, 1),
x_true ~ U(-1, 1), d = A x_true, seed 3), coefficients representable in FP32, 2^20 lines of
n = 1024 along the strided z axis. One step solves the whole grid with FP32 storage and sweeps
plus on-chip refinement (the headline ``value``); the plain FP64 solve of the same problem is
measured the same way and reported beside it. Inputs (30 GB) are far larger than L2 (129 MB),
so no flush is needed between steps.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0). Under torchrun the ranks shard the lines of one grid (lines are
independent: no collective on the data path): with ``--scaling weak`` (default) the grid has
N x 1024 y-rows and rank r solves y-rows [r 1024, (r + 1) 1024), so per-GPU work is fixed; with
``--scaling strong`` the 1024^3 grid's y-rows are split evenly. ``value`` is the unknowns of all
ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "unknowns solved/s (FP32 storage + refinement to 1e-12, vs FP64)"
UNIT = "unknowns/s"
SEED = 3
BYTES_F32R = 28.0   # a, b, c float (12) + d double (8) in, x double (8) out
BYTES_F64 = 40.0    # a, b, c, d double in, x double out
FP64_OPS_NOMINAL = 152 * 2 * 2.07e9  # FP64 pipe, nominal: 152 SMs x 2 ops/clk x 2.07 GHz (1.25 TFLOP/s)
KERNEL_OF_VARIANT = {0: "dc_kernel", 1: "thomas_kernel", 2: "refine_kernel", 3: "ragged_refine_kernel",
                     4: "refine_reg_kernel", 5: "refine_tma_fixed_kernel", 6: "refine_cluster_kernel",
                     7: "dc_kernel", 8: "refine_tree_kernel", 9: "packed_refine_kernel",
                     10: "shared_stream_kernel", 11: "refine_tree_kernel"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard_range(n_units: int, rank: int, world: int):
    """Contiguous share [lo, hi) of n_units independent units (lines, or whole grids) for a rank."""
    return n_units * rank // world, n_units * (rank + 1) // world


def reduce_max(value: float, device) -> float:
    """Maximum of a per-rank value over all ranks (any torch.distributed backend); the value itself
    when not distributed."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def traffic_record(kernel: str):
    """DRAM bytes per launch from a committed ncu summary, valid only while the kernel's own sources
    (its header and everything it includes) are unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        j = json.load(f)
    rec = j.get(kernel)
    if not rec or rec.get("source_sha") != source_sha(kernel):
        return None
    return rec


KERNEL_SOURCE = {"dc_kernel": "kernels_dc.cuh", "thomas_kernel": "kernels_thomas.cuh",
                 "refine_kernel": "kernels_refine.cuh", "ragged_refine_kernel": "kernels_ragged.cuh",
                 "refine_reg_kernel": "kernels_refine_reg.cuh", "refine_tma_fixed_kernel": "kernels_refine_tma.cuh",
                 "refine_cluster_kernel": "kernels_refine_cluster.cuh", "refine_tree_kernel": "kernels_refine_tree.cuh",
                 "packed_refine_kernel": "kernels_packed.cuh", "shared_stream_kernel": "kernels_shared.cuh"}


def source_sha(kernel: str) -> str:
    """Hash of the header that defines ``kernel`` and of the headers it includes, recursively."""
    dirs = [os.path.join(ROOT, "paper_2509_03933_gb300", "csrc"), os.path.join(ROOT, "include")]
    todo, seen = [KERNEL_SOURCE.get(kernel, "kernels_refine.cuh")], []
    while todo:
        name = todo.pop()
        if name in seen:
            continue
        path = next((os.path.join(d, name) for d in dirs if os.path.exists(os.path.join(d, name))), None)
        if path is None:
            continue
        seen.append(name)
        with open(path) as fh:
            todo += re.findall(r'^#include "([^"]+)"', fh.read(), flags=re.M)
    h = hashlib.sha256()
    for name in sorted(seen):
        path = next(os.path.join(d, name) for d in dirs if os.path.exists(os.path.join(d, name)))
        with open(path, "rb") as fh:
            h.update(name.encode() + fh.read())
    return h.hexdigest()[:16]


def pipe_batches(tune) -> int:
    return int(tune["choice"][0])


def rank_rows(ny: int, rank: int, world: int, scaling: str):
    """(y0, y1, ny_global): the y-rows [y0, y1) of the global grid that ``rank`` solves.

    Lines run along z, so a y-row is n whole lines and ranks never share a line. ``weak``: the
    global grid has world * ny y-rows, ny per rank (per-GPU work fixed as the world grows);
    ``strong``: the global grid has ny y-rows, split by shard_range."""
    if scaling == "weak":
        return rank * ny, (rank + 1) * ny, world * ny
    y0, y1 = shard_range(ny, rank, world)
    return y0, y1, ny


def make_workload(n: int, device, ny=None, y0: int = 0, ny_global=None):
    """Y-rows [y0, y0 + ny) of the general grid with n x max(n, ny_global) x n points (lines along z).
    The default is the whole n^3 grid; fewer rows give the same lines of it (profiling runs); a
    global grid taller than n (weak scaling over ranks) is one larger grid, each rank drawing its
    own block of it."""
    import synth
    ny = n if ny is None else ny
    full_ny = max(n, ny_global or 0)
    g = synth.grid_general((n, ny, n), 0, SEED, device=device, fp32_coefficients=True, full_shape=(n, full_ny, n),
                           origin=(0, y0, 0))
    g.pop("x_true")
    return g


def fp64_peak(device, sampler=None):
    """Measured FP64 FMA throughput of this GPU (the library's probe kernel: 8 independent FMA chains
    per thread, 8 blocks of 256 threads per SM), best of 5 launches timed with CUDA events after 3
    warm-up launches; with ``sampler`` running, the median SM clock gives FMAs per clock per SM."""
    import paper_2509_03933_gb300 as tdma
    props = torch.cuda.get_device_properties(device)
    sms = props.multi_processor_count
    blocks = sms * 8
    out = torch.empty(blocks, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)
    for _ in range(3):
        tdma.probe_fp64_fma(blocks, 256, 1 << 13, out, stream)
    times = []
    count = 0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        count = tdma.probe_fp64_fma(blocks, 256, 1 << 14, out, stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
    rate = count / min(times)
    res = {"fma_per_s": rate, "sms": sms, "launch_s": min(times), "fmas_per_launch": count,
           "nominal_fma_per_s": FP64_OPS_NOMINAL, "how": "tdma_probe_fp64_fma: 8 blocks x 256 threads per SM, "
           "8 independent FMA chains per thread, best of 5 (CUDA events)"}
    if sampler is not None:
        clk = sampler.summary()
        if clk.get("sm_mhz"):
            res["sm_mhz"] = clk["sm_mhz"]
            res["fma_per_clock_per_sm"] = rate / (sms * clk["sm_mhz"] * 1e6)
    return res


def cpu_oracle_baseline(n: int, ys: int, device_grid, reps_all: int = 3):
    """The C oracle (FP64 Thomas, oracle/thomas_c.c) timed on the host: one thread, then all the
    threads OpenMP gives it, on the first ``ys`` y-rows of the grid (ys n lines of n, copied to the
    host in the grid's [z][y][x] layout: lines adjacent, rows ys n apart). Returns (baseline dict,
    its solution as a [lines, n] array)."""
    from oracle import c_thomas
    host = [device_grid[k][:, :ys, :].double().cpu().numpy() for k in ("a32", "b32", "c32", "d")]
    x = np.empty_like(host[3])
    lines = ys * n
    args = (n, lines, lines, 1, *host, x)
    t0 = time.perf_counter()
    c_thomas.solve_strided(*args, threads=1)
    t1 = time.perf_counter() - t0
    threads = c_thomas.max_threads()
    best = float("inf")
    for _ in range(reps_all):
        t0 = time.perf_counter()
        c_thomas.solve_strided(*args, threads=threads)
        best = min(best, time.perf_counter() - t0)
    units = lines * n
    base = {"value": units / best, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{lines} lines x {n} (first {ys} y-rows of the grid, z axis), C FP64 Thomas "
                      f"(oracle/thomas_c.c, OpenMP over blocks of 8 adjacent lines), best of {reps_all}",
            "single_core_value": units / t1, "os_cpu_count": os.cpu_count(), "cpu_model": c_thomas.cpu_model()}
    return base, np.moveaxis(x, 0, -1).reshape(lines, n)


def sample_oracle_lines(g, ys: int):
    """Lines of the first ``ys`` y-rows (all x, full z) of the workload, as oracle inputs."""
    import synth
    sl = lambda t: synth.line_view(t[:, :ys, :].double().cpu(), 0).numpy()
    return sl(g["a32"]), sl(g["b32"]), sl(g["c32"]), sl(g["d"])


def synth_lines_check(hx, ys: int, nl: int, ref) -> float:
    """Relative L2 error of the first ``nl`` lines of the first ``ys`` y-rows of a host solution."""
    import oracle
    import synth
    return oracle.rel_l2(synth.line_view(hx[:, :ys, :], 0).numpy()[:nl], ref)


def time_steps(fn, steps, warmup, stream):
    """Device time of ``steps`` calls after ``warmup`` calls; per-launch events on ``stream``."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for s, e in ev:
        s.record(stream)
        fn()
        e.record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    total = t0.elapsed_time(t1)
    per = [s.elapsed_time(e) for s, e in ev]
    return total, per


# ---------------------------------------------------------------------------------------------
# the other workloads (reported under "suite"); each: throughput, plan, error on sampled lines

def _flush_l2(buf):
    buf.add_(1.0)  # a write larger than L2 between timed launches of small workloads


def _timed(fn, steps, warmup, stream, flush=None):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for s0, s1 in ev:
        if flush is not None:
            flush()
        s0.record(stream)
        fn()
        s1.record(stream)
    torch.cuda.synchronize()
    per = sorted(a.elapsed_time(b) for a, b in ev)
    return per[len(per) // 2]


def suite_small_grid(stream, hbm_peak, flush):
    """64^3 grid, 4096 lines of n = 64 along z, FP64, one partition (Thomas) and four."""
    import oracle
    import synth
    import paper_2509_03933_gb300 as tdma
    g = synth.grid_general((64, 64, 64), 0, 0, device="cuda")
    a, b, c, d = g["a"], g["b"], g["c"], g["d"]
    # CPU-baseline leg: the oracle on all 4096 lines (timed), its output also the reference
    inp = [synth.line_view(t.cpu(), 0).numpy() for t in (a, b, c, d)]
    t0 = time.perf_counter()
    ref = oracle.thomas(*inp)
    dt = time.perf_counter() - t0
    out = {"cpu_baseline": {"value": 64 ** 3 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": "all 4096 lines"}}
    for P in (1, 4):
        plan = tdma.Plan(*tdma.line_layout(d, 0), partitions=P)
        x = torch.empty_like(d)
        ms = _timed(lambda: plan.solve(a, b, c, d, x), 50, 5, stream, flush)
        err = oracle.rel_l2(synth.line_view(x.cpu(), 0).numpy(), ref)
        U = 64 ** 3
        out[f"P{P}"] = {"us_per_solve": ms * 1e3, "unknowns_per_s": U / (ms * 1e-3),
                        "hbm_frac": BYTES_F64 * U / (ms * 1e-3) / 1e9 / hbm_peak, "rel_l2_error": err,
                        "plan": plan.config, "l2": "flushed between launches"}
    return out


def suite_adi(stream, hbm_peak, fp64_probe=None, n=512):
    """512^3 ADI viscous sweeps x -> y -> z, one CUDA graph per step: per-element coefficients
    with 8 partitions per line, and the same operator as 1D coefficients shared by all lines
    (one factorisation per sweep, per-line right-hand-side recurrences)."""
    import oracle
    import synth
    import paper_2509_03933_gb300 as tdma
    from scipy.fft import dstn, idstn
    r = 0.5
    g = synth.grid_adi((n, n, n), seed=1, r=r, device="cuda")
    a, b, c, d = g["a"], g["b"], g["c"], g["d"]
    lam = 1 + 4 * r * np.sin(np.pi * np.arange(1, n + 1) / (2 * (n + 1))) ** 2
    L = lam[:, None, None] * lam[None, :, None] * lam[None, None, :]
    ref = idstn(dstn(d.cpu().numpy(), type=1, workers=-1) / L, type=1, workers=-1)
    U = 3 * n ** 3
    u = d.clone()
    out = {}
    # CPU-baseline leg: the oracle's Thomas (FP64) and PDD on a sample of z lines (timed)
    lines = synth.line_view(d[:, :8, :].cpu(), 0).numpy()  # 8 y-rows: 8 n lines of n
    A = np.full_like(lines, -r)
    B = np.full_like(lines, 1 + 2 * r)
    t0 = time.perf_counter()
    oracle.thomas(A, B, A, lines)
    dt = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.pdd(A, B, A, lines, 8)
    dt_pdd = time.perf_counter() - t0
    out["cpu_baseline"] = {"value": lines.size / dt, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                           "sample": f"{lines.shape[0]} z lines of n = {n} (Thomas, FP64)",
                           "pdd_P8_value": lines.size / dt_pdd}
    one = lambda v: torch.full((n,), v, dtype=torch.float64, device="cuda")
    legs = (("per_element_P8", (a, b, c), dict(partitions=8)),
            ("shared_coefficients", (one(-r), one(1 + 2 * r), one(-r)), dict(coef_broadcast=True)))
    for name, coef, kw in legs:
        plans = [tdma.Plan(*tdma.line_layout(u, ax), **kw) for ax in (2, 1, 0)]
        graph = tdma.sweep_graph([(p, coef + (u, u)) for p in plans])
        per_axis = {ax: _timed(lambda: p.solve(*coef, u, u), 10, 3, stream) for ax, p in zip("xyz", plans)}
        ms = _timed(graph.replay, 10, 3, stream)
        u.copy_(d)
        graph.replay()
        torch.cuda.synchronize()
        leg = {"ms_per_xyz_step": ms, "ms_per_sweep": per_axis, "unknowns_per_s": U / (ms * 1e-3),
               "hbm_frac": BYTES_F64 * U / (ms * 1e-3) / 1e9 / hbm_peak,
               "rel_l2_error_vs_closed_form": oracle.rel_l2(u.cpu().numpy(), ref),
               "plans": [p.config for p in plans]}
        if kw.get("coef_broadcast"):
            # d in, x out (16 B per unknown); 3 FP64-pipe operations per unknown
            leg["launches_per_step"] = 6
            leg["hbm_frac"] = 16.0 * U / (ms * 1e-3) / 1e9 / hbm_peak
            peak = fp64_probe["fma_per_s"] if fp64_probe else FP64_OPS_NOMINAL
            leg["fp64_pipe_frac"] = 3.0 * U / (ms * 1e-3) / peak
            leg["fp64_pipe_peak_kind"] = "measured (FP64 FMA probe)" if fp64_probe else "nominal"
            leg["bytes_per_unknown"] = 16.0
        else:
            leg["launches_per_step"] = 3
        out[name] = leg
        del graph, plans
    # the parallel diagonally dominant approximation against the exact reduced solve, per
    # partition count: time of an xyz step and error against the closed form
    sweep = {}
    for P in (8, 32, 64, 128):
        row = {}
        for tag, pdd in (("exact", False), ("pdd", True)):
            plans = [tdma.Plan(*tdma.line_layout(u, ax), partitions=P, pdd=pdd) for ax in (2, 1, 0)]
            graph = tdma.sweep_graph([(p, (a, b, c, u, u)) for p in plans])
            ms = _timed(graph.replay, 10, 3, stream)
            u.copy_(d)
            graph.replay()
            torch.cuda.synchronize()
            row[tag] = {"ms_per_xyz_step": ms, "rel_l2_error_vs_closed_form": oracle.rel_l2(u.cpu().numpy(), ref),
                        "variant": plans[0].config["variant"]}
            del graph, plans
        sweep[f"P{P}"] = row
    out["pdd_vs_exact_per_element"] = sweep
    return out


def suite_poisson(stream, hbm_peak):
    """1024^3 wavenumber lines along z: broadcast coefficients + per-line shift, complex RHS
    (2 interleaved real RHS), zero mode pinned and solved by its own one-line plan."""
    import oracle
    import synth
    import paper_2509_03933_gb300 as tdma
    n = 1024
    p = synth.poisson_lines(n, n, n, seed=2, device="cuda")
    d = p["d"]
    x = torch.empty_like(d)
    d3, x3 = d.view(n, n * n, 2), x.view(n, n * n, 2)
    shift = p["shift"][1:].contiguous()
    rng = np.random.default_rng(2)
    modes = np.unique(np.concatenate([[0, 1, n, n + 1, n * n - 1], rng.choice(n * n, 59, False)]))
    ha, hc, hb0, hs = (p[k].cpu().numpy() for k in ("a", "c", "b0", "shift"))
    # CPU-baseline leg: the extended-precision oracle on the sampled modes (timed)
    t0 = time.perf_counter()
    refs = []
    for m in modes:
        if m == 0:
            A, B, C = (p[k].cpu().numpy() for k in ("pin_a", "pin_b", "pin_c"))
        else:
            A, B, C = ha, hb0 + hs[m], hc
        refs.append(oracle.thomas_ext(A, B, C, d3[:, m, :].cpu().numpy()))
    refs = np.stack(refs)
    dt = time.perf_counter() - t0
    out = {"cpu_baseline": {"value": len(modes) * n / dt, "unit": "complex unknowns/s", "cores": 1,
                            "kind": "oracle (extended precision)", "sample": f"{len(modes)} modes x {n}"}}
    for prec in ("f64", "f64r"):
        main = tdma.Plan(*tdma.line_layout(d3[:, 1:, :], 0, nrhs=2), nrhs=2, coef_broadcast=True, diag_shift=shift,
                         precision=prec)
        zero = tdma.Plan(*tdma.line_layout(d3[:, :1, :], 0, nrhs=2), nrhs=2, coef_broadcast=True, precision=prec)

        def step():
            main.solve(p["a"], p["b0"], p["c"], d3[:, 1:, :], x3[:, 1:, :])
            zero.solve(p["pin_a"], p["pin_b"], p["pin_c"], d3[:, :1, :], x3[:, :1, :])
        ms = _timed(step, 8, 3, stream)
        got = np.stack([x3[:, m, :].cpu().numpy() for m in modes])
        U = n ** 3  # complex unknowns
        per_mode = np.linalg.norm((got - refs).reshape(len(modes), -1), axis=1) / \
            np.linalg.norm(refs.reshape(len(modes), -1), axis=1)
        out[prec] = {"ms_per_step": ms, "complex_unknowns_per_s": U / (ms * 1e-3),
                     "hbm_frac": 32.0 * U / (ms * 1e-3) / 1e9 / hbm_peak,
                     "rel_l2_error_vs_extended": oracle.rel_l2(got, refs), "worst_mode_error": float(per_mode.max()),
                     "modes_checked": int(len(modes)), "plan": main.config}
        if prec == "f64r":
            out[prec]["lines_corrected"] = main.corrected_lines() + zero.corrected_lines()
            out[prec]["lines"] = n * n
        del main, zero
    del p, d, x, d3, x3, shift
    torch.cuda.empty_cache()
    out["fft_pipeline"] = suite_poisson_fft(stream, n)
    return out


def suite_poisson_fft(stream, n=1024):
    """The whole FFT-based Poisson solve on an n^3 grid q[y][z][x] (periodic x, z; stretched y
    with Neumann ends): cuFFT over the (z, x) planes, the n (n/2 + 1) n wavenumber lines along y,
    cuFFT back, through tdma_poisson_solve. Error: the discrete equation on sampled y planes
    (normwise backward error; the pinned row excluded). The line solves alone are timed on a
    buffer of the spectrum's layout."""
    import synth
    import paper_2509_03933_gb300 as tdma
    import oracle
    a, c, b = synth.poisson_coefficients(n)
    dx = dz = 2 * np.pi / n
    q = synth.normal(7, synth.AID["d"], torch.arange(n ** 3, device="cuda")).reshape(n, n, n)
    phi = torch.empty_like(q)
    out = {}
    # CPU-baseline leg: the oracle's FFT-based solve (numpy FFTs + Thomas) on 32 y-rows' worth of
    # a 128 x 128 x n grid (timed), scaled to grid points per second
    ns = 128
    ac, cc, bc = synth.poisson_coefficients(32)
    qs = np.random.default_rng(7).standard_normal((32, ns, ns))
    t0 = time.perf_counter()
    oracle.poisson_fft(qs, 2 * np.pi / ns, 2 * np.pi / ns, ac, bc, cc)
    dt = time.perf_counter() - t0
    out["cpu_baseline"] = {"value": qs.size / dt, "unit": "grid points/s", "cores": 1, "kind": "oracle",
                           "sample": f"32 x {ns} x {ns} grid (numpy FFTs + Thomas)"}
    for prec in ("f64", "f64r"):
        solver = tdma.PoissonFFT(n, n, n, dx, dz, a, b, c, precision=prec)
        ms = _timed(lambda: solver.solve(q, out=phi, stream=stream), 5, 3, stream)
        solver.solve(q, out=phi, check=True)
        A, B, C = (torch.from_numpy(t).cuda() for t in (a, b, c))
        pmax = phi.abs().max().item()
        worst = 0.0
        for y in (0, 1, n // 2, n - 1):
            pl = phi[y]
            lap = (torch.roll(pl, -1, 1) - 2 * pl + torch.roll(pl, 1, 1)) / dx ** 2
            lap += (torch.roll(pl, -1, 0) - 2 * pl + torch.roll(pl, 1, 0)) / dz ** 2 + B[y] * pl
            if y > 0:
                lap += A[y] * phi[y - 1]
            if y < n - 1:
                lap += C[y] * phi[y + 1]
            r = lap - q[y]
            if y == 0:
                r = r - r.mean()
            scale = (4 / dx ** 2 + 4 / dz ** 2 + abs(a[y]) + abs(b[y]) + abs(c[y])) * pmax
            worst = max(worst, r.abs().max().item() / scale)
        out[prec] = {"ms_per_solve": ms, "grid_points_per_s": n ** 3 / (ms * 1e-3),
                     "backward_error_sampled_planes": worst, "workspace_GB": solver.workspace.numel() / 1e9}
        del solver
        torch.cuda.empty_cache()
    # the wavenumber lines alone, in the spectrum's layout [y][kz][kx] (lines 1 .. L-1)
    nkx = n // 2 + 1
    L = n * nkx
    spec = torch.zeros((n, L, 2), dtype=torch.float64, device="cuda")
    k2x = (2 - 2 * np.cos(2 * np.pi * np.arange(nkx) / n)) / dx ** 2
    k2z = (2 - 2 * np.cos(2 * np.pi * np.arange(n) / n)) / dz ** 2
    shift = torch.from_numpy(-(k2z[:, None] + k2x[None, :]).reshape(-1)[1:].copy()).cuda()
    plan = tdma.Plan(n, L - 1, elem_stride=L, inner_count=L - 1, inner_stride=1, nrhs=2, coef_broadcast=True,
                     diag_shift=shift)
    A, B, C = (torch.from_numpy(t).cuda() for t in (a, b, c))
    lines = spec[:, 1:, :]
    ms_lines = _timed(lambda: plan.solve(A, B, C, lines, lines, stream=stream), 5, 3, stream)
    out["lines_only"] = {"ms": ms_lines, "plan": plan.config, "complex_unknowns": n * (L - 1)}
    out["fft_share_f64"] = 1.0 - ms_lines / out["f64"]["ms_per_solve"]
    return out


def suite_x_axis(stream, hbm_peak, n=1024):
    """The precision workload along the unit-stride x axis: general FP32-representable coefficients
    on an n^3 grid (seed 3), lines along x, FP32 + refinement and FP64, errors against the oracle on
    the lines of the first four z-planes."""
    import oracle
    import synth
    import paper_2509_03933_gb300 as tdma
    g = synth.grid_general((n, n, n), 2, SEED, device="cuda", fp32_coefficients=True)
    g.pop("x_true")
    d = g["d"]
    x = torch.empty_like(d)
    U = n ** 3
    out = {}
    sample = lambda t: synth.line_view(t[:4].double().cpu(), 2).numpy()
    ref = oracle.thomas(*(sample(g[k]) for k in ("a32", "b32", "c32")), sample(d))
    for prec, keys, nbytes in (("f32r", ("a32", "b32", "c32"), BYTES_F32R), ("f64", ("a", "b", "c"), BYTES_F64)):
        plan = tdma.Plan(*tdma.line_layout(d, 2), precision=prec)
        coef = tuple(g[k] for k in keys)
        ms = _timed(lambda: plan.solve(*coef, d, x), 10, 3, stream)
        out[prec] = {"ms_per_solve": ms, "unknowns_per_s": U / (ms * 1e-3),
                     "hbm_frac": nbytes * U / (ms * 1e-3) / 1e9 / hbm_peak,
                     "rel_l2_error": oracle.rel_l2(sample(x), ref), "status": plan.last_error()[0],
                     "plan": plan.config}
        del plan
    out["l2"] = "inputs larger than L2"
    return out


def suite_split_line(stream, n=512):
    """The split-line stages and schedule on one rank (the multi-GPU exchange degenerates to a
    copy): n^3 FP64 lines along z, the paper's batch-size estimator against timing every candidate
    batch, and the fused one-partition Thomas kernel on the same problem."""
    import oracle
    import synth
    import paper_2509_03933_gb300 as tdma
    from paper_2509_03933_gb300.split_line import SlabStages, SplitLineSolver, choose_batch
    g = synth.grid_general((n, n, n), 0, 3, device="cuda")
    a, b, c, d = (g[k] for k in ("a", "b", "c", "d"))
    L = n * n
    x = torch.empty_like(d)
    st = SlabStages(n, L, (L, L, 1, 0))
    stage_times, measured = {}, {}
    for batch in (L, L // 2, L // 4, L // 8):
        sol = SplitLineSolver(st, L, batch)
        stage_times[batch] = sol.measure_stages(a, b, c, d, x)
        measured[batch] = _timed(lambda: sol.solve(a, b, c, d, x), 5, 3, stream)
        del sol
    best, est = choose_batch(L, stage_times)
    ref = oracle.thomas(*(synth.line_view(t[:, :1, :].cpu(), 0).numpy() for t in (a, b, c, d)))
    err = oracle.rel_l2(synth.line_view(x[:, :1, :].cpu(), 0).numpy(), ref)
    plan = tdma.Plan(*tdma.line_layout(d, 0), partitions=1)
    ms_thomas = _timed(lambda: plan.solve(a, b, c, d, x), 5, 3, stream)
    return {"ms_per_solve_by_batch": measured, "estimated_ms_by_batch": est, "stage_ms_by_batch": stage_times,
            "estimator_choice": best, "fastest_measured": min(measured, key=measured.get),
            "rel_l2_error_first_y_row": err, "fused_thomas_ms": ms_thomas, "ranks": 1}


def suite_ragged(stream, hbm_peak, n_lines=20000):
    """20000 lines, n log-uniform in [16, 16384], packed; FP32+refinement and FP64 in one
    persistent launch each; backward for loss = sum(w * x), w ~ N(0, 1)."""
    import oracle
    import synth
    import paper_2509_03933_gb300 as tdma
    lengths = synth.ragged_lengths(n_lines, 16, 16384, seed=4)
    r = synth.ragged_general(lengths, 4, device="cuda", fp32_coefficients=True)
    U = r["total"]
    rng = np.random.default_rng(4)
    lines = np.unique(np.concatenate([np.argsort(-lengths)[:10], rng.choice(n_lines, min(300, n_lines), replace=False)]))
    offs, lens = r["offsets"].cpu().numpy(), r["lengths"].cpu().numpy()
    ha, hb, hc, hd = (r[k].cpu().numpy() for k in ("a", "b", "c", "d"))
    # CPU-baseline leg: the oracle on the sampled lines (timed), its output also the reference
    t0 = time.perf_counter()
    ref = oracle.thomas_ragged(ha, hb, hc, hd, offs, lens, lines=lines)
    dt = time.perf_counter() - t0
    want = np.concatenate([ref[l] for l in sorted(ref)])
    w = synth.normal(4, synth.AID["w"], torch.arange(U, device="cuda"))
    out = {"lines": n_lines, "unknowns": int(U),
           "cpu_baseline": {"value": int(want.size) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{len(ref)} lines ({int(want.size)} unknowns), longest 10 + random"}}
    for prec, keys, fbytes, bbytes in (("f32r", ("a32", "b32", "c32"), BYTES_F32R, 8.0 * 3 + 4 * 3 + 8 * 2),
                                       ("f64", ("a", "b", "c"), BYTES_F64, 72.0)):
        a, b, c = (r[k] for k in keys)
        d = r["d"]
        x, plan = tdma.solve_ragged(a, b, c, d, r["offsets"], r["lengths"], precision=prec)
        default_cfg = plan.config
        ms_default = _timed(lambda: plan.solve(a, b, c, d, x), 10, 3, stream)
        tuned_cfg = plan.autotune(a, b, c, d, x)  # rows per partition (and chunk vs group kernel), timed
        ms = _timed(lambda: plan.solve(a, b, c, d, x), 10, 3, stream)
        st, iters = plan.last_error()
        xs = x.cpu().numpy()
        got = np.concatenate([xs[offs[l]:offs[l] + lens[l]] for l in sorted(ref)])
        ga, gb, gc, gd = (torch.empty_like(a), torch.empty_like(b), torch.empty_like(c), torch.empty_like(x))
        msb = _timed(lambda: plan.backward(a, b, c, x, w, ga, gb, gc, gd), 10, 3, stream)
        gdh, wh = gd.cpu().numpy(), w.cpu().numpy()
        l0 = sorted(ref)[:50]
        rg = [oracle.adjoint_grads(ha[o:o + n_], hb[o:o + n_], hc[o:o + n_], xs[o:o + n_], wh[o:o + n_])[3]
              for o, n_ in ((offs[l], lens[l]) for l in l0)]
        lam_err = oracle.rel_l2(np.concatenate([gdh[offs[l]:offs[l] + lens[l]] for l in l0]), np.concatenate(rg))
        out[prec] = {"forward_ms": ms, "unknowns_per_s": U / (ms * 1e-3),
                     "hbm_frac": fbytes * U / (ms * 1e-3) / 1e9 / hbm_peak, "rel_l2_error": oracle.rel_l2(got, want),
                     "status": st, "corrections_max": iters, "backward_ms": msb,
                     "backward_unknowns_per_s": U / (msb * 1e-3),
                     "backward_lambda_rel_l2_error": lam_err, "plan": plan.config,
                     "autotune": {"default_plan": default_cfg, "default_ms": ms_default, "tuned_plan": tuned_cfg,
                                  "tuned_ms": ms}}
    return out


def run_reference(args):
    """The oracle on the host's cores: the C FP64 Thomas (oracle/thomas_c.c, OpenMP over blocks of
    adjacent lines, all threads) on a bounded sample of the same workload per step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    from oracle import c_thomas
    n = args.n
    ys = max(1, args.ref_lines // n)
    g = synth.grid_general((n, ys, n), 0, SEED, fp32_coefficients=True, full_shape=(n, n, n), origin=(0, 0, 0))
    a, b, c, d = (g[k].double().numpy() for k in ("a32", "b32", "c32", "d"))  # [z][y][x]: lines adjacent
    x = np.empty_like(d)
    lines = ys * n
    threads = c_thomas.max_threads()
    step = lambda: c_thomas.solve_strided(n, lines, lines, 1, a, b, c, d, x, threads=threads)
    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t) / max(1, args.steps)
    units = lines * n
    value = units / dt
    sample = (f"{lines} lines x {n} (first {ys} y-rows of the {n}^3 grid, z axis) per step, C FP64 Thomas "
              f"(oracle/thomas_c.c), {threads} OpenMP threads")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"general-coefficient {n}^3 grid, lines along z, seed {SEED}, "
                                  "FP32-representable coefficients", "lines": n * n, "n": n},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                            "os_cpu_count": os.cpu_count(), "cpu_model": c_thomas.cpu_model()},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--ny", type=int, default=0, help="solve only the first ny y-rows (profiling runs)")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="N > 1: weak = ny y-rows per rank of a taller grid; strong = the grid's y-rows split")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--e2e-batches", type=int, default=0,
                    help="slices of lines in the pipelined host solve (0: chosen by HostPipeline.tuned)")
    ap.add_argument("--cpu-lines", type=int, default=32768, help="lines in the CPU oracle sample")
    ap.add_argument("--ref-lines", type=int, default=32768, help="lines per reference-arm step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-suite", action="store_true", help="skip the other workloads")
    ap.add_argument("--only-poisson-fft", type=int, default=0, metavar="N",
                    help="run only the FFT-based Poisson solve on an N^3 grid and print it (profiling runs)")
    ap.add_argument("--only-split-line", type=int, default=0, metavar="N",
                    help="run only the split-line stages on one rank on an N^3 grid and print them")
    ap.add_argument("--only-x-axis", type=int, default=0, metavar="N",
                    help="run only the x-axis precision workload on an N^3 grid and print it")
    ap.add_argument("--only-adi", type=int, default=0, metavar="N",
                    help="run only the ADI workload on an N^3 grid and print it (profiling runs)")
    ap.add_argument("--only-ragged", type=int, default=0, metavar="LINES",
                    help="run only the ragged workload with LINES lines (profiling runs) and print it")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.only_poisson_fft > 0:
        print(json.dumps({"poisson_fft": suite_poisson_fft(torch.cuda.current_stream(), args.only_poisson_fft)}),
              flush=True)
        return 0
    if args.only_split_line > 0:
        print(json.dumps({"split_line": suite_split_line(torch.cuda.current_stream(), args.only_split_line)}),
              flush=True)
        return 0
    if args.only_x_axis > 0:
        hbm_peak, _ = peaks()
        print(json.dumps({"x_axis": suite_x_axis(torch.cuda.current_stream(), hbm_peak, args.only_x_axis)}),
              flush=True)
        return 0
    if args.only_adi > 0:
        hbm_peak, _ = peaks()
        print(json.dumps({"adi": suite_adi(torch.cuda.current_stream(), hbm_peak, None, args.only_adi)}), flush=True)
        return 0
    if args.only_ragged > 0:
        hbm_peak, _ = peaks()
        print(json.dumps({"ragged": suite_ragged(torch.cuda.current_stream(), hbm_peak, args.only_ragged)}), flush=True)
        return 0

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    import paper_2509_03933_gb300 as tdma

    dev = torch.device("cuda", local if ws > 1 else 0)
    n = args.n
    ny_arg = args.ny if args.ny > 0 else n
    y0, y1, ny_global = rank_rows(ny_arg, rank, ws, args.scaling)
    ny = y1 - y0  # this rank's y-rows (its lines: ny n of n unknowns)
    U = n * ny * n
    U_all = n * ny_global * n  # every rank's lines, each solved by exactly one rank
    g = make_workload(n, dev, ny, y0, ny_global)
    a32, b32, c32, d = g["a32"], g["b32"], g["c32"], g["d"]
    x = torch.empty_like(d)
    stream = torch.cuda.current_stream()
    lay = tdma.line_layout(d, 0)
    plan_r = tdma.Plan(*lay, precision="f32r")
    plan_d = tdma.Plan(*lay, precision="f64")

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # ---------------- headline: FP32 storage + refinement
    barrier()
    with ClockSampler(local if ws > 1 else 0) as clk:
        total_r, per_r = time_steps(lambda: plan_r.solve(a32, b32, c32, d, x), args.steps, args.warmup, stream)
    barrier()
    st, iters = plan_r.last_error()
    ms_r = reduce_max(total_r / args.steps, dev)  # the slowest rank sets the job's time
    x_r = x.clone() if rank == 0 else None

    # ---------------- the plain FP64 solve of the same problem
    a, b, c = g["a"], g["b"], g["c"]
    k_d = max(3, args.steps // 3)
    barrier()
    total_d, per_d = time_steps(lambda: plan_d.solve(a, b, c, d, x), k_d, args.warmup, stream)
    barrier()
    st_d, _ = plan_d.last_error()
    ms_d = reduce_max(total_d / k_d, dev)
    x_d = x

    import synth
    import oracle
    hbm_peak, peak_kind = peaks()
    fp64_probe = roof = cpu = ref = None
    err = {}
    ys = min(ny, max(1, args.cpu_lines // n))
    if rank == 0:
        # the FP64 pipe's measured peak (the FP64 kernels' second roofline)
        with ClockSampler(local if ws > 1 else 0) as clk64:
            fp64_probe = fp64_peak(dev, clk64)
        kern_ms = sorted(per_r)[len(per_r) // 2]
        achieved = BYTES_F32R * U / (kern_ms * 1e-3) / 1e9
        kname = KERNEL_OF_VARIANT.get(plan_r.config["variant"], "refine_kernel")
        trec = traffic_record(kname)
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": (trec["dram_bytes"] * (U / trec["unknowns"])) if trec else None,
                "peak_kind": f"{peak_kind} (STREAM-style copy)", "algorithmic_bytes_per_unknown": BYTES_F32R,
                "kernel": kname, "kernel_ms": kern_ms}
        # ---------------- CPU oracle on a bounded sample (rank 0 at N = 1; also the error check)
        if not args.no_cpu and ws == 1:
            cpu, ref = cpu_oracle_baseline(n, ys, g)
        else:
            ys = 1
            oa, ob, oc, od = sample_oracle_lines(g, ys)
            ref = oracle.thomas(oa[:256], ob[:256], oc[:256], od[:256])
        nl = ref.shape[0]
        got_r = synth.line_view(x_r[:, :ys, :].cpu(), 0).numpy()[:nl]
        got_d = synth.line_view(x_d[:, :ys, :].cpu(), 0).numpy()[:nl]
        line_err = lambda got: float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))
        err = {"f32r": oracle.rel_l2(got_r, ref), "f64": oracle.rel_l2(got_d, ref), "lines_checked": int(nl),
               "f32r_worst_line": line_err(got_r), "f64_worst_line": line_err(got_d),
               "f32r_status": st, "f64_status": st_d, "f32r_corrections_max": iters}

    # ---------------- end to end on every rank (its own lines): pinned host buffers, copies inside
    # the timed region, through the pipelined host solve (slices of lines in flight on two streams:
    # host-to-device copies, solves and device-to-host copies of different slices overlap)
    e2e = None
    if not args.no_e2e:
        del g, a, b, c
        torch.cuda.empty_cache()
        h = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in
             (("a", a32), ("b", b32), ("c", c32), ("d", d))}
        for k, v in (("a", a32), ("b", b32), ("c", c32), ("d", d)):
            h[k].copy_(v)
        hx = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
        bi = sum(v.numel() * v.element_size() for v in (a32, b32, c32, d))
        bo = x.numel() * x.element_size()
        shape = tuple(d.shape)
        a32 = b32 = c32 = d = x = None  # the pipeline stages slices in its own device buffers
        torch.cuda.empty_cache()
        if args.e2e_batches > 0:
            pipe = tdma.HostPipeline(shape, axis=0, precision="f32r", batches=args.e2e_batches, slots=2, device=dev)
            tune = {"choice": (args.e2e_batches, 2), "tuned": False}
        else:  # slices and slots chosen on this data (timed candidates, the pipeline model beside them)
            pipe, tune = tdma.HostPipeline.tuned(shape, 0, "f32r", h["a"], h["b"], h["c"], h["d"], hx, device=dev)
        barrier()
        tot, _ = time_steps(lambda: pipe.solve(h["a"], h["b"], h["c"], h["d"], hx), args.e2e_steps, 2, stream)
        barrier()
        ms_e = reduce_max(tot / args.e2e_steps, dev)
        e2e = {"value": U_all / (ms_e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": bi * ws,
               "d2h_bytes_per_step": bo * ws, "steps": args.e2e_steps, "ms_per_step": ms_e,
               "api": f"HostPipeline(batches={pipe_batches(tune)}, slots={tune['choice'][1]}) -> tdma_solve_host",
               "pipeline_tuning": tune}
        if rank == 0:
            e2e["rel_l2_error"] = synth_lines_check(hx, ys, ref.shape[0], ref)
        del pipe, h, hx

    if rank != 0:
        barrier()
        return 0

    cfg_d = plan_d.config
    suite = None
    if not args.no_suite:
        plan_d = x_d = g = a = b = c = a32 = b32 = c32 = d = x = x_r = None  # release the 1024^3 arrays
        torch.cuda.empty_cache()
        flushbuf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
        suite = {}
        for name, fn in (("grid64_z_f64", lambda: suite_small_grid(stream, hbm_peak, lambda: _flush_l2(flushbuf))),
                         ("adi512_xyz_f64", lambda: suite_adi(stream, hbm_peak, fp64_probe)),
                         ("poisson1024_z_complex", lambda: suite_poisson(stream, hbm_peak)),
                         ("ragged20000", lambda: suite_ragged(stream, hbm_peak)),
                         ("split_line512_1rank", lambda: suite_split_line(stream)),
                         ("x_axis1024_f32r_f64", lambda: suite_x_axis(stream, hbm_peak))):
            try:
                suite[name] = fn()
            except Exception as exc:  # report, keep the headline line
                suite[name] = {"error": f"{type(exc).__name__}: {exc}"}
            torch.cuda.empty_cache()

    cfg_r = plan_r.config
    # FP64-pipe instructions per unknown: Thomas 8 (5 + a 3-FMA reciprocal), partitioned sweep 14
    fp64_ops = 8.0 if cfg_d["variant"] == 1 else 14.0
    fp64_peak_ops = fp64_probe["fma_per_s"]
    shard = (f"rank r of {ws} solves y-rows [{ny} r, {ny} (r + 1))" if args.scaling == "weak"
             else f"the {ny_global} y-rows split evenly over {ws} ranks") if ws > 1 else "one rank"
    out = {
        "metric": METRIC, "value": U_all / (ms_r * 1e-3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_r, "higher_is_better": True,
        "scaling": args.scaling if ws > 1 else "weak",
        "vs_baseline": None, "dtype": "f32 sweeps + extra-precise residual, f64 in/out", "data": "synthetic",
        "config": {"workload": f"general-coefficient {n}x{ny_global}x{n} grid, {n * ny_global} lines of n={n} along z "
                               f"(stride {n * ny} per rank), seed {SEED}, FP32-representable coefficients",
                   "lines": n * ny_global, "n": n, "sharding": shard,
                   "l2": "inputs (30 GB per rank) larger than L2", "plan": cfg_r},
        "fp64": {"value": U_all / (ms_d * 1e-3), "unit": UNIT, "ms_per_step": ms_d, "plan": cfg_d,
                 "roofline": {"bound": "alu", "achieved": fp64_ops * U / (ms_d * 1e-3) / 1e9,
                              "peak": fp64_peak_ops / 1e9, "unit": "G FP64-pipe instructions/s",
                              "peak_kind": "measured (FP64 FMA probe, this run)",
                              "frac": fp64_ops * U / (ms_d * 1e-3) / fp64_peak_ops,
                              "ops_per_unknown": fp64_ops,
                              "hbm_frac": BYTES_F64 * U / (ms_d * 1e-3) / 1e9 / hbm_peak},
                 "fp64_peak_probe": fp64_probe},
        "error": err,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk.summary(),
        "gpu_launches": args.steps,
        "suite": suite,
        "impl": "ours",
    }
    print(json.dumps(out), flush=True)
    if ws > 1:
        barrier()
    return 0


if __name__ == "__main__":
    sys.exit(main())
