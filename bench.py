#!/usr/bin/env python
"""Throughput of the batched tridiagonal solve on one GB300 per rank.

Workload: the general-coefficient 1024^3 grid (a, c ~ U(-1, 0), b = 2 + |a| + |c| + U(0, 1),
x_true ~ U(-1, 1), d = A x_true, seed 3), coefficients representable in FP32, 2^20 lines of
n = 1024 along the strided z axis. One step solves the whole grid with FP32 storage and sweeps
plus on-chip refinement (the headline ``value``); the plain FP64 solve of the same problem is
measured the same way and reported beside it. Inputs (30 GB) are far larger than L2 (129 MB),
so no flush is needed between steps.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0). Under torchrun every rank solves its own copy of the workload
(independent problems: weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
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
FP64_OPS_PEAK = 152 * 2 * 2.07e9  # FP64 pipe: 152 SMs x 2 ops/clk x 2.07 GHz (1.25 TFLOP/s, FMA = 2)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


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
    """DRAM bytes per launch from a committed ncu summary, valid only for the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        j = json.load(f)
    rec = j.get(kernel)
    if not rec or rec.get("source_sha") != source_sha():
        return None
    return rec


def source_sha() -> str:
    h = hashlib.sha256()
    cdir = os.path.join(ROOT, "paper_2509_03933_gb300", "csrc")
    for f in sorted(os.listdir(cdir)):
        with open(os.path.join(cdir, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def make_workload(n: int, device):
    import synth
    g = synth.grid_general((n, n, n), 0, SEED, device=device, fp32_coefficients=True)
    g.pop("x_true")
    return g


def sample_oracle_lines(g, ys: int):
    """Lines of the first ``ys`` y-rows (all x, full z) of the workload, as oracle inputs."""
    import synth
    sl = lambda t: synth.line_view(t[:, :ys, :].double().cpu(), 0).numpy()
    return sl(g["a32"]), sl(g["b32"]), sl(g["c32"]), sl(g["d"])


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


def run_reference(args):
    """The oracle (CPU, numpy, one core) on bounded samples of the same workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import synth
    n = args.n
    ys = max(1, args.ref_lines // n)
    g = synth.grid_general((n, ys, n), 0, SEED, fp32_coefficients=True, full_shape=(n, n, n), origin=(0, 0, 0))
    lv = lambda t: synth.line_view(t.double(), 0).numpy()
    a, b, c, d = lv(g["a32"]), lv(g["b32"]), lv(g["c32"]), lv(g["d"])
    units = a.size
    for _ in range(args.warmup):
        oracle.thomas(a, b, c, d)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.thomas(a, b, c, d)
    dt = (time.perf_counter() - t) / max(1, args.steps)
    value = units / dt
    sample = f"{ys * n} lines x {n} (first {ys} y-rows of the {n}^3 grid, z axis) per step"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"general-coefficient {n}^3 grid, lines along z, seed {SEED}, "
                                  "FP32-representable coefficients", "lines": n * n, "n": n},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-lines", type=int, default=32768, help="lines in the CPU oracle sample")
    ap.add_argument("--ref-lines", type=int, default=4096, help="lines per reference-arm step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    import paper_2509_03933_gb300 as tdma

    dev = torch.device("cuda", local if ws > 1 else 0)
    n = args.n
    U = n ** 3
    g = make_workload(n, dev)
    a32, b32, c32, d = g["a32"], g["b32"], g["c32"], g["d"]
    x = torch.empty_like(d)
    stream = torch.cuda.current_stream()
    plan_r = tdma.Plan(n, n * n, n * n, n * n, 1, 0, precision="f32r")
    plan_d = tdma.Plan(n, n * n, n * n, n * n, 1, 0, precision="f64")

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # ---------------- headline: FP32 storage + refinement
    barrier()
    with ClockSampler(local if ws > 1 else 0) as clk:
        total_r, per_r = time_steps(lambda: plan_r.solve(a32, b32, c32, d, x), args.steps, args.warmup, stream)
    barrier()
    st, iters = plan_r.last_error()
    ms_r = total_r / args.steps
    if ws > 1:
        t = torch.tensor([ms_r], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_r = float(t.item())
    x_r = x.clone() if rank == 0 else None

    # ---------------- the plain FP64 solve of the same problem
    a, b, c = g["a"], g["b"], g["c"]
    total_d, per_d = time_steps(lambda: plan_d.solve(a, b, c, d, x), max(3, args.steps // 3), args.warmup, stream)
    st_d, _ = plan_d.last_error()
    ms_d = total_d / max(3, args.steps // 3)
    x_d = x

    if rank != 0:
        barrier()
        return 0

    hbm_peak, peak_kind = peaks()
    kern_ms = sorted(per_r)[len(per_r) // 2]
    achieved = BYTES_F32R * U / (kern_ms * 1e-3) / 1e9
    trec = traffic_record("refine_kernel")
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
            "traffic": (trec["dram_bytes"] * (U / trec["unknowns"])) if trec else None,
            "peak_kind": f"{peak_kind} (STREAM-style copy)", "algorithmic_bytes_per_unknown": BYTES_F32R,
            "kernel": "refine_kernel", "kernel_ms": kern_ms}

    # ---------------- CPU oracle on a bounded sample (also the per-result error check)
    cpu = None
    err = {}
    import oracle
    ys = max(1, args.cpu_lines // n)
    oa, ob, oc, od = sample_oracle_lines(g, ys)
    if not args.no_cpu:
        t0 = time.perf_counter()
        ref = oracle.thomas(oa, ob, oc, od)
        dt = time.perf_counter() - t0
        cpu = {"value": oa.size / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{ys * n} lines x {n} (first {ys} y-rows of the grid), numpy Thomas, FP64"}
    else:
        ref = oracle.thomas(oa[:256], ob[:256], oc[:256], od[:256])
    import synth
    nl = ref.shape[0]
    got_r = synth.line_view(x_r[:, :ys, :].cpu(), 0).numpy()[:nl]
    got_d = synth.line_view(x_d[:, :ys, :].cpu(), 0).numpy()[:nl]
    err = {"f32r": oracle.rel_l2(got_r, ref), "f64": oracle.rel_l2(got_d, ref), "lines_checked": int(nl),
           "f32r_status": st, "f64_status": st_d, "f32r_corrections_max": iters}

    # ---------------- end to end: pinned host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        del g, a, b, c
        torch.cuda.empty_cache()
        h = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in
             (("a", a32), ("b", b32), ("c", c32), ("d", d))}
        for k, v in (("a", a32), ("b", b32), ("c", c32), ("d", d)):
            h[k].copy_(v)
        hx = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)

        def e2e_step():
            for k, dv in (("a", a32), ("b", b32), ("c", c32), ("d", d)):
                dv.copy_(h[k], non_blocking=True)
            plan_r.solve(a32, b32, c32, d, x)
            hx.copy_(x, non_blocking=True)

        tot, _ = time_steps(e2e_step, args.e2e_steps, 1, stream)
        bi = sum(v.numel() * v.element_size() for v in (a32, b32, c32, d))
        e2e = {"value": U / (tot / args.e2e_steps * 1e-3), "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": x.numel() * x.element_size(), "steps": args.e2e_steps,
               "ms_per_step": tot / args.e2e_steps}

    cfg_r = plan_r.config
    fp64_ops = 15.0  # FP64-pipe instructions per unknown of the fused FP64 kernel
    out = {
        "metric": METRIC, "value": ws * U / (ms_r * 1e-3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_r, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 sweeps + extra-precise residual, f64 in/out", "data": "synthetic",
        "config": {"workload": f"general-coefficient {n}^3 grid, {n * n} lines of n={n} along z (stride {n * n}), "
                               f"seed {SEED}, FP32-representable coefficients", "lines": n * n, "n": n,
                   "l2": "inputs (30 GB) larger than L2", "plan": cfg_r},
        "fp64": {"value": ws * U / (ms_d * 1e-3), "unit": UNIT, "ms_per_step": ms_d, "plan": plan_d.config,
                 "roofline": {"bound": "alu", "achieved": fp64_ops * U / (ms_d * 1e-3) / 1e9,
                              "peak": FP64_OPS_PEAK / 1e9, "unit": "Gop/s (FP64 pipe)",
                              "frac": fp64_ops * U / (ms_d * 1e-3) / FP64_OPS_PEAK,
                              "hbm_frac": BYTES_F64 * U / (ms_d * 1e-3) / 1e9 / hbm_peak}},
        "error": err,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk.summary(),
        "gpu_launches": args.steps,
        "impl": "ours",
    }
    print(json.dumps(out), flush=True)
    if ws > 1:
        barrier()
    return 0


if __name__ == "__main__":
    sys.exit(main())
