"""Autotuner: picks a valid configuration by timing, solves correctly with it, and a new plan of
the same problem class starts from the cached choice (also through the cache file)."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle as O
import synth
from parity import rel_err
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,shape,axis", [("f64", (128, 32, 64), 0), ("f64", (16, 16, 256), 2),
                                                  ("f32r", (256, 16, 64), 0), ("f32", (64, 64, 64), 1)])
def test_autotune_choice_is_valid_and_cached(precision, shape, axis):
    fp32 = precision != "f64"
    g = synth.grid_general(shape, axis, 51, device="cuda", fp32_coefficients=fp32)
    if precision == "f64":
        a, b, c, d = g["a"], g["b"], g["c"], g["d"]
    elif precision == "f32":
        a, b, c, d = g["a32"], g["b32"], g["c32"], g["d"].float()
    else:
        a, b, c, d = g["a32"], g["b32"], g["c32"], g["d"]
    lay = tdma.line_layout(d, axis)
    plan = tdma.Plan(*lay, precision=precision)
    x = torch.empty_like(d)
    cfg = plan.autotune(a, b, c, d, x)
    assert cfg["partitions"] >= 1 and cfg["threads_per_block"] >= 1
    plan.solve(a, b, c, d, x)
    assert plan.last_error()[0] == 0
    ref = O.thomas(*(synth.line_view(t.double().cpu(), axis).numpy() for t in (a, b, c, d)))
    tol = {"f64": 1e-12, "f32": 1e-5, "f32r": 1e-12}[precision]
    assert rel_err(synth.line_view(x.double().cpu(), axis).numpy(), ref) <= tol
    plan2 = tdma.Plan(*lay, precision=precision)
    assert (plan2.config["variant"], plan2.config["partitions"]) == (cfg["variant"], cfg["partitions"])


def test_autotune_cache_file_roundtrip(tmp_path):
    path = tmp_path / "tune.txt"
    code = (
        "import sys, os, torch; sys.path.insert(0, os.getcwd())\n"
        "import synth, paper_2509_03933_gb300 as tdma\n"
        "g = synth.grid_general((96, 8, 8), 0, 1, device='cuda')\n"
        "a,b,c,d = g['a'],g['b'],g['c'],g['d']\n"
        "lay = tdma.line_layout(d, 0)\n"
        "p = tdma.Plan(*lay)\n"
        "if sys.argv[1] == 'tune':\n"
        "    cfg = p.autotune(a,b,c,d,torch.empty_like(d))\n"
        "else:\n"
        "    cfg = p.config\n"
        "print(cfg['variant'], cfg['partitions'])\n")
    env = dict(os.environ, TDMA_AUTOTUNE_CACHE=str(path))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    first = subprocess.run([sys.executable, "-c", code, "tune"], env=env, cwd=root, capture_output=True, text=True,
                           timeout=600)
    assert first.returncode == 0, first.stderr
    assert path.exists() and path.read_text().strip()
    second = subprocess.run([sys.executable, "-c", code, "read"], env=env, cwd=root, capture_output=True, text=True,
                            timeout=600)
    assert second.returncode == 0, second.stderr
    assert first.stdout.split() == second.stdout.split()


@pytest.mark.parametrize("precision", ["f64", "f32r"])
def test_ragged_autotune_choice_matches_oracle(precision):
    # a ragged batch: the group kernels timed with 8..32 rows per partition (and, for FP32 +
    # refinement, the chunk kernel); the chosen plan solves and differentiates correctly, and a new
    # plan of the same batch class starts from the cached choice
    from parity import rel_err_packed
    lengths = synth.ragged_lengths(1500, 16, 16384, seed=8)
    r = synth.ragged_general(lengths, 8, device="cuda", fp32_coefficients=True)
    keys = ("a32", "b32", "c32") if precision == "f32r" else ("a", "b", "c")
    a, b, c = (r[k] for k in keys)
    d = r["d"]
    x, plan = tdma.solve_ragged(a, b, c, d, r["offsets"], r["lengths"], precision=precision)
    cfg = plan.autotune(a, b, c, d, x)
    assert cfg["variant"] in (3, 9)  # the group kernel or the chunk kernel
    if cfg["variant"] == 3:
        assert cfg["rows_per_thread"] in (8, 12, 16, 24, 32)
    x.zero_()
    plan.solve(a, b, c, d, x)
    assert plan.last_error()[0] == 0
    offs, lens = r["offsets"].cpu().numpy(), r["lengths"].cpu().numpy()
    rng = np.random.default_rng(8)
    lines = np.unique(np.concatenate([np.argsort(-lengths)[:5], rng.choice(len(lengths), 100, replace=False)]))
    ha, hb, hc, hd = (r[k].cpu().numpy() for k in ("a", "b", "c", "d"))
    ref = O.thomas_ragged(ha, hb, hc, hd, offs, lens, lines=lines)
    xs = x.cpu().numpy()
    got = np.concatenate([xs[offs[l]:offs[l] + lens[l]] for l in sorted(ref)])
    want = np.concatenate([ref[l] for l in sorted(ref)])
    assert rel_err_packed(got, want, [lens[l] for l in sorted(ref)]) <= 1e-12
    w = synth.normal(8, synth.AID["w"], torch.arange(r["total"], device="cuda"))
    ga, gb, gc, gd = (torch.empty_like(a), torch.empty_like(b), torch.empty_like(c), torch.empty_like(x))
    plan.backward(a, b, c, x, w, ga, gb, gc, gd)
    assert plan.last_error()[0] == 0
    hg, hw = gd.cpu().numpy(), w.cpu().numpy()
    for l in sorted(ref)[:20]:
        s = slice(offs[l], offs[l] + lens[l])
        assert O.rel_l2(hg[s], O.adjoint_grads(ha[s], hb[s], hc[s], xs[s], hw[s])[3]) <= 1e-12
    _, plan2 = tdma.solve_ragged(a, b, c, d, r["offsets"], r["lengths"], precision=precision)
    c2 = plan2.config
    assert (c2["variant"], c2["rows_per_thread"] if c2["variant"] == 3 else 0) == \
        (cfg["variant"], cfg["rows_per_thread"] if cfg["variant"] == 3 else 0)


def test_tuned_host_pipeline_matches_device_solve():
    # HostPipeline.tuned: slices and slots timed on the caller's host arrays with the pipeline model
    # predicted beside them; the chosen pipeline gives the on-device solve
    shape = (128, 32, 64)
    g = synth.grid_general(shape, 0, 24, device="cuda", fp32_coefficients=True)
    a, b, c, d = g["a32"], g["b32"], g["c32"], g["d"]
    x_dev = tdma.solve(a, b, c, d, axis=0, precision="f32r")
    h = [t.cpu().pin_memory() for t in (a, b, c, d)]
    hx = torch.empty(d.shape, dtype=d.dtype).pin_memory()
    pipe, rep = tdma.HostPipeline.tuned(shape, 0, "f32r", *h, hx, batches=(2, 4, 8), slots=(2, 3))
    assert rep["choice"] in [(r["batches"], r["slots"]) for r in rep["candidates"]]
    assert len(rep["candidates"]) == 6
    for row in rep["candidates"]:
        assert row["predicted_ms"] > 0 and row["measured_ms"] > 0
    hx.zero_()
    pipe.solve(*h, hx)
    torch.cuda.synchronize()
    assert torch.equal(hx, x_dev.cpu())
    again, rep2 = tdma.HostPipeline.tuned(shape, 0, "f32r", *h, hx)  # cached: no new timing
    assert rep2 is rep and (again.slots, again.layout.n_lines) == (pipe.slots, pipe.layout.n_lines)
