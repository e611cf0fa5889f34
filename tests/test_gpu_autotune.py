"""Autotuner: picks a valid configuration by timing, solves correctly with it, and a new plan of
the same problem class starts from the cached choice (also through the cache file)."""
import os
import subprocess
import sys

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
