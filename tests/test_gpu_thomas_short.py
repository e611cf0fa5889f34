"""One partition per line (Thomas) for short lines in small batches, where the P = 1 solve stages
each warp's 32 lines in shared memory before sweeping: FP64 and FP32, one and two right-hand
sides, a per-line diagonal shift, line lengths from 2 to 128, partial warps, the 64^3 grid of the
smallest workload, x written over d, and a zero pivot, against the oracle per line."""
import numpy as np
import pytest
import torch

import oracle as O
from parity import rel_err
import synth
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
THOMAS = 1  # TDMA_VARIANT_THOMAS


def _ref_lines(t, axis=0):
    """Lines on axis 0 of the returned float64 array."""
    return np.moveaxis(t.double().cpu().numpy(), axis, -1).reshape(-1, t.shape[axis])


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("n,lines", [(2, 5), (2, 31), (3, 33), (17, 64), (64, 4096), (128, 100), (128, 16384)])
def test_short_lines_match_oracle(precision, n, lines):
    g = synth.grid_general((n, lines), 0, 80 + n, device="cuda")
    dt = torch.float64 if precision == "f64" else torch.float32
    a, b, c, d = (g[k].to(dt) for k in ("a", "b", "c", "d"))
    plan = tdma.Plan(*tdma.line_layout(d, 0), precision=precision, partitions=1)
    assert plan.config["variant"] == THOMAS
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    assert plan.last_error()[0] == 0
    ref = O.thomas(*(_ref_lines(t) for t in (a, b, c, d)))
    assert rel_err(_ref_lines(x), ref) <= TOL[precision]


def test_grid64_z_lines_in_place():
    # the smallest workload's layout: 4096 lines of n = 64 along z of a 64^3 grid
    g = synth.grid_general((64, 64, 64), 0, 0, device="cuda")
    a, b, c, d = g["a"], g["b"], g["c"], g["d"]
    plan = tdma.Plan(*tdma.line_layout(d, 0), partitions=1)
    ref = O.thomas(*(_ref_lines(t) for t in (a, b, c, d)))
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    assert plan.last_error()[0] == 0
    assert rel_err(_ref_lines(x), ref) <= 1e-12
    dd = d.clone()
    plan.solve(a, b, c, dd, dd)
    assert plan.last_error()[0] == 0
    assert torch.equal(dd, x)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_two_right_hand_sides_and_shift(precision):
    # complex right-hand sides (re, im interleaved) and a per-line shift added to b
    n, lines = 96, 200
    g = synth.grid_general((n, lines), 0, 91, device="cuda")
    dt = torch.float64 if precision == "f64" else torch.float32
    a, b, c = (g[k].to(dt) for k in ("a", "b", "c"))
    d2 = torch.stack([g["d"], 0.5 - g["d"]], dim=-1).to(dt).contiguous()
    shift = (0.25 + 0.01 * torch.arange(lines, device="cuda", dtype=torch.float64)).to(dt)
    plan = tdma.Plan(*tdma.line_layout(d2, 0, nrhs=2), nrhs=2, diag_shift=shift, precision=precision, partitions=1)
    assert plan.config["variant"] == THOMAS
    x = torch.empty_like(d2)
    plan.solve(a, b, c, d2, x)
    assert plan.last_error()[0] == 0
    bs = (b + shift[None, :]).double()
    for q in range(2):
        ref = O.thomas(*(_ref_lines(t) for t in (a, bs, c, d2[..., q])))
        assert rel_err(_ref_lines(x[..., q]), ref) <= TOL[precision]


def test_zero_pivot_sets_nonfinite_status():
    n, lines = 8, 40
    a = torch.zeros(n, lines, dtype=torch.float64, device="cuda")
    c = torch.zeros_like(a)
    b = torch.ones_like(a)
    b[3, 17] = 0.0  # a zero diagonal with no coupling: pivot 0 in line 17
    d = torch.ones_like(a)
    plan = tdma.Plan(*tdma.line_layout(d, 0), partitions=1)
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    assert plan.last_error()[0] == 5
