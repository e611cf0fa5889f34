"""FP32 storage + refinement with right-hand sides outside the fast path of the merge-tree kernel's
float-pair split of d (normal magnitudes from 2^-74): lines whose d lies below 2^-74 and lines
with d = 0 (both take the general split), and ordinary lines in the same launch, along a strided
axis and along the unit-stride axis, against the oracle per line (a line whose reference is zero
is held to its absolute error)."""
import numpy as np
import pytest
import torch

import oracle as O
from parity import rel_err
import synth
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("axis", [0, 1])
def test_tiny_zero_and_ordinary_right_hand_sides(axis):
    n, L = 1024, 96
    shape = (n, L) if axis == 0 else (L, n)
    g = synth.grid_general(shape, axis, 61, device="cpu", fp32_coefficients=True)
    a, b, c = g["a32"], g["b32"], g["c32"]
    d = g["d"].clone()
    lines = d if axis == 1 else d.T  # a [L][n] view of the lines
    lines[0:32] *= 1e-28   # below 2^-74
    lines[32:48] = 0.0     # zero lines
    lines[48:52, ::7] = 0.0  # scattered zeros inside ordinary lines
    A, B, C, D = (t.cuda() for t in (a, b, c, d))
    plan = tdma.Plan(*tdma.line_layout(D, axis), precision="f32r")
    assert plan.config["variant"] == (8 if axis == 0 else 11)
    x = torch.empty_like(D)
    plan.solve(A, B, C, D, x)
    st, iters = plan.last_error()
    assert st == 0, (st, iters)
    to_lines = (lambda t: t.cpu().numpy().T) if axis == 0 else (lambda t: t.cpu().numpy())
    ref = O.thomas(*(to_lines(t).astype(np.float64) for t in (a, b, c, d)))
    got = to_lines(x)
    assert rel_err(got[:32] * 1e28, ref[:32] * 1e28) <= 1e-12  # the tiny lines, relative to their own size
    assert float(np.abs(got[32:48]).max()) == 0.0
    assert rel_err(got[48:], ref[48:]) <= 1e-12
