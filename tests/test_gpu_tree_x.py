"""FP32 storage + refinement on uniform unit-stride lines (rows adjacent in memory) with the
merge-tree cluster kernel and tiles cut along the lines, against the oracle: the three compiled
line lengths (n = 8 C M with M = 16 and clusters of 2, 4 and 8 CTAs), partial and repeated line
groups, lines addressed through two line axes, gaps between lines (left untouched), lines that
need more corrections, the stop rule run out, and x written over d."""
import numpy as np
import pytest
import torch

import oracle as O
from parity import rel_err
import synth
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu

TREE_X = 11  # TDMA_VARIANT_REFINE_TREE_X
PACKED = 9   # TDMA_VARIANT_PACKED


def _lines(t):
    """[..., n] tensor -> [lines, n] float64 numpy."""
    return t.reshape(-1, t.shape[-1]).double().cpu().numpy()


@pytest.mark.parametrize("n,L", [(1024, 300), (512, 40), (256, 32), (256, 4100), (1024, 33), (512, 6400)])
def test_unit_stride_lines_match_oracle(n, L):
    # 40 and 33 lines leave a partial last group; 4100 and 6400 lines give more groups than
    # clusters fit on the GPU, so the persistent clusters take several groups each
    g = synth.grid_general((L, n), 1, 40 + n, device="cuda", fp32_coefficients=True)
    a, b, c, d = g["a32"], g["b32"], g["c32"], g["d"]
    plan = tdma.Plan(*tdma.line_layout(d, 1), precision="f32r")
    assert plan.config["variant"] == TREE_X
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    st, iters = plan.last_error()
    assert st == 0 and iters == 1
    ref = O.thomas(*(_lines(t) for t in (a, b, c, d)))
    assert rel_err(_lines(x), ref) <= 1e-12


def test_two_line_axes_and_gaps():
    # lines along x of a [3][64 of 96][256] slice: 64 lines per plane (a multiple of the 32 lines
    # of a cluster), planes 96 x 256 elements apart; then lines of 256 in rows of 260 elements,
    # with the 4 gap elements of every row left as they were
    g = synth.grid_general((3, 96, 256), 2, 51, device="cuda", fp32_coefficients=True)
    a, b, c, d = (g[k][:, :64, :] for k in ("a32", "b32", "c32", "d"))
    plan = tdma.Plan(*tdma.line_layout(d, 2), precision="f32r")
    assert plan.config["variant"] == TREE_X
    x = torch.empty((3, 96, 256), dtype=torch.float64, device="cuda")[:, :64, :]
    plan.solve(a, b, c, d, x)
    assert plan.last_error()[0] == 0
    ref = O.thomas(*(_lines(t) for t in (a, b, c, d)))
    assert rel_err(_lines(x), ref) <= 1e-12

    L, n, gap = 200, 256, 4
    g = synth.grid_general((L, n + gap), 1, 52, device="cuda", fp32_coefficients=True)
    a, b, c = (g[k][:, :n] for k in ("a32", "b32", "c32"))
    d = g["d"][:, :n]
    plan = tdma.Plan(*tdma.line_layout(d, 1), precision="f32r")
    assert plan.config["variant"] == TREE_X
    xg = torch.full((L, n + gap), 7.0, dtype=torch.float64, device="cuda")
    plan.solve(a, b, c, d, xg[:, :n])
    assert plan.last_error()[0] == 0
    ref = O.thomas(*(_lines(t) for t in (a, b, c, d)))
    assert rel_err(_lines(xg[:, :n]), ref) <= 1e-12
    assert bool((xg[:, n:] == 7.0).all())


def test_layouts_the_tiles_cannot_describe_take_the_chunk_kernel():
    # 48 lines per plane (not a multiple of 32), or a row pitch that is not 16 bytes of floats
    g = synth.grid_general((2, 96, 256), 2, 53, device="cuda", fp32_coefficients=True)
    d = g["d"][:, :48, :]
    assert tdma.Plan(*tdma.line_layout(d, 2), precision="f32r").config["variant"] == PACKED
    g = synth.grid_general((64, 258), 1, 54, device="cuda", fp32_coefficients=True)
    d = g["d"][:, :256]
    assert tdma.Plan(*tdma.line_layout(d, 1), precision="f32r").config["variant"] == PACKED


def test_more_corrections_not_converged_and_in_place():
    # weak diagonal dominance (b = |a| + |c| + 0.02) needs several corrections; an unreachable
    # tolerance runs max_refine_iters of them and reports TDMA_ERR_NOT_CONVERGED; x may alias d
    L, n = 4100, 1024
    a = (synth.uniform(31, synth.AID["a"], torch.arange(n * L)) - 1.0).float().view(L, n)
    c = (synth.uniform(31, synth.AID["c"], torch.arange(n * L)) - 1.0).float().view(L, n)
    b = (a.abs() + c.abs() + 0.02).float()
    xt = 2.0 * synth.uniform(31, synth.AID["x_true"], torch.arange(n * L)).view(L, n) - 1.0
    d = synth.apply_tridiag(a.double(), b.double(), c.double(), xt, 1)
    a, b, c, d = a.cuda(), b.cuda(), c.cuda(), d.cuda()
    ref = O.thomas(*(_lines(t) for t in (a, b, c, d)))
    plan = tdma.Plan(*tdma.line_layout(d, 1), precision="f32r")
    assert plan.config["variant"] == TREE_X
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    st, iters = plan.last_error()
    assert st == 0 and iters >= 2
    assert rel_err(_lines(x), ref) <= 1e-12
    dd = d.clone()
    plan.solve(a, b, c, dd, dd)  # in place
    assert plan.last_error()[0] == 0
    assert rel_err(_lines(dd), ref) <= 1e-12
    stiff = tdma.Plan(*tdma.line_layout(d, 1), precision="f32r", max_refine_iters=3, refine_tol=1e-30)
    stiff.solve(a, b, c, d, x)
    st, iters = stiff.last_error()
    assert st == 7 and iters == 3
    assert rel_err(_lines(x), ref) <= 1e-12


@pytest.mark.parametrize("axis", [0, 1])
def test_cluster_variants_refuse_arrays_off_16_bytes(axis):
    # the tiles travel by TMA: an array one element off a 16-byte boundary is refused before
    # anything runs (TDMA_ERR_UNSUPPORTED); the aligned solve still works afterwards
    n, L = 256, 64
    shape = (n, L) if axis == 0 else (L, n)
    g = synth.grid_general(shape, axis, 71, device="cuda", fp32_coefficients=True)
    a, b, c, d = g["a32"], g["b32"], g["c32"], g["d"]
    plan = tdma.Plan(*tdma.line_layout(d, axis), precision="f32r")
    assert plan.config["variant"] == (8 if axis == 0 else TREE_X)
    big = torch.empty(d.numel() + 1, dtype=torch.float64, device="cuda")
    xs = big[1:].view(shape)  # 8 bytes past a 16-byte boundary
    with pytest.raises(tdma.TDMAError) as e:
        plan.solve(a, b, c, d, xs)
    assert e.value.status == 2
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    assert plan.last_error()[0] == 0
    ref = O.thomas(*(_lines(t if axis == 1 else t.T) for t in (a, b, c, d)))
    assert rel_err(_lines(x if axis == 1 else x.T), ref) <= 1e-12


@pytest.mark.parametrize("axis", [0, 1])
def test_single_correction_reports_lines_short_of_the_rule(axis):
    # With one correction allowed, a line that fails the stop rule is reported (status 7) without
    # further passes; out of place the rule of a line group is settled with the next group's
    # exchange, or, for a cluster's last group, by an exchange of its own: 4100 lines give every
    # cluster several groups. A line group that meets the rule reports status 0 with the same x.
    n, L = 256, 4100
    shape = (n, L) if axis == 0 else (L, n)
    g = synth.grid_general(shape, axis, 73, device="cuda", fp32_coefficients=True)
    a, b, c, d = g["a32"], g["b32"], g["c32"], g["d"]
    stiff = tdma.Plan(*tdma.line_layout(d, axis), precision="f32r", max_refine_iters=1, refine_tol=1e-30)
    assert stiff.config["variant"] == (8 if axis == 0 else TREE_X)
    x1 = torch.empty_like(d)
    stiff.solve(a, b, c, d, x1)
    assert stiff.last_error() == (7, 1)
    plan = tdma.Plan(*tdma.line_layout(d, axis), precision="f32r", max_refine_iters=1)
    x2 = torch.empty_like(d)
    plan.solve(a, b, c, d, x2)
    assert plan.last_error() == (0, 1)
    assert torch.equal(x1, x2)  # one correction either way
    ref = O.thomas(*(_lines(t if axis == 1 else t.T) for t in (a, b, c, d)))
    assert rel_err(_lines(x2 if axis == 1 else x2.T), ref) <= 1e-12
