"""Forward-solve parity of the CUDA path against the CPU oracle (element by element).

Tolerances (relative L2, pooled over the compared lines and for every single line): FP64 <= 1e-12,
FP32 <= 1e-5, FP32 + refinement <= 1e-12, as the FP64 oracle demands of each precision.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from parity import rel_err
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f32r": 1e-12}


def _np_lines(t, axis):
    return synth.line_view(t.detach().double().cpu(), axis).numpy()


def _grid_case(shape, axis, seed, precision, partitions):
    fp32 = precision in ("f32", "f32r")
    g = synth.grid_general(shape, axis, seed, device="cpu", fp32_coefficients=fp32)
    if precision == "f64":
        a, b, c, d = (g[k].cuda() for k in ("a", "b", "c", "d"))
    elif precision == "f32":
        a, b, c = (g[k + "32"].cuda() for k in ("a", "b", "c"))
        d = g["d"].float().cuda()
    else:
        a, b, c = (g[k + "32"].cuda() for k in ("a", "b", "c"))
        d = g["d"].cuda()
    x = tdma.solve(a, b, c, d, axis=axis, precision=precision, partitions=partitions, check=True)
    # the oracle solves the problem exactly as stored (float inputs widened to double)
    ref = O.thomas(*(_np_lines(t, axis) for t in (a, b, c, d)))
    return _np_lines(x, axis), ref


@pytest.mark.parametrize("partitions", [1, 4])
def test_config0_z_axis_f64(partitions):
    # 64^3 grid, 4096 lines of n = 64 along the strided z axis, seed 0
    x, ref = _grid_case((64, 64, 64), 0, 0, "f64", partitions)
    assert rel_err(x, ref) <= TOL["f64"]
    assert np.max(np.abs(x - ref)) <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("partitions", [0, 1, 2, 3, 5, 8])
def test_axes_and_uneven_partitions_f64(axis, partitions):
    shape = (33, 20, 41)
    n = shape[axis]
    if partitions > 1 and n // partitions < 2:
        pytest.skip("partition too small")
    x, ref = _grid_case(shape, axis, 7 + axis, "f64", partitions)
    assert rel_err(x, ref) <= TOL["f64"]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 31, 32, 33, 63, 64, 65, 257, 1000])
@pytest.mark.parametrize("precision", ["f64", "f32", "f32r"])
def test_line_lengths_and_ragged_tails(n, precision):
    # 37 lines: not a multiple of the lines per block; unit-stride rows
    x, ref = _grid_case((37, n), 1, 11 + n, precision, 0)
    assert rel_err(x, ref) <= TOL[precision]


@pytest.mark.parametrize("precision", ["f32", "f32r"])
@pytest.mark.parametrize("axis,partitions", [(0, 0), (0, 4), (2, 8), (1, 3)])
def test_float_paths_on_grid(precision, axis, partitions):
    x, ref = _grid_case((48, 24, 40), axis, 3, precision, partitions)
    assert rel_err(x, ref) <= TOL[precision]


def test_refinement_reports_corrections_and_beats_fp32():
    g = synth.grid_general((64, 16, 16), 0, 3, fp32_coefficients=True)
    a, b, c = (g[k + "32"].cuda() for k in ("a", "b", "c"))
    d = g["d"].cuda()
    plan = tdma.Plan(64, 256, 256, 256, 1, 0, precision="f32r")
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    st, iters = plan.last_error()
    assert st == 0 and 1 <= iters <= 4
    ref = O.thomas(*(_np_lines(t, 0) for t in (a, b, c, d)))
    e_r = rel_err(_np_lines(x, 0), ref)
    x32 = tdma.solve(a, b, c, d.float(), axis=0, precision="f32")
    e_32 = rel_err(_np_lines(x32, 0), ref)
    assert e_r <= 1e-12 and e_32 > 1e3 * e_r


def test_x_aliases_d():
    g = synth.grid_general((16, 8, 40), 2, 5)
    a, b, c, d = (g[k].cuda() for k in ("a", "b", "c", "d"))
    ref = O.thomas(*(_np_lines(t, 2) for t in (a, b, c, d)))
    tdma.solve(a, b, c, d, axis=2, partitions=4, out=d)
    assert rel_err(_np_lines(d, 2), ref) <= 1e-12


def test_strided_subset_of_lines():
    # every other x-line of a grid (inner stride 2) along z
    g = synth.grid_general((40, 6, 16), 0, 9)
    a, b, c, d = (g[k].cuda()[:, :, ::2] for k in ("a", "b", "c", "d"))
    ref = O.thomas(*(_np_lines(t.contiguous(), 0) for t in (a, b, c, d)))
    full = torch.zeros(40, 6, 16, dtype=torch.float64, device="cuda")
    x = full[:, :, ::2]
    tdma.solve(a, b, c, d, axis=0, partitions=4, out=x)
    assert rel_err(_np_lines(x.contiguous(), 0), ref) <= 1e-12
    assert torch.count_nonzero(full[:, :, 1::2]) == 0  # lines in between untouched


def test_zero_lines_is_a_noop():
    e = torch.empty(0, 10, dtype=torch.float64, device="cuda")
    plan = tdma.Plan(10, 0, 1, 1, 10, 0)
    plan.solve(e, e, e, e, e)
    assert plan.last_error()[0] == 0


def test_zero_pivot_sets_nonfinite_status():
    n = 16
    a = torch.zeros(4, n, dtype=torch.float64, device="cuda")
    c = torch.zeros_like(a)
    b = torch.ones_like(a)
    b[2, 5] = 0.0  # singular line
    d = torch.ones_like(a)
    plan = tdma.Plan(n, 4, 1, 4, n, 0, partitions=2)
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    st, _ = plan.last_error()
    assert st == 5
    assert plan.last_error()[0] == 0  # cleared after reading


def test_poisson_lines_broadcast_complex():
    # wavenumber lines along z of a small grid: broadcast a, c, b0 plus per-line shift,
    # complex right-hand side as two interleaved right-hand sides; the zero mode is skipped
    nx, ny, nz = 8, 6, 64
    p = synth.poisson_lines(nx, ny, nz, seed=2, device="cuda")
    d = p["d"].reshape(nz, ny * nx, 2)[:, 1:, :]
    shift = p["shift"][1:].contiguous()
    x = tdma.solve(p["a"], p["b0"], p["c"], d, axis=0, nrhs=2, coef_broadcast=True, diag_shift=shift,
                   partitions=4, check=True)
    L = ny * nx - 1
    a = np.broadcast_to(p["a"].cpu().numpy(), (L, nz))
    c = np.broadcast_to(p["c"].cpu().numpy(), (L, nz))
    b = p["b0"].cpu().numpy()[None, :] + shift.cpu().numpy()[:, None]
    dn = d.cpu().numpy().transpose(1, 0, 2)  # [lines, n, 2]
    ref = O.thomas_ext(a, b, c, dn)
    got = x.cpu().numpy().transpose(1, 0, 2)
    assert rel_err(got, ref) <= 1e-12


@pytest.mark.parametrize("n,lines", [(1024, 64), (512, 48), (256, 40), (64, 100), (1024, 37), (256, 6)])
def test_refine_tile_kernels_z_lines(n, lines):
    # lines along the strided axis of an [n][lines] grid: element stride = line count. Line
    # counts divisible by 4 take the TMA-staged tile; others the plain-load fallback; 6 lines
    # leave a partial last block.
    x, ref = _grid_case((n, lines), 0, 17 + n, "f32r", 0)
    assert rel_err(x, ref) <= TOL["f32r"]
    x, ref = _grid_case((n, lines), 0, 17 + n, "f32", 0)
    assert rel_err(x, ref) <= TOL["f32"]


@pytest.mark.parametrize("tree", [True, False])
@pytest.mark.parametrize("n,lines", [(1024, 96), (512, 40), (256, 32), (512, 4100), (256, 6400)])
def test_cluster_refine_kernels(monkeypatch, tree, n, lines):
    # lines of n = 8 C M rows spread over a CTA cluster: the merge-tree kernel (default) and,
    # with it switched off, the kernel with a serial Stage B; 40 and 4100 lines leave a partial
    # group; 4100 and 6400 lines give more groups than clusters fit on the GPU, so the persistent
    # clusters of the merge-tree kernel take several groups each
    if not tree:
        monkeypatch.setenv("TDMA_DISABLE_TREE", "1")
    g = synth.grid_general((n, lines), 0, 23 + n, device="cpu", fp32_coefficients=True)
    a, b, c = (g[k + "32"].cuda() for k in ("a", "b", "c"))
    d = g["d"].cuda()
    plan = tdma.Plan(*tdma.line_layout(d, 0), precision="f32r")
    assert plan.config["variant"] == (8 if tree else 6)
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    st, iters = plan.last_error()
    assert st == 0 and iters == 1
    ref = O.thomas(*(_np_lines(t, 0) for t in (a, b, c, d)))
    assert rel_err(_np_lines(x, 0), ref) <= TOL["f32r"]


@pytest.mark.parametrize("tree", [True, False])
def test_cluster_refine_more_corrections_and_in_place(monkeypatch, tree):
    # weak diagonal dominance (b = |a| + |c| + 0.02) needs several corrections; an unreachable
    # tolerance runs max_refine_iters of them and reports TDMA_ERR_NOT_CONVERGED; x may alias d
    if not tree:
        monkeypatch.setenv("TDMA_DISABLE_TREE", "1")
    n, lines = 1024, 4100
    a = (synth.uniform(29, synth.AID["a"], torch.arange(n * lines)) - 1.0).float().view(n, lines)
    c = (synth.uniform(29, synth.AID["c"], torch.arange(n * lines)) - 1.0).float().view(n, lines)
    b = (a.abs() + c.abs() + 0.02).float()
    xt = 2.0 * synth.uniform(29, synth.AID["x_true"], torch.arange(n * lines)).view(n, lines) - 1.0
    d = synth.apply_tridiag(a.double(), b.double(), c.double(), xt, 0)
    a, b, c, d = a.cuda(), b.cuda(), c.cuda(), d.cuda()
    ref = O.thomas(*(_np_lines(t, 0) for t in (a, b, c, d)))
    plan = tdma.Plan(*tdma.line_layout(d, 0), precision="f32r")
    assert plan.config["variant"] == (8 if tree else 6)
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    st, iters = plan.last_error()
    assert st == 0 and iters >= 2
    assert rel_err(_np_lines(x, 0), ref) <= TOL["f32r"]
    dd = d.clone()
    plan.solve(a, b, c, dd, dd)  # in place
    assert plan.last_error()[0] == 0
    assert rel_err(_np_lines(dd, 0), ref) <= TOL["f32r"]
    stiff = tdma.Plan(*tdma.line_layout(d, 0), precision="f32r", max_refine_iters=3, refine_tol=1e-30)
    stiff.solve(a, b, c, d, x)
    st, iters = stiff.last_error()
    assert st == 7 and iters == 3
    assert rel_err(_np_lines(x, 0), ref) <= TOL["f32r"]


@pytest.mark.parametrize("partitions", [1, 4])
def test_fp64_refine_mode_general_and_badly_conditioned(partitions):
    # general lines: at least as accurate as plain FP64
    x, ref = _grid_case((64, 8, 24), 0, 61, "f64", partitions)
    g = synth.grid_general((64, 8, 24), 0, 61)
    a, b, c, d = (g[k].cuda() for k in ("a", "b", "c", "d"))
    xr = tdma.solve(a, b, c, d, axis=0, precision="f64r", partitions=partitions, check=True)
    assert rel_err(_np_lines(xr, 0), ref) <= 1e-14
    # the pinned Poisson zero mode (condition number ~1e9) against extended precision
    pz = synth.poisson_lines(2, 2, 1024, seed=2, device="cuda", rhs=True)
    dz = pz["d"].view(1024, 4, 2)[:, :1, :]
    xz = tdma.solve(pz["pin_a"], pz["pin_b"], pz["pin_c"], dz, axis=0, nrhs=2, coef_broadcast=True,
                    precision="f64r", partitions=partitions, check=True)
    ref = O.thomas_ext(pz["pin_a"].cpu().numpy(), pz["pin_b"].cpu().numpy(), pz["pin_c"].cpu().numpy(),
                       dz[:, 0, :].cpu().numpy())
    assert O.rel_l2(xz[:, 0, :].cpu().numpy(), ref) <= 1e-13


def test_fp64_refine_rejects_in_place():
    g = synth.grid_general((16, 4, 4), 0, 62)
    a, b, c, d = (g[k].cuda() for k in ("a", "b", "c", "d"))
    with pytest.raises(tdma.TDMAError):
        tdma.solve(a, b, c, d, axis=0, precision="f64r", out=d)
