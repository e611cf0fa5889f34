"""The FFT-based Poisson pipeline (cuFFT over the (z, x) planes, the wavenumber lines along y,
cuFFT back) through the C ABI against the oracle's FFT-based solve element by element, and at the
full 1024^3 size by the discrete equation itself on sampled planes."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu


def _problem(ny, nz, nx, seed, beta=2.0):
    a, c, b = synth.poisson_coefficients(ny, beta)
    q = torch.from_numpy(np.random.default_rng(seed).standard_normal((ny, nz, nx)))
    return a, b, c, 2 * np.pi / nx, 2 * np.pi / nz, q


@pytest.mark.parametrize("shape", [(40, 24, 32), (33, 16, 18), (9, 4, 2), (64, 30, 64), (128, 2, 2)])
@pytest.mark.parametrize("precision", ["f64", "f64r"])
def test_pipeline_matches_oracle(shape, precision):
    ny, nz, nx = shape
    a, b, c, dx, dz, q = _problem(ny, nz, nx, sum(shape))
    solver = tdma.PoissonFFT(nx, ny, nz, dx, dz, a, b, c, precision=precision)
    phi = solver.solve(q.cuda(), check=True)
    ref = O.poisson_fft(q.numpy(), dx, dz, a, b, c)
    assert O.rel_l2(phi.cpu().numpy(), ref) <= 1e-12


def test_in_place_and_repeated():
    a, b, c, dx, dz, q = _problem(48, 20, 36, 5)
    ref = O.poisson_fft(q.numpy(), dx, dz, a, b, c)
    solver = tdma.PoissonFFT(36, 48, 20, dx, dz, a, b, c)
    qd = q.cuda()
    p1 = solver.solve(qd)
    p2 = solver.solve(qd)
    assert torch.equal(p1, p2)
    solver.solve(qd, out=qd)  # phi over q
    assert O.rel_l2(qd.cpu().numpy(), ref) <= 1e-12


def test_dirichlet_operator_without_pin():
    ny, nz, nx = 30, 12, 16
    a, b, c = np.ones(ny), np.full(ny, -2.0), np.ones(ny)
    q = torch.from_numpy(np.random.default_rng(6).standard_normal((ny, nz, nx)))
    solver = tdma.PoissonFFT(nx, ny, nz, 0.5, 0.25, a, b, c, pin_zero_mode=False)
    phi = solver.solve(q.cuda(), check=True)
    ref = O.poisson_fft(q.numpy(), 0.5, 0.25, a, b, c, pin_zero_mode=False)
    assert O.rel_l2(phi.cpu().numpy(), ref) <= 1e-12


def test_invalid_descriptors():
    a, b, c = np.ones(8), np.full(8, -2.0), np.ones(8)
    for kw in (dict(nx=7), dict(nz=1), dict(dx=0.0)):
        args = dict(nx=8, ny=8, nz=4, dx=1.0, dz=1.0)
        args.update(kw)
        with pytest.raises(tdma.TDMAError):
            tdma.PoissonFFT(args["nx"], args["ny"], args["nz"], args["dx"], args["dz"], a, b, c)
    with pytest.raises(tdma.TDMAError):
        tdma.PoissonFFT(8, 8, 4, 1.0, 1.0, a, b, c, precision="f32")


def test_full_size_1024_cubed_by_the_discrete_equation():
    # the bench workload: 1024^3 grid, stretched y (Neumann ends), periodic x and z. Checked on
    # sampled y planes by applying the discrete operator with plain differences: every equation
    # holds except row 0 of the (0, 0) mode, which the pin replaces (a constant over plane y = 0)
    n = 1024
    a, c, b = synth.poisson_coefficients(n)
    dx = dz = 2 * np.pi / n
    q = synth.normal(7, synth.AID["d"], torch.arange(n ** 3, device="cuda")).reshape(n, n, n)
    solver = tdma.PoissonFFT(n, n, n, dx, dz, a, b, c)
    phi = solver.solve(q, check=True)
    A, B, C = (torch.from_numpy(t).cuda() for t in (a, b, c))
    pmax = phi.abs().max().item()
    for y in (0, 1, 2, 511, 1022, 1023):
        p = phi[y]
        lap = (torch.roll(p, -1, 1) - 2 * p + torch.roll(p, 1, 1)) / dx ** 2
        lap += (torch.roll(p, -1, 0) - 2 * p + torch.roll(p, 1, 0)) / dz ** 2
        lap += B[y] * p
        if y > 0:
            lap += A[y] * phi[y - 1]
        if y < n - 1:
            lap += C[y] * phi[y + 1]
        r = lap - q[y]
        if y == 0:
            r = r - r.mean()
            assert abs(p.mean().item()) <= 1e-9 * pmax
        # normwise backward error: |r| against |operator| |phi|
        scale = (4 / dx ** 2 + 4 / dz ** 2 + abs(A[y].item()) + abs(B[y].item()) + abs(C[y].item())) * pmax
        assert r.abs().max().item() <= 1e-12 * scale
