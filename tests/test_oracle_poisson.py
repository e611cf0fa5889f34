"""Pins for the oracle's FFT-based Poisson solve, by the discrete equation itself (applied with
plain finite differences in physical space, not through any transform) and by manufactured
solutions. A planted wrong wavenumber, a wrong axis, a missing pin and a transform scaling
mistake each fail a pin."""
import inspect

import numpy as np
import pytest

import oracle as O
import oracle.tdma_oracle as T
import synth


def _operator(phi, dx, dz, a, b, c):
    """D_xx phi + D_zz phi + D_yy phi by direct differences (periodic x, z; rows (a, b, c) along y)."""
    lap = (np.roll(phi, -1, 2) - 2 * phi + np.roll(phi, 1, 2)) / dx ** 2
    lap += (np.roll(phi, -1, 1) - 2 * phi + np.roll(phi, 1, 1)) / dz ** 2
    yy = b[:, None, None] * phi
    yy[1:] += a[1:, None, None] * phi[:-1]
    yy[:-1] += c[:-1, None, None] * phi[1:]
    return lap + yy


def _problem(ny, nz, nx, seed):
    a, c, b = synth.poisson_coefficients(ny)           # stretched y grid, Neumann ends
    dx, dz = 2 * np.pi / nx, 2 * np.pi / nz
    rng = np.random.default_rng(seed)
    phi = rng.standard_normal((ny, nz, nx))
    phi[0] -= phi[0].mean()                             # the pinned row: zero mode of plane y = 0 is 0
    return phi, _operator(phi, dx, dz, a, b, c), dx, dz, a, b, c


@pytest.mark.parametrize("shape", [(16, 8, 12), (33, 10, 6), (9, 4, 2), (40, 24, 32)])
def test_manufactured_solution_is_recovered(shape):
    phi, q, dx, dz, a, b, c = _problem(*shape, seed=sum(shape))
    got = O.poisson_fft(q, dx, dz, a, b, c)
    assert O.rel_l2(got, phi) < 1e-9  # the y operator's condition number (Neumann, stretched) ~ 1e5


def test_solution_satisfies_the_discrete_equation():
    ny, nz, nx = 24, 12, 16
    a, c, b = synth.poisson_coefficients(ny)
    dx, dz = 0.3, 0.7
    q = np.random.default_rng(3).standard_normal((ny, nz, nx))
    phi = O.poisson_fft(q, dx, dz, a, b, c)
    r = _operator(phi, dx, dz, a, b, c) - q
    # every equation holds except row 0 of the (0, 0) mode, which the pin replaced: the residual
    # is a constant over the plane y = 0 and zero elsewhere
    assert np.abs(r[1:]).max() < 1e-10 * np.abs(q).max()
    assert np.abs(r[0] - r[0].mean()).max() < 1e-10 * np.abs(q).max()
    assert abs(phi[0].mean()) < 1e-12                  # the pin itself


def test_unpinned_dirichlet_operator():
    # Dirichlet ends make D_yy nonsingular: nothing is pinned and every equation holds
    ny, nz, nx = 20, 8, 10
    a = np.full(ny, 1.0)
    c = np.full(ny, 1.0)
    b = np.full(ny, -2.0)
    q = np.random.default_rng(4).standard_normal((ny, nz, nx))
    phi = O.poisson_fft(q, 0.5, 0.25, a, b, c, pin_zero_mode=False)
    assert np.abs(_operator(phi, 0.5, 0.25, a, b, c) - q).max() < 1e-10 * np.abs(q).max()


def _mutant(old, new):
    src = inspect.getsource(T.poisson_fft)
    assert old in src
    ns = dict(T.__dict__)
    exec(src.replace(old, new), ns)
    return ns["poisson_fft"]


@pytest.mark.parametrize("old,new", [
    ("np.arange(nkx) / nx", "np.arange(nkx) / (2 * nx)"),            # wrong wavenumber
    ("k2z[:, None] + k2x[None, :]", "k2z[:, None] + 0.0 * k2x[None, :]"),  # x wavenumber dropped
    ("lines_b[0, 0], lines_c[0, 0] = 1.0, 0.0", "pass"),                # pin missing
    ("D[0, 0, :] = 0.0", "D[0, 1, :] = 0.0"),                          # pin on the wrong row
    ("return np.fft.irfft2(Phi, s=(nz, nx), axes=(1, 2))", "return np.fft.irfft2(Phi, s=(nz, nx), axes=(1, 2)) * 2"),
])
def test_pins_catch_planted_mistakes(old, new):
    bad = _mutant(old, new)
    phi, q, dx, dz, a, b, c = _problem(16, 8, 12, seed=36)
    with np.errstate(all="ignore"):
        got = bad(q, dx, dz, a, b, c)
    assert not (np.all(np.isfinite(got)) and O.rel_l2(got, phi) < 1e-9)
