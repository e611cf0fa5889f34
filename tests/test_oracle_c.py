"""Pins for the C Thomas oracle (oracle/thomas_c.c), the solve the CPU baseline times on all host
cores: dense LU and exact rational arithmetic, the sine-mode closed form of tridiag(-r, 1 + 2r, -r)
(DST-I), strided layouts of a 3D grid along every axis, in-place solves, and the result being
independent of the thread count. Also bit for bit equal to the numpy sweep, which performs the same
IEEE operations in the same order."""
from fractions import Fraction

import numpy as np
import pytest
from scipy.fft import dst, idst

import oracle as O
from oracle import c_thomas as C


def _system(rng, lines, n):
    a = rng.uniform(-1, 0, (lines, n))
    c = rng.uniform(-1, 0, (lines, n))
    b = 2 + np.abs(a) + np.abs(c) + rng.uniform(0, 1, (lines, n))
    d = rng.uniform(-1, 1, (lines, n))
    return a, b, c, d


@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 33, 64])
def test_c_thomas_matches_dense_lu(n):
    rng = np.random.default_rng(500 + n)
    a, b, c, d = _system(rng, 61, n)
    x = C.thomas(a, b, c, d)
    ref = O.dense_solve(a, b, c, d)
    assert np.max(np.abs(x - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_c_thomas_matches_exact_rational():
    rng = np.random.default_rng(12)
    for trial in range(10):
        n = 9
        a = rng.integers(-3, 4, n).astype(float)
        c = rng.integers(-3, 4, n).astype(float)
        b = np.abs(a) + np.abs(c) + rng.integers(1, 4, n)
        d = rng.integers(-9, 10, n).astype(float)
        # exact: Cramer-free elimination over the rationals
        cp, dp = [Fraction(0)] * n, [Fraction(0)] * n
        cp[0], dp[0] = Fraction(c[0]) / Fraction(b[0]), Fraction(d[0]) / Fraction(b[0])
        for i in range(1, n):
            w = Fraction(b[i]) - Fraction(a[i]) * cp[i - 1]
            cp[i] = Fraction(c[i]) / w
            dp[i] = (Fraction(d[i]) - Fraction(a[i]) * dp[i - 1]) / w
        xs = [Fraction(0)] * n
        xs[-1] = dp[-1]
        for i in range(n - 2, -1, -1):
            xs[i] = dp[i] - cp[i] * xs[i + 1]
        ref = np.array([float(v) for v in xs])
        x = C.thomas(a[None], b[None], c[None], d[None])[0]
        assert np.allclose(x, ref, rtol=1e-14, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("n,r", [(31, 0.5), (64, 2.0)])
def test_c_thomas_sine_modes(n, r):
    rng = np.random.default_rng(n)
    d = rng.uniform(-1, 1, (5, n))
    lam = 1 + 4 * r * np.sin(np.pi * np.arange(1, n + 1) / (2 * (n + 1))) ** 2
    ref = idst(dst(d, type=1, axis=-1) / lam, type=1, axis=-1)
    A = np.full((5, n), -r)
    x = C.thomas(A, np.full((5, n), 1 + 2 * r), A, d)
    assert O.rel_l2(x, ref) <= 1e-13


def test_c_thomas_is_bitwise_the_numpy_sweep_and_thread_independent():
    rng = np.random.default_rng(3)
    a, b, c, d = _system(rng, 203, 77)
    ref = O.thomas(a, b, c, d)
    for threads in (1, 2, 3, max(1, C.max_threads())):
        assert np.array_equal(C.thomas(a, b, c, d, threads=threads), ref)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_c_thomas_strided_grid_axes_and_in_place(axis):
    rng = np.random.default_rng(40 + axis)
    shape = (12, 10, 9)  # [z][y][x]
    a, b, c, d = (rng.uniform(-1, 0, shape), None, rng.uniform(-1, 0, shape), rng.uniform(-1, 1, shape))
    b = 2 + np.abs(a) + np.abs(c)
    n = shape[axis]
    lines = np.moveaxis(np.stack([a, b, c, d]), axis + 1, -1).reshape(4, -1, n)
    ref = O.thomas(*lines)
    x = d.copy()
    if axis == 2:  # contiguous lines
        C.solve_strided(n, a.size // n, 1, n, a, b, c, x, x)
        got = x.reshape(-1, n)
    elif axis == 0:  # adjacent lines, rows one plane apart
        C.solve_strided(n, a.size // n, shape[1] * shape[2], 1, a, b, c, x, x)
        got = np.moveaxis(x, 0, -1).reshape(-1, n)
    else:  # y lines: handled one z-plane at a time (adjacent lines, rows one x-row apart)
        for z in range(shape[0]):
            xp = x[z].copy()
            C.solve_strided(n, shape[2], shape[2], 1, a[z], b[z], c[z], xp, xp)
            x[z] = xp
        got = np.moveaxis(x, 1, -1).reshape(-1, n)
    assert np.array_equal(got, ref)
