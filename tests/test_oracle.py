"""Pins for the CPU oracle against facts fixed by mathematics, not by the oracle itself.

Dense LU (LAPACK) and exact rational elimination pin the Thomas sweep; the closed-form sine
eigenvectors of tridiag(-r, 1+2r, -r) (DST-I, a library routine) pin the constant-coefficient
case and the 3D x->y->z sweep; manufactured solutions and the backward-error bound of Thomas
on diagonally dominant matrices pin accuracy; central finite differences and the adjoint
identity pin the gradients. The mutation tests plant plausible mistakes in copies of the
oracle and check that the pins catch each one.
"""
from fractions import Fraction

import numpy as np
import pytest
from scipy.fft import dst, dstn, idst, idstn

import oracle as O

U64 = np.finfo(np.float64).eps / 2


def dd_system(rng, lines, n, dominant=True):
    a = rng.uniform(-1, 0, (lines, n))
    c = rng.uniform(-1, 0, (lines, n))
    b = 2 + np.abs(a) + np.abs(c) + rng.uniform(0, 1, (lines, n)) if dominant else \
        rng.uniform(1.0, 1.5, (lines, n)) * rng.choice([-1, 1], (lines, n))
    d = rng.uniform(-1, 1, (lines, n))
    return a, b, c, d


# ---------------------------------------------------------------- Thomas vs brute force
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 16, 31, 32, 33, 63, 64])
def test_thomas_matches_dense_lu(n):
    rng = np.random.default_rng(100 + n)
    a, b, c, d = dd_system(rng, 200, n)
    x = O.thomas(a, b, c, d)
    ref = O.dense_solve(a, b, c, d)
    assert np.max(np.abs(x - ref) / np.maximum(1e-300, np.abs(ref).max(axis=1, keepdims=True))) < 1e-13


def _exact_solve(a, b, c, d):
    """Gaussian elimination in exact rational arithmetic (no rounding at all)."""
    n = len(b)
    A = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        A[i][i] = Fraction(b[i])
        if i > 0:
            A[i][i - 1] = Fraction(a[i])
        if i < n - 1:
            A[i][i + 1] = Fraction(c[i])
    r = [Fraction(v) for v in d]
    for k in range(n):
        p = max(range(k, n), key=lambda i: abs(A[i][k]))
        A[k], A[p] = A[p], A[k]
        r[k], r[p] = r[p], r[k]
        for i in range(k + 1, n):
            f = A[i][k] / A[k][k]
            if f:
                for j in range(k, n):
                    A[i][j] -= f * A[k][j]
                r[i] -= f * r[k]
    x = [Fraction(0)] * n
    for i in range(n - 1, -1, -1):
        s = r[i] - sum(A[i][j] * x[j] for j in range(i + 1, n))
        x[i] = s / A[i][i]
    return np.array([float(v) for v in x])


@pytest.mark.parametrize("n", [1, 2, 3, 6, 12])
def test_thomas_matches_exact_rational(n):
    # small integer coefficients, including a non-dominant (but nonsingular, pivot-free) case
    rng = np.random.default_rng(7 * n + 1)
    for trial in range(20):
        a = rng.integers(-3, 4, n).astype(float)
        c = rng.integers(-3, 4, n).astype(float)
        b = np.abs(a) + np.abs(c) + rng.integers(1, 4, n)
        if trial % 2:
            b = b * rng.choice([-1.0, 1.0], n)
        d = rng.integers(-9, 10, n).astype(float)
        x = O.thomas(a, b, c, d)
        ref = _exact_solve(a, b, c, d)
        assert np.allclose(x, ref, rtol=1e-14, atol=1e-14 * np.abs(ref).max())


def test_thomas_multiple_rhs_axis():
    rng = np.random.default_rng(3)
    a, b, c, _ = dd_system(rng, 17, 40)
    d2 = rng.normal(size=(17, 40, 2))
    x2 = O.thomas(a, b, c, d2)
    for k in range(2):
        assert np.array_equal(x2[..., k], O.thomas(a, b, c, d2[..., k]))


def test_first_a_and_last_c_are_ignored():
    rng = np.random.default_rng(4)
    a, b, c, d = dd_system(rng, 5, 9)
    a2, c2 = a.copy(), c.copy()
    a2[:, 0] = 123.0
    c2[:, -1] = -77.0
    assert np.array_equal(O.thomas(a, b, c, d), O.thomas(a2, b, c2, d))


# ---------------------------------------------------------------- divide and conquer
@pytest.mark.parametrize("n,p", [(2, 1), (4, 2), (5, 2), (7, 3), (16, 4), (31, 4), (33, 8), (64, 8),
                                 (65, 8), (64, 1), (64, 4), (9, 4), (40, 16)])
def test_dc_spike_matches_dense_lu(n, p):
    rng = np.random.default_rng(n * 31 + p)
    a, b, c, d = dd_system(rng, 50, n)
    x = O.dc_spike(a, b, c, d, p)
    ref = O.dense_solve(a, b, c, d)
    assert O.rel_l2(x, ref) < 1e-13


def test_partition_rows_rule():
    assert O.partition_rows(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert O.partition_rows(64, 4) == [(0, 16), (16, 32), (32, 48), (48, 64)]
    with pytest.raises(ValueError):
        O.partition_rows(7, 4)  # a part of one row
    b = O.partition_rows(16384, 512)
    assert b[-1][1] == 16384 and all(e - s == 32 for s, e in b)


def test_dc_interface_equations_hold_for_true_solution():
    # Invariant of Stage B: every interface row x_i + v_i x_{e_{k-1}} + w_i x_{s_{k+1}} = x~_i
    # holds for the true x. Checked through the end result: the dc solution reproduces d.
    rng = np.random.default_rng(11)
    a, b, c, d = dd_system(rng, 20, 48)
    x = O.dc_spike(a, b, c, d, 6)
    r = O.residual(a, b, c, d, x)
    assert np.abs(r).max() < 1e-14 * np.abs(d).max() * 48


# ---------------------------------------------------------------- closed forms
def _dst_solve(d, r):
    n = d.shape[-1]
    k = np.arange(1, n + 1)
    lam = 1.0 + 4.0 * r * np.sin(np.pi * k / (2.0 * (n + 1))) ** 2
    return idst(dst(d, type=1, axis=-1) / lam, type=1, axis=-1)


@pytest.mark.parametrize("n,r", [(8, 0.5), (64, 0.5), (512, 0.5), (100, 3.0)])
def test_constant_coefficient_sine_modes(n, r):
    rng = np.random.default_rng(n)
    d = rng.uniform(-1, 1, (6, n))
    a = np.full((6, n), -r)
    c = np.full((6, n), -r)
    b = np.full((6, n), 1 + 2 * r)
    assert O.rel_l2(O.thomas(a, b, c, d), _dst_solve(d, r)) < 1e-13


def test_adi_xyz_sweep_closed_form():
    # three successive line solves along x, y, z of tridiag(-r, 1+2r, -r) invert the
    # product operator, diagonal in the 3D DST-I basis with eigenvalues lam_i lam_j lam_k
    rng = np.random.default_rng(5)
    nz, ny, nx, r = 12, 10, 14, 0.5
    d = rng.uniform(-1, 1, (nz, ny, nx))
    u = d.copy()
    for axis in (2, 1, 0):
        v = np.moveaxis(u, axis, -1)
        n = v.shape[-1]
        a = np.full(v.shape, -r)
        b = np.full(v.shape, 1 + 2 * r)
        u = np.moveaxis(O.thomas(a, b, a, v), -1, axis)
    lam = [1 + 4 * r * np.sin(np.pi * np.arange(1, m + 1) / (2 * (m + 1))) ** 2 for m in (nz, ny, nx)]
    L = lam[0][:, None, None] * lam[1][None, :, None] * lam[2][None, None, :]
    ref = idstn(dstn(d, type=1) / L, type=1)
    assert O.rel_l2(u, ref) < 1e-13


# ---------------------------------------------------------------- accuracy bounds
@pytest.mark.parametrize("n", [8, 64, 1024])
def test_manufactured_solution_and_backward_error(n):
    rng = np.random.default_rng(n + 9)
    a, b, c, _ = dd_system(rng, 64, n)
    x_true = rng.uniform(-1, 1, (64, n))
    d = b * x_true
    d[:, 1:] += a[:, 1:] * x_true[:, :-1]
    d[:, :-1] += c[:, :-1] * x_true[:, 1:]
    x = O.thomas(a, b, c, d)
    # forward error: ||x - x_true|| <= 10 n u kappa with kappa <= (max row sum)/(min dominance margin)
    kappa = np.max(b + 2) / np.min(b - np.abs(a) - np.abs(c))
    assert O.rel_l2(x, x_true) < 10 * n * U64 * kappa
    # backward error of Thomas on diagonally dominant A (Higham, Accuracy and Stability, ch. 9)
    r = O.residual(a, b, c, d, x)
    normA = np.max(np.abs(a) + np.abs(b) + np.abs(c))
    be = np.linalg.norm(r, axis=1) / (normA * np.linalg.norm(x, axis=1) + np.linalg.norm(d, axis=1))
    assert be.max() < 4 * n * U64


def test_extended_precision_sweep_agrees_and_is_tighter():
    from synth import poisson_coefficients
    a, c, b0 = poisson_coefficients(1024, 2.0)
    rng = np.random.default_rng(2)
    # a well-conditioned high-wavenumber line: both sweeps agree to rounding
    d = rng.normal(size=1024)
    x64 = O.thomas(a, b0 - 2e5, c, d)
    xe = O.thomas_ext(a, b0 - 2e5, c, d)
    assert O.rel_l2(x64, xe) < 1e-14
    # the pinned zero mode (kappa ~ 1e9): extended precision has a smaller residual
    pa, pb, pc = a.copy(), b0.copy(), c.copy()
    pb[0], pc[0] = 1.0, 0.0
    d[0] = 0.0
    x64 = O.thomas(pa, pb, pc, d)
    xe = O.thomas_ext(pa, pb, pc, d)
    r64 = np.abs(O.residual(pa, pb, pc, d, x64, dtype=np.longdouble)).max()
    re = np.abs(O.residual(pa, pb, pc, d, xe, dtype=np.longdouble)).max()
    assert re <= r64
    assert O.rel_l2(x64, xe) < 1e-10


def _exact_thomas(a, b, c, d):
    """The Thomas recurrences in exact rational arithmetic (every float input is a rational)."""
    n = len(b)
    a, b, c, d = ([Fraction(float(v)) for v in t] for t in (a, b, c, d))
    cp, dp = [Fraction(0)] * n, [Fraction(0)] * n
    cp[0], dp[0] = c[0] / b[0], d[0] / b[0]
    for i in range(1, n):
        w = b[i] - a[i] * cp[i - 1]
        cp[i] = c[i] / w if i < n - 1 else Fraction(0)
        dp[i] = (d[i] - a[i] * dp[i - 1]) / w
    x = [Fraction(0)] * n
    x[-1] = dp[-1]
    for i in range(n - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    return np.array([float(v) for v in x])


def _pinned_zero_mode(n, seed):
    from synth import poisson_coefficients
    a, c, b = poisson_coefficients(n, 2.0)
    b, c = b.copy(), c.copy()
    b[0], c[0] = 1.0, 0.0
    d = np.random.default_rng(seed).normal(size=n)
    d[0] = 0.0
    return a, b, c, d


@pytest.mark.parametrize("n,seed", [(64, 1), (96, 2), (128, 3), (256, 4)])
def test_extended_precision_is_tighter_than_fp64_against_exact_rationals(n, seed):
    # The pinned Poisson zero mode (Neumann ends on the tanh-stretched grid, row 0 replaced by
    # x_0 = 0) shrunk to n rows: badly conditioned enough that FP64 elimination is visibly off the
    # exact solution, which exact rational arithmetic gives. The extended sweep must be at least
    # 10x closer; it fails if it silently runs in float64.
    if np.finfo(np.longdouble).nmant <= 52:
        pytest.skip("numpy.longdouble is float64 on this platform: no extended precision to pin")
    a, b, c, d = _pinned_zero_mode(n, seed)
    exact = _exact_thomas(a, b, c, d)
    e64 = O.rel_l2(O.thomas(a, b, c, d), exact)
    eext = O.rel_l2(O.thomas_ext(a, b, c, d), exact)
    assert e64 > 5e-15  # the case discriminates: FP64 is measurably off
    assert eext <= e64 / 10
    assert eext <= 4e-16  # only the final rounding to float64 is left


def test_extended_pin_catches_a_float64_sweep(monkeypatch):
    # planted mistake: the extended sweep loses its precision (dtype dropped to float64)
    import oracle.tdma_oracle as T
    monkeypatch.setattr(T, "thomas_ext", lambda a, b, c, d: T.thomas(a, b, c, d).astype(np.float64))
    a, b, c, d = _pinned_zero_mode(128, 3)
    exact = _exact_thomas(a, b, c, d)
    e64 = O.rel_l2(O.thomas(a, b, c, d), exact)
    assert not O.rel_l2(T.thomas_ext(a, b, c, d), exact) <= e64 / 10


# ---------------------------------------------------------------- gradients
def test_adjoint_grads_match_central_differences():
    rng = np.random.default_rng(21)
    L, n = 3, 12
    a, b, c, d = dd_system(rng, L, n)
    w = rng.normal(size=(L, n))
    def loss(a_, b_, c_, d_):
        return float(np.sum(w * O.thomas(a_, b_, c_, d_)))
    x = O.thomas(a, b, c, d)
    ga, gb, gc, gd = O.adjoint_grads(a, b, c, x, w)
    for arr, g, skip in ((a, ga, 0), (b, gb, None), (c, gc, n - 1), (d, gd, None)):
        for l in range(L):
            for i in range(n):
                base = arr[l, i]
                h = 1e-6 * max(1.0, abs(base))
                arr[l, i] = base + h
                fp = loss(a, b, c, d)
                arr[l, i] = base - h
                fm = loss(a, b, c, d)
                arr[l, i] = base
                fd = (fp - fm) / (2 * h)
                if skip is not None and i == skip:
                    assert g[l, i] == 0.0 and abs(fd) < 1e-8
                else:
                    assert abs(fd - g[l, i]) < 1e-7 * max(1.0, abs(g[l, i]))


def test_adjoint_identity():
    rng = np.random.default_rng(22)
    a, b, c, d = dd_system(rng, 30, 77)
    w = rng.normal(size=(30, 77))
    lhs = np.sum(w * O.thomas(a, b, c, d), axis=1)
    at, bt, ct = O.transpose_coefficients(a, b, c)
    rhs = np.sum(O.thomas(at, bt, ct, w) * d, axis=1)
    assert np.max(np.abs(lhs - rhs) / np.abs(lhs).max()) < 1e-13
    # A^T really is the transpose
    assert np.array_equal(O.dense_matrix(at, bt, ct)[0], O.dense_matrix(a, b, c)[0].T)


def test_ragged_matches_per_line():
    rng = np.random.default_rng(23)
    lengths = np.array([5, 17, 5, 2, 33])
    offsets = np.concatenate([[0], np.cumsum(lengths)[:-1]])
    tot = lengths.sum()
    a, b, c, d = (v[0] for v in dd_system(rng, 1, tot))
    out = O.thomas_ragged(a, b, c, d, offsets, lengths)
    for li, (o, n) in enumerate(zip(offsets, lengths)):
        s = slice(o, o + n)
        assert np.allclose(out[li], O.dense_solve(a[s], b[s], c[s], d[s]), rtol=1e-13, atol=1e-14)


# ---------------------------------------------------------------- planted mistakes
def _thomas_mutant(kind):
    def solve(a, b, c, d):
        n = b.shape[-1]
        cp = np.zeros_like(b)
        dp = np.zeros_like(d)
        cp[..., 0] = c[..., 0] / b[..., 0]
        dp[..., 0] = d[..., 0] / b[..., 0]
        for i in range(1, n):
            ai = a[..., i - 1] if kind == "index" else a[..., i]
            w = b[..., i] + ai * cp[..., i - 1] if kind == "sign" else b[..., i] - ai * cp[..., i - 1]
            cp[..., i] = c[..., i] / w if i < n - 1 else 0.0
            dp[..., i] = d[..., i] / w if kind == "drop" else (d[..., i] - ai * dp[..., i - 1]) / w
        x = np.zeros_like(d)
        x[..., -1] = dp[..., -1]
        for i in range(n - 2, -1, -1):
            cpi = c[..., i] if kind == "transpose" else cp[..., i]
            x[..., i] = dp[..., i] - cpi * x[..., i + 1]
        return x
    return solve


@pytest.mark.parametrize("kind", ["sign", "index", "drop", "transpose"])
def test_pins_catch_planted_mistakes(kind):
    rng = np.random.default_rng(99)
    a, b, c, d = dd_system(rng, 20, 16)
    bad = _thomas_mutant(kind)(a, b, c, d)
    assert O.rel_l2(bad, O.dense_solve(a, b, c, d)) > 1e-6
    if kind == "index":
        return  # a shifted index is invisible when all coefficients are equal
    # the constant-coefficient closed form catches the others as well
    r = 0.5
    ac = np.full((4, 16), -r)
    bc = np.full((4, 16), 1 + 2 * r)
    dc = rng.uniform(-1, 1, (4, 16))
    assert O.rel_l2(_thomas_mutant(kind)(ac, bc, ac.copy(), dc), _dst_solve(dc, r)) > 1e-6


def test_pins_catch_bad_partitioning(monkeypatch):
    rng = np.random.default_rng(98)
    a, b, c, d = dd_system(rng, 10, 24)
    good = O.partition_rows
    def overlapping(n, p):  # a plausible off-by-one in the split
        return [(s, min(n, e + 1)) if k < p - 1 else (s, e) for k, (s, e) in enumerate(good(n, p))]
    import oracle.tdma_oracle as T
    monkeypatch.setattr(T, "partition_rows", overlapping)
    assert O.rel_l2(T.dc_spike(a, b, c, d, 4), O.dense_solve(a, b, c, d)) > 1e-6
