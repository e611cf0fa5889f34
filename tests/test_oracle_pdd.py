"""Pins for the oracle's parallel diagonally dominant (PDD) approximation.

PDD is not the exact solve, so it is pinned by what the method fixes: with one partition it is
the Thomas solve; when the partitions are decoupled (a at every partition start and c at every
partition end zero) it is exact; every row away from a partition boundary holds exactly (the
correction of Stage A is exact inside a partition, only the interface values are approximate);
and on a Toeplitz diagonally dominant line the error falls geometrically with the partition
length, at the rate rho = (b - sqrt(b^2 - 4 a c)) / (2 |c|) of the spikes' decay. The mutation
tests plant plausible mistakes in copies of the oracle and check that the pins catch each one.
"""
import inspect

import numpy as np
import pytest

import oracle as O
import oracle.tdma_oracle as T


def _system(rng, lines, n):
    a = rng.uniform(-1, 0, (lines, n))
    c = rng.uniform(-1, 0, (lines, n))
    b = 2 + np.abs(a) + np.abs(c) + rng.uniform(0, 1, (lines, n))
    d = rng.uniform(-1, 1, (lines, n))
    return a, b, c, d


def _boundary_rows(n, p):
    rows = set()
    for k, (s, e) in enumerate(O.partition_rows(n, p)):
        if k > 0:
            rows.add(s)
        if k < p - 1:
            rows.add(e - 1)
    return sorted(rows)


def _toeplitz_error(solve, m, p=6, lines=3, seed=5):
    # tridiag(-1, 2.5, -1): spikes decay as rho^t with rho = 0.5
    n = m * p
    a = np.full((lines, n), -1.0)
    c = np.full((lines, n), -1.0)
    b = np.full((lines, n), 2.5)
    d = np.random.default_rng(seed).uniform(-1, 1, (lines, n))
    x = O.dense_solve(a, b, c, d)
    return np.abs(solve(a, b, c, d, p) - x).max() / np.abs(x).max()


def _pins_hold(pdd):
    """True if every pin below holds for the given implementation."""
    rng = np.random.default_rng(21)
    a, b, c, d = _system(rng, 8, 40)
    if O.rel_l2(pdd(a, b, c, d, 1), O.dense_solve(a, b, c, d)) > 1e-13:
        return False
    r = O.residual(a, b, c, d, pdd(a, b, c, d, 5))
    interior = np.setdiff1d(np.arange(40), _boundary_rows(40, 5))
    if np.abs(r[:, interior]).max() > 1e-13:
        return False
    a, b, c, d = _system(rng, 8, 160)  # nonsymmetric, partitions of 40 rows: spike tips < 1e-12
    if O.rel_l2(pdd(a, b, c, d, 4), O.dense_solve(a, b, c, d)) > 1e-12:
        return False
    errs = [_toeplitz_error(pdd, m) for m in (8, 16, 24)]
    if any(e > 0.5 ** m for e, m in zip(errs, (8, 16, 24))):
        return False
    return all(2 ** 6 <= errs[i] / errs[i + 1] <= 2 ** 11 for i in range(2))


def test_one_partition_is_the_exact_solve():
    rng = np.random.default_rng(1)
    for n in (1, 2, 3, 17, 64):
        a, b, c, d = _system(rng, 20, n)
        assert O.rel_l2(O.pdd(a, b, c, d, 1), O.dense_solve(a, b, c, d)) < 1e-14


@pytest.mark.parametrize("n,p", [(16, 4), (33, 8), (40, 5), (9, 4)])
def test_decoupled_partitions_are_exact(n, p):
    rng = np.random.default_rng(n + p)
    a, b, c, d = _system(rng, 20, n)
    for k, (s, e) in enumerate(O.partition_rows(n, p)):
        a[:, s] = 0.0
        c[:, e - 1] = 0.0
    assert O.rel_l2(O.pdd(a, b, c, d, p), O.dense_solve(a, b, c, d)) < 1e-14


@pytest.mark.parametrize("n,p", [(40, 5), (64, 8), (33, 8), (100, 3)])
def test_rows_off_the_partition_boundaries_hold_exactly(n, p):
    rng = np.random.default_rng(3 * n + p)
    a, b, c, d = _system(rng, 30, n)
    # weakly dominant lines so that the approximation is visible at the boundaries
    b = np.abs(a) + np.abs(c) + 0.05
    x = O.pdd(a, b, c, d, p)
    r = O.residual(a, b, c, d, x)
    bnd = _boundary_rows(n, p)
    interior = np.setdiff1d(np.arange(n), bnd)
    scale = np.abs(d).max() + np.abs(x).max() * 4
    assert np.abs(r[:, interior]).max() < 1e-14 * scale * n
    assert np.abs(r[:, bnd]).max() > 1e-8  # the dropped couplings are really dropped


def test_error_decays_geometrically_with_the_partition_length():
    errs = {m: _toeplitz_error(O.pdd, m) for m in (8, 16, 24, 32)}
    for m, e in errs.items():
        assert e <= 0.5 ** m  # below the spike tip rho^m
    for m in (8, 16, 24):
        assert 2 ** 6 <= errs[m] / errs[m + 8] <= 2 ** 11  # about rho^-8 = 256 per 8 rows
    assert _toeplitz_error(O.pdd, 64) < 1e-16 * 64


@pytest.mark.parametrize("p", [2, 4, 8])
def test_long_partitions_of_dominant_lines_reach_the_exact_solution(p):
    # b >= 2 + |a| + |c| and |a|, |c| < 1: the spikes fall by at least 3x per row, so with 40
    # rows per partition the dropped couplings are far below rounding
    rng = np.random.default_rng(40 + p)
    a, b, c, d = _system(rng, 16, 40 * p)
    assert O.rel_l2(O.pdd(a, b, c, d, p), O.dense_solve(a, b, c, d)) < 1e-14


def test_pins_hold_for_the_oracle():
    assert _pins_hold(O.pdd)


def _mutant(old, new):
    src = inspect.getsource(T.pdd)
    assert old in src
    ns = dict(T.__dict__)
    exec(src.replace(old, new), ns)
    return ns["pdd"]


@pytest.mark.parametrize("old,new", [
    ("x[:, s:e] -= w[:, s:e] * y2[:, k][:, None]", "x[:, s:e] -= w[:, s:e] * y1[:, k][:, None]"),
    ("x[:, s:e] -= v[:, s:e] * y1[:, k - 1][:, None]", "x[:, s:e] -= v[:, s:e] * y2[:, k - 1][:, None]"),
    ("det = 1.0 - wl * vr", "det = 1.0 + wl * vr"),
    ("eL = parts[k][1] - 1", "eL = parts[k][1] - 2"),
    ("rhs[:, 0] = a[:, s]", "rhs[:, 0] = c[:, s]"),
    ("rhs[:, -1] = c[:, e - 1]", "rhs[:, -1] = a[:, e - 1]"),
    ("y2[:, k] = (xt[:, sR] - vr * xt[:, eL]) / det", "y2[:, k] = (xt[:, sR] - vr * xt[:, eL])"),
    ("y1[:, k] = (xt[:, eL] - wl * xt[:, sR]) / det", "y1[:, k] = (xt[:, eL] - vr * xt[:, sR]) / det"),
    ("sR = parts[k + 1][0]", "sR = parts[k + 1][0] + 1"),
])
def test_pins_catch_planted_mistakes(old, new):
    assert not _pins_hold(_mutant(old, new))
