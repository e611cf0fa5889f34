"""Pins for the oracle's stage-level divide-and-conquer solve in the modified-Thomas form
(Section 2.1: Stage A reduces each partition to its two end unknowns, Stage B solves the reduced
system of the end rows, Stage C recovers the interior).

What fixes them, other than the oracle itself:
  - dense LU (LAPACK) for the whole solve, for every partition count and uneven splits, m = 2
    included, one and two right-hand sides;
  - the relations Stage A returns, checked row by row on the exact solution of the line (dense
    LU): every row of the final form (alpha x_0 + x_i + gamma x_{m-1} = delta, row 0 in x_{-1},
    row m-1 in x_m) and of the forward form (alpha x_0 + x_i + gamma x_{i+1} = delta) must hold
    for the true x -- these relations are what a partition hands to Stage B, so a wrong sign,
    index or dropped term in any step of the sweep breaks one of them;
  - a partition of two rows, where the form is just each row divided by its diagonal;
  - planted mistakes in a copy of the sweep, each caught by the relation pin.
"""
import numpy as np
import pytest

import oracle as O


def _system(rng, lines, n, nrhs=1, dominant=True):
    a = rng.uniform(-1, 0, (lines, n))
    c = rng.uniform(-1, 0, (lines, n))
    if dominant:
        b = 2 + np.abs(a) + np.abs(c) + rng.uniform(0, 1, (lines, n))
    else:  # pivots stay away from zero, no dominance
        b = rng.uniform(1.0, 1.5, (lines, n)) * rng.choice([-1.0, 1.0], (lines, n))
        a, c = a * 0.45, c * 0.45
    d = rng.uniform(-1, 1, (lines, n) + ((nrhs,) if nrhs > 1 else ()))
    return a, b, c, d


def _dense(a, b, c, d):
    if d.ndim == b.ndim + 1:
        return np.stack([O.dense_solve(a, b, c, d[..., q]) for q in range(d.shape[-1])], axis=-1)
    return O.dense_solve(a, b, c, d)


CASES = [(n, p) for n in (2, 3, 4, 5, 7, 16, 31, 33, 64, 65) for p in (1, 2, 3, 4, 8) if n // p >= 2]


@pytest.mark.parametrize("n,p", CASES)
@pytest.mark.parametrize("nrhs", [1, 2])
def test_dc_modified_matches_dense_lu(n, p, nrhs):
    rng = np.random.default_rng(1000 + 10 * n + p + 7 * nrhs)
    a, b, c, d = _system(rng, 40, n, nrhs)
    x = O.dc_modified(a, b, c, d, p)
    ref = _dense(a, b, c, d)
    assert x.shape == ref.shape
    assert np.max(np.abs(x - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("n,p", [(16, 4), (33, 3), (64, 8)])
def test_dc_modified_without_dominance(n, p):
    rng = np.random.default_rng(5 * n + p)
    a, b, c, d = _system(rng, 30, n, dominant=False)
    assert O.rel_l2(O.dc_modified(a, b, c, d, p), O.dense_solve(a, b, c, d)) <= 1e-12


def _check_relations(st, a, b, c, d, x, s, e, tol):
    """Every Stage A relation of partition [s, e) holds for the exact solution x of the line."""
    m = e - s
    xs, xe = x[:, s], x[:, e - 1]
    xm1 = x[:, s - 1] if s > 0 else np.zeros(len(x))
    xp1 = x[:, e] if e < x.shape[1] else np.zeros(len(x))
    al, ga, de = st["alpha"], st["gamma"], st["delta"]
    scale = np.max(np.abs(x)) + np.max(np.abs(de))
    worst = np.max(np.abs(al[:, 0] * xm1 + xs + ga[:, 0] * xe - de[:, 0]))
    for i in range(1, m - 1):
        worst = max(worst, np.max(np.abs(al[:, i] * xs + x[:, s + i] + ga[:, i] * xe - de[:, i])))
    if m >= 2:
        worst = max(worst, np.max(np.abs(al[:, m - 1] * xs + xe + ga[:, m - 1] * xp1 - de[:, m - 1])))
    af, gf, df = st["alpha_fwd"], st["gamma_fwd"], st["delta_fwd"]
    for i in range(1, m):
        nxt = x[:, s + i + 1] if i < m - 1 else xp1
        worst = max(worst, np.max(np.abs(af[:, i] * xs + x[:, s + i] + gf[:, i] * nxt - df[:, i])))
    assert worst <= tol * scale, worst / scale


@pytest.mark.parametrize("n,p", [(2, 1), (3, 1), (9, 3), (10, 4), (64, 8), (65, 8), (40, 20)])
def test_stage_a_relations_hold_for_the_exact_solution(n, p):
    rng = np.random.default_rng(77 + n + p)
    a, b, c, d = _system(rng, 25, n)
    a[:, 0] = 0.0
    c[:, -1] = 0.0
    x = O.dense_solve(a, b, c, d)
    for k, (s, e) in enumerate(O.partition_rows(n, p)):
        st = O.modified_thomas_partition(a[:, s:e], b[:, s:e], c[:, s:e], d[:, s:e])
        _check_relations(st, a, b, c, d, x, s, e, 1e-13)


def test_two_row_partition_is_the_normalised_rows():
    rng = np.random.default_rng(4)
    a, b, c, d = _system(rng, 10, 2)
    st = O.modified_thomas_partition(a, b, c, d)
    assert np.array_equal(st["alpha"], a / b)
    assert np.array_equal(st["gamma"], c / b)
    assert np.array_equal(st["delta"], d / b)


def test_reduced_system_gives_the_true_end_values():
    rng = np.random.default_rng(8)
    n, p = 48, 6
    a, b, c, d = _system(rng, 12, n, nrhs=2)
    a[:, 0] = 0.0
    c[:, -1] = 0.0
    x = _dense(a, b, c, d)
    parts = O.partition_rows(n, p)
    stages = [O.modified_thomas_partition(a[:, s:e], b[:, s:e], c[:, s:e], d[:, s:e]) for s, e in parts]
    sub, sup, rhs = O.reduced_system(stages)
    assert sub.shape == (12, 2 * p) and rhs.shape == (12, 2 * p, 2)
    ends = np.stack([O.dense_solve(sub, np.ones_like(sub), sup, rhs[..., q]) for q in range(2)], axis=-1)
    want = np.stack([x[:, s if j % 2 == 0 else e - 1] for s, e in parts for j in (0, 1)], axis=1)
    assert np.max(np.abs(ends - want)) <= 1e-13 * np.max(np.abs(want))


# ---------------------------------------------------------------- planted mistakes
def _mutant(kind):
    """A copy of the Stage A sweep with one plausible mistake."""
    def stage_a(a, b, c, d):
        m = b.shape[-1]
        al, ga, de = a / b, c / b, d / b
        al, ga, de = al.copy(), ga.copy(), de.copy()
        for i in range(2, m):
            r = 1.0 / (b[:, i] - a[:, i] * ga[:, i - 1])
            al[:, i] = (r if kind == "sign" else -r) * a[:, i] * al[:, i - 1]
            ga[:, i] = r * c[:, i]
            de[:, i] = r * d[:, i] if kind == "drop" else r * (d[:, i] - a[:, i] * de[:, i - 1])
        fwd = {"alpha_fwd": al.copy(), "gamma_fwd": ga.copy(), "delta_fwd": de.copy()}
        for i in range(m - 3, 0, -1):
            j = i + 2 if (kind == "index" and i + 2 < m) else i + 1
            de[:, i] -= ga[:, i] * de[:, j]
            al[:, i] -= ga[:, i] * al[:, j]
            ga[:, i] = -ga[:, i] * ga[:, j]
        if m >= 3:
            r = 1.0 / (1.0 - ga[:, 0] * al[:, 1])
            de[:, 0] = r * (de[:, 0] - ga[:, 0] * de[:, 1])
            if kind == "transpose":
                al[:, 0], ga[:, 0] = -r * ga[:, 0] * ga[:, 1], r * al[:, 0]
            else:
                al[:, 0], ga[:, 0] = r * al[:, 0], -r * ga[:, 0] * ga[:, 1]
        out = {"alpha": al, "gamma": ga, "delta": de}
        out.update(fwd)
        return out
    return stage_a


@pytest.mark.parametrize("kind", ["sign", "drop", "index", "transpose"])
def test_relation_pin_catches_planted_mistakes(kind):
    rng = np.random.default_rng(31)
    n, p = 24, 2
    a, b, c, d = _system(rng, 8, n)
    a[:, 0] = 0.0
    c[:, -1] = 0.0
    x = O.dense_solve(a, b, c, d)
    caught = False
    for s, e in O.partition_rows(n, p):
        st = _mutant(kind)(a[:, s:e], b[:, s:e], c[:, s:e], d[:, s:e])
        try:
            _check_relations(st, a, b, c, d, x, s, e, 1e-13)
        except AssertionError:
            caught = True
    assert caught
