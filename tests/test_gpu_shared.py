"""Lines that share one set of coefficients (1D a, b, c broadcast to every line, no per-line
shift): the factorisation is computed once per solve and every line runs the right-hand-side
recurrences only. Parity against the oracle's Thomas sweep on the broadcast arrays, for both
precisions, one and two right-hand sides, every axis of a grid, the adjoint solve with the
coefficient gradients summed over lines, and the FP64 solve with the exact-residual correction."""
import os

import numpy as np
import pytest
import torch

import oracle as O
from parity import rel_err
import synth
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu

SHARED = 10   # TDMA_VARIANT_SHARED
THOMAS = 1    # TDMA_VARIANT_THOMAS
TOL = {"f64": 1e-12, "f32": 1e-5}


def _coefficients(n, seed, dtype=torch.float64):
    # nonsymmetric, diagonally dominant, as the per-element general coefficients
    g = synth.grid_general((n, 1), 0, seed)
    a, b, c = (g[k][:, 0].contiguous() for k in ("a", "b", "c"))
    return tuple(t.to(dtype).cuda() for t in (a, b, c))


def _rhs(shape, seed, dtype, nrhs):
    full = shape + ((nrhs,) if nrhs > 1 else ())
    d = synth.normal(seed, synth.AID["d"], torch.arange(int(np.prod(full)))).reshape(full)
    return d.to(dtype).cuda()


def _lines(t, axis, nrhs):
    """[lines, n(, nrhs)] view of a grid for the oracle."""
    t = t.detach().double().cpu()
    if nrhs == 1:
        return synth.line_view(t, axis).numpy()
    return np.stack([synth.line_view(t[..., r], axis).numpy() for r in range(nrhs)], axis=-1)


def _plan(d, axis, precision, nrhs, partitions=1, refine_kappa=0.0):
    return tdma.Plan(*tdma.line_layout(d, axis, nrhs=nrhs), precision=precision, partitions=partitions, nrhs=nrhs,
                     coef_broadcast=True, refine_kappa=refine_kappa)


def _oracle(a, b, c, d, axis, nrhs, ext=False):
    D = _lines(d, axis, nrhs)
    L = D.shape[0]
    A, B, C = (np.broadcast_to(t.double().cpu().numpy(), (L, t.numel())) for t in (a, b, c))
    return (O.thomas_ext if ext else O.thomas)(A, B, C, D)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("nrhs", [1, 2])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_shared_matches_oracle_every_axis(precision, nrhs, axis):
    shape = (48, 40, 36)  # 1440 - 1920 lines: several blocks and a partial last one
    n = shape[axis]
    dt = torch.float64 if precision == "f64" else torch.float32
    a, b, c = _coefficients(n, 21 + axis, dt)
    d = _rhs(shape, 22 + axis, dt, nrhs)
    plan = _plan(d, axis, precision, nrhs)
    assert plan.config["variant"] == SHARED
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    assert plan.last_error()[0] == 0
    assert rel_err(_lines(x, axis, nrhs), _oracle(a, b, c, d, axis, nrhs)) <= TOL[precision]


@pytest.mark.parametrize("shape,nrhs", [((5, 7, 45), 1), ((5, 7, 45), 2), ((3, 11, 2), 1), ((1, 9, 1000), 2),
                                         ((2, 1, 33), 1), ((64, 33, 31), 2)])
def test_shared_unit_stride_ragged_chunks_and_partial_warps(shape, nrhs):
    # lines along the contiguous axis go through shared memory in chunks of 32 values per line,
    # one warp per 32 lines: line counts that leave a warp partly empty and lengths whose last
    # chunk is partial
    n = shape[2]
    a, b, c = _coefficients(n, 80 + n)
    d = _rhs(shape, 81, torch.float64, nrhs)
    plan = _plan(d, 2, "f64", nrhs)
    assert plan.config["variant"] == SHARED
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    assert plan.last_error()[0] == 0
    ref = _oracle(a, b, c, d, 2, nrhs)
    assert rel_err(_lines(x, 2, nrhs), ref) <= 1e-12
    plan.solve(a, b, c, d, d)  # x over d
    assert rel_err(_lines(d, 2, nrhs), ref) <= 1e-12


@pytest.mark.parametrize("n", [2, 3, 5, 1000])
def test_shared_short_and_long_lines(n):
    a, b, c = _coefficients(n, 30 + n)
    d = _rhs((n, 131), 31, torch.float64, 1)
    plan = _plan(d, 0, "f64", 1)
    assert plan.config["variant"] == SHARED
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    assert rel_err(_lines(x, 0, 1), _oracle(a, b, c, d, 0, 1)) <= 1e-12


def test_shared_in_place_and_repeated():
    n = 200
    a, b, c = _coefficients(n, 40)
    d = _rhs((n, 300), 41, torch.float64, 2)
    ref = _oracle(a, b, c, d, 0, 2)
    plan = _plan(d, 0, "f64", 2)
    x1 = torch.empty_like(d)
    plan.solve(a, b, c, d, x1)
    x2 = torch.empty_like(d)
    plan.solve(a, b, c, d, x2)
    assert torch.equal(x1, x2)
    plan.solve(a, b, c, d, d)  # x over d
    assert rel_err(_lines(d, 0, 2), ref) <= 1e-12


def test_many_lines_choose_shared_automatically_and_agree_with_thomas():
    # 65536 lines of n = 64 along the strided axis: the automatic choice is one partition per
    # line, and with shared coefficients the shared factorisation replaces the per-line one
    n, L = 64, 65536
    a, b, c = _coefficients(n, 50)
    d = _rhs((n, L), 51, torch.float64, 1)
    p1 = _plan(d, 0, "f64", 1, partitions=0)
    os.environ["TDMA_DISABLE_SHARED"] = "1"
    try:
        p2 = _plan(d, 0, "f64", 1, partitions=0)
    finally:
        del os.environ["TDMA_DISABLE_SHARED"]
    assert (p1.config["variant"], p2.config["variant"]) == (SHARED, THOMAS)
    x1, x2 = torch.empty_like(d), torch.empty_like(d)
    p1.solve(a, b, c, d, x1)
    p2.solve(a, b, c, d, x2)
    torch.cuda.synchronize()
    assert O.rel_l2(x1.cpu().numpy(), x2.cpu().numpy()) <= 1e-14
    idx = np.random.default_rng(0).choice(L, 64, replace=False)
    ref = _oracle(a, b, c, d[:, idx].contiguous(), 0, 1)
    assert rel_err(x1[:, idx].cpu().numpy().T, ref) <= 1e-12


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("nrhs", [1, 2])
def test_shared_backward_sums_gradients_over_lines(precision, nrhs):
    n, L = 96, 700
    dt = torch.float64 if precision == "f64" else torch.float32
    a, b, c = _coefficients(n, 60, dt)
    d = _rhs((n, L), 61, dt, nrhs)
    plan = _plan(d, 0, precision, nrhs)
    assert plan.config["variant"] == SHARED
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    w = _rhs((n, L), 62, dt, nrhs)
    ga, gb, gc = (torch.zeros_like(t) for t in (a, b, c))
    gd = torch.empty_like(x)
    plan.backward(a, b, c, x, w, ga, gb, gc, gd)
    torch.cuda.synchronize()
    A, B, C = (np.broadcast_to(t.double().cpu().numpy(), (L, n)) for t in (a, b, c))
    X, W = _lines(x, 0, nrhs), _lines(w, 0, nrhs)
    if nrhs == 1:
        X, W = X[..., None], W[..., None]
    sums = [np.zeros(n) for _ in range(3)]
    lam = np.zeros_like(X)
    for r in range(nrhs):
        ra, rb, rc, rl = O.adjoint_grads(A, B, C, X[..., r], W[..., r])
        for k, gk in enumerate((ra, rb, rc)):
            sums[k] += gk.sum(axis=0)
        lam[..., r] = rl
    got = _lines(gd, 0, nrhs)
    assert rel_err(got, lam[..., 0] if nrhs == 1 else lam) <= TOL[precision]
    tol = 1e-11 if precision == "f64" else 1e-4
    for g, want in zip((ga, gb, gc), sums):
        assert O.rel_l2(g.double().cpu().numpy(), want) <= tol


def test_shared_with_exact_residual_correction():
    # tridiag(-1, 2.001, -1) shared by all lines (condition number about 4000): the FP64 solve
    # followed by the exact-residual correction (an FP32 solve, which gains a factor of about
    # 4000 x 6e-8 per step) against the extended-precision oracle. Its condition-number bound
    # (4001) is below the default selection threshold (1e5), so by default no line is corrected and
    # the result is the plain FP64 solve bit for bit; refine_kappa < 0 corrects every line.
    n, L = 2048, 256
    a = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    c = a.clone()
    b = torch.full((n,), 2.001, dtype=torch.float64, device="cuda")
    d = _rhs((n, L), 71, torch.float64, 1)
    ref = _oracle(a, b, c, d, 0, 1, ext=True)
    plain = _plan(d, 0, "f64", 1)
    x64 = torch.empty_like(d)
    plain.solve(a, b, c, d, x64)
    plan = _plan(d, 0, "f64r", 1, refine_kappa=-1.0)
    assert plan.config["variant"] == SHARED
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    assert plan.last_error()[0] == 0
    assert plan.corrected_lines() == L
    e_corr = rel_err(_lines(x, 0, 1), ref)
    assert e_corr <= 1e-14
    assert e_corr <= rel_err(_lines(x64, 0, 1), ref)
    default = _plan(d, 0, "f64r", 1)
    xd = torch.empty_like(d)
    default.solve(a, b, c, d, xd)
    assert default.last_error()[0] == 0 and default.corrected_lines() == 0
    assert torch.equal(xd, x64)
    assert rel_err(_lines(xd, 0, 1), ref) <= 1e-12


def test_shared_singular_pivot_sets_status():
    n = 16
    a = torch.zeros(n, dtype=torch.float64, device="cuda")
    c = torch.zeros_like(a)
    b = torch.ones_like(a)
    b[5] = 0.0
    d = torch.ones(n, 200, dtype=torch.float64, device="cuda")
    plan = _plan(d, 0, "f64", 1)
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    assert plan.last_error()[0] == 5
    assert plan.last_error()[0] == 0


@pytest.mark.parametrize("axis", [0, 2])
def test_factorisation_over_several_chunks(axis):
    # 5000 rows: the factorisation runs over three chunks of staged coefficients, each cut into
    # 32 segments whose start values are estimated and then made exact by passes
    n = 5000
    a, b, c = _coefficients(n, 90)
    shape = (n, 40, 1) if axis == 0 else (1, 70, n)
    d = _rhs(shape, 91, torch.float64, 1)
    plan = _plan(d, axis, "f64", 1)
    assert plan.config["variant"] == SHARED
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    assert plan.last_error()[0] == 0
    assert rel_err(_lines(x, axis, 1), _oracle(a, b, c, d, axis, 1)) <= 1e-12


@pytest.mark.parametrize("diag", [2.0001, 2.5])
def test_factorisation_equals_the_serial_recurrence(diag):
    # tridiag(-1, diag, -1) over 4100 rows: on the weakly dominant line the segment estimates
    # are far off and many passes run; either way the factors are those of the serial recurrence,
    # so the solve agrees with the per-line Thomas kernel to rounding of the same operations
    n, L = 4100, 256
    a = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    b = torch.full((n,), diag, dtype=torch.float64, device="cuda")
    d = _rhs((n, L), 92, torch.float64, 1)
    p1 = _plan(d, 0, "f64", 1)
    os.environ["TDMA_DISABLE_SHARED"] = "1"
    try:
        p2 = _plan(d, 0, "f64", 1)
    finally:
        del os.environ["TDMA_DISABLE_SHARED"]
    assert (p1.config["variant"], p2.config["variant"]) == (SHARED, THOMAS)
    x1, x2 = torch.empty_like(d), torch.empty_like(d)
    p1.solve(a, b, a, d, x1)
    p2.solve(a, b, a, d, x2)  # the per-line Thomas kernel on the same broadcast coefficients
    torch.cuda.synchronize()
    assert O.rel_l2(x1.cpu().numpy(), x2.cpu().numpy()) <= 1e-15
