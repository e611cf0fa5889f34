"""Backward pass (hand-written adjoint kernels) against the oracle's adjoint gradients and
against finite differences of the forward solve (torch.autograd.gradcheck)."""
import numpy as np
import pytest
import torch

import oracle as O
from parity import rel_err
import synth
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu


def _lines(t, axis):
    return synth.line_view(t.detach().double().cpu(), axis).numpy()


@pytest.mark.parametrize("axis,partitions", [(0, 1), (0, 4), (2, 3), (1, 0)])
def test_f64_gradients_match_oracle(axis, partitions):
    g = synth.grid_general((24, 12, 20), axis, 41)
    a, b, c, d = (g[k].cuda() for k in ("a", "b", "c", "d"))
    x = tdma.solve(a, b, c, d, axis=axis, partitions=partitions, check=True)
    w = torch.randn_like(x)
    ga, gb, gc, gd = tdma.solve_backward(a, b, c, x, w, axis=axis, partitions=partitions)
    ref = O.adjoint_grads(_lines(a, axis), _lines(b, axis), _lines(c, axis), _lines(x, axis), _lines(w, axis))
    for got, want in zip((ga, gb, gc, gd), ref):
        assert rel_err(_lines(got, axis), want) <= 1e-12


def test_f32_and_refined_gradients():
    g = synth.grid_general((64, 8, 8), 0, 42, fp32_coefficients=True)
    a32, b32, c32 = (g[k + "32"].cuda() for k in ("a", "b", "c"))
    d = g["d"].cuda()
    la = lambda t: _lines(t, 0)
    x = tdma.solve(a32, b32, c32, d, axis=0, precision="f32r", check=True)
    w = torch.randn_like(x)
    ref = O.adjoint_grads(la(a32), la(b32), la(c32), la(x), la(w))
    ga, gb, gc, gd = tdma.solve_backward(a32, b32, c32, x, w, axis=0, precision="f32r")
    assert rel_err(la(gd), ref[3]) <= 1e-12          # lambda, refined in FP64
    for got, want in zip((ga, gb, gc), ref[:3]):      # stored as float
        assert rel_err(la(got), want) <= 1e-6
    x32 = tdma.solve(a32, b32, c32, d.float(), axis=0, precision="f32")
    ga, gb, gc, gd = tdma.solve_backward(a32, b32, c32, x32, w.float(), axis=0, precision="f32")
    ref = O.adjoint_grads(la(a32), la(b32), la(c32), la(x32), la(w))
    for got, want in zip((ga, gb, gc, gd), ref):
        assert rel_err(la(got), want) <= 1e-5


def test_broadcast_complex_gradients_are_summed_over_lines():
    nx, ny, nz = 4, 4, 32
    p = synth.poisson_lines(nx, ny, nz, seed=2, device="cuda")
    d = p["d"].reshape(nz, ny * nx, 2)[:, 1:, :].contiguous()
    shift = p["shift"][1:].contiguous()
    a, b0, c = p["a"], p["b0"], p["c"]
    x = tdma.solve(a, b0, c, d, axis=0, nrhs=2, coef_broadcast=True, diag_shift=shift, partitions=4, check=True)
    w = torch.randn_like(x)
    ga, gb, gc, gd = tdma.solve_backward(a, b0, c, x, w, axis=0, nrhs=2, coef_broadcast=True, diag_shift=shift,
                                         partitions=4)
    L = ny * nx - 1
    A = np.broadcast_to(a.cpu().numpy(), (L, nz))
    C = np.broadcast_to(c.cpu().numpy(), (L, nz))
    B = b0.cpu().numpy()[None, :] + shift.cpu().numpy()[:, None]
    X = x.cpu().numpy().transpose(1, 0, 2)
    W = w.cpu().numpy().transpose(1, 0, 2)
    sums = [np.zeros(nz) for _ in range(3)]
    lam = np.zeros_like(X)
    for r in range(2):
        ra, rb, rc, rl = O.adjoint_grads(A, B, C, X[..., r], W[..., r])
        for k, gk in enumerate((ra, rb, rc)):
            sums[k] += gk.sum(axis=0)
        lam[..., r] = rl
    assert rel_err(gd.cpu().numpy().transpose(1, 0, 2), lam) <= 1e-12
    for got, want in zip((ga, gb, gc), sums):
        assert O.rel_l2(got.cpu().numpy(), want) <= 1e-11


def test_autograd_function_gradcheck():
    torch.manual_seed(0)
    n, L = 12, 5
    a = (-torch.rand(L, n, dtype=torch.float64, device="cuda")).requires_grad_()
    c = (-torch.rand(L, n, dtype=torch.float64, device="cuda")).requires_grad_()
    b = (3.0 + torch.rand(L, n, dtype=torch.float64, device="cuda")).requires_grad_()
    d = torch.randn(L, n, dtype=torch.float64, device="cuda").requires_grad_()
    for P in (1, 3):
        f = lambda a_, b_, c_, d_: tdma.TDMASolve.apply(a_, b_, c_, d_, -1, "f64", P)
        assert torch.autograd.gradcheck(f, (a, b, c, d), eps=1e-6, atol=1e-7, rtol=1e-6)


def test_loss_gradient_against_central_differences():
    # loss = sum(w * x) for one line; gradients through TDMASolve vs central differences
    # of the oracle's forward solve
    rng = np.random.default_rng(5)
    n = 16
    a = rng.uniform(-1, 0, n); c = rng.uniform(-1, 0, n); b = 2 + abs(a) + abs(c) + rng.uniform(0, 1, n)
    d = rng.uniform(-1, 1, n); w = rng.normal(size=n)
    ts = [torch.tensor(v[None, :], device="cuda", requires_grad=True) for v in (a, b, c, d)]
    x = tdma.TDMASolve.apply(*ts, -1, "f64", 2)
    (x * torch.tensor(w[None, :], device="cuda")).sum().backward()
    loss = lambda a_, b_, c_, d_: float(np.sum(w * O.thomas(a_, b_, c_, d_)))
    arrs = [a, b, c, d]
    for k in range(4):
        for i in range(n):
            if (k == 0 and i == 0) or (k == 2 and i == n - 1):
                assert float(ts[k].grad[0, i]) == 0.0
                continue
            h = 1e-6 * max(1.0, abs(arrs[k][i]))
            arrs[k][i] += h; fp = loss(*arrs)
            arrs[k][i] -= 2 * h; fm = loss(*arrs)
            arrs[k][i] += h
            assert abs((fp - fm) / (2 * h) - float(ts[k].grad[0, i])) < 1e-7 * max(1.0, abs((fp - fm) / (2 * h)))
