"""Parity at the full workload sizes, in the launch configurations bench.py times, on sampled
lines the oracle solves one by one (the whole grids are too large for the CPU oracle). Errors are
bounded pooled over the sampled lines and for every sampled line."""
import numpy as np
import pytest
import torch
from scipy.fft import dstn, idstn

import oracle as O
import synth
from parity import rel_err, rel_err_packed
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu


def _lines_of(t, axis, idx):
    """Rows of the lines with flat line indices idx (lines along `axis`) as an [k, n] array."""
    v = t.movedim(axis, -1)
    flat = v.reshape(-1, v.shape[-1])
    return flat[torch.as_tensor(idx, device=t.device)].double().cpu().numpy()


def test_general_1024_cubed_fp32_refine_and_fp64():
    n = 1024
    g = synth.grid_general((n, n, n), 0, 3, device="cuda", fp32_coefficients=True)
    g.pop("x_true")
    a32, b32, c32, d = g["a32"], g["b32"], g["c32"], g["d"]
    lay = tdma.line_layout(d, 0)
    rng = np.random.default_rng(3)
    idx = np.concatenate([[0, 1, n - 1, n * n - 1], rng.choice(n * n, 1020, replace=False)])
    ref = O.thomas(*(_lines_of(t, 0, idx) for t in (a32, b32, c32, d)))
    x = torch.empty_like(d)
    pr = tdma.Plan(*lay, precision="f32r")
    pr.solve(a32, b32, c32, d, x)
    st, iters = pr.last_error()
    assert st == 0 and iters >= 1
    assert rel_err(_lines_of(x, 0, idx), ref) <= 1e-12
    pd = tdma.Plan(*lay, precision="f64")
    pd.solve(g["a"], g["b"], g["c"], d, x)
    assert pd.last_error()[0] == 0
    assert rel_err(_lines_of(x, 0, idx), ref) <= 1e-12


def test_adi_512_cubed_sweeps_match_closed_form():
    n, r = 512, 0.5
    g = synth.grid_adi((n, n, n), seed=1, r=r, device="cuda")
    a, b, c, d = g["a"], g["b"], g["c"], g["d"]
    u = d.clone()
    plans = [tdma.Plan(*tdma.line_layout(u, ax), precision="f64", partitions=8) for ax in (2, 1, 0)]
    graph = tdma.sweep_graph([(p, (a, b, c, u, u)) for p in plans])
    u.copy_(d)
    graph.replay()
    torch.cuda.synchronize()
    for p in plans:
        assert p.last_error()[0] == 0
    lam = 1 + 4 * r * np.sin(np.pi * np.arange(1, n + 1) / (2 * (n + 1))) ** 2
    L = lam[:, None, None] * lam[None, :, None] * lam[None, None, :]
    ref = idstn(dstn(d.cpu().numpy(), type=1, workers=-1) / L, type=1, workers=-1)
    assert rel_err(u.cpu().numpy(), ref) <= 1e-12  # pooled and per z-plane


@pytest.mark.parametrize("precision,tol", [("f64r", 1e-12), ("f64", 1e-11)])
def test_poisson_wavenumber_lines_1024_cubed(precision, tol):
    # Against the extended-precision oracle. Plain FP64 elimination is a few 1e-12 off on the
    # lowest modes (so is the FP64 CPU Thomas: 3e-12 on the pinned zero mode), hence its looser
    # bound; f64r corrects the lines whose condition-number bound reaches 1e5 (the lowest modes,
    # a few thousand of the 2^20) from an exact residual, solved in FP32, and meets 1e-12.
    n = 1024
    p = synth.poisson_lines(n, n, n, seed=2, device="cuda")
    d = p["d"]
    x = torch.empty_like(d)
    d3, x3 = d.view(n, n * n, 2), x.view(n, n * n, 2)
    shift = p["shift"][1:].contiguous()
    main = tdma.Plan(*tdma.line_layout(d3[:, 1:, :], 0, nrhs=2), nrhs=2, coef_broadcast=True, diag_shift=shift,
                     precision=precision)
    zero = tdma.Plan(*tdma.line_layout(d3[:, :1, :], 0, nrhs=2), nrhs=2, coef_broadcast=True, precision=precision)
    main.solve(p["a"], p["b0"], p["c"], d3[:, 1:, :], x3[:, 1:, :])
    zero.solve(p["pin_a"], p["pin_b"], p["pin_c"], d3[:, :1, :], x3[:, :1, :])
    assert main.last_error()[0] == 0 and zero.last_error()[0] == 0
    if precision == "f64r":
        assert 0 < main.corrected_lines() < (n * n) // 100 and zero.corrected_lines() == 1
    # sampled modes: the pinned zero mode, the lowest and highest wavenumbers, random ones
    rng = np.random.default_rng(2)
    modes = np.unique(np.concatenate([[0, 1, n, n + 1, n * n - 1, n * n // 2 + n // 2], rng.choice(n * n, 58, False)]))
    a = p["a"].cpu().numpy(); c = p["c"].cpu().numpy(); b0 = p["b0"].cpu().numpy()
    sh = p["shift"].cpu().numpy()
    got, want = [], []
    for m in modes:
        if m == 0:
            A, B, C = p["pin_a"].cpu().numpy(), p["pin_b"].cpu().numpy(), p["pin_c"].cpu().numpy()
        else:
            A, B, C = a, b0 + sh[m], c
        dm = d3[:, m, :].cpu().numpy()
        want.append(O.thomas_ext(A, B, C, dm))
        got.append(x3[:, m, :].cpu().numpy())
    err = rel_err(np.stack(got), np.stack(want))  # pooled and per mode
    assert err <= tol, err


@pytest.mark.parametrize("precision", ["f32r", "f64"])
def test_ragged_20000_lines(precision):
    lengths = synth.ragged_lengths(20000, 16, 16384, seed=4)
    r = synth.ragged_general(lengths, 4, device="cuda", fp32_coefficients=True)
    keys = ("a32", "b32", "c32") if precision == "f32r" else ("a", "b", "c")
    a, b, c = (r[k] for k in keys)
    d = r["d"]
    x, plan = tdma.solve_ragged(a, b, c, d, r["offsets"], r["lengths"], precision=precision, check=True)
    rng = np.random.default_rng(4)
    lines = np.unique(np.concatenate([np.argsort(-lengths)[:10], rng.choice(20000, 300, replace=False)]))
    offs, lens = r["offsets"].cpu().numpy(), r["lengths"].cpu().numpy()
    ref = O.thomas_ragged(r["a"].cpu().numpy(), r["b"].cpu().numpy(), r["c"].cpu().numpy(), d.cpu().numpy(), offs,
                          lens, lines=lines)
    xs = x.cpu().numpy()
    got = np.concatenate([xs[offs[l]:offs[l] + lens[l]] for l in sorted(ref)])
    want = np.concatenate([ref[l] for l in sorted(ref)])
    assert rel_err_packed(got, want, [lens[l] for l in sorted(ref)]) <= 1e-12
    # backward with loss = sum(w * x), w ~ N(0, 1)
    w = synth.normal(4, synth.AID["w"], torch.arange(r["total"], device="cuda"))
    ga, gb, gc, gd = (torch.empty_like(a), torch.empty_like(b), torch.empty_like(c), torch.empty_like(x))
    plan.backward(a, b, c, x, w, ga, gb, gc, gd)
    assert plan.last_error()[0] == 0
    ws = w.cpu().numpy()
    ha, hb, hc = (r[k].cpu().numpy() for k in ("a", "b", "c"))
    hgd, hgb = gd.cpu().numpy(), gb.double().cpu().numpy()
    for l in list(sorted(ref))[:60]:
        s = slice(offs[l], offs[l] + lens[l])
        rg = O.adjoint_grads(ha[s], hb[s], hc[s], xs[s], ws[s])
        assert O.rel_l2(hgd[s], rg[3]) <= 1e-12
        assert O.rel_l2(hgb[s], rg[1]) <= (1e-12 if precision == "f64" else 1e-6)
