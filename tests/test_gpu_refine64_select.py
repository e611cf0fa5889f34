"""TDMA_F64_REFINE with coefficients shared by all lines: only the lines whose condition-number
bound ||A||_inf / delta (delta: the smallest diagonal-dominance margin of a row) reaches
refine_kappa are corrected; the others keep the plain FP64 result. Checked on wavenumber lines
of the FFT-Poisson solve (Section 5.2: one operator, a per-line shift by the modified wavenumbers)
against the extended-precision oracle, per line: every line meets 1e-12, the number of corrected
lines lies between the count the bound demands and the count with the selection's factor-two
slack, and refine_kappa < 0 corrects every line."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from parity import per_line, rel_err
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu


def _kappa_bound(a, b0, c, shift):
    """||A||_inf / min_i (|b_i| - |a_i| - |c_i|) per line (a_0 = c_{n-1} = 0), inf without dominance."""
    ac = np.abs(a).copy()
    ac[0] = 0.0
    cc = np.abs(c).copy()
    cc[-1] = 0.0
    B = np.abs(b0[None, :] + shift[:, None])
    margin = (B - ac[None, :] - cc[None, :]).min(axis=1)
    norm = (B + ac[None, :] + cc[None, :]).max(axis=1)
    return np.where(margin > 0, norm / np.where(margin > 0, margin, 1.0), np.inf)


@pytest.mark.parametrize("kappa", [0.0, 3e4, -1.0])
def test_selected_lines_meet_1e12(kappa):
    nx, nz, n = 128, 64, 256  # 128 x 64 wavenumber pairs, lines of n = 256 along y
    p = synth.poisson_lines(nx, nz, n, seed=5, device="cuda")
    L = nx * nz
    d = p["d"].view(n, L, 2)[:, 1:, :].contiguous()  # the (0, 0) mode has its own plan
    shift = p["shift"][1:].contiguous()
    plan = tdma.Plan(*tdma.line_layout(d, 0, nrhs=2), nrhs=2, coef_broadcast=True, diag_shift=shift,
                     precision="f64r", refine_kappa=kappa)
    x = torch.empty_like(d)
    plan.solve(p["a"], p["b0"], p["c"], d, x)
    assert plan.last_error()[0] == 0
    corrected = plan.corrected_lines()
    a, c, b0, sh = (p[k].cpu().numpy() for k in ("a", "c", "b0", "shift"))
    sh = sh[1:]
    kb = _kappa_bound(a, b0, c, sh)
    if kappa < 0:
        assert corrected == L - 1
    else:
        k = 1e5 if kappa == 0 else kappa
        assert int(np.sum(kb >= k)) <= corrected <= int(np.sum(kb >= 0.49 * k))
        assert corrected < (L - 1) // 4  # a small share of the lines
    A = np.broadcast_to(a, (L - 1, n))
    C = np.broadcast_to(c, (L - 1, n))
    B = b0[None, :] + sh[:, None]
    ref = O.thomas_ext(A, B, C, d.cpu().numpy().transpose(1, 0, 2))
    got = x.cpu().numpy().transpose(1, 0, 2)
    assert rel_err(got, ref) <= 1e-12
    # the lines left uncorrected keep the plain FP64 solve bit for bit
    plain = tdma.Plan(*tdma.line_layout(d, 0, nrhs=2), nrhs=2, coef_broadcast=True, diag_shift=shift, precision="f64")
    x64 = torch.empty_like(d)
    plain.solve(p["a"], p["b0"], p["c"], d, x64)
    changed = (x != x64).reshape(n, L - 1, 2).any(dim=2).any(dim=0).cpu().numpy()
    assert int(changed.sum()) <= corrected
    if kappa >= 0:
        k = 1e5 if kappa == 0 else kappa
        assert not changed[kb < 0.49 * k].any()


def test_zero_mode_line_without_dominance_is_corrected():
    # the pinned zero mode: rows 1..n-1 have no dominance margin, so the line is always corrected
    pz = synth.poisson_lines(2, 2, 1024, seed=2, device="cuda", rhs=True)
    dz = pz["d"].view(1024, 4, 2)[:, :1, :].contiguous()
    plan = tdma.Plan(*tdma.line_layout(dz, 0, nrhs=2), nrhs=2, coef_broadcast=True, precision="f64r")
    x = torch.empty_like(dz)
    plan.solve(pz["pin_a"], pz["pin_b"], pz["pin_c"], dz, x)
    assert plan.last_error()[0] == 0
    assert plan.corrected_lines() == 1
    ref = O.thomas_ext(pz["pin_a"].cpu().numpy(), pz["pin_b"].cpu().numpy(), pz["pin_c"].cpu().numpy(),
                       dz[:, 0, :].cpu().numpy())
    assert O.rel_l2(x[:, 0, :].cpu().numpy(), ref) <= 1e-13
    assert float(per_line(x[:, 0, :].cpu().numpy()[None], ref[None]).max()) <= 1e-13
