"""The allocation-free entry point tdma_solve_thomas_static, called through the C ABI.

It serves callers that may not allocate device memory once running (a solver loop with its
GPU memory fixed at start-up, a host program whose pool owns the device heap): it keeps the
Thomas elimination factors in a fixed array inside the library instead of a plan and a
workspace. Its result must match the plan-based solve of the same problem and the oracle's
Thomas solve, on two calls in a row (the shared array keeps the previous call's contents), for
per-element and broadcast coefficients with a per-line shift, one and two (interleaved complex)
right-hand sides, and in place (x is d). This file is collected last so a run that stops at the
first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
import synth
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu


def _desc(n, lines, precision=0, nrhs=1, partitions=0, broadcast=False, shift=None):
    return tdma.Desc(n=n, n_lines=lines, elem_stride=lines, inner_count=lines, inner_stride=1, outer_stride=0,
                     nrhs=nrhs, precision=precision, partitions=partitions, coef_broadcast=int(broadcast),
                     diag_shift=None if shift is None else ctypes.c_void_p(shift.data_ptr()))


def _static_solve(a, b, c, d, x, desc):
    lib = tdma.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    return lib.tdma_solve_thomas_static(ctypes.byref(desc), ptr(a), ptr(b), ptr(c), ptr(d), ptr(x), stream)


def _np(t):
    return t.double().cpu().numpy()


def _case(kind, precision, seed, n, lines):
    """(a, b, c, d, shift, nrhs, broadcast, oracle lines (a, b, c, d) with lines on axis 0)."""
    g = synth.grid_general((n, lines), 0, seed, device="cuda", fp32_coefficients=(precision == "f32"))
    dt = torch.float64 if precision == "f64" else torch.float32
    pick = (lambda k: g[k]) if precision == "f64" else (lambda k: g[k + "32"])
    if kind == "broadcast_shift":
        a1, b1, c1 = (pick(k)[:, 0].contiguous() for k in ("a", "b", "c"))
        shift = torch.from_numpy(np.random.default_rng(seed).uniform(0.0, 2.0, lines)).to("cuda", dt)
        d = g["d"].to(dt)
        A = np.broadcast_to(_np(a1), (lines, n))
        B = _np(b1)[None, :] + _np(shift)[:, None]
        C = np.broadcast_to(_np(c1), (lines, n))
        return a1, b1, c1, d, shift, 1, True, (A, B, C, _np(d).T)
    a, b, c = pick("a"), pick("b"), pick("c")
    if kind == "nrhs2":
        im = synth.normal(seed, synth.AID["im"], torch.arange(n * lines, device="cuda")).reshape(n, lines)
        d = torch.stack([g["d"], im], dim=-1).to(dt).contiguous()
        return a, b, c, d, None, 2, False, (_np(a).T, _np(b).T, _np(c).T, _np(d).transpose(1, 0, 2))
    d = g["d"].to(dt)
    return a, b, c, d, None, 1, False, (_np(a).T, _np(b).T, _np(c).T, _np(d).T)


@pytest.mark.parametrize("kind", ["per_element", "broadcast_shift", "nrhs2", "in_place"])
@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_static_entry_matches_plan_solve_twice(kind, precision, tol):
    n, lines = 300, 512  # lines along the strided axis of an [n][lines] grid
    for call, seed in enumerate((31, 32)):
        a, b, c, d, shift, nrhs, bcast, ref_in = _case(kind, precision, seed, n, lines)
        x_ref = tdma.solve(a, b, c, d, axis=0, precision=precision, partitions=1, nrhs=nrhs,
                           coef_broadcast=bcast, diag_shift=shift, check=True)
        desc = _desc(n, lines, 0 if precision == "f64" else 1, nrhs=nrhs, broadcast=bcast, shift=shift)
        if kind == "in_place":
            x = d.clone()
            st = _static_solve(a, b, c, x, x, desc)
        else:
            x = torch.full_like(d, float("nan"))
            st = _static_solve(a, b, c, d, x, desc)
        torch.cuda.synchronize()
        assert st == 0, f"call {call}: status {st}"
        assert O.rel_l2(_np(x), _np(x_ref)) <= tol
        got = _np(x).transpose(1, 0, 2) if nrhs == 2 else _np(x).T
        ref = O.thomas(*ref_in)
        assert O.rel_l2(got, ref) <= tol
        worst = max(O.rel_l2(got[i], ref[i]) for i in range(0, lines, 7))
        assert worst <= tol


def test_static_entry_rejects_oversized_problem():
    lib = tdma.load_library()
    desc = _desc(1 << 20, 1 << 10)  # 2^30 FP64 factors, far beyond the fixed array
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(one.data_ptr())
    assert lib.tdma_solve_thomas_static(ctypes.byref(desc), p, p, p, p, p, None) == 3


def test_static_entry_rejects_bad_and_unsupported_descriptors():
    lib = tdma.load_library()
    one = torch.zeros(64, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(one.data_ptr())
    bad = _desc(8, 4, partitions=-1)
    assert lib.tdma_solve_thomas_static(ctypes.byref(bad), p, p, p, p, p, None) == 1
    for prec in (tdma.F32_REFINE, tdma.F64_REFINE):  # valid for a plan, not for this entry
        desc = _desc(8, 4, precision=prec)
        assert lib.tdma_solve_thomas_static(ctypes.byref(desc), p, p, p, p, p, None) == 2
    split = _desc(8, 4, partitions=2)
    assert lib.tdma_solve_thomas_static(ctypes.byref(split), p, p, p, p, p, None) == 2
