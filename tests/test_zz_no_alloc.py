"""The allocation-free entry point tdma_solve_thomas_static, called through the C ABI.

It serves callers that may not allocate device memory once running (a solver loop with its
GPU memory fixed at start-up, a host program whose pool owns the device heap): it keeps the
Thomas elimination factors in a fixed array inside the library instead of a plan and a
workspace. Its result must match the plan-based solve of the same problem, on two calls in a
row (the shared array keeps the previous call's contents). This file is collected last so a
run that stops at the first failure has run every other test before it.
"""
import ctypes

import pytest
import torch

import oracle as O
import synth
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu


def _desc(n, lines, precision=0, nrhs=1):
    return tdma.Desc(n=n, n_lines=lines, elem_stride=lines, inner_count=lines, inner_stride=1, outer_stride=0,
                     nrhs=nrhs, precision=precision, partitions=0)


def _static_solve(a, b, c, d, x, n, lines, precision=0):
    lib = tdma.load_library()
    desc = _desc(n, lines, precision)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    return lib.tdma_solve_thomas_static(ctypes.byref(desc), ptr(a), ptr(b), ptr(c), ptr(d), ptr(x), stream)


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_static_entry_matches_plan_solve_twice(precision, tol):
    n, lines = 300, 512  # lines along the strided axis of an [n][lines] grid
    for call, seed in enumerate((31, 32)):
        g = synth.grid_general((n, lines), 0, seed, device="cuda", fp32_coefficients=(precision == "f32"))
        if precision == "f64":
            a, b, c, d = g["a"], g["b"], g["c"], g["d"]
        else:
            a, b, c, d = g["a32"], g["b32"], g["c32"], g["d"].float()
        x_ref = tdma.solve(a, b, c, d, axis=0, precision=precision, partitions=1, check=True)
        x = torch.full_like(d, float("nan"))
        st = _static_solve(a, b, c, d, x, n, lines, 0 if precision == "f64" else 1)
        torch.cuda.synchronize()
        assert st == 0, f"call {call}: status {st}"
        assert O.rel_l2(x.double().cpu().numpy(), x_ref.double().cpu().numpy()) <= tol
        ref = O.thomas(*(synth.line_view(t.double().cpu(), 0).numpy() for t in (a, b, c, d)))
        assert O.rel_l2(synth.line_view(x.double().cpu(), 0).numpy(), ref) <= tol


def test_static_entry_rejects_oversized_problem():
    lib = tdma.load_library()
    desc = _desc(1 << 20, 1 << 10)  # 2^30 FP64 factors, far beyond the fixed array
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(one.data_ptr())
    assert lib.tdma_solve_thomas_static(ctypes.byref(desc), p, p, p, p, p, None) == 3
