"""The C-ABI library builds, loads and exports every symbol include/tdma.h declares, and its
host-side validation rejects bad descriptors (no GPU needed: validation runs before any CUDA call)."""
import ctypes

import pytest

import paper_2509_03933_gb300 as tdma


def test_library_exports_declared_symbols():
    lib = tdma.load_library()
    names = tdma.declared_symbols()
    assert {"tdma_plan_create", "tdma_solve", "tdma_solve_backward", "tdma_plan_destroy",
            "tdma_last_device_error", "tdma_status_string", "tdma_plan_autotune",
            "tdma_plan_get_config"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings():
    lib = tdma.load_library()
    for code, text in tdma.STATUS.items():
        assert lib.tdma_status_string(code).decode() == text
    assert lib.tdma_status_string(99).decode() == "unknown status"


def _create(**kw):
    lib = tdma.load_library()
    base = dict(n=64, n_lines=16, elem_stride=1, inner_count=16, inner_stride=64, outer_stride=0, nrhs=1,
                precision=0, partitions=0)
    base.update(kw)
    d = tdma.Desc(**base)
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t(0)
    return lib.tdma_plan_create(ctypes.byref(h), ctypes.byref(d), ctypes.byref(ws))


@pytest.mark.parametrize("kw,code", [
    (dict(n=-1), 1), (dict(n_lines=-5), 1), (dict(nrhs=3), 1), (dict(precision=7), 1),
    (dict(partitions=-1), 1), (dict(partitions=40), 1),  # 64 / 40 < 2 rows per partition
    (dict(inner_count=0), 1), (dict(elem_stride=-1), 1),
    (dict(n=0, ragged_max_n=0), 1),                       # ragged without offsets/lengths
    (dict(precision=2, nrhs=2), 2), (dict(precision=2, coef_broadcast=1), 2),
    (dict(pdd=1), 1), (dict(pdd=2, partitions=4), 1),   # PDD needs explicit partitions; flag 0/1
    (dict(pdd=1, partitions=4, precision=2), 2), (dict(pdd=1, partitions=4, precision=3), 2),
    (dict(pdd=1, partitions=4, n=0, n_lines=0), 2),      # ragged batches have no PDD mode
])
def test_invalid_descriptors_are_rejected_on_the_host(kw, code):
    assert _create(**kw) == code


def test_null_arguments():
    lib = tdma.load_library()
    assert lib.tdma_plan_create(None, None, None) == 1
    assert lib.tdma_plan_destroy(None) == 0
    assert lib.tdma_solve(None, None, None, None, None, None, None, 0, None) == 1
    assert lib.tdma_last_device_error(None, None, None) == 1


def test_line_layout_of_grid_axes():
    import torch
    g = torch.empty(4, 5, 6)
    assert tdma.line_layout(g, 0) == (4, 30, 30, 30, 1, 0)       # z lines: merged (y, x)
    assert tdma.line_layout(g, 1) == (5, 24, 6, 6, 1, 30)         # y lines
    assert tdma.line_layout(g, 2) == (6, 20, 1, 20, 6, 0)         # x lines: merged (z, y)
    c = torch.empty(4, 5, 6, 2)
    assert tdma.line_layout(c, 0, nrhs=2) == (4, 30, 30, 30, 1, 0)


def test_poisson_descriptor_validation_on_the_host():
    import numpy as np
    lib = tdma.load_library()
    coef = np.ones(8)
    ptr = coef.ctypes.data

    def create(**kw):
        base = dict(nx=8, ny=8, nz=4, dx=1.0, dz=1.0, a=ptr, b=ptr, c=ptr, pin_zero_mode=1, precision=0)
        base.update(kw)
        h = ctypes.c_void_p()
        ws = ctypes.c_size_t(0)
        return lib.tdma_poisson_create(ctypes.byref(h), ctypes.byref(tdma.PoissonDesc(**base)), ctypes.byref(ws))

    assert create(nx=7) == 1          # odd nx (real-to-complex transform of even length)
    assert create(nz=1) == 1
    assert create(ny=1) == 1
    assert create(dx=0.0) == 1
    assert create(a=None) == 1
    assert create(pin_zero_mode=2) == 1
    assert create(precision=1) == 2   # FP32 lines are not offered
    assert lib.tdma_poisson_solve(None, None, None, None, 0, None) == 1
    assert lib.tdma_poisson_destroy(None) == 0


def test_slab_stage_validation_on_the_host():
    from paper_2509_03933_gb300.split_line import SlabDesc, _bind
    lib = _bind(tdma.load_library())
    ok = dict(n_local=8, n_lines=10, elem_stride=10, inner_count=10, inner_stride=1, outer_stride=0, nrhs=1,
              first=1, last=0)
    d = SlabDesc(**ok)
    assert lib.tdma_slab_scratch_bytes(ctypes.byref(d), 10) == 6 * 3 * 10 * 8
    assert lib.tdma_slab_pairs_work_bytes(4, 10, 2) == 2 * 4 * 10 * 3 * 8
    bad = SlabDesc(**dict(ok, n_local=1))
    assert lib.tdma_slab_reduce(ctypes.byref(bad), None, None, None, None, 0, 10, None, None, None, None) == 1
    assert lib.tdma_slab_reduce(ctypes.byref(d), None, None, None, None, 5, 10, None, None, None, None) == 1
    assert lib.tdma_slab_reduce(ctypes.byref(d), None, None, None, None, 0, 0, None, None, None, None) == 0
    assert lib.tdma_slab_pairs_solve(0, 10, 1, None, None, None, None, None) == 1
    assert lib.tdma_slab_pairs_solve(2, 10, 3, None, None, None, None, None) == 1
    assert lib.tdma_slab_finish(ctypes.byref(d), 0, 11, None, None, None, None) == 1
