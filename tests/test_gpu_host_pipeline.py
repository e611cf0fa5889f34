"""Pipelined solves of grids held in host memory (tdma_solve_host): slices of lines through device
staging slots on several streams must give exactly the on-device solve of the whole grid."""
import pytest
import torch

import oracle as O
import synth
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu


def _grid(shape, axis, precision, seed):
    g = synth.grid_general(shape, axis, seed, device="cuda", fp32_coefficients=precision == "f32r")
    if precision == "f32r":
        return g["a32"], g["b32"], g["c32"], g["d"]
    return g["a"], g["b"], g["c"], g["d"]


@pytest.mark.parametrize("precision", ["f64", "f32r", "f32"])
@pytest.mark.parametrize("axis", [0, 2])
def test_pipeline_matches_device_solve(precision, axis):
    shape = (64, 16, 64)
    a, b, c, d = _grid(shape, axis, "f32r" if precision == "f32r" else "f64", 21)
    if precision == "f32":
        a, b, c, d = a.float(), b.float(), c.float(), d.float()
    x_dev = tdma.solve(a, b, c, d, axis=axis, precision=precision)
    pipe = tdma.HostPipeline(shape, axis=axis, precision=precision, batches=8, slots=3)
    h = [t.cpu().pin_memory() for t in (a, b, c, d)]
    hx = torch.empty(d.shape, dtype=d.dtype).pin_memory()
    pipe.solve(*h, hx)
    torch.cuda.synchronize()
    # a slice solves whole lines with the same kernels as the full grid: identical results, except
    # for FP32 + refinement along the contiguous axis, where the chunk kernel cuts the lines it is
    # given into chunks (a slice's chunks differ from the full grid's): equal to rounding there
    if precision == "f32r" and axis == 2:
        assert O.rel_l2(hx.numpy(), x_dev.cpu().numpy()) <= 1e-14
    else:
        assert torch.equal(hx, x_dev.cpu())
    assert pipe.plan.last_error()[0] == 0


def test_pipeline_one_slot_and_repeated_use():
    shape = (32, 8, 32)
    a, b, c, d = _grid(shape, 0, "f32r", 22)
    x_dev = tdma.solve(a, b, c, d, axis=0, precision="f32r")
    pipe = tdma.HostPipeline(shape, axis=0, precision="f32r", batches=4, slots=1)
    h = [t.cpu().pin_memory() for t in (a, b, c, d)]
    for _ in range(2):
        hx = torch.zeros(d.shape, dtype=d.dtype).pin_memory()
        pipe.solve(*h, hx)
        torch.cuda.synchronize()
        assert torch.equal(hx, x_dev.cpu())


def test_pipeline_rejects_bad_arguments():
    with pytest.raises(ValueError):
        tdma.HostPipeline((32, 3, 5), axis=0, batches=4)  # 15 lines do not split into 4 slices
    with pytest.raises(ValueError):
        tdma.HostPipeline((8, 8, 8), axis=1)
    shape = (16, 4, 8)
    pipe = tdma.HostPipeline(shape, axis=0, precision="f64", batches=2, slots=2)
    h = [torch.ones(shape, dtype=torch.float64).pin_memory() for _ in range(4)]
    with pytest.raises(tdma.TDMAError) as e:
        pipe.solve(h[0], h[1], h[2], h[3], h[3])  # x over d
    assert e.value.status == 1
