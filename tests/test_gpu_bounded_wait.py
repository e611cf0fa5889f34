"""Failure detection without a GPU fault: the bounded mbarrier wait of the solver kernels, made to
run out on a barrier nothing arrives on (tdma_probe_bounded_wait), reports TDMA_ERR_TIMEOUT through a
status word the host reads, ends in bounded time, and leaves the context usable: a solve afterwards
is correct."""
import ctypes
import time

import pytest
import torch

import oracle as O
import synth
from parity import rel_err
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu


def _wait(polls):
    lib = tdma.load_library()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    t0 = time.perf_counter()
    st = lib.tdma_probe_bounded_wait(polls, ctypes.c_void_p(status.data_ptr()), stream)
    torch.cuda.synchronize()
    return st, int(status.item()), time.perf_counter() - t0


@pytest.mark.parametrize("polls", [1, 100, 20000])
def test_bounded_wait_runs_out_and_reports_timeout(polls):
    st, word, seconds = _wait(polls)
    assert st == 0
    assert word == 6  # TDMA_ERR_TIMEOUT
    assert seconds < 5.0
    # the context still works: a solve right after is correct
    g = synth.grid_general((64, 4, 8), 0, 9, device="cuda")
    a, b, c, d = g["a"], g["b"], g["c"], g["d"]
    x = tdma.solve(a, b, c, d, axis=0, partitions=4, check=True)
    lines = lambda t: synth.line_view(t.cpu(), 0).numpy()
    assert rel_err(lines(x), O.thomas(lines(a), lines(b), lines(c), lines(d))) <= 1e-12


def test_bounded_wait_rejects_bad_arguments():
    lib = tdma.load_library()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.tdma_probe_bounded_wait(0, ctypes.c_void_p(status.data_ptr()), None) == 1
    assert lib.tdma_probe_bounded_wait(1 << 21, ctypes.c_void_p(status.data_ptr()), None) == 1
    assert lib.tdma_probe_bounded_wait(10, None, None) == 1
