"""The parallel diagonally dominant (PDD) approximation on the fused divide-and-conquer kernel
against the oracle's PDD (the same approximation, element by element), on lines dominant enough
to be solved by PDD in practice but weak enough that PDD differs visibly from the exact solve.
Also: one partition is exact, the long-partition (workspace scratch) kernel, two right-hand
sides, float, and the accuracy against the exact solve as the partitions get shorter."""
import numpy as np
import pytest
import torch

import oracle as O
from parity import rel_err
import synth
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu

DC, DC_GLOBAL = 0, 7


def _grid(n, lines, seed, weak=0.3, dtype=torch.float64):
    # a, c ~ U(-1, 0), b = |a| + |c| + weak + U(0, 0.1): spikes fall by a few per cent a row
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1, 0, (n, lines))
    c = rng.uniform(-1, 0, (n, lines))
    b = np.abs(a) + np.abs(c) + weak + rng.uniform(0, 0.1, (n, lines))
    d = rng.uniform(-1, 1, (n, lines))
    return [torch.from_numpy(t).to(dtype).cuda() for t in (a, b, c, d)]


def _lines(t):
    return t.double().cpu().numpy().T  # [lines, n] for grids laid out [n][lines]


@pytest.mark.parametrize("n,P", [(64, 2), (64, 4), (67, 8), (40, 16), (33, 16), (256, 32), (9, 4)])
def test_pdd_matches_oracle_pdd(n, P):
    a, b, c, d = _grid(n, 300, n + P)
    x = tdma.solve(a, b, c, d, axis=0, partitions=P, pdd=True, check=True)
    A, B, C, D = (_lines(t) for t in (a, b, c, d))
    ref = O.pdd(A, B, C, D, P)
    assert rel_err(_lines(x), ref) <= 1e-12
    exact = O.dense_solve(A, B, C, D) if n <= 128 else O.thomas(A, B, C, D)
    if P > 1 and n // P <= 16:
        assert O.rel_l2(ref, exact) > 1e-8  # the approximation is really exercised


def test_one_partition_is_exact():
    a, b, c, d = _grid(50, 200, 3)
    x = tdma.solve(a, b, c, d, axis=0, partitions=1, pdd=True, check=True)
    assert rel_err(_lines(x), O.thomas(*(_lines(t) for t in (a, b, c, d)))) <= 1e-12


def test_long_partitions_use_workspace_scratch():
    # 512 rows, 8 partitions of 64 (the ADI configuration): Stage A scratch in the workspace
    a, b, c, d = _grid(512, 1000, 5, weak=0.05)
    plan = tdma.Plan(*tdma.line_layout(d, 0), partitions=8, pdd=True)
    assert plan.config["variant"] == DC_GLOBAL
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    assert plan.last_error()[0] == 0
    ref = O.pdd(*(_lines(t) for t in (a, b, c, d)), 8)
    assert rel_err(_lines(x), ref) <= 1e-12


def test_unit_stride_lines_and_in_place():
    a, b, c, d = (t.T.contiguous() for t in _grid(48, 120, 7))  # [lines][n]: unit stride
    ref = O.pdd(*(t.double().cpu().numpy() for t in (a, b, c, d)), 6)
    plan = tdma.Plan(*tdma.line_layout(d, 1), partitions=6, pdd=True)
    assert plan.config["variant"] == DC
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    assert rel_err(x.cpu().numpy(), ref) <= 1e-12
    plan.solve(a, b, c, d, d)
    assert rel_err(d.cpu().numpy(), ref) <= 1e-12


def test_two_right_hand_sides():
    a, b, c, d = _grid(96, 150, 9)
    d2 = torch.stack([d, torch.flip(d, [0]) * 0.5], dim=-1).contiguous()
    x = tdma.solve(a, b, c, d2, axis=0, nrhs=2, partitions=8, pdd=True, check=True)
    A, B, C = (_lines(t) for t in (a, b, c))
    for q in range(2):
        ref = O.pdd(A, B, C, _lines(d2[..., q]), 8)
        assert rel_err(_lines(x[..., q]), ref) <= 1e-12


def test_float():
    a, b, c, d = _grid(128, 256, 11, dtype=torch.float32)
    x = tdma.solve(a, b, c, d, axis=0, precision="f32", partitions=8, pdd=True, check=True)
    ref = O.pdd(*(_lines(t) for t in (a, b, c, d)), 8)
    assert rel_err(_lines(x), ref) <= 1e-5


def test_accuracy_against_exact_falls_with_partition_length():
    # the ADI operator tridiag(-r, 1 + 2r, -r), r = 0.5: spikes fall by 2 - sqrt(3) = 0.27 a row
    n, L, r = 512, 64, 0.5
    a = torch.full((n, L), -r, dtype=torch.float64, device="cuda")
    b = torch.full((n, L), 1 + 2 * r, dtype=torch.float64, device="cuda")
    d = torch.from_numpy(np.random.default_rng(2).uniform(-1, 1, (n, L))).cuda()
    exact = O.thomas(*(_lines(t) for t in (a, b, a, d)))
    errs = {}
    for P in (8, 32, 64, 128):
        x = tdma.solve(a, b, a, d, axis=0, partitions=P, pdd=True, check=True)
        errs[P] = O.rel_l2(_lines(x), exact)
    # oracle PDD on the same lines: 1.0e-16, 6.9e-11, 3.7e-6, 1.0e-3 for P = 8, 32, 64, 128
    assert errs[8] <= 1e-14              # 64-row partitions: spike tips (0.27^64) below rounding
    assert errs[32] <= 1e-9              # 16 rows
    assert 1e-8 <= errs[64] <= 1e-4      # 8 rows
    assert 1e-4 <= errs[128] <= 1e-2     # 4 rows


def test_backward_is_unsupported():
    a, b, c, d = _grid(32, 40, 13)
    plan = tdma.Plan(*tdma.line_layout(d, 0), partitions=4, pdd=True)
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    with pytest.raises(tdma.TDMAError):
        plan.backward(a, b, c, x, x.clone(), None, None, None, torch.empty_like(x))
