"""The one-partition Thomas sweep on unit-stride lines (staged through shared memory in chunks of
8 rows, 32 lines per warp) against the oracle: both precisions, one and two right-hand sides,
line lengths with a partial last chunk, line counts that leave a warp partly empty, gaps between
lines, and x written over d."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from parity import rel_err
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu

THOMAS = 1
TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("nrhs", [1, 2])
@pytest.mark.parametrize("L,n,gap", [(100, 37, 0), (33, 1024, 0), (70, 2, 0), (65, 300, 5), (1, 17, 0)])
def test_staged_thomas_matches_oracle(precision, nrhs, L, n, gap):
    dt = torch.float64 if precision == "f64" else torch.float32
    g = synth.grid_general((L, n + gap), 1, L + n, device="cpu")
    a, b, c = (g[k].to(dt).cuda()[:, :n] for k in ("a", "b", "c"))
    dfull = synth.normal(3, synth.AID["d"], torch.arange(L * (n + gap) * nrhs)).reshape(
        (L, n + gap) + ((nrhs,) if nrhs > 1 else ())).to(dt).cuda()
    d = dfull[:, :n]
    plan = tdma.Plan(*tdma.line_layout(d, 1, nrhs=nrhs), precision=precision, partitions=1, nrhs=nrhs)
    assert plan.config["variant"] == THOMAS
    x = torch.full_like(dfull, 7.0)
    plan.solve(a, b, c, d, x[:, :n])
    assert plan.last_error()[0] == 0
    A, B, C = (t.double().cpu().numpy() for t in (a, b, c))
    D = d.double().cpu().numpy()
    ref = O.thomas(A, B, C, D)
    assert rel_err(x[:, :n].double().cpu().numpy(), ref) <= TOL[precision]
    if gap:
        assert bool((x[:, n:] == 7.0).all())
    dd = dfull.clone()  # the plan's layout (line pitch n + gap)
    plan.solve(a, b, c, dd[:, :n], dd[:, :n])  # x over d
    assert rel_err(dd[:, :n].double().cpu().numpy(), ref) <= TOL[precision]


def test_staged_thomas_singular_pivot_sets_status():
    L, n = 40, 50
    a = torch.zeros(L, n, dtype=torch.float64, device="cuda")
    c = torch.zeros_like(a)
    b = torch.ones_like(a)
    b[7, 20] = 0.0
    d = torch.ones_like(a)
    plan = tdma.Plan(*tdma.line_layout(d, 1), partitions=1)
    x = torch.empty_like(d)
    plan.solve(a, b, c, d, x)
    assert plan.last_error()[0] == 5
