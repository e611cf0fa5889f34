"""Ragged batches (lines of uneven length in one persistent launch) against the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from parity import rel_err, rel_err_packed
import synth
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f32r": 1e-12}


def _run(lengths, seed, precision, check_lines=None):
    r = synth.ragged_general(lengths, seed, device="cuda", fp32_coefficients=precision != "f64")
    if precision == "f64":
        a, b, c, d = r["a"], r["b"], r["c"], r["d"]
    elif precision == "f32":
        a, b, c, d = r["a32"], r["b32"], r["c32"], r["d"].float()
    else:
        a, b, c, d = r["a32"], r["b32"], r["c32"], r["d"]
    x, plan = tdma.solve_ragged(a, b, c, d, r["offsets"], r["lengths"], precision=precision, check=True)
    offs, lens = r["offsets"].cpu().numpy(), r["lengths"].cpu().numpy()
    ref = O.thomas_ragged(a.double().cpu().numpy(), b.double().cpu().numpy(), c.double().cpu().numpy(),
                          d.double().cpu().numpy(), offs, lens, lines=check_lines)
    xs = x.double().cpu().numpy()
    got = np.concatenate([xs[offs[l]:offs[l] + lens[l]] for l in sorted(ref)])
    want = np.concatenate([ref[l] for l in sorted(ref)])
    return rel_err_packed(got, want, [lens[l] for l in sorted(ref)]), plan


@pytest.mark.parametrize("precision", ["f64", "f32", "f32r"])
def test_small_ragged_mix(precision):
    lengths = np.array([1, 2, 3, 4, 5, 7, 16, 17, 31, 33, 100, 257, 1000, 4097, 2, 64, 65, 1, 12, 300], np.int32)
    err, plan = _run(lengths, 4, precision)
    assert err <= TOL[precision]
    assert plan.config["variant"] == (9 if precision == "f32r" else 3)  # f32r: the chunk kernel


@pytest.mark.parametrize("precision", ["f64", "f32r"])
def test_log_uniform_batch_sampled(precision):
    # 3000 lines, n log-uniform in [16, 16384] as in the 20000-line workload; 200 lines checked
    lengths = synth.ragged_lengths(3000, 16, 16384, seed=4)
    rng = np.random.default_rng(0)
    lines = np.concatenate([np.argsort(-lengths)[:20], rng.choice(len(lengths), 180, replace=False)])
    err, plan = _run(lengths, 4, precision, check_lines=np.unique(lines))
    assert err <= TOL[precision]
    st, iters = plan.last_error()
    assert st == 0


def test_many_short_lines_share_blocks():
    lengths = np.full(5000, 5, np.int32)
    err, plan = _run(lengths, 7, "f64")
    assert err <= 1e-12
    assert plan.config["lines_per_block"] > 1


@pytest.mark.parametrize("precision", ["f64", "f32r"])
def test_ragged_backward_matches_oracle_adjoint(precision):
    lengths = np.array([3, 700, 16, 5000, 33, 2, 129], np.int32)
    r = synth.ragged_general(lengths, 9, device="cuda", fp32_coefficients=precision != "f64")
    keys = ("a", "b", "c") if precision == "f64" else ("a32", "b32", "c32")
    a, b, c = (r[k] for k in keys)
    d = r["d"]
    x, plan = tdma.solve_ragged(a, b, c, d, r["offsets"], r["lengths"], precision=precision, check=True)
    w = torch.randn_like(x)
    ga, gb, gc, gd = (torch.empty_like(a), torch.empty_like(b), torch.empty_like(c), torch.empty_like(x))
    plan.backward(a, b, c, x, w, ga, gb, gc, gd)
    torch.cuda.synchronize()
    offs, lens = r["offsets"].cpu().numpy(), r["lengths"].cpu().numpy()
    h = lambda t: t.double().cpu().numpy()
    for l, (o, n) in enumerate(zip(offs, lens)):
        s = slice(o, o + n)
        ref = O.adjoint_grads(h(a)[s], h(b)[s], h(c)[s], h(x)[s], h(w)[s])
        assert O.rel_l2(h(gd)[s], ref[3]) <= 1e-12
        tol = 1e-12 if precision == "f64" else 1e-6
        for got, want in zip((ga, gb, gc), ref[:3]):
            assert O.rel_l2(h(got)[s], want) <= tol
