"""Ragged batches in FP32 storage + refinement on the chunk kernel (packed unit-stride lines, one
chunk of whole lines per CTA cluster) against the oracle, including the layouts that change how
chunks are cut: lines out of memory order, gaps between lines, the longest line a chunk holds,
thousands of one-row lines, lines that need a second correction, and x written over d."""
import os

import numpy as np
import pytest
import torch

import oracle as O
from parity import rel_err, rel_err_packed
import synth
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu

PACKED = 9        # TDMA_VARIANT_PACKED
RAGGED = 3        # TDMA_VARIANT_RAGGED
CHUNK_ROWS = 18816  # longest line the chunk kernel takes (4 CTAs x 224 partitions x 21 rows)


def _oracle(a, b, c, d, offs, lens, lines=None, dtype=np.float64):
    h = lambda t: t.double().cpu().numpy()
    return O.thomas_ragged(h(a), h(b), h(c), h(d), offs, lens, lines=lines, dtype=dtype)


def _err(x, ref, offs, lens):
    xs = x.double().cpu().numpy()
    got = np.concatenate([xs[offs[l]:offs[l] + lens[l]] for l in sorted(ref)])
    want = np.concatenate([ref[l] for l in sorted(ref)])
    return rel_err_packed(got, want, [lens[l] for l in sorted(ref)])


def _problem(lengths, seed):
    r = synth.ragged_general(np.asarray(lengths, np.int32), seed, device="cuda", fp32_coefficients=True)
    return r["a32"], r["b32"], r["c32"], r["d"], r["offsets"], r["lengths"]


def _solve(a, b, c, d, offs, lens, out=None, check=True, **kw):
    x, plan = tdma.solve_ragged(a, b, c, d, offs, lens, precision="f32r", out=out, check=check, **kw)
    return x, plan


@pytest.mark.parametrize("lengths", [
    [1, 2, 3, 4, 5, 7, 16, 17, 31, 33, 100, 257, 1000, 4097, 2, 64, 65, 1, 12, 300],
    [CHUNK_ROWS],
    [CHUNK_ROWS, CHUNK_ROWS, 1, CHUNK_ROWS - 1],
    [5],
    [895, 896, 897, 1792, 1793, 3583, 8961],
    [20] * 900,
])
def test_packed_matches_oracle(lengths):
    a, b, c, d, offs, lens = _problem(lengths, 11)
    x, plan = _solve(a, b, c, d, offs, lens)
    assert plan.config["variant"] == PACKED
    err = _err(x, _oracle(a, b, c, d, offs.cpu().numpy(), lens.cpu().numpy()), offs.cpu().numpy(),
               lens.cpu().numpy())
    assert err <= 1e-12


def test_packed_many_one_row_lines():
    lengths = np.ones(5000, np.int32)
    lengths[::7] = 3
    a, b, c, d, offs, lens = _problem(lengths, 12)
    x, plan = _solve(a, b, c, d, offs, lens)
    assert plan.config["variant"] == PACKED
    o, n = offs.cpu().numpy(), lens.cpu().numpy()
    assert _err(x, _oracle(a, b, c, d, o, n), o, n) <= 1e-12


def test_packed_log_uniform_batch_sampled():
    lengths = synth.ragged_lengths(3000, 16, 16384, seed=4)
    a, b, c, d, offs, lens = _problem(lengths, 4)
    x, plan = _solve(a, b, c, d, offs, lens, check=False)
    assert plan.config["variant"] == PACKED
    o, n = offs.cpu().numpy(), lens.cpu().numpy()
    rng = np.random.default_rng(0)
    lines = np.unique(np.concatenate([np.argsort(-lengths)[:20], rng.choice(len(lengths), 180, replace=False)]))
    assert _err(x, _oracle(a, b, c, d, o, n, lines=lines), o, n) <= 1e-12
    st, iters = plan.last_error()
    assert st == 0 and iters >= 1


def test_packed_lines_out_of_memory_order_and_gaps():
    # the same lines described in a shuffled order, then with gaps between them in memory
    lengths = np.array([40, 3000, 7, 17000, 1, 900, 2, 5000, 64], np.int32)
    a, b, c, d, offs, lens = _problem(lengths, 13)
    perm = np.random.default_rng(1).permutation(len(lengths))
    offs_p, lens_p = offs[torch.from_numpy(perm).cuda()], lens[torch.from_numpy(perm).cuda()]
    x, plan = _solve(a, b, c, d, offs_p, lens_p)
    assert plan.config["variant"] == PACKED
    o, n = offs.cpu().numpy(), lens.cpu().numpy()
    ref = _oracle(a, b, c, d, o, n)
    assert _err(x, ref, o, n) <= 1e-12
    # gaps: every line shifted by 3 elements per preceding line; the gap elements stay untouched
    gap = 3
    o2 = o + gap * np.arange(len(o))
    total = int(o2[-1] + n[-1])
    sp = lambda t, fill: torch.full((total,), fill, dtype=t.dtype, device="cuda")
    a2, b2, c2, d2 = sp(a, 0.0), sp(b, 1.0), sp(c, 0.0), sp(d, 0.0)
    for l in range(len(o)):
        for src, dst in ((a, a2), (b, b2), (c, c2), (d, d2)):
            dst[o2[l]:o2[l] + n[l]] = src[o[l]:o[l] + n[l]]
    x2 = torch.full_like(d2, 7.0)
    offs2 = torch.from_numpy(o2).cuda()
    x2, plan2 = _solve(a2, b2, c2, d2, offs2, lens, out=x2)
    assert plan2.config["variant"] == PACKED
    assert _err(x2, ref, o2, n) <= 1e-12
    mask = torch.ones(total, dtype=torch.bool, device="cuda")
    for l in range(len(o)):
        mask[o2[l]:o2[l] + n[l]] = False
    assert bool((x2[mask] == 7.0).all())  # nothing outside the lines is written


def test_packed_in_place_and_repeated_solves():
    lengths = synth.ragged_lengths(400, 16, 16384, seed=5)
    a, b, c, d, offs, lens = _problem(lengths, 14)
    o, n = offs.cpu().numpy(), lens.cpu().numpy()
    ref = _oracle(a, b, c, d, o, n)
    x1, plan = _solve(a, b, c, d, offs, lens)
    x2, _ = _solve(a, b, c, d, offs, lens, plan=plan)
    assert torch.equal(x1, x2)  # the per-line maxima are back at zero after every launch
    dd = d.clone()
    _solve(a, b, c, dd, offs, lens, out=dd, plan=plan)  # x over d
    assert _err(dd, ref, o, n) <= 1e-12


def test_packed_second_correction_for_weakly_dominant_lines():
    # tridiag(-1, 2.01, -1) has condition number about 400: the float solve is good to about 1e-5,
    # one correction leaves about 1e-10 and the stop rule asks for more (the rare path that reads x
    # back); the rows' dominance (1 - 2 / 2.01 = 5e-3) certifies the float-pair residual's floor
    # below the tolerance, so the line converges; the reference is the extended-precision oracle
    lengths = np.array([3000, 50, 17000, 700], np.int32)
    a, b, c, d, offs, lens = _problem(lengths, 15)
    o, n = offs.cpu().numpy(), lens.cpu().numpy()
    a.fill_(-1.0)
    c.fill_(-1.0)
    b.fill_(2.01)
    A, B, C = a.double(), b.double(), c.double()
    xt = torch.sin(torch.arange(a.numel(), device="cuda", dtype=torch.float64) * 0.37)
    dn = B * xt
    for l in range(len(o)):
        s, e = o[l], o[l] + n[l]
        dn[s + 1:e] += A[s + 1:e] * xt[s:e - 1]
        dn[s:e - 1] += C[s:e - 1] * xt[s + 1:e]
    x, plan = _solve(a, b, c, dn, offs, lens, check=False)
    assert plan.config["variant"] == PACKED
    st, iters = plan.last_error()
    assert st == 0
    assert iters >= 2
    assert _err(x, _oracle(a, b, c, dn, o, n, dtype=np.longdouble), o, n) <= 1e-12


def _weak(lengths, seed):
    """tridiag(-1, 2.01, -1) lines (condition number about 400: the stop rule asks for a second
    correction) with the right-hand side of a known smooth solution."""
    a, b, c, d, offs, lens = _problem(lengths, seed)
    o, n = offs.cpu().numpy(), lens.cpu().numpy()
    a.fill_(-1.0)
    c.fill_(-1.0)
    b.fill_(2.01)
    xt = torch.sin(torch.arange(a.numel(), device="cuda", dtype=torch.float64) * 0.37)
    dn = 2.01 * xt
    for l in range(len(o)):
        s, e = o[l], o[l] + n[l]
        dn[s + 1:e] -= xt[s:e - 1]
        dn[s:e - 1] -= xt[s + 1:e]
    return a, b, c, dn, offs, lens, o, n


def test_packed_second_correction_in_place():
    # x over d: the chunk kernel keeps d's float pairs and makes the further corrections itself
    a, b, c, dn, offs, lens, o, n = _weak(np.array([3000, 50, 17000, 700], np.int32), 15)
    ref = _oracle(a, b, c, dn, o, n, dtype=np.longdouble)
    xd = dn.clone()
    _, plan = _solve(a, b, c, xd, offs, lens, out=xd, check=False)
    assert plan.config["variant"] == PACKED
    st, iters = plan.last_error()
    assert st == 0 and iters >= 2
    assert _err(xd, ref, o, n) <= 1e-12


def test_packed_every_chunk_corrected_again():
    # Out of place every chunk is listed for the further-correction launch, more chunks than
    # clusters, so each cluster of that launch takes several; in place the same in the chunk kernel
    lengths = synth.ragged_lengths(3000, 16, 16384, seed=12)
    a, b, c, dn, offs, lens, o, n = _weak(lengths, 16)
    x, plan = _solve(a, b, c, dn, offs, lens, check=False)
    assert plan.config["variant"] == PACKED
    assert int(n.sum()) > CHUNK_ROWS * (plan.config["blocks"] // 4)  # more chunks than clusters
    st, iters = plan.last_error()
    assert st == 0 and iters >= 2
    lines = sorted(set(np.random.default_rng(3).choice(len(o), 40, replace=False).tolist()) | {int(np.argmax(n))})
    ref = _oracle(a, b, c, dn, o, n, lines=lines, dtype=np.longdouble)
    assert _err(x, ref, o, n) <= 1e-12
    xd = dn.clone()
    _solve(a, b, c, xd, offs, lens, out=xd, check=False, plan=plan)
    st2, iters2 = plan.last_error()
    assert st2 == 0 and iters2 >= 2
    assert torch.equal(xd, x)  # the same passes in either kernel


def test_packed_stop_rule_run_out_and_nonfinite_values():
    # Chunks whose lines fail the local stop test go to the rule on the line maxima after the last
    # chunk: an unreachable tolerance runs max_refine_iters corrections and reports
    # TDMA_ERR_NOT_CONVERGED (7), with x still as good as the corrections make it; a NaN in d
    # reports TDMA_ERR_NONFINITE (5); the plan's next launch, on clean data, reports 0 again.
    lengths = synth.ragged_lengths(300, 16, 16384, seed=9)
    a, b, c, d, offs, lens = _problem(lengths, 21)
    o, n = offs.cpu().numpy(), lens.cpu().numpy()
    ref = _oracle(a, b, c, d, o, n)
    x, plan = _solve(a, b, c, d, offs, lens, check=False, max_refine_iters=3, refine_tol=1e-30)
    assert plan.config["variant"] == PACKED
    assert plan.last_error() == (7, 3)
    assert _err(x, ref, o, n) <= 1e-12
    x, plan = _solve(a, b, c, d, offs, lens, check=False, max_refine_iters=1, refine_tol=1e-30)
    assert plan.last_error() == (7, 1)
    bad = d.clone()
    bad[int(o[5]) + int(n[5]) // 2] = float("nan")
    x, plan = _solve(a, b, c, bad, offs, lens, check=False)
    assert plan.last_error()[0] == 5
    x, _ = _solve(a, b, c, d, offs, lens, check=False, plan=plan)
    assert plan.last_error()[0] == 0
    assert _err(x, ref, o, n) <= 1e-12


def test_packed_agrees_with_group_kernel():
    lengths = synth.ragged_lengths(500, 16, 16384, seed=6)
    a, b, c, d, offs, lens = _problem(lengths, 16)
    x1, p1 = _solve(a, b, c, d, offs, lens)
    os.environ["TDMA_DISABLE_PACKED"] = "1"
    try:
        x2, p2 = _solve(a, b, c, d, offs, lens)
    finally:
        del os.environ["TDMA_DISABLE_PACKED"]
    assert (p1.config["variant"], p2.config["variant"]) == (PACKED, RAGGED)
    assert O.rel_l2(x1.cpu().numpy(), x2.cpu().numpy()) <= 2e-12


def test_line_longer_than_a_chunk_uses_group_kernel():
    lengths = np.array([CHUNK_ROWS + 1, 10], np.int32)
    a, b, c, d, offs, lens = _problem(lengths, 17)
    x, plan = _solve(a, b, c, d, offs, lens)
    assert plan.config["variant"] == RAGGED
    o, n = offs.cpu().numpy(), lens.cpu().numpy()
    assert _err(x, _oracle(a, b, c, d, o, n), o, n) <= 1e-12


def _grads(a, b, c, x, w, plan):
    ga, gb, gc, gd = (torch.empty_like(a), torch.empty_like(b), torch.empty_like(c), torch.empty_like(x))
    plan.backward(a, b, c, x, w, ga, gb, gc, gd)
    torch.cuda.synchronize()
    return ga, gb, gc, gd


def test_packed_backward_matches_group_kernel_and_oracle():
    # the adjoint solve A^T lambda = w on the chunk kernel (transposed rows) against the group
    # kernel and, on sampled lines, against the oracle's adjoint
    lengths = synth.ragged_lengths(400, 16, 16384, seed=7)
    a, b, c, d, offs, lens = _problem(lengths, 18)
    x, p1 = _solve(a, b, c, d, offs, lens)
    w = synth.normal(18, synth.AID["w"], torch.arange(x.numel(), device="cuda"))
    g1 = _grads(a, b, c, x, w, p1)
    assert p1.last_error()[0] == 0
    os.environ["TDMA_DISABLE_PACKED"] = "1"
    try:
        _, p2 = _solve(a, b, c, d, offs, lens)
    finally:
        del os.environ["TDMA_DISABLE_PACKED"]
    g2 = _grads(a, b, c, x, w, p2)
    assert O.rel_l2(g1[3].cpu().numpy(), g2[3].cpu().numpy()) <= 2e-12
    o, n = offs.cpu().numpy(), lens.cpu().numpy()
    h = lambda t: t.double().cpu().numpy()
    for l in list(np.argsort(-n)[:3]) + [int(np.argmin(n)), 17, 200]:
        s = slice(o[l], o[l] + n[l])
        ref = O.adjoint_grads(h(a)[s], h(b)[s], h(c)[s], h(x)[s], h(w)[s])
        assert O.rel_l2(h(g1[3])[s], ref[3]) <= 1e-12
        for got, want in zip(g1[:3], ref[:3]):
            assert O.rel_l2(h(got)[s], want) <= 1e-6  # float gradients of float coefficients


def test_packed_backward_second_correction():
    # tridiag(-1, 2.01, -1) (condition number about 400, its own transpose): the adjoint solve on
    # the transposed rows needs more than one correction too; the nonsymmetric case is covered
    # against the group kernel above
    lengths = np.array([4000, 9000, 31], np.int32)
    a, b, c, d, offs, lens = _problem(lengths, 19)
    a.fill_(-1.0)
    c.fill_(-1.0)
    b.fill_(2.01)
    x, plan = _solve(a, b, c, d, offs, lens)
    w = torch.cos(torch.arange(x.numel(), device="cuda", dtype=torch.float64) * 0.11)
    g = _grads(a, b, c, x, w, plan)
    st, iters = plan.last_error()
    assert st == 0 and iters >= 2
    o, n = offs.cpu().numpy(), lens.cpu().numpy()
    h = lambda t: t.double().cpu().numpy()
    for l in range(len(o)):
        s = slice(o[l], o[l] + n[l])
        at, bt, ct = O.transpose_coefficients(h(a)[s], h(b)[s], h(c)[s])
        assert O.rel_l2(h(g[3])[s], O.thomas_ext(at, bt, ct, h(w)[s])) <= 1e-12


@pytest.mark.parametrize("n,L,gap", [(1000, 300, 0), (CHUNK_ROWS, 3, 0), (5000, 40, 16), (37, 2000, 0), (2, 9, 3)])
def test_uniform_unit_stride_lines_use_the_chunk_kernel(n, L, gap):
    # uniform lines along the contiguous axis in FP32 + refinement whose length is not one the
    # merge-tree kernel takes (n = 256, 512, 1024): whole contiguous lines form the chunks (a gap
    # between lines ends a chunk); x between the lines stays untouched
    g = synth.grid_general((L, n + gap), 1, 20 + n, device="cuda", fp32_coefficients=True)
    a, b, c = (g[k][:, :n] for k in ("a32", "b32", "c32"))
    d = g["d"][:, :n]
    plan = tdma.Plan(*tdma.line_layout(d, 1), precision="f32r")
    assert plan.config["variant"] == PACKED
    x = torch.full((L, n + gap), 7.0, dtype=torch.float64, device="cuda")
    plan.solve(a, b, c, d, x[:, :n])
    assert plan.last_error()[0] == 0
    ref = O.thomas(*(t.double().cpu().numpy() for t in (a, b, c, d)))
    assert rel_err(x[:, :n].cpu().numpy(), ref) <= 1e-12
    if gap:
        assert bool((x[:, n:] == 7.0).all())
    if n <= 5000:  # explicit partitions keep the partition kernels
        fixed = tdma.Plan(*tdma.line_layout(d, 1), precision="f32r", partitions=1 if n < 4 else 2)
        assert fixed.config["variant"] != PACKED


def test_backward_with_group_kernel_forward_and_chunk_tables(tmp_path):
    # A ragged FP32 + refinement plan whose forward pass runs the group kernel (a cached choice, as
    # after an autotune that picked it) while the chunk kernel's tables exist: the adjoint solve
    # runs the chunk kernel with the chunk kernel's own configuration. The choice is seeded through
    # the tuning cache file, read once per process, so the check runs in a child process.
    import subprocess
    import sys
    lengths = synth.ragged_lengths(300, 16, 16384, seed=21)
    lb = lambda v: int(max(1, int(v))).bit_length() - 1
    key = f"ragged p2 l{lb(len(lengths))} m{lb(lengths.max())} t{lb(lengths.sum())}"
    path = tmp_path / "tune.txt"
    path.write_text(f"{key}|{RAGGED}|16\n")
    code = (
        "import sys, os, numpy as np, torch; sys.path.insert(0, os.getcwd())\n"
        "import oracle as O, synth, paper_2509_03933_gb300 as tdma\n"
        "lengths = synth.ragged_lengths(300, 16, 16384, seed=21)\n"
        "r = synth.ragged_general(lengths, 21, device='cuda', fp32_coefficients=True)\n"
        "a, b, c, d = r['a32'], r['b32'], r['c32'], r['d']\n"
        "x, plan = tdma.solve_ragged(a, b, c, d, r['offsets'], r['lengths'], precision='f32r')\n"
        f"assert plan.config['variant'] == {RAGGED}, plan.config\n"
        "assert plan.last_error()[0] == 0\n"
        "w = synth.normal(21, synth.AID['w'], torch.arange(r['total'], device='cuda'))\n"
        "ga, gb, gc, gd = (torch.empty_like(a), torch.empty_like(b), torch.empty_like(c), torch.empty_like(x))\n"
        "plan.backward(a, b, c, x, w, ga, gb, gc, gd)\n"
        "assert plan.last_error()[0] == 0\n"
        "offs, lens = r['offsets'].cpu().numpy(), r['lengths'].cpu().numpy()\n"
        "ha, hb, hc = (r[k].cpu().numpy() for k in ('a', 'b', 'c'))\n"
        "xs, hw, hg = x.cpu().numpy(), w.cpu().numpy(), gd.cpu().numpy()\n"
        "worst = 0.0\n"
        "for l in list(np.argsort(-lengths)[:3]) + list(range(0, 300, 29)):\n"
        "    s = slice(offs[l], offs[l] + lens[l])\n"
        "    worst = max(worst, O.rel_l2(hg[s], O.adjoint_grads(ha[s], hb[s], hc[s], xs[s], hw[s])[3]))\n"
        "print('worst', worst)\n"
        "assert worst <= 1e-12, worst\n")
    env = dict(os.environ, TDMA_AUTOTUNE_CACHE=str(path))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    run = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=600)
    assert run.returncode == 0, run.stdout + run.stderr
