"""The seeded input generators: counter-based draws agree across backends and match the
distributions the workloads name."""
import numpy as np
import torch

import synth


def test_uniform_torch_equals_numpy_bitwise():
    idx = np.concatenate([np.arange(5000), np.array([2**30 - 1, 2**30, 2**39 + 17])])
    for seed, aid in ((0, 1), (3, 4), (4, 9), (65535, 255)):
        u_np = synth.uniform_np(seed, aid, idx)
        u_t = synth.uniform(seed, aid, torch.from_numpy(idx.astype(np.int64))).numpy()
        assert np.array_equal(u_np, u_t)
        assert u_np.min() >= 0.0 and u_np.max() < 1.0


def test_uniform_moments_and_independence():
    u = synth.uniform_np(0, 1, np.arange(200000))
    v = synth.uniform_np(0, 2, np.arange(200000))
    assert abs(u.mean() - 0.5) < 5e-3 and abs(u.var() - 1 / 12) < 2e-3
    assert abs(np.corrcoef(u, v)[0, 1]) < 1e-2


def test_general_grid_distribution_and_rhs():
    g = synth.grid_general((8, 8, 8), axis=0, seed=0)
    a, b, c = g["a"], g["b"], g["c"]
    assert (a < 0).all() and (a >= -1).all() and (c < 0).all()
    margin = b - a.abs() - c.abs()
    assert (margin >= 2.0).all() and (margin <= 3.0).all()
    # d = A x_true along z
    x = g["x_true"]
    ref = b * x
    ref[1:] += a[1:] * x[:-1]
    ref[:-1] += c[:-1] * x[1:]
    assert torch.equal(g["d"], ref)


def test_fp32_coefficients_define_the_problem():
    g = synth.grid_general((4, 4, 16), axis=2, seed=3, fp32_coefficients=True)
    assert torch.equal(g["a"], g["a32"].double()) and torch.equal(g["b"], g["b32"].double())


def test_ragged_lengths_log_uniform():
    n = synth.ragged_lengths(20000, 16, 16384, seed=4)
    assert n.min() >= 16 and n.max() <= 16384
    # log-uniform: mean of ln n near the midpoint of [ln 16, ln 16385]
    assert abs(np.log(n).mean() - 0.5 * (np.log(16) + np.log(16385))) < 0.05
    r = synth.ragged_general(n[:50], seed=4)
    assert r["total"] == int(n[:50].sum())


def test_poisson_lines_shapes():
    p = synth.poisson_lines(8, 8, 32, seed=2)
    assert p["d"].shape == (32, 8, 8, 2) and p["shift"].shape == (64,)
    assert p["shift"][0] == 0.0 and (p["shift"][1:] < 0).all()
    assert float(p["d"][0, 0, 0, 0]) == 0.0


def test_sampled_block_equals_full_draw():
    full = synth.grid_general((16, 12, 10), 0, 3, fp32_coefficients=True)
    part = synth.grid_general((16, 4, 3), 0, 3, fp32_coefficients=True, full_shape=(16, 12, 10), origin=(0, 5, 6))
    for k in ("a32", "b32", "c32", "d", "x_true"):
        assert torch.equal(part[k], full[k][:, 5:9, 6:9])
