"""FP64 pivots outside the normal range of the reciprocal seed, checked on the host.

The FP64 sweeps form 1/w from the hardware's approximate reciprocal, which flushes subnormals
to zero in its input and output: a pivot at or beyond 2^1022 (reciprocal below the normal range)
would give 0, a finite value that no finiteness check sees, and a subnormal pivot would look like
a zero. Such pivots take the IEEE division: a huge pivot gives its correctly rounded reciprocal,
and a subnormal pivot (reciprocal beyond the double range) is reported as TDMA_ERR_NONFINITE."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2509_03933_gb300 as tdma

pytestmark = pytest.mark.gpu


def _lines(n, lines, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1, 0, (n, lines))
    c = rng.uniform(-1, 0, (n, lines))
    b = 2 + np.abs(a) + np.abs(c) + rng.uniform(0, 1, (n, lines))
    x = rng.uniform(1, 2, (n, lines))
    return a, b, c, x


def _apply(a, b, c, x):
    d = b * x
    d[1:] += a[1:] * x[:-1]
    d[:-1] += c[:-1] * x[1:]
    return d


@pytest.mark.parametrize("partitions", [1, 4])
def test_pivots_beyond_2_pow_1022_are_solved(partitions):
    n, lines = 16, 300
    a, b, c, x = _lines(n, lines, 3 + partitions)
    huge = np.arange(0, lines, 5)  # every fifth line: decoupled rows with pivots near the top
    a[:, huge], c[:, huge] = 0.0, 0.0
    b[:, huge] = np.ldexp(1.0 + np.random.default_rng(1).uniform(0, 0.9, (n, len(huge))), 1022)
    d = _apply(a, b, c, x)
    assert np.all(np.isfinite(d))
    t = [torch.from_numpy(v).cuda() for v in (a, b, c, d)]
    got = tdma.solve(*t, axis=0, partitions=partitions, check=True).cpu().numpy()
    ref = O.thomas(a.T, b.T, c.T, d.T).T
    assert np.max(np.abs(got[:, huge] - x[:, huge]) / x[:, huge]) <= 1e-14
    assert O.rel_l2(got, ref) <= 1e-12
    per_line = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert per_line.max() <= 1e-12


@pytest.mark.parametrize("partitions", [1, 4])
def test_subnormal_pivot_is_reported(partitions):
    n, lines = 16, 64
    a, b, c, x = _lines(n, lines, 11)
    a[:, 9], c[:, 9] = 0.0, 0.0
    b[5, 9] = np.ldexp(1.0, -1060)  # subnormal: its reciprocal is beyond the double range
    d = _apply(a, b, c, x)
    t = [torch.from_numpy(v).cuda() for v in (a, b, c, d)]
    with pytest.raises(tdma.TDMAError) as exc:
        tdma.solve(*t, axis=0, partitions=partitions, check=True)
    assert exc.value.status == 5
