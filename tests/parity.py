"""Error measures of the GPU parity tests.

A pooled relative L2 error over many lines can hide one bad line among many good ones, so the
parity tests bound both the pooled error and the worst relative L2 error of any single line:
``rel_err(got, ref)`` is the larger of the two, with lines on axis 0 (any trailing axes, such as
rows and right-hand sides, belong to the line). Lines packed back to back (ragged batches) are
split by their lengths first (``rel_err_packed``).
"""
import numpy as np

import oracle as O


def per_line(got, ref) -> np.ndarray:
    """Relative L2 error of every line (axis 0); a line whose reference is zero gets its absolute
    error."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if got.size != ref.size:
        raise ValueError(f"shapes differ: {got.shape} vs {ref.shape}")
    got = got.reshape(ref.shape)
    if ref.ndim <= 1:
        return np.array([O.rel_l2(got, ref)])
    g = got.reshape(ref.shape[0], -1)
    r = ref.reshape(ref.shape[0], -1)
    num = np.linalg.norm(g - r, axis=1)
    den = np.linalg.norm(r, axis=1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def rel_err(got, ref) -> float:
    """max(pooled relative L2 error, worst per-line relative L2 error); lines on axis 0."""
    return max(O.rel_l2(got, ref), float(per_line(got, ref).max()))


def rel_err_packed(got, ref, lengths) -> float:
    """As rel_err for 1D arrays holding lines of the given lengths back to back."""
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    if got.size != ref.size or int(np.sum(lengths)) != ref.size:
        raise ValueError("lengths do not cover the arrays")
    worst, s = 0.0, 0
    for n in lengths:
        n = int(n)
        worst = max(worst, O.rel_l2(got[s:s + n], ref[s:s + n]))
        s += n
    return max(O.rel_l2(got, ref), worst)
