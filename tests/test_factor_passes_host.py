"""The segmented factorisation of the shared-coefficient kernels, emulated in numpy: the warp's 32
segments start from estimates composed from 2x2 matrix products of the fractional map
c'_i = sup_i / (b_i - sub_i c'_{i-1}), then rerun the plain recurrence with each segment's start
taken from the previous segment's end until no start changes. The fixed point is the serial
recurrence bit for bit, reached within 32 passes, and within 2 on diagonally dominant lines."""
import math

import numpy as np
import pytest


def _serial(sub, b, sup):
    c = 0.0
    out = np.zeros(len(b))
    for i in range(len(b)):
        w = 1.0 / (b[i] - sub[i] * c)
        c = sup[i] * w
        out[i] = c
    return out


def _rescale(P):
    m = np.abs(P).max()
    if m > 0 and np.isfinite(m):
        P = P * 2.0 ** (-(math.frexp(m)[1] - 1))
    return P


def _segmented(sub, b, sup, chunk=2016):
    n = len(b)
    cp = np.zeros(n)
    carry = 0.0
    passes = []
    for i0 in range(0, n, chunk):
        rows = min(chunk, n - i0)
        seg = (rows + 31) // 32
        bounds = [(min(k * seg, rows), min(min(k * seg, rows) + seg, rows)) for k in range(32)]
        prods = []
        for r0, r1 in bounds:
            P = np.eye(2)
            for r in range(r0, r1):
                P = _rescale(np.array([[0.0, sup[i0 + r]], [-sub[i0 + r], b[i0 + r]]])) @ P
            prods.append(_rescale(P))
        scan = [prods[0]]
        for k in range(1, 32):
            scan.append(_rescale(prods[k] @ scan[-1]))
        start = [carry] + [(E[0, 0] * carry + E[0, 1]) / (E[1, 0] * carry + E[1, 1]) for E in scan[:-1]]
        for p in range(33):
            ends = []
            for k, (r0, r1) in enumerate(bounds):
                c = start[k]
                for r in range(r0, r1):
                    w = 1.0 / (b[i0 + r] - sub[i0 + r] * c)
                    c = sup[i0 + r] * w
                    cp[i0 + r] = c
                ends.append(c if r1 > r0 else start[k])
            nxt = [carry] + ends[:-1]
            changed = any(r1 > r0 and nxt[k] != start[k] for k, (r0, r1) in enumerate(bounds))
            start = nxt
            if not changed:
                break
        passes.append(p + 1)
        carry = ends[max(k for k, (r0, r1) in enumerate(bounds) if r1 > r0)]
    return cp, passes


@pytest.mark.parametrize("n", [5, 100, 512, 3000])
@pytest.mark.parametrize("kind", ["general", "weak", "laplacian"])
def test_segmented_factorisation_is_the_serial_recurrence(n, kind):
    rng = np.random.default_rng(n)
    if kind == "general":
        a, c = -rng.random(n), -rng.random(n)
        b = 2 + np.abs(a) + np.abs(c) + rng.random(n)
    else:
        a, c = -np.ones(n), -np.ones(n)
        b = np.full(n, 2.001 if kind == "weak" else 2.0)
    sub = np.r_[0.0, a[1:]]
    sup = np.r_[c[:-1], 0.0]
    cp, passes = _segmented(sub, b, sup)
    assert np.array_equal(cp, _serial(sub, b, sup))  # bit for bit
    assert max(passes) <= 33
    if kind == "general":
        assert max(passes) <= 2
