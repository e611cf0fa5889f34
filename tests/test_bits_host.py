"""The integer-pipe FP64 <-> float-pair paths of the refinement kernels (csrc/bits.cuh), compiled
for the host and checked bit for bit against the plain conversions on millions of values."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_split_and_widen_match_plain_conversions():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "bits_check")
        subprocess.run([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2509_03933_gb300", "csrc"),
                        "-I", os.path.join(ROOT, "include"), "-o", exe, os.path.join(ROOT, "tests", "bits_check.cu")],
                       check=True, capture_output=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("OK"), out.stdout


def _exact_trunc_float(v):
    """(sign, value) of the Fraction v truncated to 24 significant bits (0 below 2^-126)."""
    from fractions import Fraction
    if v == 0:
        return 0.0
    s = -1.0 if v < 0 else 1.0
    a = abs(v)
    p = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** p > a:
        p -= 1
    if p < -126:  # below the normal float range: flushed to zero
        return s * 0.0
    m = int(a / Fraction(2) ** (p - 23))  # floor: 24-bit significand
    return s * float(Fraction(m) * Fraction(2) ** (p - 23))


def test_exact_residual_matches_rational_arithmetic():
    import random
    import struct
    from fractions import Fraction
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    rng = random.Random(5)
    cases = []
    for k in range(3000):
        mag = 10.0 ** rng.uniform(-30, 30)
        a, b, c = (rng.uniform(-2, 2) * mag for _ in range(3))
        xm, x, xp = (rng.uniform(-3, 3) * 10.0 ** rng.uniform(-5, 5) for _ in range(3))
        if k % 3 == 0:  # a row nearly satisfied in FP64: the residual cancels to a few ulps
            d = a * xm + b * x + c * xp
        elif k % 3 == 1:
            d = (a * xm + b * x + c * xp) * (1 + rng.uniform(-1e-9, 1e-9))
        else:
            d = rng.uniform(-5, 5) * mag
        if k % 50 == 7:
            a = 0.0
        if k % 50 == 11:
            xp = -0.0
        cases.append((d, a, xm, b, x, c, xp))
    cases.append((1.0, float("inf"), 1.0, 1.0, 1.0, 1.0, 1.0))
    hexd = lambda v: format(struct.unpack("<Q", struct.pack("<d", v))[0], "x")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "residual_check")
        subprocess.run([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2509_03933_gb300", "csrc"),
                        "-I", os.path.join(ROOT, "include"), "-o", exe, os.path.join(ROOT, "tests", "residual_check.cu")],
                       check=True, capture_output=True)
        inp = "\n".join(" ".join(hexd(v) for v in cs) for cs in cases) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, timeout=120).stdout.split()
    assert len(out) == len(cases)
    got = [struct.unpack("<f", struct.pack("<I", int(h, 16)))[0] for h in out]
    assert got[-1] != got[-1]  # NaN for a non-finite operand
    for (d, a, xm, b, x, c, xp), g in zip(cases[:-1], got[:-1]):
        F = Fraction
        terms = [F(d), -F(a) * F(xm), -F(b) * F(x), -F(c) * F(xp)]
        exact = sum(terms)
        want = _exact_trunc_float(exact)
        big = max(abs(t) for t in terms)
        tol = abs(exact) * F(2) ** -22 + big * F(2) ** -103
        assert abs(F(g) - F(want)) <= tol, (d, a, xm, b, x, c, xp, g, want)
        if abs(exact) > big * F(2) ** -75:  # the truncated tail is far below the result: the same bits
            assert g == want or abs(F(g) - exact) <= abs(exact) * F(2) ** -23
