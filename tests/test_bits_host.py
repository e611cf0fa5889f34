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
