"""ctypes binding of the C FP64 Thomas oracle (``thomas_c.c``), built with gcc on first use.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the CPU baseline leg and reference arm of
``bench.py`` time it on the host's cores; the tests pin it. It computes what ``thomas`` in
``tdma_oracle.py`` computes (Section 1, the Thomas algorithm), in plain C with OpenMP over
blocks of adjacent lines.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "thomas_c.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle_thomas.so")

_lib = None
_openmp = None


def build(force: bool = False) -> str:
    """Compile thomas_c.c into _build/liboracle_thomas.so (gcc, OpenMP when available)."""
    global _openmp
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", tmp]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:  # no OpenMP runtime: one thread
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"gcc failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.oracle_thomas.argtypes = [ctypes.c_int64] * 4 + [dp] * 5 + [ctypes.c_int]
        _lib.oracle_thomas.restype = ctypes.c_int
        _lib.oracle_max_threads.restype = ctypes.c_int
    return _lib


def max_threads() -> int:
    """Threads the C oracle can use (the OpenMP default: the host's cores)."""
    return int(_load().oracle_max_threads())


# Arm CPU part numbers (MIDR part field) of the server cores this runs on
_ARM_PARTS = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1",
              "0xd49": "Arm Neoverse N2", "0xd84": "Arm Neoverse V3"}


def cpu_model() -> str:
    """The host CPU's model name: /proc/cpuinfo's model name (x86), else lscpu's, else the Arm part
    number, else the machine type."""
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields.setdefault(k.strip().lower(), v.strip())
    except OSError:
        pass
    if fields.get("model name"):
        return fields["model name"]
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                name = line.split(":", 1)[1].strip()
                if name and name != "-":
                    return name
    except (OSError, subprocess.SubprocessError):
        pass
    part = fields.get("cpu part", "").lower()
    if part:
        return _ARM_PARTS.get(part, f"Arm CPU part {part}")
    return platform.processor() or platform.machine()


def _ptr(t):
    return t.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def solve_strided(n, n_lines, row_stride, line_stride, a, b, c, d, x, threads=None):
    """x = A^{-1} d for n_lines lines of n unknowns; unknown i of line l at element
    l * line_stride + i * row_stride of the flat float64 arrays a, b, c, d, x (x may be d)."""
    arrs = [np.ascontiguousarray(t, dtype=np.float64) if t is not x else t for t in (a, b, c, d)]
    assert x.dtype == np.float64 and x.flags.c_contiguous
    threads = max_threads() if threads is None else int(threads)
    st = _load().oracle_thomas(int(n), int(n_lines), int(row_stride), int(line_stride), *(_ptr(t) for t in arrs),
                               _ptr(x), threads)
    if st != 0:
        raise RuntimeError("oracle_thomas failed")
    return x


def thomas(a, b, c, d, threads=None):
    """Lines on axis 0, rows on axis 1 (arrays of shape (lines, n)); returns x."""
    a, b, c, d = (np.ascontiguousarray(t, dtype=np.float64) for t in (a, b, c, d))
    lines, n = b.shape
    x = np.empty_like(d)
    return solve_strided(n, lines, 1, n, a, b, c, d, x, threads)
