"""Builds the CUDA library (libtdma.so) in-tree for sm_103a with nvcc."""
from __future__ import annotations

import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libtdma.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _sources():
    out = []
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            if f.endswith((".cu", ".cuh", ".h")):
                out.append(os.path.join(d, f))
    return out


def nvcc_path() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    for cand in ("/usr/local/cuda/bin/nvcc",):
        if os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtdma.so")


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the csrc/*.cu translation units into _build/libtdma.so (skipped when up to date)."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tag = f".tmp{os.getpid()}"
    units = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith(".cu")]
    # every translation unit compiles in its own nvcc process, all at once; then one link
    jobs = []
    for u in units:
        obj = os.path.join(OUT_DIR, os.path.basename(u)[:-3] + tag + ".o")
        cmd = [nvcc_path(), *NVCC_FLAGS, "-I", INCLUDE, "-I", CSRC, "-c", "-o", obj, u]
        if verbose:
            print(" ".join(cmd))
        jobs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True), obj))
    failed = []
    for proc, obj in jobs:
        out, err = proc.communicate()
        if proc.returncode != 0:
            failed.append(f"{obj}: nvcc failed ({proc.returncode}):\n{out}\n{err}")
    objs = [obj for _, obj in jobs]
    try:
        if failed:
            raise RuntimeError("\n".join(failed))
        tmp = LIB + tag
        cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc_path())), "lib64")
        cmd = [nvcc_path(), *ARCH, "-shared", "-o", tmp, *objs,
               "-lcufft", "-Xlinker", f"-rpath={cuda_lib}"]  # cuFFT for the FFT-Poisson pipeline
        if verbose:
            print(" ".join(cmd))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed ({r.returncode}):\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    finally:
        for obj in objs:
            if os.path.exists(obj):
                os.remove(obj)
    return LIB
