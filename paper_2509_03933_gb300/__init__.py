"""Batched divide-and-conquer tridiagonal solves on one GB300 (Pipelined-TDMA hot path).

Thin ctypes binding over the C ABI in include/tdma.h (libtdma.so, built in-tree by
``_build.build``): argument marshalling only, every step of a solve runs in the library's
CUDA kernels. PyTorch provides device memory and streams. There is no CPU fallback: without
the library or a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import torch

from . import _build

__all__ = ["PoissonFFT", "Plan", "solve", "solve_ragged", "solve_backward", "TDMASolve", "line_layout", "TDMAError", "F64", "F32",
           "F32_REFINE", "load_library", "declared_symbols", "probe_fp64_fma", "sweep_graph", "HostPipeline", "HostLayout"]

F64, F32, F32_REFINE, F64_REFINE = 0, 1, 2, 3
_PREC = {"f64": F64, "f32": F32, "f32r": F32_REFINE, "f64r": F64_REFINE, F64: F64, F32: F32, F32_REFINE: F32_REFINE,
         F64_REFINE: F64_REFINE}
STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported configuration", 3: "workspace too small",
          4: "CUDA runtime error", 5: "zero or non-finite pivot", 6: "bounded wait timed out",
          7: "refinement did not converge"}


class TDMAError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} (status {status})")
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_lines", ctypes.c_int64), ("elem_stride", ctypes.c_int64),
                ("inner_count", ctypes.c_int64), ("inner_stride", ctypes.c_int64),
                ("outer_stride", ctypes.c_int64), ("ragged_offsets", ctypes.c_void_p),
                ("ragged_lengths", ctypes.c_void_p), ("ragged_max_n", ctypes.c_int64),
                ("ragged_total", ctypes.c_int64), ("nrhs", ctypes.c_int32), ("coef_broadcast", ctypes.c_int32),
                ("diag_shift", ctypes.c_void_p), ("precision", ctypes.c_int32), ("partitions", ctypes.c_int32),
                ("max_refine_iters", ctypes.c_int32), ("refine_tol", ctypes.c_double), ("pdd", ctypes.c_int32),
                ("refine_kappa", ctypes.c_double)]


class PoissonDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64), ("dx", ctypes.c_double),
                ("dz", ctypes.c_double), ("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("c", ctypes.c_void_p),
                ("pin_zero_mode", ctypes.c_int32), ("precision", ctypes.c_int32)]


class Config(ctypes.Structure):
    _fields_ = [("partitions", ctypes.c_int32), ("rows_per_thread", ctypes.c_int32),
                ("lines_per_block", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("blocks", ctypes.c_int32), ("smem_bytes", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_int64)]


class HostLayout(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_lines", ctypes.c_int64), ("line_stride", ctypes.c_int64),
                ("row_stride", ctypes.c_int64)]


_LIB = None
_VP = ctypes.c_void_p


def load_library(build: bool = True) -> ctypes.CDLL:
    """Load libtdma.so (building it first if it is missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libtdma.so not found at {path}; run paper_2509_03933_gb300._build.build()")
    lib = ctypes.CDLL(path)
    st = ctypes.c_int
    lib.tdma_plan_create.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(Desc), ctypes.POINTER(ctypes.c_size_t)]
    lib.tdma_plan_create.restype = st
    lib.tdma_plan_destroy.argtypes = [_VP]
    lib.tdma_plan_destroy.restype = st
    lib.tdma_solve.argtypes = [_VP] + [_VP] * 6 + [ctypes.c_size_t, _VP]
    lib.tdma_solve.restype = st
    lib.tdma_solve_backward.argtypes = [_VP] + [_VP] * 10 + [ctypes.c_size_t, _VP]
    lib.tdma_solve_backward.restype = st
    lib.tdma_plan_autotune.argtypes = [_VP] + [_VP] * 6 + [ctypes.c_size_t, _VP]
    lib.tdma_plan_autotune.restype = st
    lib.tdma_plan_get_config.argtypes = [_VP, ctypes.POINTER(Config)]
    lib.tdma_plan_get_config.restype = st
    lib.tdma_last_device_error.argtypes = [_VP, _VP, ctypes.POINTER(ctypes.c_int32)]
    lib.tdma_last_device_error.restype = st
    lib.tdma_status_string.argtypes = [ctypes.c_int]
    lib.tdma_status_string.restype = ctypes.c_char_p
    lib.tdma_solve_thomas_static.argtypes = [ctypes.POINTER(Desc)] + [_VP] * 6
    lib.tdma_solve_thomas_static.restype = st
    lib.tdma_solve_host.argtypes = [_VP, ctypes.POINTER(HostLayout)] + [_VP] * 5 + [ctypes.c_int32, _VP, _VP,
                                                                                     ctypes.c_size_t, _VP]
    lib.tdma_solve_host.restype = st
    lib.tdma_poisson_create.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(PoissonDesc),
                                        ctypes.POINTER(ctypes.c_size_t)]
    lib.tdma_poisson_create.restype = st
    lib.tdma_poisson_solve.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]
    lib.tdma_poisson_solve.restype = st
    lib.tdma_poisson_last_error.argtypes = [_VP, _VP]
    lib.tdma_poisson_last_error.restype = st
    lib.tdma_poisson_destroy.argtypes = [_VP]
    lib.tdma_poisson_destroy.restype = st
    lib.tdma_probe_fp64_fma.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _VP,
                                        ctypes.POINTER(ctypes.c_int64), _VP]
    lib.tdma_probe_fp64_fma.restype = st
    lib.tdma_probe_bounded_wait.argtypes = [ctypes.c_uint32, _VP, _VP]
    lib.tdma_probe_bounded_wait.restype = st
    lib.tdma_plan_corrected_lines.argtypes = [_VP, _VP, ctypes.POINTER(ctypes.c_int64)]
    lib.tdma_plan_corrected_lines.restype = st
    _LIB = lib
    return lib


def probe_fp64_fma(blocks: int, threads: int = 256, iters: int = 1 << 14, out=None, stream=None) -> int:
    """Enqueue the library's FP64 FMA throughput probe on ``stream``; returns the number of FMAs it
    runs (the caller times the launch). ``out``: a CUDA float64 tensor of >= ``blocks`` values."""
    lib = load_library()
    if out is None:
        out = torch.empty(blocks, dtype=torch.float64, device="cuda")
    count = ctypes.c_int64(0)
    st = lib.tdma_probe_fp64_fma(int(blocks), int(threads), int(iters), _ptr(out), ctypes.byref(count), _stream(stream))
    if st != 0:
        raise TDMAError(st, "tdma_probe_fp64_fma")
    return int(count.value)


def declared_symbols() -> list:
    """Function names declared in include/*.h."""
    names = []
    inc = _build.INCLUDE
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(tdma_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def line_layout(t: torch.Tensor, axis: int, nrhs: int = 1):
    """(n, n_lines, elem_stride, inner_count, inner_stride, outer_stride) of lines along ``axis``.

    For nrhs = 2 the tensor carries a trailing axis of 2 interleaved values (re, im) per element.
    """
    shape, strides = list(t.shape), list(t.stride())
    if nrhs == 2:
        if shape[-1] != 2 or strides[-1] != 1:
            raise ValueError("nrhs = 2 needs a trailing axis of 2 contiguous values")
        shape, strides = shape[:-1], strides[:-1]
        if any(s % 2 for s in strides):
            raise ValueError("element strides must be whole (re, im) pairs")
        strides = [s // 2 for s in strides]
    nd = len(shape)
    axis = axis % nd
    n, es = shape[axis], strides[axis]
    dims = [(shape[i], strides[i]) for i in range(nd) if i != axis and shape[i] != 1]
    merged = []
    for sz, st in dims:  # merge dims that are contiguous with the previous one
        if merged and merged[-1][1] == st * sz:
            psz, _ = merged[-1]
            merged[-1] = (psz * sz, st)
        else:
            merged.append((sz, st))
    if len(merged) == 0:
        return n, 1, es, 1, 0, 0
    if len(merged) == 1:
        return n, merged[0][0], es, merged[0][0], merged[0][1], 0
    if len(merged) == 2:
        (so, sto), (si, sti) = merged
        return n, so * si, es, si, sti, sto
    raise ValueError("lines must be addressable with at most two line axes")


class Plan:
    """A solve plan for one layout (wraps tdma_plan_t)."""

    def __init__(self, n, n_lines, elem_stride=1, inner_count=None, inner_stride=None, outer_stride=0,
                 precision="f64", partitions=0, nrhs=1, coef_broadcast=False, diag_shift=None,
                 ragged_offsets=None, ragged_lengths=None, ragged_max_n=0, ragged_total=0,
                 max_refine_iters=0, refine_tol=0.0, pdd=False, refine_kappa=0.0):
        self._lib = load_library()
        if inner_count is None:
            inner_count = max(1, n_lines)
        if inner_stride is None:
            inner_stride = n
        self._keep = (diag_shift, ragged_offsets, ragged_lengths)
        self.desc = Desc(n=n, n_lines=n_lines, elem_stride=elem_stride, inner_count=inner_count,
                         inner_stride=inner_stride, outer_stride=outer_stride,
                         ragged_offsets=_ptr(ragged_offsets), ragged_lengths=_ptr(ragged_lengths),
                         ragged_max_n=ragged_max_n, ragged_total=ragged_total, nrhs=nrhs,
                         coef_broadcast=int(bool(coef_broadcast)), diag_shift=_ptr(diag_shift),
                         precision=_PREC[precision], partitions=partitions,
                         max_refine_iters=max_refine_iters, refine_tol=refine_tol, pdd=int(bool(pdd)),
                         refine_kappa=refine_kappa)
        self._h = ctypes.c_void_p()
        ws = ctypes.c_size_t(0)
        st = self._lib.tdma_plan_create(ctypes.byref(self._h), ctypes.byref(self.desc), ctypes.byref(ws))
        if st != 0:
            raise TDMAError(st, "tdma_plan_create")
        self.workspace_bytes = ws.value
        self._ws = None

    def __del__(self):
        try:
            if getattr(self, "_h", None) and self._h.value:
                self._lib.tdma_plan_destroy(self._h)
        except Exception:
            pass

    @property
    def config(self) -> dict:
        c = Config()
        self._lib.tdma_plan_get_config(self._h, ctypes.byref(c))
        return {f: getattr(c, f) for f, _ in Config._fields_}

    def workspace(self, device) -> torch.Tensor:
        if self._ws is None or self._ws.numel() < self.workspace_bytes:
            self._ws = torch.empty(max(1, self.workspace_bytes), dtype=torch.uint8, device=device)
        return self._ws

    def solve(self, a, b, c, d, x, workspace=None, stream=None):
        ws = workspace if workspace is not None else (self.workspace(d.device) if self.workspace_bytes else None)
        st = self._lib.tdma_solve(self._h, _ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(x), _ptr(ws),
                                  ctypes.c_size_t(ws.numel() if ws is not None else 0), _stream(stream))
        if st != 0:
            raise TDMAError(st, "tdma_solve")
        return x

    def backward(self, a, b, c, x, grad_x, grad_a=None, grad_b=None, grad_c=None, grad_d=None,
                 workspace=None, stream=None):
        ws = workspace if workspace is not None else (self.workspace(x.device) if self.workspace_bytes else None)
        st = self._lib.tdma_solve_backward(self._h, _ptr(a), _ptr(b), _ptr(c), _ptr(x), _ptr(grad_x),
                                           _ptr(grad_a), _ptr(grad_b), _ptr(grad_c), _ptr(grad_d), _ptr(ws),
                                           ctypes.c_size_t(ws.numel() if ws is not None else 0), _stream(stream))
        if st != 0:
            raise TDMAError(st, "tdma_solve_backward")

    def autotune(self, a, b, c, d, x, workspace=None, stream=None):
        """Time the candidate configurations on these buffers and keep the fastest. Without an
        explicit workspace, one large enough for every candidate is offered (3 words per unknown;
        ragged batches: 5 words per unknown plus padding for the shortest partitions)."""
        if workspace is None:
            if self.desc.n == 0:
                unknowns = self.desc.ragged_total + 256 * self.desc.n_lines
                words = 5
            else:
                unknowns = self.desc.n * self.desc.n_lines * self.desc.nrhs
                words = 3
            workspace = torch.empty(max(1, unknowns * 8 * words), dtype=torch.uint8, device=d.device)
        ws = workspace
        st = self._lib.tdma_plan_autotune(self._h, _ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(x), _ptr(ws),
                                          ctypes.c_size_t(ws.numel()), _stream(stream))
        if st != 0:
            raise TDMAError(st, "tdma_plan_autotune")
        cfg = self.config
        self.workspace_bytes = cfg["workspace_bytes"]
        if self.workspace_bytes and (self._ws is None or self._ws.numel() < self.workspace_bytes):
            self._ws = ws if ws.numel() >= self.workspace_bytes else None
        return cfg

    def corrected_lines(self, stream=None) -> int:
        """Lines the last TDMA_F64_REFINE solve corrected (the rest kept the plain FP64 result);
        synchronises the stream."""
        lines = ctypes.c_int64(0)
        st = self._lib.tdma_plan_corrected_lines(self._h, _stream(stream), ctypes.byref(lines))
        if st != 0:
            raise TDMAError(st, "tdma_plan_corrected_lines")
        return int(lines.value)

    def last_error(self, stream=None):
        """(status, max refinement corrections used); synchronises the stream."""
        info = ctypes.c_int32(0)
        st = self._lib.tdma_last_device_error(self._h, _stream(stream), ctypes.byref(info))
        return st, info.value


class PoissonFFT:
    """FFT-based Poisson solve on one GPU (tdma_poisson_*): D_xx phi + D_yy phi + D_zz phi = q on an
    (ny, nz, nx) grid stored [y][z][x], periodic in x and z with spacings dx, dz, and D_yy the
    tridiagonal operator (a, b, c) along y (1D arrays of length ny, host or CPU tensors). cuFFT over
    every (z, x) plane, one tridiagonal line per wavenumber pair along y, cuFFT back. With
    ``pin_zero_mode`` the (0, 0) line's row 0 becomes Phi_0 = 0 (needed when D_yy has Neumann ends).
    ``precision`` "f64r" (default: the wavenumber lines whose condition-number bound reaches 1e5, the
    lowest modes, corrected from an exact residual) or "f64" (plain FP64 elimination)."""

    def __init__(self, nx, ny, nz, dx, dz, a, b, c, pin_zero_mode=True, precision="f64r", device="cuda"):
        self._lib = load_library()
        ha, hb, hc = (np.ascontiguousarray(np.asarray(t.cpu() if torch.is_tensor(t) else t, dtype=np.float64))
                      for t in (a, b, c))
        if not (ha.shape == hb.shape == hc.shape == (ny,)):
            raise ValueError("a, b, c must be 1D of length ny")
        self.desc = PoissonDesc(nx=nx, ny=ny, nz=nz, dx=dx, dz=dz, a=ha.ctypes.data, b=hb.ctypes.data,
                                c=hc.ctypes.data, pin_zero_mode=int(bool(pin_zero_mode)), precision=_PREC[precision])
        self._h = ctypes.c_void_p()
        ws = ctypes.c_size_t(0)
        with torch.cuda.device(torch.device(device)):
            st = self._lib.tdma_poisson_create(ctypes.byref(self._h), ctypes.byref(self.desc), ctypes.byref(ws))
        if st != 0:
            raise TDMAError(st, "tdma_poisson_create")
        self.shape = (ny, nz, nx)
        self.workspace = torch.empty(max(1, ws.value), dtype=torch.uint8, device=device)

    def __del__(self):
        try:
            if getattr(self, "_h", None) and self._h.value:
                self._lib.tdma_poisson_destroy(self._h)
        except Exception:
            pass

    def solve(self, q, out=None, stream=None, check=False):
        """phi for right-hand side q (a contiguous float64 CUDA tensor of shape (ny, nz, nx))."""
        if not q.is_cuda or q.dtype != torch.float64 or tuple(q.shape) != self.shape or not q.is_contiguous():
            raise ValueError(f"q must be a contiguous float64 CUDA tensor of shape {self.shape}")
        phi = torch.empty_like(q) if out is None else out
        st = self._lib.tdma_poisson_solve(self._h, _ptr(q), _ptr(phi), _ptr(self.workspace),
                                          ctypes.c_size_t(self.workspace.numel()), _stream(stream))
        if st != 0:
            raise TDMAError(st, "tdma_poisson_solve")
        if check:
            st = self._lib.tdma_poisson_last_error(self._h, _stream(stream))
            if st != 0:
                raise TDMAError(st, "device")
        return phi


class HostPipeline:
    """Solve a grid held in host memory as a pipeline of slices (tdma_solve_host): slices of lines
    move through ``slots`` device staging buffers, each on its own stream, so that host-to-device
    copies, solves and device-to-host copies of different slices run at the same time.

    ``shape`` is a C-order grid and ``axis`` the solve axis: 0 (lines adjacent in memory, rows
    strided) or the last axis (contiguous lines). ``batches`` slices split the lines evenly. The
    staging buffers, streams and the slice plan are made once; ``solve`` takes host tensors
    (pinned for full copy speed) of the precision's types and enqueues everything; ``synchronize``
    waits for it."""

    def __init__(self, shape, axis=0, precision="f64", batches=8, slots=3, device="cuda"):
        self._lib = load_library()
        shape = tuple(int(v) for v in shape)
        axis = axis % len(shape)
        if axis not in (0, len(shape) - 1):
            raise ValueError("HostPipeline solves along the first or the last axis")
        n = shape[axis]
        lines = 1
        for k, v in enumerate(shape):
            if k != axis:
                lines *= v
        if lines % batches:
            raise ValueError("batches must divide the number of lines")
        L = lines // batches
        if axis == 0:
            self.layout = HostLayout(n=n, n_lines=lines, line_stride=1, row_stride=lines)
            self.plan = Plan(n, L, elem_stride=L, inner_count=L, inner_stride=1, precision=precision)
        else:
            self.layout = HostLayout(n=n, n_lines=lines, line_stride=n, row_stride=1)
            self.plan = Plan(n, L, elem_stride=1, inner_count=L, inner_stride=n, precision=precision)
        cdt = torch.float64 if precision in ("f64", "f64r") else torch.float32
        ddt = torch.float32 if precision == "f32" else torch.float64
        dev = torch.device(device)
        self.buffers = [[torch.empty(n * L, dtype=t, device=dev) for t in (cdt, cdt, cdt, ddt, ddt)]
                        for _ in range(slots)]
        self.workspaces = [self.plan.workspace(dev) if k == 0 else
                           torch.empty(max(1, self.plan.workspace_bytes), dtype=torch.uint8, device=dev)
                           for k in range(slots)] if self.plan.workspace_bytes else None
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(slots)]
        self._bufs = (_VP * (5 * slots))(*[t.data_ptr() for bl in self.buffers for t in bl])
        self._ws = (_VP * slots)(*[w.data_ptr() for w in self.workspaces]) if self.workspaces else None
        self._st = (_VP * slots)(*[s.cuda_stream for s in self.streams])
        self.slots = slots

    def solve(self, a, b, c, d, x):
        """Enqueue the pipelined solve of host arrays a, b, c, d into host array x (x must not be d)."""
        for s in self.streams:
            s.wait_stream(torch.cuda.current_stream())
        st = self._lib.tdma_solve_host(self.plan._h, ctypes.byref(self.layout), _ptr(a), _ptr(b), _ptr(c), _ptr(d),
                                       _ptr(x), self.slots, self._bufs, self._ws,
                                       ctypes.c_size_t(self.plan.workspace_bytes), self._st)
        if st != 0:
            raise TDMAError(st, "tdma_solve_host")
        for s in self.streams:  # work queued on the caller's stream afterwards follows the pipeline
            torch.cuda.current_stream().wait_stream(s)
        return x

    def synchronize(self):
        for s in self.streams:
            s.synchronize()

    @staticmethod
    def predict(h, s, o, batches, slots):
        """Pipelined time of ``batches`` slices whose host-to-device copy, solve and device-to-host
        copy take h, s and o each (the three stages of Section 4.2's pipeline; the copies in the two
        directions run on separate copy engines): the first slice passes all three stages, then one
        slice leaves every max(h, s, o), or every (h + s + o) / slots when the slots, each holding one
        slice through its three stages, are the limit."""
        return h + s + o + (batches - 1) * max(h, s, o, (h + s + o) / slots)

    @classmethod
    def tuned(cls, shape, axis, precision, a, b, c, d, x, device="cuda", batches=(4, 8, 16), slots=(2, 3),
              reps=2):
        """A pipeline with ``batches`` and ``slots`` chosen for this grid on the caller's host arrays
        (overwriting x), cached per (shape, axis, precision) for the process. Like the batch-size
        estimator of Section 4.2.3, the stages of one slice are timed once per slice count on one slot
        (so nothing overlaps: the solve alone, and the copies as the rest of the serial time, split by
        bytes in and out) and the pipelined time is predicted (``predict``); every candidate is then
        also measured, and the fastest measured is kept. Returns (pipeline, report) with the choice and
        the predicted and measured milliseconds of every candidate."""
        key = (tuple(int(v) for v in shape), axis, precision)
        dev = torch.device(device)
        if key in _PIPE_CACHE:
            k, sl = _PIPE_CACHE[key]["choice"]
            return cls(shape, axis, precision, k, sl, device), _PIPE_CACHE[key]
        lines = 1
        for i, v in enumerate(shape):
            if i != axis % len(shape):
                lines *= int(v)
        bin_ = sum(t.numel() * t.element_size() for t in (a, b, c, d))
        bout = x.numel() * x.element_size()

        def timed(fn):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            fn()
            torch.cuda.synchronize(dev)
            best = float("inf")
            for _ in range(reps):
                e0.record()
                fn()
                e1.record()
                torch.cuda.synchronize(dev)
                best = min(best, e0.elapsed_time(e1))
            return best

        rows = []
        for k in batches:
            if lines % k:
                continue
            one = cls(shape, axis, precision, k, 1, device)
            serial = timed(lambda: one.solve(a, b, c, d, x))  # one slot: every stage in turn
            bufs = one.buffers[0]
            ws = one.workspaces[0] if one.workspaces else None
            solve = timed(lambda: one.plan.solve(*bufs[:4], bufs[4], workspace=ws)) * k
            copies = max(0.0, serial - solve)
            h, o = copies * bin_ / (bin_ + bout) / k, copies * bout / (bin_ + bout) / k
            del one, bufs, ws
            for sl in slots:
                pred = cls.predict(h, solve / k, o, k, sl)
                pipe = cls(shape, axis, precision, k, sl, device)
                meas = timed(lambda: pipe.solve(a, b, c, d, x))
                rows.append({"batches": k, "slots": sl, "predicted_ms": pred, "measured_ms": meas,
                             "stage_ms": [h, solve / k, o]})
                del pipe
                torch.cuda.empty_cache()
        if not rows:
            raise ValueError("no candidate slice count divides the number of lines")
        best = min(rows, key=lambda r: r["measured_ms"])
        est = min(rows, key=lambda r: r["predicted_ms"])
        report = {"choice": (best["batches"], best["slots"]), "estimator_choice": (est["batches"], est["slots"]),
                  "estimator_choice_measured_ms": est["measured_ms"], "best_measured_ms": best["measured_ms"],
                  "candidates": rows}
        _PIPE_CACHE[key] = report
        return cls(shape, axis, precision, best["batches"], best["slots"], device), report


_PIPE_CACHE = {}


def _check_same_layout(ref, *ts):
    for t in ts:
        if t is not None and (t.shape != ref.shape or t.stride() != ref.stride()):
            return False
    return True


_PLAN_CACHE = {}


def _plan_for(d, axis, precision, partitions, nrhs, coef_broadcast, diag_shift, max_refine_iters, refine_tol,
              pdd=False):
    lay = line_layout(d, axis, nrhs)
    key = (lay, precision, partitions, nrhs, coef_broadcast,
           None if diag_shift is None else diag_shift.data_ptr(), max_refine_iters, refine_tol, bool(pdd), d.device)
    p = _PLAN_CACHE.get(key)
    if p is None:
        n, nl, es, ic, isd, osd = lay
        p = Plan(n, nl, es, ic, isd, osd, precision=precision, partitions=partitions, nrhs=nrhs,
                 coef_broadcast=coef_broadcast, diag_shift=diag_shift, max_refine_iters=max_refine_iters,
                 refine_tol=refine_tol, pdd=pdd)
        _PLAN_CACHE[key] = p
    return p


def solve(a, b, c, d, axis=-1, precision="f64", partitions=0, out=None, nrhs=1, coef_broadcast=False,
          diag_shift=None, max_refine_iters=0, refine_tol=0.0, check=False, pdd=False):
    """Solve a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i along ``axis`` of every line of ``d``.

    a, b, c have d's layout (or are 1D of length n with ``coef_broadcast``); ``out`` may be d.
    ``check`` synchronises and raises on device-side numerical errors. ``pdd`` selects the
    parallel diagonally dominant approximation with ``partitions`` partitions per line.
    """
    if not d.is_cuda:
        raise RuntimeError("tdma.solve needs CUDA tensors (no CPU fallback)")
    if not coef_broadcast and not _check_same_layout(d if nrhs == 1 else d[..., 0], a, b, c):
        a, b, c = (t.contiguous() for t in (a, b, c))
        d = d.contiguous()
    if out is None:
        x = torch.empty_like(d)
        if not _check_same_layout(d, x):  # d is a view with gaps: solve a dense copy
            d = d.contiguous()
            if not coef_broadcast:
                a, b, c = (t.contiguous() for t in (a, b, c))
            x = torch.empty_like(d)
    else:
        x = out
        if not _check_same_layout(d, x):
            raise ValueError("out must have d's layout")
    p = _plan_for(d, axis, precision, partitions, nrhs, coef_broadcast, diag_shift, max_refine_iters, refine_tol,
                  pdd)
    p.solve(a, b, c, d, x)
    if check:
        st, _ = p.last_error()
        if st != 0:
            raise TDMAError(st, "device")
    return x


def solve_ragged(a, b, c, d, offsets, lengths, precision="f64", out=None, max_n=None, max_refine_iters=0,
                 refine_tol=0.0, check=False, plan=None):
    """Solve lines of uneven length packed in 1D arrays: line l has lengths[l] unknowns starting at
    offsets[l] (device int64 / int32 tensors). One persistent launch over a device work queue.
    Returns (x, plan); pass the plan back to reuse its sorted tables for the same batch."""
    if not d.is_cuda:
        raise RuntimeError("tdma.solve_ragged needs CUDA tensors (no CPU fallback)")
    if plan is None:
        n_max = int(lengths.max().item()) if max_n is None else int(max_n)
        plan = Plan(0, int(lengths.numel()), precision=precision, ragged_offsets=offsets, ragged_lengths=lengths,
                    ragged_max_n=n_max, ragged_total=int(d.numel()), max_refine_iters=max_refine_iters,
                    refine_tol=refine_tol)
    x = torch.empty_like(d) if out is None else out
    plan.solve(a, b, c, d, x)
    if check:
        st, _ = plan.last_error()
        if st != 0:
            raise TDMAError(st, "device")
    return x, plan


def solve_backward(a, b, c, x, grad_x, axis=-1, precision="f64", partitions=0, nrhs=1, coef_broadcast=False,
                   diag_shift=None, need=(True, True, True, True)):
    """Gradients (grad_a, grad_b, grad_c, grad_d) of a loss with dL/dx = grad_x through x = A^{-1} d."""
    p = _plan_for(x, axis, precision, partitions, nrhs, coef_broadcast, diag_shift, 0, 0.0)
    if coef_broadcast:
        ga, gb, gc = (torch.zeros_like(t) if f else None for t, f in zip((a, b, c), need[:3]))
    else:
        ga, gb, gc = (torch.empty_like(t) if f else None for t, f in zip((a, b, c), need[:3]))
    gd = torch.empty_like(x)  # lambda = A^{-T} grad_x, always computed
    p.backward(a, b, c, x, grad_x.contiguous() if grad_x.stride() != x.stride() else grad_x, ga, gb, gc, gd)
    return ga, gb, gc, (gd if need[3] else None)


class TDMASolve(torch.autograd.Function):
    """x = A^{-1} d along ``axis`` with a hand-written adjoint (tdma_solve_backward)."""

    @staticmethod
    def forward(ctx, a, b, c, d, axis=-1, precision="f64", partitions=0):
        x = solve(a, b, c, d, axis=axis, precision=precision, partitions=partitions)
        ctx.save_for_backward(a, b, c, x)
        ctx.cfg = (axis, precision, partitions)
        return x

    @staticmethod
    def backward(ctx, grad_x):
        a, b, c, x = ctx.saved_tensors
        axis, precision, partitions = ctx.cfg
        need = ctx.needs_input_grad[:4]
        ga, gb, gc, gd = solve_backward(a, b, c, x, grad_x, axis=axis, precision=precision,
                                        partitions=partitions, need=tuple(bool(v) for v in need))
        return ga, gb, gc, gd, None, None, None


def sweep_graph(plans_and_args, stream=None):
    """Capture a sequence of solves (e.g. the x, y, z sweeps of an ADI step) in one CUDA graph.

    ``plans_and_args`` is a list of (Plan, (a, b, c, d, x)) run in order on one stream; the
    returned torch.cuda.CUDAGraph replays them with a single launch.
    """
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream() if stream is None else stream
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for p, args in plans_and_args:  # warm-up outside capture
            p.solve(*args, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(g, stream=s):
        for p, args in plans_and_args:
            p.solve(*args, stream=s)
    return g
