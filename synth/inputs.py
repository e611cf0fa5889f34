"""Seeded synthetic problems shaped like the paper's workloads.

Every random value is a pure function of (seed, array id, element index): a
splitmix64 hash of the counter, mapped to a double in [0, 1) (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014). Any
line of a 1024^3 grid can therefore be regenerated on its own, on the host or
on the device, without drawing the rest.

The module only builds inputs (coefficients, right-hand sides, manufactured
solutions); it contains none of the tridiagonal solver's arithmetic.

Grids are C-ordered ``[nz][ny][nx]`` (x has unit stride). A tridiagonal line
along ``axis`` couples neighbouring elements along that axis; ``a`` is the
sub-diagonal, ``b`` the diagonal and ``c`` the super-diagonal (Section 3.2.1,
where a, b and c are the sub-, main and super-diagonal of A). The first ``a``
and the last ``c`` of each line are drawn but never used.
"""
from __future__ import annotations

import math

import numpy as np
import torch

__all__ = [
    "uniform_np", "uniform", "normal", "grid_general", "grid_adi", "ragged_lengths",
    "ragged_general", "tanh_grid", "poisson_coefficients", "modified_wavenumbers",
    "poisson_lines", "apply_tridiag", "line_view", "AID",
]

# array ids of the counter-based generator
AID = dict(a=1, b=2, c=3, x_true=4, d=5, re=6, im=7, w=8, length=9, b_extra=10)

_C0 = 0x9E3779B97F4A7C15
_C1 = 0xBF58476D1CE4E5B9
_C2 = 0x94D049BB133111EB


def _key(seed: int, array_id: int) -> int:
    return ((array_id & 0xFF) << 56) | ((seed & 0xFFFF) << 40)


def uniform_np(seed: int, array_id: int, idx) -> np.ndarray:
    """Uniform doubles in [0, 1) for element indices ``idx`` (< 2^40), numpy uint64 arithmetic."""
    z = np.asarray(idx, dtype=np.uint64) ^ np.uint64(_key(seed, array_id))
    with np.errstate(over="ignore"):
        z = z + np.uint64(_C0)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_C1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_C2)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _s64(v: int) -> int:
    v &= (1 << 64) - 1
    return v - (1 << 64) if v >= (1 << 63) else v


def _srl(z: torch.Tensor, s: int) -> torch.Tensor:
    # logical right shift of int64 two's complement values
    return (z >> s) & ((1 << (64 - s)) - 1)


def uniform(seed: int, array_id: int, idx: torch.Tensor) -> torch.Tensor:
    """Same generator as :func:`uniform_np` on int64 torch tensors (CPU or CUDA); wraps mod 2^64."""
    z = idx ^ _s64(_key(seed, array_id))
    z = z + _s64(_C0)
    z = (z ^ _srl(z, 30)) * _s64(_C1)
    z = (z ^ _srl(z, 27)) * _s64(_C2)
    z = z ^ _srl(z, 31)
    return _srl(z, 11).to(torch.float64) * (2.0 ** -53)


def _fill(out: torch.Tensor, fn, chunk: int = 1 << 25) -> torch.Tensor:
    """Fill flat ``out`` with fn(idx) chunk by chunk (bounded temporaries)."""
    flat = out.view(-1)
    n = flat.numel()
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        idx = torch.arange(s, e, dtype=torch.int64, device=out.device)
        flat[s:e] = fn(idx).to(out.dtype)
    return out


def normal(seed: int, array_id: int, idx: torch.Tensor) -> torch.Tensor:
    """Standard normal variates by the Box-Muller transform of two counter draws."""
    u1 = uniform(seed, array_id, 2 * idx)
    u2 = uniform(seed, array_id, 2 * idx + 1)
    return torch.sqrt(-2.0 * torch.log1p(-u1)) * torch.cos((2.0 * math.pi) * u2)


def line_view(t: torch.Tensor, axis: int) -> torch.Tensor:
    """View a grid as [lines, n] with the solve axis last (a copy if not already contiguous)."""
    return t.movedim(axis, -1).reshape(-1, t.shape[axis])


def apply_tridiag(a: torch.Tensor, b: torch.Tensor, c: torch.Tensor, x: torch.Tensor, axis: int) -> torch.Tensor:
    """d = A x along ``axis`` as (b*x + a*x_prev) + c*x_next, each operation rounded on its own.

    Used only to manufacture right-hand sides from a chosen solution.
    """
    n = x.shape[axis]
    d = b * x
    if n > 1:
        d.narrow(axis, 1, n - 1).add_(a.narrow(axis, 1, n - 1) * x.narrow(axis, 0, n - 1))
        d.narrow(axis, 0, n - 1).add_(c.narrow(axis, 0, n - 1) * x.narrow(axis, 1, n - 1))
    return d


def _global_index(shape, full_shape, origin):
    """Map flat indices of a sub-block ``shape`` at ``origin`` to flat indices of ``full_shape``."""
    if full_shape is None:
        return lambda i: i
    full_shape = tuple(int(s) for s in full_shape)
    strides_full = [1] * len(full_shape)
    for k in range(len(full_shape) - 2, -1, -1):
        strides_full[k] = strides_full[k + 1] * full_shape[k + 1]
    def g(i):
        out = torch.zeros_like(i)
        rem = i
        for k in range(len(shape) - 1, -1, -1):
            q = rem % shape[k]
            rem = rem // shape[k]
            out += (q + origin[k]) * strides_full[k]
        return out
    return g


def grid_general(shape, axis: int, seed: int, device="cpu", fp32_coefficients: bool = False,
                 with_solution: bool = True, full_shape=None, origin=None):
    """General diagonally dominant problem (the distribution of the 64^3 and 1024^3 workloads).

    a, c ~ U(-1, 0); b = 2 + |a| + |c| + U(0, 1); x_true ~ U(-1, 1); d = A x_true along ``axis``.
    With ``fp32_coefficients`` the drawn a, b, c are rounded to float32 and those rounded values
    define the problem (returned both as float64 and float32); d is formed in float64 from them.
    With ``full_shape``/``origin`` the block ``shape`` at ``origin`` of that larger grid is drawn
    (identical values to the full draw; the block must span the whole solve axis).
    Returns a dict of tensors shaped like the grid.
    """
    shape = tuple(int(s) for s in shape)
    if full_shape is not None:
        origin = tuple(origin or (0,) * len(shape))
        if shape[axis] != full_shape[axis] or origin[axis] != 0:
            raise ValueError("a sampled block must span the whole solve axis")
    gi = _global_index(shape, full_shape, origin)
    f64 = dict(dtype=torch.float64, device=device)
    a = _fill(torch.empty(shape, **f64), lambda i: uniform(seed, AID["a"], gi(i)) - 1.0)
    c = _fill(torch.empty(shape, **f64), lambda i: uniform(seed, AID["c"], gi(i)) - 1.0)
    b = _fill(torch.empty(shape, **f64), lambda i: uniform(seed, AID["b"], gi(i)))
    b.add_(2.0).add_(a.abs()).add_(c.abs())  # 2 + |a| + |c| + U, evaluated as ((U + 2) + |a|) + |c|
    out = {}
    if fp32_coefficients:
        a32, b32, c32 = a.float(), b.float(), c.float()
        out.update(a32=a32, b32=b32, c32=c32)
        a, b, c = a32.double(), b32.double(), c32.double()
    out.update(a=a, b=b, c=c)
    if with_solution:
        x = _fill(torch.empty(shape, **f64), lambda i: 2.0 * uniform(seed, AID["x_true"], gi(i)) - 1.0)
        out["x_true"] = x
        out["d"] = apply_tridiag(a, b, c, x, axis)
    return out


def grid_adi(shape, seed: int, r: float = 0.5, device="cpu"):
    """Constant-coefficient ADI viscous operator tridiag(-r, 1 + 2r, -r) stored as full arrays.

    Homogeneous Dirichlet ends (the first a and last c of a line are unused); d ~ U(-1, 1).
    """
    shape = tuple(int(s) for s in shape)
    f64 = dict(dtype=torch.float64, device=device)
    a = torch.full(shape, -r, **f64)
    c = torch.full(shape, -r, **f64)
    b = torch.full(shape, 1.0 + 2.0 * r, **f64)
    d = _fill(torch.empty(shape, **f64), lambda i: 2.0 * uniform(seed, AID["d"], i) - 1.0)
    return dict(a=a, b=b, c=c, d=d)


def ragged_lengths(n_lines: int = 20000, n_min: int = 16, n_max: int = 16384, seed: int = 4) -> np.ndarray:
    """Line lengths log-uniform in [n_min, n_max]: n = min(n_max, floor(exp(U(ln n_min, ln(n_max + 1)))))."""
    u = uniform_np(seed, AID["length"], np.arange(n_lines))
    lo, hi = math.log(n_min), math.log(n_max + 1)
    n = np.floor(np.exp(lo + (hi - lo) * u)).astype(np.int64)
    return np.clip(n, n_min, n_max).astype(np.int32)


def ragged_general(lengths, seed: int, device="cpu", fp32_coefficients: bool = False,
                   with_solution: bool = True):
    """Lines of uneven length packed back to back with unit stride, config-0 distributions.

    Returns a dict with flat tensors a, b, c (float64, plus float32 copies when requested),
    d and x_true, and int64 ``offsets`` / int32 ``lengths`` describing the packing.
    """
    lengths = np.asarray(lengths, dtype=np.int64)
    offsets = np.zeros(len(lengths), dtype=np.int64)
    if len(lengths) > 1:
        offsets[1:] = np.cumsum(lengths)[:-1]
    total = int(lengths.sum())
    f64 = dict(dtype=torch.float64, device=device)
    a = _fill(torch.empty(total, **f64), lambda i: uniform(seed, AID["a"], i) - 1.0)
    c = _fill(torch.empty(total, **f64), lambda i: uniform(seed, AID["c"], i) - 1.0)
    b = _fill(torch.empty(total, **f64), lambda i: uniform(seed, AID["b"], i))
    b.add_(2.0).add_(a.abs()).add_(c.abs())
    out = dict(offsets=torch.from_numpy(offsets).to(device),
               lengths=torch.from_numpy(lengths.astype(np.int32)).to(device), total=total)
    if fp32_coefficients:
        a32, b32, c32 = a.float(), b.float(), c.float()
        out.update(a32=a32, b32=b32, c32=c32)
        a, b, c = a32.double(), b32.double(), c32.double()
    out.update(a=a, b=b, c=c)
    if with_solution:
        x = _fill(torch.empty(total, **f64), lambda i: 2.0 * uniform(seed, AID["x_true"], i) - 1.0)
        start = torch.zeros(total, dtype=torch.bool, device=device)
        start[out["offsets"]] = True
        end = torch.zeros(total, dtype=torch.bool, device=device)
        end[out["offsets"] + out["lengths"].to(torch.int64) - 1] = True
        d = b * x
        if total > 1:
            lo = a[1:] * x[:-1]
            lo[start[1:]] = 0.0
            d[1:] += lo
            up = c[:-1] * x[1:]
            up[end[:-1]] = 0.0
            d[:-1] += up
        out.update(x_true=x, d=d)
    return out


def tanh_grid(n: int, beta: float = 2.0) -> np.ndarray:
    """Wall-normal nodes y_k = tanh(beta (2k/(n-1) - 1)) / tanh(beta), k = 0..n-1 (hyperbolic-tangent stretching)."""
    k = np.arange(n, dtype=np.float64)
    return np.tanh(beta * (2.0 * k / (n - 1) - 1.0)) / math.tanh(beta)


def poisson_coefficients(n: int, beta: float = 2.0):
    """Second-difference coefficients on the stretched grid, Neumann ends by ghost reflection.

    Interior: a_k = 2 / (h_{k-1}(h_{k-1}+h_k)), c_k = 2 / (h_k(h_{k-1}+h_k)).
    Row 0: a_0 = 0, c_0 = 2/h_0^2. Row n-1: a = 2/h_{n-2}^2, c = 0. The base diagonal is -(a_k + c_k).
    Returns float64 numpy arrays (a, c, b0).
    """
    y = tanh_grid(n, beta)
    h = np.diff(y)
    a = np.zeros(n)
    c = np.zeros(n)
    hm, hp = h[:-1], h[1:]
    a[1:-1] = 2.0 / (hm * (hm + hp))
    c[1:-1] = 2.0 / (hp * (hm + hp))
    c[0] = 2.0 / h[0] ** 2
    a[-1] = 2.0 / h[-1] ** 2
    b0 = -(a + c)
    return a, c, b0


def modified_wavenumbers(N: int, length: float = 2.0 * math.pi) -> np.ndarray:
    """k'^2(l) = (2 - 2 cos(2 pi l / N)) / dx^2 with dx = length / N (second-order periodic differences)."""
    dx = length / N
    l = np.arange(N, dtype=np.float64)
    return (2.0 - 2.0 * np.cos(2.0 * math.pi * l / N)) / dx ** 2


def poisson_lines(nx: int, ny: int, nz: int, seed: int = 2, beta: float = 2.0, device="cpu",
                  rhs: bool = True):
    """Wavenumber lines of an FFT Poisson solver: lines along z, one per (kx, ky) = (x, y) index.

    Broadcast coefficients a_k, c_k, b0_k (length nz) and a per-line diagonal shift
    -(k'^2_x + k'^2_y). The right-hand side is complex, stored as interleaved (re, im) float64
    pairs of shape [nz][ny][nx][2], re and im ~ N(0, 1). Line 0 is the kx = ky = 0 mode, which
    is singular until pinned: its pinned form (row 0 replaced by x_0 = 0) is returned as
    general per-element arrays ``pin_a/pin_b/pin_c`` of length nz, and its right-hand side
    row 0 is set to zero.
    """
    a, c, b0 = poisson_coefficients(nz, beta)
    kx2 = modified_wavenumbers(nx)
    ky2 = modified_wavenumbers(ny)
    shift = -(ky2[:, None] + kx2[None, :]).reshape(-1)
    out = dict(a=torch.from_numpy(a).to(device), c=torch.from_numpy(c).to(device),
               b0=torch.from_numpy(b0).to(device), shift=torch.from_numpy(shift).to(device))
    pa, pb, pc = a.copy(), b0.copy(), c.copy()
    pb[0], pc[0] = 1.0, 0.0
    out.update(pin_a=torch.from_numpy(pa).to(device), pin_b=torch.from_numpy(pb).to(device),
               pin_c=torch.from_numpy(pc).to(device))
    if rhs:
        d = torch.empty((nz, ny, nx, 2), dtype=torch.float64, device=device)
        re =_fill(torch.empty((nz, ny, nx), dtype=torch.float64, device=device),
                   lambda i: normal(seed, AID["re"], i))
        d[..., 0] = re
        del re
        im = _fill(torch.empty((nz, ny, nx), dtype=torch.float64, device=device),
                   lambda i: normal(seed, AID["im"], i))
        d[..., 1] = im
        del im
        d[0, 0, 0, :] = 0.0  # pinned row of the zero mode
        out["d"] = d
    return out
