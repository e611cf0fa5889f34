"""Plain, slow, obviously correct CPU reference for batched tridiagonal solves.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py``; never by the CUDA library, with which it shares no code.

Problem (Algorithm 1, "Problem: Ax = d (N times)"; Section 3.2.1: a, b and c are the
sub-, main and super-diagonal of A): for every line,
    a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i,   i = 0..n-1,
with a_0 and c_{n-1} ignored (no coupling outside the line). Arrays are numpy float64 of
shape (lines, n) (or (n,)); ``d`` may carry extra trailing right-hand-side axes.

Functions and the passage each follows:
  thomas          -- the Thomas algorithm (Section 1), the plain definition x = A^{-1} d.
  thomas_ext      -- the same sweep in numpy.longdouble (extended precision) for badly
                     conditioned lines (the pinned Poisson zero mode).
  dense_solve     -- x = A^{-1} d by dense LU with partial pivoting (numpy.linalg.solve).
  partition_rows  -- split of a line into p contiguous partitions (Section 2.2; the paper
                     is silent on uneven splits: the first n mod p partitions take one
                     extra row, and every partition needs at least 2 rows).
  dc_spike        -- the divide-and-conquer solve in the paper's own three-stage form
                     (Section 2.1 stages 1-5; Algorithm 1: solve the decoupled system
                     A~ x~ = d~, solve the reduced system Z y = E^T x~ of size 2p - 2
                     (Section 2.2), correct x = x~ - Y y).
  modified_thomas_partition
                  -- Stage A in the modified-Thomas form (Section 2.1: each partition reduced
                     to its two end unknowns; the paper defers the stage equations to Sun 1989
                     and to the PaScaL_TDMA form it cites): a forward sweep that keeps x_0 as a
                     parameter, a backward sweep that expresses every row in x_0 and x_{m-1},
                     and the elimination of x_1 from row 0.
  reduced_system  -- the 2p-row unit-diagonal system of the partitions' end rows (the on-chip
                     analogue of the paper's A2B step), stacked in partition order.
  dc_modified     -- the three stages in that form: Stage A per partition, Stage B by Thomas on
                     the reduced system, Stage C x_i = delta_i - alpha_i x_0 - gamma_i x_{m-1}.
  pdd             -- the parallel diagonally dominant (PDD) approximation the paper's
                     momentum solver uses for its diagonally dominant ADI lines (Section 5.1,
                     Section 6.2.2; Sun's method): Stage A as in dc_spike, then one 2x2 system
                     per interface that keeps only the couplings between the two end unknowns
                     of the interface, then the correction of dc_spike. The paper prints no
                     PDD values; it is pinned by the cases the method fixes (p = 1 and
                     decoupled partitions are exact, rows off the partition boundaries hold
                     exactly, the error falls geometrically with the partition length).
  poisson_fft     -- the FFT-based Poisson solve (Section 5.2): real FFT over every periodic
                     (z, x) plane, one tridiagonal line per wavenumber pair along y with the
                     diagonal shifted by the modified wavenumbers, inverse FFT (numpy.fft and
                     thomas as the steps).
  residual        -- r = d - A x.
  adjoint_grads   -- gradients of a scalar loss through x = A^{-1} d: lambda = A^{-T} g,
                     grad_d = lambda, grad_b = -lambda*x, grad_a_i = -lambda_i x_{i-1},
                     grad_c_i = -lambda_i x_{i+1} (standard adjoint of a linear solve;
                     the paper has no backward pass).
  thomas_ragged   -- Thomas over lines of uneven length packed back to back.
"""
from __future__ import annotations

import numpy as np

__all__ = ["thomas", "thomas_ext", "dense_matrix", "dense_solve", "partition_rows", "dc_spike",
           "modified_thomas_partition", "reduced_system", "dc_modified", "pdd", "poisson_fft",
           "residual", "adjoint_grads", "transpose_coefficients", "thomas_ragged", "rel_l2"]


def _as2d(*arrs):
    return [np.asarray(x) for x in arrs]


def thomas(a, b, c, d, dtype=np.float64):
    """Thomas algorithm (Section 1): LU without pivoting, forward elimination then back substitution.

    c'_0 = c_0/b_0, d'_0 = d_0/b_0; for i >= 1: w = b_i - a_i c'_{i-1}, c'_i = c_i/w,
    d'_i = (d_i - a_i d'_{i-1})/w; then x_{n-1} = d'_{n-1}, x_i = d'_i - c'_i x_{i+1}.
    Vectorised over lines (leading axes); loops over rows. ``d`` may have trailing RHS axes.
    """
    a, b, c, d = (np.asarray(t, dtype=dtype) for t in (a, b, c, d))
    n = b.shape[-1]
    extra = d.ndim - b.ndim  # trailing right-hand-side axes of d
    rows_d = d.shape[b.ndim - 1]
    assert rows_d == n
    def col(t, i):
        return t[..., i]
    def rhs(t, i):
        return t[(Ellipsis, i) + (slice(None),) * extra] if extra else t[..., i]
    def bc(v):  # broadcast a per-row coefficient over the RHS axes
        return v.reshape(v.shape + (1,) * extra) if extra else v
    cp = np.empty(b.shape, dtype=dtype)
    dp = np.empty(d.shape, dtype=dtype)
    cp[..., 0] = col(c, 0) / col(b, 0) if n > 1 else 0.0
    if extra:
        dp[(Ellipsis, 0) + (slice(None),) * extra] = rhs(d, 0) / bc(col(b, 0))
    else:
        dp[..., 0] = d[..., 0] / b[..., 0]
    for i in range(1, n):
        w = col(b, i) - col(a, i) * cp[..., i - 1]
        cp[..., i] = (col(c, i) / w) if i < n - 1 else 0.0
        if extra:
            sl = (Ellipsis, i) + (slice(None),) * extra
            slp = (Ellipsis, i - 1) + (slice(None),) * extra
            dp[sl] = (d[sl] - bc(col(a, i)) * dp[slp]) / bc(w)
        else:
            dp[..., i] = (d[..., i] - a[..., i] * dp[..., i - 1]) / w
    x = np.empty(d.shape, dtype=dtype)
    if extra:
        last = (Ellipsis, n - 1) + (slice(None),) * extra
        x[last] = dp[last]
        for i in range(n - 2, -1, -1):
            sl = (Ellipsis, i) + (slice(None),) * extra
            sln = (Ellipsis, i + 1) + (slice(None),) * extra
            x[sl] = dp[sl] - bc(cp[..., i]) * x[sln]
    else:
        x[..., n - 1] = dp[..., n - 1]
        for i in range(n - 2, -1, -1):
            x[..., i] = dp[..., i] - cp[..., i] * x[..., i + 1]
    return x


def thomas_ext(a, b, c, d):
    """The Thomas sweep of :func:`thomas` in numpy.longdouble; returns float64.

    longdouble is the 80-bit x87 format on x86-64 and IEEE binary128 on AArch64; both carry
    more than 53 significant bits, which is all this reference needs.
    """
    return thomas(a, b, c, d, dtype=np.longdouble).astype(np.float64)


def dense_matrix(a, b, c):
    """The dense n x n matrix of one line (a_0 and c_{n-1} dropped)."""
    a, b, c = (np.asarray(t, dtype=np.float64) for t in (a, b, c))
    n = b.shape[-1]
    A = np.zeros(b.shape[:-1] + (n, n))
    idx = np.arange(n)
    A[..., idx, idx] = b
    if n > 1:
        A[..., idx[1:], idx[:-1]] = a[..., 1:]
        A[..., idx[:-1], idx[1:]] = c[..., :-1]
    return A


def dense_solve(a, b, c, d):
    """x = A^{-1} d by LAPACK LU with partial pivoting, line by line (brute-force pin)."""
    A = dense_matrix(a, b, c)
    d = np.asarray(d, dtype=np.float64)
    return np.linalg.solve(A, d[..., None])[..., 0]


def partition_rows(n: int, p: int):
    """Contiguous partitions [start, end) of a line of n rows into p parts.

    The first (n mod p) partitions hold ceil(n/p) rows, the rest floor(n/p). Raises if a
    partition would hold fewer than 2 rows (the two-endpoint reduction needs m >= 2).
    """
    if p < 1:
        raise ValueError("p must be >= 1")
    q, r = divmod(n, p)
    sizes = [q + 1] * r + [q] * (p - r)
    if min(sizes) < 2 and not (p == 1 and n >= 1):
        raise ValueError(f"partition of {n} rows into {p} parts leaves a part with < 2 rows")
    bounds, s = [], 0
    for m in sizes:
        bounds.append((s, s + m))
        s += m
    return bounds


def dc_spike(a, b, c, d, p: int):
    """Divide-and-conquer solve in the paper's three computation stages (Section 2.1, Algorithm 1).

    Stage A (decoupled solve, A~ x~ = d~): each partition k = [s, e] is solved on its own with
    its outer couplings a_s and c_e removed, for the right-hand side d and for the two coupling
    columns: v = A_k^{-1}(a_s e_first) (k > 0) and w = A_k^{-1}(c_e e_last) (k < p-1). Then
    inside partition k, x_i = x~_i - v_i x_{s-1} - w_i x_{e+1}.
    Stage B (reduced system Z y = E^T x~, size 2p - 2, Section 2.2): the interface unknowns
    y = [x_{e_0}, x_{s_1}, x_{e_1}, ..., x_{e_{p-2}}, x_{s_{p-1}}] satisfy, for each interface
    row i in {s_k (k > 0), e_k (k < p-1)}: x_i + v_i x_{e_{k-1}} + w_i x_{s_{k+1}} = x~_i.
    Solved here by dense LU (numpy.linalg.solve).
    Stage C (correction, x = x~ - Y y): apply the relation above to every row.
    Works on (lines, n) arrays; returns x with the shape of d.
    """
    a, b, c, d = (np.atleast_2d(np.asarray(t, dtype=np.float64)) for t in (a, b, c, d))
    squeeze = np.asarray(b).ndim == 1
    L, n = b.shape
    parts = partition_rows(n, p)
    xt = np.zeros((L, n))
    v = np.zeros((L, n))
    w = np.zeros((L, n))
    for k, (s, e) in enumerate(parts):  # Stage A
        ak, bk, ck = a[:, s:e].copy(), b[:, s:e], c[:, s:e].copy()
        ak[:, 0] = 0.0
        ck[:, -1] = 0.0
        xt[:, s:e] = thomas(ak, bk, ck, d[:, s:e])
        if k > 0:
            rhs = np.zeros((L, e - s))
            rhs[:, 0] = a[:, s]
            v[:, s:e] = thomas(ak, bk, ck, rhs)
        if k < p - 1:
            rhs = np.zeros((L, e - s))
            rhs[:, -1] = c[:, e - 1]
            w[:, s:e] = thomas(ak, bk, ck, rhs)
    if p == 1:
        x = xt
    else:
        # interface unknown j: 2k-1 -> x_{s_k} (k >= 1), 2k -> x_{e_k} (k <= p-2)
        m = 2 * p - 2
        iface_row = []
        for k, (s, e) in enumerate(parts):
            if k > 0:
                iface_row.append((2 * k - 1, s, k))
            if k < p - 1:
                iface_row.append((2 * k, e - 1, k))
        Z = np.zeros((L, m, m))
        rhs = np.zeros((L, m))
        for j, row, k in iface_row:  # Stage B assembly
            Z[:, j, j] = 1.0
            if k > 0:
                Z[:, j, 2 * (k - 1)] += v[:, row]        # coefficient of x_{e_{k-1}}
            if k < p - 1:
                Z[:, j, 2 * (k + 1) - 1] += w[:, row]    # coefficient of x_{s_{k+1}}
            rhs[:, j] = xt[:, row]
        y = np.linalg.solve(Z, rhs[..., None])[..., 0]
        x = xt.copy()
        for k, (s, e) in enumerate(parts):  # Stage C
            if k > 0:
                x[:, s:e] -= v[:, s:e] * y[:, 2 * (k - 1)][:, None]
            if k < p - 1:
                x[:, s:e] -= w[:, s:e] * y[:, 2 * (k + 1) - 1][:, None]
    return x[0] if squeeze else x


def _rhs_row(t, i, extra):
    """Row i of a right-hand-side array (one optional trailing RHS axis)."""
    return t[..., i, :] if extra else t[..., i]


def modified_thomas_partition(a, b, c, d):
    """Stage A of one partition in the modified-Thomas form (Section 2.1, stages 1-2: each
    partition is reduced to relations in its two end unknowns; Algorithm 1's decoupled solve).

    Input: the m >= 2 rows of one partition (lines on the leading axes; d may carry one trailing
    right-hand-side axis). a[..., 0] couples row 0 to the unknown just before the partition
    (x_{-1}) and c[..., m-1] couples row m-1 to the one just after it (x_m); pass 0 at a line
    end. Every row is divided by its diagonal and x_1 .. x_{m-2} are eliminated, so that
        row 0:          alpha_0 x_{-1} + x_0 + gamma_0 x_{m-1} = delta_0
        row i, 1..m-2:  alpha_i x_0 + x_i + gamma_i x_{m-1} = delta_i
        row m-1:        alpha_{m-1} x_0 + x_{m-1} + gamma_{m-1} x_m = delta_{m-1}
    Steps, in this order:
      1. rows 0 and 1 divided by their diagonal: alpha = a / b, gamma = c / b, delta = d / b;
      2. forward, i = 2..m-1, x_{i-1} eliminated with row i-1 (alpha_{i-1} x_0 + x_{i-1} +
         gamma_{i-1} x_i = delta_{i-1}):  r = 1 / (b_i - a_i gamma_{i-1}),
         alpha_i = -r a_i alpha_{i-1},  gamma_i = r c_i,  delta_i = r (d_i - a_i delta_{i-1});
         after this step row i (i >= 1) reads alpha_i x_0 + x_i + gamma_i x_{i+1} = delta_i
         (returned as the forward form);
      3. backward, i = m-3 down to 1, x_{i+1} eliminated with row i+1 (already in x_0 and
         x_{m-1}):  delta_i -= gamma_i delta_{i+1},  alpha_i -= gamma_i alpha_{i+1},
         gamma_i = -gamma_i gamma_{i+1};
      4. row 0, when m >= 3, x_1 eliminated with row 1:  r = 1 / (1 - gamma_0 alpha_1),
         delta_0 = r (delta_0 - gamma_0 delta_1),  alpha_0 = r alpha_0,  gamma_0 = -r gamma_0 gamma_1.
    Returns a dict of arrays shaped like b (delta like d): alpha, gamma, delta (the final form)
    and alpha_fwd, gamma_fwd, delta_fwd (the forward form after step 2; row 0 as after step 1).
    """
    a, b, c, d = (np.asarray(t, dtype=np.float64) for t in (a, b, c, d))
    m = b.shape[-1]
    if m < 2:
        raise ValueError("a partition needs at least 2 rows")
    extra = d.ndim - b.ndim
    if extra not in (0, 1):
        raise ValueError("d may carry at most one trailing right-hand-side axis")
    ex = (lambda v: v[..., None]) if extra else (lambda v: v)
    al = np.empty(b.shape)
    ga = np.empty(b.shape)
    de = np.empty(d.shape)
    for i in (0, 1):  # step 1
        al[..., i] = a[..., i] / b[..., i]
        ga[..., i] = c[..., i] / b[..., i]
        de[(Ellipsis, i) + (slice(None),) * extra] = _rhs_row(d, i, extra) / ex(b[..., i])
    for i in range(2, m):  # step 2
        r = 1.0 / (b[..., i] - a[..., i] * ga[..., i - 1])
        al[..., i] = -r * a[..., i] * al[..., i - 1]
        ga[..., i] = r * c[..., i]
        de[(Ellipsis, i) + (slice(None),) * extra] = ex(r) * (_rhs_row(d, i, extra)
                                                              - ex(a[..., i]) * _rhs_row(de, i - 1, extra))
    fwd = {"alpha_fwd": al.copy(), "gamma_fwd": ga.copy(), "delta_fwd": de.copy()}
    for i in range(m - 3, 0, -1):  # step 3
        de[(Ellipsis, i) + (slice(None),) * extra] = _rhs_row(de, i, extra) - ex(ga[..., i]) * _rhs_row(de, i + 1, extra)
        al[..., i] = al[..., i] - ga[..., i] * al[..., i + 1]
        ga[..., i] = -ga[..., i] * ga[..., i + 1]
    if m >= 3:  # step 4
        r = 1.0 / (1.0 - ga[..., 0] * al[..., 1])
        de[(Ellipsis, 0) + (slice(None),) * extra] = ex(r) * (_rhs_row(de, 0, extra)
                                                              - ex(ga[..., 0]) * _rhs_row(de, 1, extra))
        al[..., 0] = r * al[..., 0]
        ga[..., 0] = -r * ga[..., 0] * ga[..., 1]
    out = {"alpha": al, "gamma": ga, "delta": de}
    out.update(fwd)
    return out


def reduced_system(stages):
    """The reduced system of a line split into partitions (Section 2.2; its assembly is the
    paper's A2B step, here on one device): for partition k with Stage A result ``stages[k]``
    (modified_thomas_partition), unknown 2k is its first unknown and 2k+1 its last; row 2k is
    the partition's row 0 and row 2k+1 its row m-1, both with unit diagonal:
        row 2k:    alpha_0 y_{2k-1} + y_{2k} + gamma_0 y_{2k+1} = delta_0
        row 2k+1:  alpha_{m-1} y_{2k} + y_{2k+1} + gamma_{m-1} y_{2k+2} = delta_{m-1}
    Returns (sub, sup, rhs) with the rows on the last axis (rhs with its trailing RHS axis).
    """
    sub, sup, rhs = [], [], []
    for st in stages:
        extra = st["delta"].ndim - st["alpha"].ndim
        for i in (0, -1):
            sub.append(st["alpha"][..., i])
            sup.append(st["gamma"][..., i])
            rhs.append(_rhs_row(st["delta"], i, extra))
    rows_axis = -2 if rhs[0].ndim > sub[0].ndim else -1
    return np.stack(sub, axis=-1), np.stack(sup, axis=-1), np.stack(rhs, axis=rows_axis)


def dc_modified(a, b, c, d, p: int):
    """Divide-and-conquer solve in the modified-Thomas form (Section 2.1's three stages):
    Stage A, modified_thomas_partition on every partition of partition_rows(n, p) with the
    line's a_0 and c_{n-1} set to 0; Stage B, thomas on the 2p-row reduced_system (unit
    diagonal); Stage C, x_i = delta_i - alpha_i x_0 - gamma_i x_{m-1} inside every partition
    (its two end unknowns taken from Stage B). Lines on the leading axes; d may carry one
    trailing right-hand-side axis. Returns x shaped like d.
    """
    a, b, c, d = (np.asarray(t, dtype=np.float64) for t in (a, b, c, d))
    n = b.shape[-1]
    extra = d.ndim - b.ndim
    if n == 1:
        return d / (b[..., None] if extra else b)
    parts = partition_rows(n, p)
    stages = []
    for k, (s, e) in enumerate(parts):  # Stage A
        ak, ck = a[..., s:e].copy(), c[..., s:e].copy()
        if k == 0:
            ak[..., 0] = 0.0
        if k == len(parts) - 1:
            ck[..., -1] = 0.0
        dk = d[..., s:e, :] if extra else d[..., s:e]
        stages.append(modified_thomas_partition(ak, b[..., s:e], ck, dk))
    sub, sup, rhs = reduced_system(stages)  # Stage B
    ends = thomas(sub, np.ones(sub.shape), sup, rhs)
    x = np.empty(d.shape)
    ex = (lambda v: v[..., None]) if extra else (lambda v: v)
    for k, ((s, e), st) in enumerate(zip(parts, stages)):  # Stage C
        x0 = _rhs_row(ends, 2 * k, extra)
        xl = _rhs_row(ends, 2 * k + 1, extra)
        for i in range(e - s):
            if i == 0:
                v = x0
            elif i == e - s - 1:
                v = xl
            else:
                v = _rhs_row(st["delta"], i, extra) - ex(st["alpha"][..., i]) * x0 - ex(st["gamma"][..., i]) * xl
            x[(Ellipsis, s + i) + (slice(None),) * extra] = v
    return x


def pdd(a, b, c, d, p: int):
    """Parallel diagonally dominant approximation (Section 5.1 and Section 6.2.2 name it for the
    diagonally dominant momentum systems; the steps are Sun's PDD method).

    Stage A, as in dc_spike: per partition k = [s, e], with its outer couplings a_s and c_e
    removed, x~ = A_k^{-1} d, v = A_k^{-1}(a_s e_first) (k > 0), w = A_k^{-1}(c_e e_last)
    (k < p-1), so that inside the partition x_i = x~_i - v_i x_{s-1} - w_i x_{e+1} exactly.
    Reduced step: at the interface between partitions k and k+1 (rows e_k and s_{k+1}) the exact
    relations of its two unknowns are
        x_{e_k} + v_{e_k} x_{e_{k-1}} + w_{e_k} x_{s_{k+1}} = x~_{e_k},
        x_{s_{k+1}} + v_{s_{k+1}} x_{e_k} + w_{s_{k+1}} x_{s_{k+2}} = x~_{s_{k+1}}.
    PDD drops v_{e_k} (the left coupling seen at the far end of partition k) and w_{s_{k+1}} (the
    right coupling seen at the far end of partition k+1), which leaves the 2x2 system
        [1, w_{e_k}; v_{s_{k+1}}, 1] [y1; y2] = [x~_{e_k}; x~_{s_{k+1}}]
    for y1 ~ x_{e_k}, y2 ~ x_{s_{k+1}}, solved by Cramer's rule.
    Correction: x = x~ - v y1(left interface) - w y2(right interface) in every partition.
    p = 1 is the Thomas solve. Works on (lines, n) arrays; returns x with the shape of d.
    """
    a, b, c, d = (np.atleast_2d(np.asarray(t, dtype=np.float64)) for t in (a, b, c, d))
    squeeze = np.asarray(b).ndim == 1
    L, n = b.shape
    parts = partition_rows(n, p)
    xt = np.zeros((L, n))
    v = np.zeros((L, n))
    w = np.zeros((L, n))
    for k, (s, e) in enumerate(parts):  # Stage A
        ak, bk, ck = a[:, s:e].copy(), b[:, s:e], c[:, s:e].copy()
        ak[:, 0] = 0.0
        ck[:, -1] = 0.0
        xt[:, s:e] = thomas(ak, bk, ck, d[:, s:e])
        if k > 0:
            rhs = np.zeros((L, e - s))
            rhs[:, 0] = a[:, s]
            v[:, s:e] = thomas(ak, bk, ck, rhs)
        if k < p - 1:
            rhs = np.zeros((L, e - s))
            rhs[:, -1] = c[:, e - 1]
            w[:, s:e] = thomas(ak, bk, ck, rhs)
    y1 = np.zeros((L, p))  # y1[:, k]: x_{e_k} at interface k (k = 0..p-2)
    y2 = np.zeros((L, p))  # y2[:, k]: x_{s_{k+1}}
    for k in range(p - 1):
        eL = parts[k][1] - 1
        sR = parts[k + 1][0]
        wl, vr = w[:, eL], v[:, sR]
        det = 1.0 - wl * vr
        y1[:, k] = (xt[:, eL] - wl * xt[:, sR]) / det
        y2[:, k] = (xt[:, sR] - vr * xt[:, eL]) / det
    x = xt.copy()
    for k, (s, e) in enumerate(parts):  # correction with the neighbours' interface values
        if k > 0:
            x[:, s:e] -= v[:, s:e] * y1[:, k - 1][:, None]
        if k < p - 1:
            x[:, s:e] -= w[:, s:e] * y2[:, k][:, None]
    return x[0] if squeeze else x


def poisson_fft(q, dx, dz, a, b, c, pin_zero_mode=True):
    """Discrete Poisson solve D_xx phi + D_yy phi + D_zz phi = q on a grid q[y][z][x] periodic in
    x and z (Section 5.2: Fourier transforms in the two periodic directions leave
    (D_yy - k_x'^2 - k_z'^2) Phi = Q, one tridiagonal system along y per wavenumber pair).

    D_xx, D_zz are the periodic second differences (u_{i+1} - 2 u_i + u_{i-1}) / h^2, whose Fourier
    symbols are -k'^2(l) = -(2 - 2 cos(2 pi l / N)) / h^2; D_yy is the tridiagonal (a, b, c) of
    length ny. Steps: Q = rfft2(q) over (z, x); for every (kz, kx) solve the complex line with
    Thomas (real and imaginary parts as two right-hand sides); phi = irfft2(Phi). With
    pin_zero_mode the (0, 0) line's row 0 is replaced by Phi_0 = 0 (its system is singular when
    D_yy has Neumann ends).
    """
    q = np.asarray(q, dtype=np.float64)
    ny, nz, nx = q.shape
    a, b, c = (np.asarray(t, dtype=np.float64) for t in (a, b, c))
    Q = np.fft.rfft2(q, axes=(1, 2))                      # [ny][nz][nkx]
    nkx = Q.shape[2]
    k2x = (2.0 - 2.0 * np.cos(2.0 * np.pi * np.arange(nkx) / nx)) / dx ** 2
    k2z = (2.0 - 2.0 * np.cos(2.0 * np.pi * np.arange(nz) / nz)) / dz ** 2
    shift = -(k2z[:, None] + k2x[None, :]).reshape(-1)   # line l = kz * nkx + kx
    L = nz * nkx
    lines_a = np.broadcast_to(a, (L, ny)).copy()
    lines_b = b[None, :] + shift[:, None]
    lines_c = np.broadcast_to(c, (L, ny)).copy()
    rhs = Q.reshape(ny, L).T                             # [L][ny] complex
    D = np.stack([rhs.real, rhs.imag], axis=-1)          # [L][ny][2]
    if pin_zero_mode:
        lines_b[0, 0], lines_c[0, 0] = 1.0, 0.0
        D[0, 0, :] = 0.0
    X = thomas(lines_a, lines_b, lines_c, D)
    Phi = (X[..., 0] + 1j * X[..., 1]).T.reshape(ny, nz, nkx)
    return np.fft.irfft2(Phi, s=(nz, nx), axes=(1, 2))


def residual(a, b, c, d, x, dtype=np.float64):
    """r = d - A x along the last axis (a_0 and c_{n-1} ignored)."""
    a, b, c, d, x = (np.asarray(t, dtype=dtype) for t in (a, b, c, d, x))
    ax = b * x
    ax[..., 1:] += a[..., 1:] * x[..., :-1]
    ax[..., :-1] += c[..., :-1] * x[..., 1:]
    return d - ax


def transpose_coefficients(a, b, c):
    """Diagonals of A^T: sub'_i = c_{i-1}, diag'_i = b_i, super'_i = a_{i+1} (ends zero)."""
    a, b, c = (np.asarray(t, dtype=np.float64) for t in (a, b, c))
    at = np.zeros_like(a)
    ct = np.zeros_like(c)
    at[..., 1:] = c[..., :-1]
    ct[..., :-1] = a[..., 1:]
    return at, b.copy(), ct


def adjoint_grads(a, b, c, x, g):
    """Gradients of L with dL/dx = g through x = A^{-1} d (standard adjoint: dL/dA = -lambda x^T).

    lambda = A^{-T} g (Thomas on the transposed diagonals); grad_d = lambda;
    grad_b = -lambda x; grad_a_i = -lambda_i x_{i-1} (0 at i = 0);
    grad_c_i = -lambda_i x_{i+1} (0 at i = n-1).
    """
    at, bt, ct = transpose_coefficients(a, b, c)
    lam = thomas(at, bt, ct, g)
    x = np.asarray(x, dtype=np.float64)
    ga = np.zeros_like(lam)
    gc = np.zeros_like(lam)
    ga[..., 1:] = -lam[..., 1:] * x[..., :-1]
    gc[..., :-1] = -lam[..., :-1] * x[..., 1:]
    return ga, -lam * x, gc, lam


def thomas_ragged(a, b, c, d, offsets, lengths, lines=None, dtype=np.float64):
    """Thomas over packed lines of uneven length; solves ``lines`` (default all) and returns
    {line index: x}. Lines of equal length are solved together.
    """
    offsets = np.asarray(offsets, dtype=np.int64)
    lengths = np.asarray(lengths, dtype=np.int64)
    lines = np.arange(len(lengths)) if lines is None else np.asarray(lines)
    out = {}
    for n in np.unique(lengths[lines]):
        sel = lines[lengths[lines] == n]
        idx = offsets[sel][:, None] + np.arange(n)[None, :]
        x = thomas(a[idx], b[idx], c[idx], d[idx], dtype=dtype)
        for k, li in enumerate(sel):
            out[int(li)] = x[k].astype(np.float64)
    return out


def rel_l2(x, ref):
    """Relative L2 error ||x - ref|| / ||ref||."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref.ravel())
    return float(np.linalg.norm((x - ref).ravel()) / (den if den > 0 else 1.0))
