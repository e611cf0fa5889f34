// FP64 solve followed by a correction from an exact residual (TDMA_F64_REFINE).
//
// For badly conditioned lines (the pinned zero mode of the Poisson wavenumber lines has
// condition number about 1e9) a plain FP64 elimination is a few 1e-12 away from the exact
// solution. Mixed-precision iterative refinement (Wilkinson 1963; Moler 1967; Carson and Higham
// 2018) removes that: with the residual r = d - A x evaluated more precisely than the solve and a
// correction solve whose relative error is well below one, x + dx is accurate to the residual's
// precision. Here the residual is exact (residual_exact in exact_residual.cuh: 106-bit products and a
// 128-bit fixed-point sum on the integer pipes) and the correction is solved in FP32 with the
// coefficients truncated to float: its relative error, about kappa 2^-23, stays near 1e-3 even on
// the worst Poisson modes, so one correction takes their error from about 2e-12 to the 1e-15
// range. GB300 runs FP64 arithmetic at 1/64 of the FP32 rate; this correction uses three FP64 adds
// per unknown (b + shift, and x += dx per right-hand side) where a double-double residual and a
// second FP64 solve took about 70.
//
// The residual is one thread per unknown (no dependence along the line); the FP32 correction is
// one thread per line, with its factors c' and the residuals / forward right-hand sides in the
// workspace ([row][line], coalesced across adjacent lines). Residuals
// below the float range (right-hand sides under about 1e-22) are flushed to zero: such lines keep
// the plain FP64 accuracy.
#pragma once
#include "layout.cuh"
#include "exact_residual.cuh"

namespace tdma {

// r = d - A x exactly for every (line, row), one thread each (adjacent threads on adjacent lines),
// into R ([row][line], nrhs floats each).
template <int NR>
__global__ void __launch_bounds__(256) residual_exact_kernel(const Args A, float* __restrict__ R) {
  const Layout& L = A.lay;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L.n * L.n_lines) return;
  const int64_t line = idx % L.n_lines, i = idx / L.n_lines;
  const int64_t e = L.off(line) + i * L.es, ci = A.bcast ? i : e;
  const double shift = A.shift ? ldg((const double*)A.shift + line) : 0.0;
  const DecF64 da = dec_f64(i > 0 ? ldg((const double*)A.a + ci) : 0.0);
  const DecF64 db = dec_f64(ldg((const double*)A.b + ci) + shift);  // the b of the FP64 solve
  const DecF64 dc = dec_f64(i < L.n - 1 ? ldg((const double*)A.c + ci) : 0.0);
  const double* X = (const double*)A.x;
  const double* D = (const double*)A.d;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    const DecF64 dxm = dec_f64(i > 0 ? X[(e - L.es) * NR + q] : 0.0);
    const DecF64 dxp = dec_f64(i < L.n - 1 ? X[(e + L.es) * NR + q] : 0.0);
    R[idx * NR + q] = residual_exact_dec(dec_f64(ldg(D + e * NR + q)), da, dxm, db, dec_f64(X[e * NR + q]), dc, dxp);
  }
}

// The FP32 correction A32 dx = r (A32: coefficients truncated to float) and x += dx, one thread
// per line: forward elimination over R in place (c' to cw), back substitution into x. Rows are
// loaded kCorrAhead ahead of the recurrence in both sweeps (the loads of later rows are issued
// before this row's stores, which the compiler may not reorder across: R, cw and x may alias).
constexpr int kCorrAhead = 4;

template <int NR>
__global__ void __launch_bounds__(128) correction32_kernel(const Args A, float* __restrict__ cw, float* __restrict__ R) {
  constexpr int K = kCorrAhead;
  const int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= A.lay.n_lines) return;
  const int64_t n = A.lay.n, es = A.lay.es, L = A.lay.n_lines;
  const int64_t base = A.lay.off(line);
  const double shift = A.shift ? ldg((const double*)A.shift + line) : 0.0;
  double* X = (double*)A.x;
  float* Rl = R + line * NR;   // row i at Rl[i * L * NR + q]
  float* cwl = cw + line;      // row i at cwl[i * L]
  float cp = 0.f, rp[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) rp[q] = 0.f;
  float rb[K][NR];
#pragma unroll
  for (int u = 0; u < K; ++u)
    if (u < n) {
#pragma unroll
      for (int q = 0; q < NR; ++q) rb[u][q] = Rl[(int64_t)u * L * NR + q];
    }
  for (int64_t i0 = 0; i0 < n; i0 += K) {
    float nb[K][NR];
#pragma unroll
    for (int u = 0; u < K; ++u)
      if (i0 + K + u < n) {
#pragma unroll
        for (int q = 0; q < NR; ++q) nb[u][q] = Rl[(i0 + K + u) * L * NR + q];
      }
#pragma unroll
    for (int u = 0; u < K; ++u) {
      const int64_t i = i0 + u;
      if (i < n) {
        const int64_t ci = A.bcast ? i : base + i * es;
        const float a32 = i > 0 ? f64_to_f32_trunc(ldg((const double*)A.a + ci)) : 0.f;
        const float b32 = f64_to_f32_trunc(ldg((const double*)A.b + ci) + shift);
        const float c32 = i < n - 1 ? f64_to_f32_trunc(ldg((const double*)A.c + ci)) : 0.f;
        const float w = rcp(fmaf(-a32, cp, b32));
        cp = c32 * w;
        cwl[i * L] = cp;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          rp[q] = fmaf(-a32, rp[q], rb[u][q]) * w;
          Rl[i * L * NR + q] = rp[q];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < K; ++u)
#pragma unroll
      for (int q = 0; q < NR; ++q) rb[u][q] = nb[u][q];
  }
  // back substitution from row n-1 (dn = its d') down to row 0, rows K ahead
  float dn[NR];
  bool ok = true;
#pragma unroll
  for (int q = 0; q < NR; ++q) dn[q] = rp[q];
  float cb[K], db[K][NR];
  double xb[K][NR];
  auto load_row = [&](int64_t i, float& c, float* d, double* xv) {
    c = i < n - 1 ? cwl[i * L] : 0.f;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      d[q] = Rl[i * L * NR + q];
      xv[q] = X[(base + i * es) * NR + q];
    }
  };
#pragma unroll
  for (int u = 0; u < K; ++u)
    if (n - 1 - u >= 0) load_row(n - 1 - u, cb[u], db[u], xb[u]);
  for (int64_t i0 = n - 1; i0 >= 0; i0 -= K) {
    float nc[K], nd[K][NR];
    double nx[K][NR];
#pragma unroll
    for (int u = 0; u < K; ++u)
      if (i0 - K - u >= 0) load_row(i0 - K - u, nc[u], nd[u], nx[u]);
#pragma unroll
    for (int u = 0; u < K; ++u) {
      const int64_t i = i0 - u;
      if (i >= 0) {
        const int64_t e = base + i * es;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          if (i < n - 1) dn[q] = fmaf(-cb[u], dn[q], db[u][q]);
          ok &= isfinite(dn[q]);
          X[e * NR + q] = xb[u][q] + f2d_fast(dn[q]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < K; ++u) {
      cb[u] = nc[u];
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        db[u][q] = nd[u][q];
        xb[u][q] = nx[u][q];
      }
    }
  }
  if (!ok) report_error(A.st, 5);
}

}  // namespace tdma
