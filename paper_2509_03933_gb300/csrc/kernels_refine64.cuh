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
// per line: forward elimination over R in place (c' to cw), back substitution into x.
template <int NR>
__global__ void __launch_bounds__(128) correction32_kernel(const Args A, float* __restrict__ cw, float* __restrict__ R) {
  const int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= A.lay.n_lines) return;
  const int64_t n = A.lay.n, es = A.lay.es, L = A.lay.n_lines;
  const int64_t base = A.lay.off(line);
  const double shift = A.shift ? ldg((const double*)A.shift + line) : 0.0;
  double* X = (double*)A.x;
  float cp = 0.f, rp[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) rp[q] = 0.f;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t ci = A.bcast ? i : base + i * es;
    const float a32 = i > 0 ? f64_to_f32_trunc(ldg((const double*)A.a + ci)) : 0.f;
    const float b32 = f64_to_f32_trunc(ldg((const double*)A.b + ci) + shift);
    const float c32 = i < n - 1 ? f64_to_f32_trunc(ldg((const double*)A.c + ci)) : 0.f;
    const float w = rcp(fmaf(-a32, cp, b32));
    cp = c32 * w;
    cw[i * L + line] = cp;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      float* r = R + (i * L + line) * NR + q;
      rp[q] = fmaf(-a32, rp[q], *r) * w;
      *r = rp[q];
    }
  }
  float dn[NR];
  bool ok = true;
#pragma unroll
  for (int q = 0; q < NR; ++q) dn[q] = rp[q];
  for (int64_t i = n - 1; i >= 0; --i) {
    const int64_t e = base + i * es;
    if (i < n - 1) {
      const float cpi = cw[i * L + line];
#pragma unroll
      for (int q = 0; q < NR; ++q) dn[q] = fmaf(-cpi, dn[q], R[(i * L + line) * NR + q]);
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      ok &= isfinite(dn[q]);
      X[e * NR + q] += f2d_fast(dn[q]);
    }
  }
  if (!ok) report_error(A.st, 5);
}

}  // namespace tdma
