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

// Lines to correct (coefficients broadcast to all lines, optional per-line shift): line l is listed
// unless its condition-number bound is below kappa_max. For a row-diagonally-dominant A,
// ||A^-1||_inf <= 1 / delta with delta = min_i (|b_i| - |a_i| - |c_i|) (Varah 1975), so
// kappa_inf(A) <= ||A||_inf / delta. Both are evaluated in float (rounding about 2^-24 of the row
// sums, far inside the factor of two of slack taken below: a line is kept off the list only if
// ||A|| < delta kappa_max / 2). Lines without a positive margin are always listed. The rows are
// staged in shared memory as floats (b_i, |a_i| + |c_i|), kSelectRows at a time; one thread per
// line, grid-stride. Listed lines go to list[0 .. *count) (order unspecified).
constexpr int kSelectRows = 2048;

__global__ void __launch_bounds__(256) select_lines_kernel(const Args A, float kappa_max, int32_t* __restrict__ list,
                                                           int32_t* count) {
  __shared__ float sb[kSelectRows], sac[kSelectRows];
  const int64_t n = A.lay.n, L = A.lay.n_lines;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // every block walks the same number of line rounds (the barriers below need all its threads)
  const int64_t rounds = (L + stride - 1) / stride;
  for (int64_t r = 0; r < rounds; ++r) {
    const int64_t line = first + r * stride;
    const bool active = line < L;
    const float s = (active && A.shift) ? (float)ldg((const double*)A.shift + line) : 0.f;
    float margin = INFINITY, norm = 0.f;
    for (int64_t i0 = 0; i0 < n; i0 += kSelectRows) {
      const int rows = (int)(n - i0 < kSelectRows ? n - i0 : kSelectRows);
      __syncthreads();
      for (int t = threadIdx.x; t < rows; t += blockDim.x) {
        const int64_t i = i0 + t;
        const double av = i > 0 ? fabs(ldg((const double*)A.a + i)) : 0.0;
        const double cv = i < n - 1 ? fabs(ldg((const double*)A.c + i)) : 0.0;
        sb[t] = (float)ldg((const double*)A.b + i);
        sac[t] = (float)(av + cv);
      }
      __syncthreads();
      if (active) {
        for (int t = 0; t < rows; ++t) {
          const float bb = fabsf(sb[t] + s);
          margin = fminf(margin, bb - sac[t]);
          norm = fmaxf(norm, bb + sac[t]);
        }
      }
    }
    if (active && !(margin > 0.f && norm < 0.5f * kappa_max * margin)) list[atomicAdd(count, 1)] = (int32_t)line;
  }
}

// r = d - A x exactly for every (line, row) of the corrected lines, one thread each (adjacent
// threads on adjacent lines), grid-stride, into R ([row][k], nrhs floats each, row pitch n_lines).
// Line k is list[k] for k < *count, or every line k when list is null (then n_lines is written to
// *count, the number of corrected lines the plan reports).
template <int NR>
__global__ void __launch_bounds__(256) residual_exact_kernel(const Args A, float* __restrict__ R,
                                                             const int32_t* __restrict__ list, int32_t* count) {
  const Layout& L = A.lay;
  const int64_t cnt = list ? (int64_t)*count : L.n_lines;
  if (!list && blockIdx.x == 0 && threadIdx.x == 0) *count = (int32_t)L.n_lines;
  const int64_t total = L.n * cnt;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = idx % cnt, i = idx / cnt;
    const int64_t line = list ? (int64_t)list[k] : k;
    const int64_t e = L.off(line) + i * L.es, ci = A.bcast ? i : e;
    const double shift = A.shift ? ldg((const double*)A.shift + line) : 0.0;
    const DecF64 da = dec_f64(i > 0 ? ldg((const double*)A.a + ci) : 0.0);
    const DecF64 db = dec_f64(ldg((const double*)A.b + ci) + shift);  // the b of the FP64 solve
    const DecF64 dc = dec_f64(i < L.n - 1 ? ldg((const double*)A.c + ci) : 0.0);
    const double* X = (const double*)A.x;
    const double* D = (const double*)A.d;
    const int64_t r = i * L.n_lines + k;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const DecF64 dxm = dec_f64(i > 0 ? X[(e - L.es) * NR + q] : 0.0);
      const DecF64 dxp = dec_f64(i < L.n - 1 ? X[(e + L.es) * NR + q] : 0.0);
      R[r * NR + q] = residual_exact_dec(dec_f64(ldg(D + e * NR + q)), da, dxm, db, dec_f64(X[e * NR + q]), dc, dxp);
    }
  }
}

// The FP32 correction A32 dx = r (A32: coefficients truncated to float) and x += dx, one thread
// per line: forward elimination over R in place (c' to cw), back substitution into x. Rows are
// loaded kCorrAhead ahead of the recurrence in both sweeps (the loads of later rows are issued
// before this row's stores, which the compiler may not reorder across: R, cw and x may alias).
constexpr int kCorrAhead = 4;

template <int NR>
TDMA_DEV void correct_line(const Args& A, float* __restrict__ cw, float* __restrict__ R, int64_t k, int64_t line);

// Line k (as in residual_exact_kernel) uses column k of R and cw; grid-stride over k.
template <int NR>
__global__ void __launch_bounds__(128) correction32_kernel(const Args A, float* __restrict__ cw, float* __restrict__ R,
                                                           const int32_t* __restrict__ list, const int32_t* count) {
  const int64_t cnt = list ? (int64_t)*count : A.lay.n_lines;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += (int64_t)gridDim.x * blockDim.x)
    correct_line<NR>(A, cw, R, k, list ? (int64_t)list[k] : k);
}

// The correction of one line: column k of R and cw.
template <int NR>
TDMA_DEV void correct_line(const Args& A, float* __restrict__ cw, float* __restrict__ R, int64_t k, int64_t line) {
  constexpr int K = kCorrAhead;
  const int64_t n = A.lay.n, es = A.lay.es, L = A.lay.n_lines;
  const int64_t base = A.lay.off(line);
  const double shift = A.shift ? ldg((const double*)A.shift + line) : 0.0;
  double* X = (double*)A.x;
  float* Rl = R + k * NR;   // row i at Rl[i * L * NR + q]
  float* cwl = cw + k;      // row i at cwl[i * L]
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
