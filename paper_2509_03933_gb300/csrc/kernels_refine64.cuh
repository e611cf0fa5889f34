// FP64 solve followed by iterative refinement with a double-double residual (TDMA_F64_REFINE).
//
// For badly conditioned lines (the pinned zero mode of the Poisson wavenumber lines has
// condition number about 1e9) a plain FP64 elimination is a few 1e-12 away from the exact
// solution. Mixed-precision refinement with an extra-precise residual (Wilkinson 1963; Demmel
// et al. 2006) removes that: r = d - A x evaluated in double-double arithmetic (FMA-based
// TwoProduct and Knuth's TwoSum, accurate as if computed with twice the precision; Ogita, Rump
// and Oishi 2005), one more FP64 solve for the correction, x += correction. The FP64 solve
// contracts the error by its own relative error (about 1e-12 here), so one correction leaves
// only the rounding of x itself.
//
// The residual and correction live in a workspace buffer R. With broadcast coefficients the
// correction solve does not depend on the layout of the right-hand side, so R is compact
// ([row][line]); otherwise R uses the plan's layout.
#pragma once
#include "layout.cuh"

namespace tdma {

struct dd { double h, l; };

TDMA_DEV dd two_sum_d(double a, double b) {
  const double s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  return {s, __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb))};
}
TDMA_DEV dd two_prod_d(double a, double b) {
  const double p = __dmul_rn(a, b);
  return {p, __fma_rn(a, b, -p)};
}

// r_i = d_i - (a_i x_{i-1} + b_i x_i + c_i x_{i+1}) accumulated in double-double (Dot2-style).
TDMA_DEV double residual_dd(double a, double b, double c, double d, double xm, double x0, double xp) {
  const dd p1 = two_prod_d(b, x0), p2 = two_prod_d(a, xm), p3 = two_prod_d(c, xp);
  const dd s1 = two_sum_d(d, -p1.h);
  const dd s2 = two_sum_d(s1.h, -p2.h);
  const dd s3 = two_sum_d(s2.h, -p3.h);
  const double err = ((s1.l + s2.l) + s3.l) - ((p1.l + p2.l) + p3.l);
  return __dadd_rn(s3.h, err);
}

// One thread per (line, row); `lr` is the layout of R (compact or the plan's).
template <int NR>
__global__ void __launch_bounds__(256) residual64_kernel(const Args A, const Layout lr, double* __restrict__ R) {
  const Layout& L = A.lay;
  const int64_t total = L.n * L.n_lines;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int64_t line = idx % L.n_lines, i = idx / L.n_lines;  // adjacent threads: adjacent lines
  const int64_t e = L.off(line) + i * L.es, er = lr.off(line) + i * lr.es;
  const int64_t ci = A.bcast ? i : e;
  const double shift = A.shift ? ldg((const double*)A.shift + line) : 0.0;
  const double a = i > 0 ? ldg((const double*)A.a + ci) : 0.0;
  const double b = ldg((const double*)A.b + ci) + shift;
  const double c = i < L.n - 1 ? ldg((const double*)A.c + ci) : 0.0;
  const double* X = (const double*)A.x;
  const double* D = (const double*)A.d;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    const double xm = i > 0 ? X[(e - L.es) * NR + q] : 0.0;
    const double xp = i < L.n - 1 ? X[(e + L.es) * NR + q] : 0.0;
    R[er * NR + q] = residual_dd(a, b, c, D[e * NR + q], xm, X[e * NR + q], xp);
  }
}

template <int NR>
__global__ void __launch_bounds__(256) update64_kernel(const Layout L, const Layout lr, double* __restrict__ X,
                                                       const double* __restrict__ R) {
  const int64_t total = L.n * L.n_lines;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int64_t line = idx % L.n_lines, i = idx / L.n_lines;
  const int64_t e = L.off(line) + i * L.es, er = lr.off(line) + i * lr.es;
#pragma unroll
  for (int q = 0; q < NR; ++q) X[e * NR + q] += R[er * NR + q];
}

}  // namespace tdma
