// Lines split across devices (the paper's 1D slab decomposition along the solve axis; Section 2.1
// and Algorithm 2): every rank holds a slab of consecutive rows of every line. The three stages
// become three kernels with an exchange between them:
//   slab_reduce_kernel   Stage A over the rank's slab (the slab is one partition): the modified
//                        Thomas sweep leaves the slab's first and last rows as a unit-diagonal
//                        pair in the neighbours' end unknowns (the reduced rows sent to the rank
//                        that solves Stage B for the line) and the interior relations in a
//                        scratch array;
//   pairs_solve_kernel   Stage B on the gathered pairs of all slabs of a line: the 2W-row
//                        unit-diagonal system by Thomas, giving every slab's two end values;
//   slab_finish_kernel   Stage C over the slab from its two end values.
// FP64 throughout (Stage B in FP64 as everywhere on the path). One thread per line; the scratch
// and the line arrays are [row][line], so a warp's accesses to one row are coalesced when the
// lines are adjacent in memory.
#pragma once
#include "layout.cuh"

namespace tdma {

// Values per line in the reduced buffer: sub0, sup0, sub1, sup1, rhs0[NR], rhs1[NR].
template <int NR> __host__ __device__ constexpr int slab_k() { return 4 + 2 * NR; }

struct SlabArgs {
  const double* a;
  const double* b;
  const double* c;
  const double* d;
  double* x;
  Layout lay;        // n = rows of the slab
  int first, last;   // the slab holds the line's first / last row
  int64_t line0, count;
  double* red;       // [count][K]
  double* scratch;   // (n - 2) x (2 + NR) x count, [array][row][line]
  const double* ends;  // [count][2 NR]
  DevStatus* st;
};

template <int NR>
__global__ void __launch_bounds__(128) slab_reduce_kernel(const SlabArgs S) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= S.count) return;
  const int64_t line = S.line0 + j, m = S.lay.n, es = S.lay.es, base = S.lay.off(line);
  const int64_t slots = m - 2, cnt = S.count;
  double* s_alpha = S.scratch;
  double* s_gamma = s_alpha + slots * cnt;
  double* s_delta = s_gamma + slots * cnt;  // NR arrays
  auto ld = [&](const double* p, int64_t i) { return __ldg(p + base + i * es); };
  auto ldd = [&](int64_t i, int q) { return __ldg(S.d + (base + i * es) * NR + q); };
  // row 0 of the slab
  const double a0 = S.first ? 0.0 : ld(S.a, 0), b0 = ld(S.b, 0), c0 = ld(S.c, 0);
  double d0[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) d0[q] = ldd(0, q);
  // rows 1 .. m-1: forward modified-Thomas recurrences (alpha: coefficient of x_0, gamma: of the
  // next row, delta: right-hand side), with the row-0 relation accumulated in F, G, Q
  double alpha = -1.0, gamma = 0.0, delta[NR], F[NR], G = 0.0, Q = 1.0;
#pragma unroll
  for (int q = 0; q < NR; ++q) { delta[q] = 0.0; F[q] = 0.0; }
  bool ok = true;
  for (int64_t t = 1; t < m; ++t) {
    const double a = ld(S.a, t), b = ld(S.b, t);
    const double c = (S.last && t == m - 1) ? 0.0 : ld(S.c, t);
    const double r = rcp(b - a * gamma);
    ok &= finite(r);
    const double ar = a * r;
    alpha = -ar * alpha;
    gamma = c * r;
#pragma unroll
    for (int q = 0; q < NR; ++q) delta[q] = r * ldd(t, q) - ar * delta[q];
    if (t <= m - 2) {
      const int64_t o = (t - 1) * cnt + j;
      s_alpha[o] = alpha;
      s_gamma[o] = gamma;
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        s_delta[q * slots * cnt + o] = delta[q];
        F[q] += Q * delta[q];
      }
      G += Q * alpha;
      Q = -Q * gamma;
    }
  }
  const double rho = rcp(b0 - c0 * G);
  ok &= finite(rho);
  double* r = S.red + j * slab_k<NR>();
  r[0] = rho * a0;       // row 0: sub (x of the previous slab's last row)
  r[1] = rho * c0 * Q;   //        sup (x of this slab's last row)
  r[2] = alpha;          // row m-1: sub (x of this slab's first row)
  r[3] = gamma;          //          sup (x of the next slab's first row)
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    r[4 + q] = rho * (d0[q] - c0 * F[q]);
    r[4 + NR + q] = delta[q];
  }
  if (!ok) report_error(S.st, 5);
}

// gathered: [W][count][K] (slab-major, as an all-to-all delivers it); ends: [W][count][2 NR].
template <int NR>
__global__ void __launch_bounds__(128) pairs_solve_kernel(int W, int64_t count, const double* __restrict__ gathered,
                                                          double* __restrict__ ends, double* __restrict__ work,
                                                          DevStatus* st) {
  constexpr int K = slab_k<NR>();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= count) return;
  // forward Thomas over the 2W unit-diagonal rows; c' and d' to the work array [row][count]
  const int64_t R = 2 * (int64_t)W;
  double* cpw = work;                  // R x count
  double* dpw = work + R * count;      // NR x R x count
  double cp = 0.0, dp[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) dp[q] = 0.0;
  bool ok = true;
  for (int64_t i = 0; i < R; ++i) {
    const double* g = gathered + ((i >> 1) * count + j) * K;
    const int h = (int)(i & 1);
    const double sub = i == 0 ? 0.0 : g[2 * h];
    const double sup = i == R - 1 ? 0.0 : g[2 * h + 1];
    const double iw = rcp(1.0 - sub * cp);
    ok &= finite(iw);
    cp = sup * iw;
    cpw[i * count + j] = cp;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      dp[q] = (g[4 + h * NR + q] - sub * dp[q]) * iw;
      dpw[(q * R + i) * count + j] = dp[q];
    }
  }
  double xn[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) xn[q] = dp[q];
  for (int64_t i = R - 1; i >= 0; --i) {
    if (i < R - 1) {
      const double c = cpw[i * count + j];
#pragma unroll
      for (int q = 0; q < NR; ++q) xn[q] = dpw[(q * R + i) * count + j] - c * xn[q];
    }
    double* e = ends + ((i >> 1) * count + j) * (2 * NR) + (i & 1) * NR;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      e[q] = xn[q];
      ok &= finite(xn[q]);
    }
  }
  if (!ok) report_error(st, 5);
}

// ends: [count][2 NR] (the slab's own first and last values).
template <int NR>
__global__ void __launch_bounds__(128) slab_finish_kernel(const SlabArgs S) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= S.count) return;
  const int64_t line = S.line0 + j, m = S.lay.n, es = S.lay.es, base = S.lay.off(line);
  const int64_t slots = m - 2, cnt = S.count;
  const double* s_alpha = S.scratch;
  const double* s_gamma = s_alpha + slots * cnt;
  const double* s_delta = s_gamma + slots * cnt;
  double x0[NR], xn[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    x0[q] = S.ends[j * 2 * NR + q];
    xn[q] = S.ends[j * 2 * NR + NR + q];
    S.x[base * NR + q] = x0[q];
    S.x[(base + (m - 1) * es) * NR + q] = xn[q];
  }
  for (int64_t t = m - 2; t >= 1; --t) {
    const int64_t o = (t - 1) * cnt + j;
    const double al = s_alpha[o], ga = s_gamma[o];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      xn[q] = s_delta[q * slots * cnt + o] - al * x0[q] - ga * xn[q];
      S.x[(base + t * es) * NR + q] = xn[q];
    }
  }
}

}  // namespace tdma
