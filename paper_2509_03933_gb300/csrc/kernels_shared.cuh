// Lines that share one set of coefficients (coef_broadcast without a per-line shift): the Thomas
// factorisation c'_i, 1 / w_i depends on the coefficients only, so it is computed once for all
// lines and every line runs just the right-hand-side recurrences:
//     d'_i = (d_i - a_i d'_{i-1}) / w_i,    x_i = d'_i - c'_i x_{i+1},
// three FP64 operations per unknown and right-hand side instead of nine (GB300's FP64 pipe bounds
// the Thomas sweep). In the paper's momentum solver all systems of a batch share one coefficient
// matrix, which depends on the grid spacing only (Section 6.2.1); here that matrix is factorised
// once per solve for all lines of the batch. With TR the factors are those of A^T (the adjoint).
#pragma once
#include "layout.cuh"
#include "kernels_dc.cuh"

namespace tdma {

// Factors of the shared coefficients, one thread (a recurrence along the line).
template <class CT, bool TR>
__global__ void shared_factor_kernel(const Args A, CT* __restrict__ cp, CT* __restrict__ wi) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int64_t n = A.lay.n;
  const CT* pa = (const CT*)A.a;
  const CT* pb = (const CT*)A.b;
  const CT* pc = (const CT*)A.c;
  CT c_prev = CT(0);
  bool ok = true;
  for (int64_t i = 0; i < n; ++i) {
    const CT sub = i == 0 ? CT(0) : (TR ? pc[i - 1] : pa[i]);
    const CT sup = i == n - 1 ? CT(0) : (TR ? pa[i + 1] : pc[i]);
    const CT w = rcp(pb[i] - sub * c_prev);
    ok &= finite(w);
    c_prev = sup * w;
    cp[i] = c_prev;
    wi[i] = w;
  }
  if (!ok) report_error(A.st, 5);
}

// One thread per line: forward recurrence into x, back substitution in place.
template <class CT, int NR, bool TR>
__global__ void __launch_bounds__(128) shared_solve_kernel(const Args A, const CT* __restrict__ cp,
                                                           const CT* __restrict__ wi) {
  const int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= A.lay.n_lines) return;
  const int64_t n = A.lay.n, es = A.lay.es, base = A.lay.off(line);
  const CT* pa = (const CT*)A.a;
  const CT* pc = (const CT*)A.c;
  const CT* D = (const CT*)A.d;
  CT* X = (CT*)A.x;
  CT dp[NR], nd[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    dp[q] = CT(0);
    nd[q] = ldg(D + base * NR + q);  // row 0, loaded ahead
  }
  for (int64_t i = 0; i < n; ++i) {
    const int64_t e = base + i * es;
    CT d[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      d[q] = nd[q];
      if (i + 1 < n) nd[q] = ldg(D + (e + es) * NR + q);
    }
    const CT sub = i == 0 ? CT(0) : (TR ? ldg(pc + i - 1) : ldg(pa + i));
    const CT w = ldg(wi + i);
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      dp[q] = (d[q] - sub * dp[q]) * w;
      X[e * NR + q] = dp[q];
    }
  }
  CT xn[NR];
  bool ok = true;
#pragma unroll
  for (int q = 0; q < NR; ++q) xn[q] = dp[q];
  for (int64_t i = n - 2; i >= 0; --i) {
    const int64_t e = base + i * es;
    const CT c = ldg(cp + i);
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      xn[q] = X[e * NR + q] - c * xn[q];
      X[e * NR + q] = xn[q];
    }
  }
#pragma unroll
  for (int q = 0; q < NR; ++q) ok &= finite(xn[q]);
  if (!ok) report_error(A.st, 5);
}

template <class CT, int NR, bool TR>
inline cudaError_t launch_shared(const Args& A, cudaStream_t s) {
  CT* cp = (CT*)A.ws;
  CT* wi = cp + A.lay.n;
  shared_factor_kernel<CT, TR><<<1, 32, 0, s>>>(A, cp, wi);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  shared_solve_kernel<CT, NR, TR><<<(unsigned)((A.lay.n_lines + 127) / 128), 128, 0, s>>>(A, cp, wi);
  return cudaGetLastError();
}

inline cudaError_t launch_shared_any(tdma_precision_t p, int nrhs, bool tr, const Args& A, cudaStream_t s) {
  if (p == TDMA_F64) {
    if (nrhs == 1) return tr ? launch_shared<double, 1, true>(A, s) : launch_shared<double, 1, false>(A, s);
    return tr ? launch_shared<double, 2, true>(A, s) : launch_shared<double, 2, false>(A, s);
  }
  if (nrhs == 1) return tr ? launch_shared<float, 1, true>(A, s) : launch_shared<float, 1, false>(A, s);
  return tr ? launch_shared<float, 2, true>(A, s) : launch_shared<float, 2, false>(A, s);
}

}  // namespace tdma
