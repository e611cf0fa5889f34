// Backward pass of x = A^{-1} d (adjoint method; the paper has no backward pass).
//
// For a scalar loss L with g = dL/dx: lambda = A^{-T} g, dL/dd = lambda and, since
// dL/dA = -lambda x^T restricted to the three diagonals,
//   dL/db_i = -lambda_i x_i,  dL/da_i = -lambda_i x_{i-1} (i >= 1),  dL/dc_i = -lambda_i x_{i+1} (i <= n-2).
// The adjoint solve reuses the forward kernels with transposed row reads (TR = true); this file
// holds the elementwise epilogue that turns lambda and x into the coefficient gradients. With
// nrhs = 2 the coefficients are real and shared by both right-hand sides, so their gradients
// sum the two components. With broadcast coefficients the gradients of the 1D arrays are sums
// over lines (warp-reduced, then atomically accumulated).
#pragma once
#include "tdma.h"
#include "layout.cuh"
#include "bits.cuh"

namespace tdma {

// 0 - l x in the gradient type (+0 for a zero product): in the precision of x (for float x exact
// before its one rounding: the product of two floats fits in a double, so its float rounding is
// the float product), narrowed to float on the integer pipe for double x and float gradients (the
// FP64 pipe converts at its own low rate). The results equal those of 0 - l x formed in double and
// rounded once to the gradient type.
template <class GT, class XT> TDMA_DEV GT neg_prod(XT l, XT x) { return (GT)(XT(0) - l * x); }
template <> TDMA_DEV float neg_prod<float, double>(double l, double x) { return d2f_fast(0.0 - l * x); }

template <class GT, class XT, int NR>
__global__ void __launch_bounds__(256) adjoint_epilogue(const Layout lay, const int bcast, const int line_fastest,
                                                        const XT* __restrict__ x, const XT* __restrict__ lam,
                                                        GT* __restrict__ ga, GT* __restrict__ gb,
                                                        GT* __restrict__ gc) {
  const int64_t total = lay.n * lay.n_lines;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = idx < total;
  int64_t line = 0, i = 0;
  if (line_fastest) { i = idx / lay.n_lines; line = idx % lay.n_lines; }
  else { line = idx / lay.n; i = idx % lay.n; }
  if (!live) { line = 0; i = 0; }
  const int64_t e = lay.off(line) + i * lay.es;
  if constexpr (NR == 1) {  // one product per gradient: no sum to carry in double
    if (!bcast) {
      if (live) {
        const XT l = lam[e];
        if (ga) ga[e] = i > 0 ? neg_prod<GT>(l, x[e - lay.es]) : GT(0);
        if (gb) gb[e] = neg_prod<GT>(l, x[e]);
        if (gc) gc[e] = i < lay.n - 1 ? neg_prod<GT>(l, x[e + lay.es]) : GT(0);
      }
      return;
    }
  }
  double sa = 0.0, sb = 0.0, sc = 0.0;
  if (live) {
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const double l = (double)lam[e * NR + q];
      sb -= l * (double)x[e * NR + q];
      if (i > 0) sa -= l * (double)x[(e - lay.es) * NR + q];
      if (i < lay.n - 1) sc -= l * (double)x[(e + lay.es) * NR + q];
    }
  }
  if (!bcast) {
    if (live) {
      if (ga) ga[e] = (GT)sa;
      if (gb) gb[e] = (GT)sb;
      if (gc) gc[e] = (GT)sc;
    }
    return;
  }
  // broadcast coefficients: one gradient per row index i, summed over lines
  const unsigned full = 0xffffffffu;
  const long long i0 = __shfl_sync(full, (long long)i, 0);
  const bool same_row = __all_sync(full, !live || (long long)i == i0);
  if (same_row) {
    for (int off = 16; off > 0; off >>= 1) {
      sa += __shfl_xor_sync(full, sa, off);
      sb += __shfl_xor_sync(full, sb, off);
      sc += __shfl_xor_sync(full, sc, off);
    }
    if ((threadIdx.x & 31) == 0) {
      if (ga) atomicAdd(ga + i0, (GT)sa);
      if (gb) atomicAdd(gb + i0, (GT)sb);
      if (gc) atomicAdd(gc + i0, (GT)sc);
    }
  } else if (live) {
    if (ga) atomicAdd(ga + i, (GT)sa);
    if (gb) atomicAdd(gb + i, (GT)sb);
    if (gc) atomicAdd(gc + i, (GT)sc);
  }
}

template <class GT, class XT, int NR>
inline cudaError_t launch_epilogue(const Layout& lay, int bcast, const void* x, const void* lam, void* ga, void* gb,
                                   void* gc, cudaStream_t s) {
  const int64_t total = lay.n * lay.n_lines;
  if (total == 0) return cudaSuccess;
  const int line_fastest = lay.es != 1;  // adjacent threads on adjacent lines on strided axes
  const int64_t blocks = (total + 255) / 256;
  adjoint_epilogue<GT, XT, NR><<<(unsigned)blocks, 256, 0, s>>>(lay, bcast, line_fastest, (const XT*)x, (const XT*)lam,
                                                               (GT*)ga, (GT*)gb, (GT*)gc);
  return cudaGetLastError();
}

}  // namespace tdma
