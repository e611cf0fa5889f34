// One partition per line (P = 1): the Thomas sweep, one thread per line, elimination factors
// kept in the workspace.
//
// The Thomas algorithm (Section 1; the paper's Stage A with p = 1) needs fewer operations per
// unknown than the partitioned sweep: w = b_i - a_i c'_{i-1}, c'_i = c_i / w,
// d'_i = (d_i - a_i d'_{i-1}) / w, then x_i = d'_i - c'_i x_{i+1}. On GB300 the FP64 pipe bounds
// the FP64 solve, so when a batch has enough lines to fill the GPU with one thread per line
// this is the fastest FP64 form (8 FP64-pipe operations per unknown against about 14). The
// forward sweep stores c' in the workspace (row-major [row][line], coalesced across adjacent
// lines) and d' in x; the backward sweep reads both back in reverse order.
#pragma once
#include "tdma.h"
#include "layout.cuh"
#include "kernels_dc.cuh"

namespace tdma {

constexpr int kThomasBlock = 128;
constexpr int kThomasAhead = 2;  // rows loaded ahead of the forward sweep (4 cost occupancy: 27.7 -> 23.4 ms)

template <class CT, int NR, bool TR = false>
__global__ void __launch_bounds__(kThomasBlock) thomas_kernel(const Args A, CT* __restrict__ cws) {
  const int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= A.lay.n_lines) return;
  const int64_t n = A.lay.n, es = A.lay.es, L = A.lay.n_lines;
  const int64_t base = A.lay.off(line);
  const CT shift = A.shift ? ldg((const CT*)A.shift + line) : CT(0);
  CT* cw = cws + line;  // c'_i at cw[i * L]

  Row<CT, NR> buf[kThomasAhead];
#pragma unroll
  for (int u = 0; u < kThomasAhead; ++u)
    if (u < n) load_row<CT, NR, TR>(buf[u], A, base + u * es, u, shift);
  CT cp = CT(0), dp[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) dp[q] = CT(0);
  bool ok = true;
  for (int64_t i0 = 0; i0 < n; i0 += kThomasAhead) {
    Row<CT, NR> nxt[kThomasAhead];
#pragma unroll
    for (int u = 0; u < kThomasAhead; ++u) {
      const int64_t i = i0 + kThomasAhead + u;
      if (i < n) load_row<CT, NR, TR>(nxt[u], A, base + i * es, i, shift);
    }
#pragma unroll
    for (int u = 0; u < kThomasAhead; ++u) {
      const int64_t i = i0 + u;
      if (i < n) {
        Row<CT, NR>& rw = buf[u];
        const CT a = (i == 0) ? CT(0) : rw.a;
        const CT cc = (i == n - 1) ? CT(0) : rw.c;
        const CT r = rcp(rw.b - a * cp);
        ok &= finite(r);
        cp = cc * r;
        CT v[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) v[q] = dp[q] = (rw.d[q] - a * dp[q]) * r;
        cw[i * L] = cp;
        store_x<CT, NR>(A, base + i * es, v);
      }
    }
#pragma unroll
    for (int u = 0; u < kThomasAhead; ++u) buf[u] = nxt[u];
  }
  // backward: x_i = d'_i - c'_i x_{i+1}; dp holds x_{n-1} = d'_{n-1}
  CT xn[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) xn[q] = dp[q];
  for (int64_t i0 = n - 2; i0 >= 0; i0 -= kThomasAhead) {
    CT cpv[kThomasAhead];
    Row<CT, NR> dv[kThomasAhead];
#pragma unroll
    for (int u = 0; u < kThomasAhead; ++u) {
      const int64_t i = i0 - u;
      if (i >= 0) {
        cpv[u] = cw[i * L];
        const int64_t e = base + i * es;
        if constexpr (NR == 1) {
          dv[u].d[0] = ((const CT*)A.x)[e];
        } else if constexpr (sizeof(CT) == 8) {
          const double2 t = ((const double2*)A.x)[e];
          dv[u].d[0] = t.x; dv[u].d[1] = t.y;
        } else {
          const float2 t = ((const float2*)A.x)[e];
          dv[u].d[0] = t.x; dv[u].d[1] = t.y;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kThomasAhead; ++u) {
      const int64_t i = i0 - u;
      if (i >= 0) {
#pragma unroll
        for (int q = 0; q < NR; ++q) xn[q] = dv[u].d[q] - cpv[u] * xn[q];
        store_x<CT, NR>(A, base + i * es, xn);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NR; ++q) ok &= finite(xn[q]);
  if (!ok) report_error(A.st, 5);
}

// The Thomas form is used when P = 1 is requested (or chosen) and the batch has lines to
// fill the GPU; its workspace is one coefficient per unknown.
inline bool use_thomas_variant(const tdma_desc_t& d) { return d.n > 1 && d.precision != TDMA_F32_REFINE; }

inline void thomas_config(const tdma_desc_t& d, tdma_config_t& c) {
  c = tdma_config_t{};
  c.partitions = 1;
  c.rows_per_thread = (int32_t)d.n;
  c.lines_per_block = kThomasBlock;
  c.threads_per_block = kThomasBlock;
  c.blocks = (int32_t)((d.n_lines + kThomasBlock - 1) / kThomasBlock);
  c.smem_bytes = 0;
  c.variant = TDMA_VARIANT_THOMAS;
}

inline size_t thomas_workspace(const tdma_desc_t& d) {
  return (size_t)d.n * (size_t)d.n_lines * (d.precision == TDMA_F64 ? 8 : 4);
}

inline cudaError_t launch_thomas(tdma_precision_t p, int nrhs, const Args& A, const tdma_config_t& c,
                                 cudaStream_t s) {
  const dim3 grid(c.blocks), block(c.threads_per_block);
  if (p == TDMA_F64) {
    if (nrhs == 1) thomas_kernel<double, 1><<<grid, block, 0, s>>>(A, (double*)A.ws);
    else thomas_kernel<double, 2><<<grid, block, 0, s>>>(A, (double*)A.ws);
  } else {
    if (nrhs == 1) thomas_kernel<float, 1><<<grid, block, 0, s>>>(A, (float*)A.ws);
    else thomas_kernel<float, 2><<<grid, block, 0, s>>>(A, (float*)A.ws);
  }
  return cudaGetLastError();
}
inline cudaError_t prepare_thomas(tdma_precision_t, int, size_t) { return cudaSuccess; }

}  // namespace tdma
