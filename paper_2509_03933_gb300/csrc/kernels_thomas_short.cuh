// One partition per line (P = 1) for short lines in small batches: the Thomas sweep (Section 1)
// with the whole line staged in shared memory first.
//
// A batch of a few thousand short lines gives the GPU one thread per line and a few warps per
// SM; a sweep that reads its rows as it goes then waits a memory latency per row. Here one warp
// takes 32 lines whose elements of a row are adjacent in memory (a strided solve axis, lines along
// the unit-stride axis of the rest of the grid), and every thread issues asynchronous copies of all
// n rows of its line (a, b, c, d) into its own column of a [row][lane] shared-memory tile before it
// sweeps: the latency is paid once. The forward sweep keeps c' over c and d' over d in the tile, the
// backward sweep writes x, row by row, coalesced across the warp. Each thread reads and writes its
// own column only, so the warp needs no barrier; x may alias d (all of d is in the tile before any
// x is written). Same arithmetic as thomas_kernel (8 FP64-pipe operations per unknown in FP64).
#pragma once
#include "tdma.h"
#include "layout.cuh"
#include "kernels_dc.cuh"

namespace tdma {

constexpr int kShortMaxN = 128;           // longest line staged (FP64, two right-hand sides: 160 KB)
constexpr int64_t kShortMaxLines = 16384;  // larger batches fill the GPU with thomas_kernel

template <int B> TDMA_DEV void cp_async_bytes(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src),
               "n"(B)
               : "memory");
}

template <class CT, int NR>
__global__ void __launch_bounds__(32) thomas_short_kernel(const Args A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = (int)A.lay.n, lane = threadIdx.x;
  const int64_t line = (int64_t)blockIdx.x * 32 + lane;
  if (line >= A.lay.n_lines) return;
  const int64_t es = A.lay.es, base = A.lay.off(line);
  CT* sa = reinterpret_cast<CT*>(smem_raw) + lane;  // row i of this line at [i * 32]
  CT* sb = sa + n * 32;
  CT* sc = sb + n * 32;
  CT* sd = reinterpret_cast<CT*>(smem_raw) + 3 * n * 32 + lane * NR;  // row i at [i * 32 * NR]
  for (int i = 0; i < n; ++i) {
    const int64_t e = base + i * es;
    cp_async_bytes<sizeof(CT)>(sa + i * 32, (const CT*)A.a + e);
    cp_async_bytes<sizeof(CT)>(sb + i * 32, (const CT*)A.b + e);
    cp_async_bytes<sizeof(CT)>(sc + i * 32, (const CT*)A.c + e);
    cp_async_bytes<sizeof(CT) * NR>(sd + i * 32 * NR, (const CT*)A.d + e * NR);
  }
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
  const CT shift = A.shift ? ldg((const CT*)A.shift + line) : CT(0);
  CT cp = CT(0), dp[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) dp[q] = CT(0);
  bool ok = true;
  for (int i = 0; i < n; ++i) {
    const CT a = i == 0 ? CT(0) : sa[i * 32];
    const CT c = i == n - 1 ? CT(0) : sc[i * 32];
    const CT r = rcp(sb[i * 32] + shift - a * cp);
    ok &= finite(r);
    cp = c * r;
    sc[i * 32] = cp;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      dp[q] = (sd[i * 32 * NR + q] - a * dp[q]) * r;
      sd[i * 32 * NR + q] = dp[q];
    }
  }
  // backward: x_i = d'_i - c'_i x_{i+1}; dp holds x_{n-1} = d'_{n-1}
  store_x<CT, NR>(A, base + (int64_t)(n - 1) * es, dp);
  for (int i = n - 2; i >= 0; --i) {
    const CT cpi = sc[i * 32];
#pragma unroll
    for (int q = 0; q < NR; ++q) dp[q] = sd[i * 32 * NR + q] - cpi * dp[q];
    store_x<CT, NR>(A, base + i * es, dp);
  }
#pragma unroll
  for (int q = 0; q < NR; ++q) ok &= finite(dp[q]);
  if (!ok) report_error(A.st, 5);
}

// Shared memory of one warp's tile.
inline size_t thomas_short_smem(int64_t n, int nrhs, size_t elem) { return (size_t)n * 32 * (3 + nrhs) * elem; }

// Does a P = 1 solve of this layout take the staged form? Short lines, adjacent lines (a row of
// 32 lines is one contiguous run), per-line coefficient arrays, a batch too small to fill the GPU
// with one thread per line.
inline bool thomas_short_ok(const tdma_desc_t& d) {
  return d.n >= 1 && d.n <= kShortMaxN && d.n_lines >= 1 && d.n_lines <= kShortMaxLines && d.inner_stride == 1 &&
         d.elem_stride != 1 && !d.coef_broadcast;
}

}  // namespace tdma
