// One partition per line (the Thomas sweep) on unit-stride lines, through shared memory.
//
// With the lines along the contiguous axis, one thread per line reads rows that are a line apart
// across the warp (no coalescing). Here each warp owns 32 lines and moves them through shared
// memory in chunks of kTsRows rows: a quarter-warp (a half-warp for two interleaved right-hand
// sides) copies one line's chunk of an array with cp.async (coalesced segments), the next chunk in
// flight while lane j sweeps line j over the current one. Chunks of 8 rows keep the tiles small
// enough for 12 warps per SM (1024^3 FP64 along x: 21.2 ms; 16 rows: 26.4 ms; 4 rows: 26.8 ms). The forward sweep leaves c' in the
// workspace ([line][row]) and d' in x; the backward sweep reads both back the same way. The
// arithmetic is that of the strided Thomas kernel (8 FP64-pipe operations per unknown).
#pragma once
#include "layout.cuh"

namespace tdma {

constexpr int kTsWarps = 2;   // warps per block
constexpr int kTsRows = 8;    // rows per chunk
constexpr int kTsPitchC = kTsRows + 1;  // odd pitches: lane j's row of a tile in its own banks

template <int NR> __host__ __device__ constexpr int ts_pitch_d() { return kTsRows * NR + 1; }

// Per warp: two buffers of the a, b, c tiles [32][kTsPitchC] and the d tile [32][pitch_d], then
// the warps' 32 line offsets.
template <class CT, int NR> __host__ __device__ constexpr size_t ts_buffer_elems() {
  return (size_t)3 * 32 * kTsPitchC + (size_t)32 * ts_pitch_d<NR>();
}
template <class CT, int NR> inline size_t thomas_staged_smem() {
  return (size_t)kTsWarps * (2 * ts_buffer_elems<CT, NR>() * sizeof(CT) + 32 * sizeof(int64_t));
}

TDMA_DEV void ts_copy(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
TDMA_DEV void ts_copy(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
TDMA_DEV void ts_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> TDMA_DEV void ts_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Copies of one chunk between global memory and a tile: V values per line per chunk (V = 16 or
// 32), value k of line j at src + base_j + first + k (first + k < limit), lane l on value l mod V
// of lines l / V, l / V + 32 / V, ...
template <class CT, int V, bool TO_SMEM>
TDMA_DEV void ts_move(CT* tile, int pitch, CT* g, const int64_t* base, int64_t mult, int lines, int64_t first,
                      int64_t limit, int lane) {
  constexpr int LPI = 32 / V;
  const int e = lane % V, sub = lane / V;
  const int64_t k = first + e;
  if (k >= limit) return;
  for (int j = sub; j < lines; j += LPI) {
    CT* t = tile + j * pitch + e;
    CT* p = g + base[j] * mult + k;
    if (TO_SMEM) ts_copy(t, p);
    else *p = *t;
  }
}

template <class CT, int NR>
__global__ void __launch_bounds__(kTsWarps * 32) thomas_staged_kernel(const Args A, CT* __restrict__ ws) {
  constexpr int R = kTsRows, PC = kTsPitchC, PD = ts_pitch_d<NR>(), VD = R * NR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  CT* tiles = (CT*)smem_raw + (size_t)warp * 2 * ts_buffer_elems<CT, NR>();
  int64_t* s_off = (int64_t*)((CT*)smem_raw + (size_t)kTsWarps * 2 * ts_buffer_elems<CT, NR>()) + warp * 32;
  const int64_t line0 = ((int64_t)blockIdx.x * kTsWarps + warp) * 32;
  const int64_t L = A.lay.n_lines, n = A.lay.n;
  if (line0 >= L) return;
  const int lines = L - line0 < 32 ? (int)(L - line0) : 32;
  s_off[lane] = lane < lines ? A.lay.off(line0 + lane) : 0;
  __syncwarp();
  // workspace rows of this warp's lines: line * n + row
  CT* W = ws + line0 * n;
  auto tile = [&](int b, int arr) -> CT* {  // arr 0..2: a, b, c; 3: d
    CT* t = tiles + (size_t)b * ts_buffer_elems<CT, NR>();
    return arr < 3 ? t + (size_t)arr * 32 * PC : t + (size_t)3 * 32 * PC;
  };
  const int nc = (int)((n + R - 1) / R);
  const CT* Ca = (const CT*)A.a;
  const CT* Cb = (const CT*)A.b;
  const CT* Cc = (const CT*)A.c;
  const CT* D = (const CT*)A.d;
  CT* X = (CT*)A.x;
  // offsets of the workspace lines relative to W, in the same form as s_off (line index * n)
  __shared__ int64_t s_wl[kTsWarps][32];
  s_wl[warp][lane] = (int64_t)lane * n;
  __syncwarp();
  auto issue_fwd = [&](int c, int b) {
    const int64_t r0 = (int64_t)c * R;
    ts_move<CT, R, true>(tile(b, 0), PC, const_cast<CT*>(Ca), s_off, 1, lines, r0, n, lane);
    ts_move<CT, R, true>(tile(b, 1), PC, const_cast<CT*>(Cb), s_off, 1, lines, r0, n, lane);
    ts_move<CT, R, true>(tile(b, 2), PC, const_cast<CT*>(Cc), s_off, 1, lines, r0, n, lane);
    ts_move<CT, VD, true>(tile(b, 3), PD, const_cast<CT*>(D), s_off, NR, lines, r0 * NR, n * NR, lane);
    ts_commit();
  };
  const bool mine = lane < lines;
  CT cp = CT(0), dp[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) dp[q] = CT(0);
  bool ok = true;
  // forward sweep: c' into the c tile, d' into the d tile, then out to the workspace and x
  issue_fwd(0, 0);
  for (int c = 0; c < nc; ++c) {
    const int b = c & 1;
    if (c + 1 < nc) { issue_fwd(c + 1, b ^ 1); ts_wait<1>(); } else { ts_wait<0>(); }
    __syncwarp();
    if (mine) {
      const CT* ta = tile(b, 0) + lane * PC;
      const CT* tb = tile(b, 1) + lane * PC;
      CT* tc = tile(b, 2) + lane * PC;
      CT* td = tile(b, 3) + lane * PD;
      const int64_t r0 = (int64_t)c * R;
      const int rows = n - r0 < R ? (int)(n - r0) : R;
      for (int r = 0; r < rows; ++r) {
        const int64_t i = r0 + r;
        const CT a = i == 0 ? CT(0) : ta[r];
        const CT cc = i == n - 1 ? CT(0) : tc[r];
        const CT w = rcp(tb[r] - a * cp);
        ok &= finite(w);
        cp = cc * w;
        tc[r] = cp;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          dp[q] = (td[r * NR + q] - a * dp[q]) * w;
          td[r * NR + q] = dp[q];
        }
      }
    }
    __syncwarp();
    const int64_t r0 = (int64_t)c * R;
    ts_move<CT, R, false>(tile(b, 2), PC, W, s_wl[warp], 1, lines, r0, n, lane);
    ts_move<CT, VD, false>(tile(b, 3), PD, X, s_off, NR, lines, r0 * NR, n * NR, lane);
    __syncwarp();
  }
  // backward sweep, chunks nc-1 .. 0: x_i = d'_i - c'_i x_{i+1}; x_{n-1} = d'_{n-1} is in place
  auto issue_bwd = [&](int c, int b) {
    const int64_t r0 = (int64_t)c * R;
    ts_move<CT, R, true>(tile(b, 2), PC, W, s_wl[warp], 1, lines, r0, n, lane);
    ts_move<CT, VD, true>(tile(b, 3), PD, X, s_off, NR, lines, r0 * NR, n * NR, lane);
    ts_commit();
  };
  CT xn[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) xn[q] = dp[q];
  issue_bwd(nc - 1, 0);
  for (int c = nc - 1, s = 0; c >= 0; --c, ++s) {
    const int b = s & 1;
    if (c > 0) { issue_bwd(c - 1, b ^ 1); ts_wait<1>(); } else { ts_wait<0>(); }
    __syncwarp();
    if (mine) {
      const CT* tc = tile(b, 2) + lane * PC;
      CT* td = tile(b, 3) + lane * PD;
      const int64_t r0 = (int64_t)c * R;
      const int rows = n - r0 < R ? (int)(n - r0) : R;
      for (int r = rows - 1; r >= 0; --r) {
        if (r0 + r == n - 1) continue;
        const CT cc = tc[r];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          xn[q] = td[r * NR + q] - cc * xn[q];
          td[r * NR + q] = xn[q];
        }
      }
    }
    __syncwarp();
    const int64_t r0 = (int64_t)c * R;
    ts_move<CT, VD, false>(tile(b, 3), PD, X, s_off, NR, lines, r0 * NR, n * NR, lane);
    __syncwarp();
  }
#pragma unroll
  for (int q = 0; q < NR; ++q) ok &= finite(xn[q]);
  if (mine && !ok) report_error(A.st, 5);
}

template <class CT, int NR> inline cudaError_t prepare_thomas_staged_one() {
  return cudaFuncSetAttribute(thomas_staged_kernel<CT, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)thomas_staged_smem<CT, NR>());
}
inline cudaError_t prepare_thomas_staged(tdma_precision_t p, int nrhs) {
  if (p == TDMA_F64) return nrhs == 1 ? prepare_thomas_staged_one<double, 1>() : prepare_thomas_staged_one<double, 2>();
  return nrhs == 1 ? prepare_thomas_staged_one<float, 1>() : prepare_thomas_staged_one<float, 2>();
}

inline cudaError_t launch_thomas_staged(tdma_precision_t p, int nrhs, const Args& A, cudaStream_t s) {
  const unsigned blocks = (unsigned)((A.lay.n_lines + kTsWarps * 32 - 1) / (kTsWarps * 32));
  const unsigned T = kTsWarps * 32;
  if (p == TDMA_F64) {
    if (nrhs == 1) thomas_staged_kernel<double, 1><<<blocks, T, thomas_staged_smem<double, 1>(), s>>>(A, (double*)A.ws);
    else thomas_staged_kernel<double, 2><<<blocks, T, thomas_staged_smem<double, 2>(), s>>>(A, (double*)A.ws);
  } else {
    if (nrhs == 1) thomas_staged_kernel<float, 1><<<blocks, T, thomas_staged_smem<float, 1>(), s>>>(A, (float*)A.ws);
    else thomas_staged_kernel<float, 2><<<blocks, T, thomas_staged_smem<float, 2>(), s>>>(A, (float*)A.ws);
  }
  return cudaGetLastError();
}

}  // namespace tdma
