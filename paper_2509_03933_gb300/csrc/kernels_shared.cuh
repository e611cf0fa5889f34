// Lines that share one set of coefficients (coef_broadcast without a per-line shift): the Thomas
// factorisation c'_i, 1 / w_i depends on the coefficients only, so it is computed once for all
// lines and every line runs just the right-hand-side recurrences:
//     d'_i = (d_i - a_i d'_{i-1}) / w_i,    x_i = d'_i - c'_i x_{i+1},
// three FP64 operations per unknown and right-hand side instead of nine (GB300's FP64 pipe bounds
// the Thomas sweep). In the paper's momentum solver all systems of a batch share one coefficient
// matrix, which depends on the grid spacing only (Section 6.2.1); here that matrix is factorised
// once per solve for all lines of the batch. With TR the factors are those of A^T (the adjoint).
//
// Two line kernels, one thread per line, both writing d' to x in the forward sweep and reading it
// back in the backward sweep:
//   stream: adjacent lines are adjacent in memory (a strided axis), so one warp's access to a row
//           is coalesced; rows are loaded kSharedAhead ahead of the recurrence in both sweeps.
//   staged: unit-stride lines (the contiguous axis). Each warp owns 32 lines and moves them
//           through shared memory in chunks of 16 elements per line: a half-warp copies one
//           line's chunk (coalesced 128-byte segments, cp.async, the next chunk in flight during
//           the recurrence over the current one), lane j runs the recurrence of line j.
#pragma once
#include "layout.cuh"
#include "kernels_dc.cuh"

namespace tdma {

constexpr int kSharedBlock = 128;
constexpr int kSharedAhead = 4;   // rows in flight per thread in the stream kernel
constexpr int kStageElems = 16;   // elements per line per chunk in the staged kernel (34 KB per
                                  // block: 6 blocks per SM; 32 elements held 3)
constexpr int kStagePitch = 17;   // odd pitch: lane j's row of the chunk falls in its own banks

template <class CT> struct alignas(2 * sizeof(CT)) Pair { CT sub, w; };

// Shared-coefficient workspace: n (sub-diagonal, 1 / w) pairs, then n values c'.
template <class CT> inline size_t shared_workspace_bytes(int64_t n) { return (size_t)3 * n * sizeof(CT); }

template <class CT> inline size_t shared_staged_smem() {
  return (size_t)(kSharedBlock / 32) * 2 * 32 * kStagePitch * sizeof(CT) + (size_t)kSharedBlock * sizeof(int64_t);
}

// Factors of the shared coefficients: the Thomas recurrence w_i = 1 / (b_i - sub_i c'_{i-1}),
// c'_i = sup_i w_i, with the results of the serial recurrence bit for bit (the arithmetic of the
// per-line Thomas kernel, backward stable where Thomas is). One FP64 operation depends on the
// previous one along the whole line, and a dependent FP64 operation of a single thread takes
// about 85 cycles on GB300 (one thread over a 512-row line: 148 us), so the chain is cut into
// 32 segments, one per lane of warp 0, over a chunk of coefficients staged in shared memory:
//   1. start values: c'_i is a linear fractional map of c'_{i-1}, i.e. with c' = N / D,
//      [N_i; D_i] = M_i [N_{i-1}; D_{i-1}], M_i = [[0, sup_i], [-sub_i, b_i]]; each lane forms
//      the product of its segment's matrices (rescaled by powers of two, which leaves N / D
//      unchanged), a scan over the warp composes them, and the composition applied to the
//      value entering the chunk estimates the value entering each segment;
//   2. every lane runs the serial recurrence over its segment from its start value;
//   3. each lane takes the end value of the lane before as its new start (lane 0 keeps the
//      exact one); while any start changed (bit for bit), repeat 2.
// At the fixed point every segment starts from the exact serial value, so every value is the
// serial recurrence's; after pass t at least lanes 0..t are final, so at most 32 passes run, and
// on diagonally dominant lines the estimate's error dies out within a segment, so two or three
// passes suffice.
constexpr int kFactorThreads = 256;
constexpr int kFactorChunk = 2016;  // 3 arrays of 2016 doubles + the carry: under 48 KB static

template <class CT> struct M2 { CT a, b, c, d; };  // [[a, b], [c, d]]

template <class CT> TDMA_DEV M2<CT> mul2(const M2<CT>& x, const M2<CT>& y) {  // x y
  return M2<CT>{fma(x.a, y.a, x.b * y.c), fma(x.a, y.b, x.b * y.d), fma(x.c, y.a, x.d * y.c),
                fma(x.c, y.b, x.d * y.d)};
}
template <class CT> TDMA_DEV M2<CT> shfl_up2(const M2<CT>& x, int dl) {
  return M2<CT>{__shfl_up_sync(0xffffffffu, x.a, dl), __shfl_up_sync(0xffffffffu, x.b, dl),
                __shfl_up_sync(0xffffffffu, x.c, dl), __shfl_up_sync(0xffffffffu, x.d, dl)};
}
// Multiply by the power of two that brings the largest entry into [1, 2) (exact).
template <class CT> TDMA_DEV void rescale(M2<CT>& x) {
  const CT m = fmax(fmax(fabs(x.a), fabs(x.b)), fmax(fabs(x.c), fabs(x.d)));
  if (m > CT(0) && isfinite(m)) {
    const int k = ilogb(m);
    x.a = scalbn(x.a, -k); x.b = scalbn(x.b, -k); x.c = scalbn(x.c, -k); x.d = scalbn(x.d, -k);
  }
}
TDMA_DEV uint64_t value_bits(double v) { return (uint64_t)__double_as_longlong(v); }
TDMA_DEV uint64_t value_bits(float v) { return (uint64_t)__float_as_uint(v); }

template <class CT, bool TR>
__global__ void __launch_bounds__(kFactorThreads) shared_factor_kernel(const Args A, Pair<CT>* __restrict__ sw,
                                                                       CT* __restrict__ cp) {
  __shared__ CT s_sub[kFactorChunk], s_b[kFactorChunk], s_sup[kFactorChunk];
  __shared__ CT s_carry;
  const int64_t n = A.lay.n;
  const CT* pa = (const CT*)A.a;
  const CT* pb = (const CT*)A.b;
  const CT* pc = (const CT*)A.c;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) s_carry = CT(0);
  bool ok = true;
  for (int64_t i0 = 0; i0 < n; i0 += kFactorChunk) {
    const int rows = n - i0 < kFactorChunk ? (int)(n - i0) : kFactorChunk;
    for (int r = threadIdx.x; r < rows; r += kFactorThreads) {
      const int64_t i = i0 + r;
      s_sub[r] = i == 0 ? CT(0) : (TR ? ldg(pc + i - 1) : ldg(pa + i));
      s_sup[r] = i == n - 1 ? CT(0) : (TR ? ldg(pa + i + 1) : ldg(pc + i));
      s_b[r] = ldg(pb + i);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int seg = (rows + 31) / 32;
      const int r0 = lane * seg < rows ? lane * seg : rows;
      const int r1 = r0 + seg < rows ? r0 + seg : rows;
      // 1. estimates of the values entering the segments
      M2<CT> P{CT(1), CT(0), CT(0), CT(1)};
      for (int r = r0; r < r1; ++r) {
        M2<CT> Mi{CT(0), s_sup[r], -s_sub[r], s_b[r]};
        rescale(Mi);
        P = mul2(Mi, P);
        if (((r - r0) & 7) == 7) rescale(P);
      }
      rescale(P);
      for (int dl = 1; dl < 32; dl <<= 1) {  // inclusive scan, later segments on the left
        const M2<CT> o = shfl_up2(P, dl);
        if (lane >= dl) {
          P = mul2(P, o);
          rescale(P);
        }
      }
      const M2<CT> E = shfl_up2(P, 1);
      const CT carry = s_carry;
      CT start = carry;
      if (lane > 0) start = fma(E.a, carry, E.b) / fma(E.c, carry, E.d);
      // 2./3. serial passes until the start values stop changing
      CT end = start;
      bool lane_ok = true;
      for (int pass = 0; pass < 33; ++pass) {
        CT c_prev = start;
        lane_ok = true;
#pragma unroll 4
        for (int r = r0; r < r1; ++r) {
          const CT sub = s_sub[r];
          const CT w = rcp(s_b[r] - sub * c_prev);
          lane_ok &= finite(w);
          c_prev = s_sup[r] * w;
          sw[i0 + r] = Pair<CT>{sub, w};
          cp[i0 + r] = c_prev;
        }
        end = r1 > r0 ? c_prev : start;  // an empty segment passes its start on
        CT next = __shfl_up_sync(0xffffffffu, end, 1);
        if (lane == 0) next = carry;
        const bool changed = r1 > r0 && value_bits(next) != value_bits(start);
        start = next;
        if (!__any_sync(0xffffffffu, changed)) break;
      }
      ok &= lane_ok;
      __syncwarp();
      if (r1 == rows && r0 < r1) s_carry = end;  // the value leaving the chunk
    }
    __syncthreads();
  }
  if (!ok) report_error(A.st, 5);
}

template <class CT, int NR> struct Vals { CT v[NR]; };

template <class CT, int NR, bool NC>
TDMA_DEV void load_vals(Vals<CT, NR>& r, const CT* p) {
  if constexpr (NR == 1) {
    r.v[0] = NC ? ldg(p) : *p;
  } else if constexpr (sizeof(CT) == 8) {
    const double2 t = NC ? __ldg((const double2*)p) : *(const double2*)p;
    r.v[0] = t.x; r.v[1] = t.y;
  } else {
    const float2 t = NC ? __ldg((const float2*)p) : *(const float2*)p;
    r.v[0] = t.x; r.v[1] = t.y;
  }
}

template <class CT, int NR>
TDMA_DEV void store_vals(CT* p, const CT* v) {
  if constexpr (NR == 1) {
    *p = v[0];
  } else if constexpr (sizeof(CT) == 8) {
    *(double2*)p = make_double2(v[0], v[1]);
  } else {
    *(float2*)p = make_float2(v[0], v[1]);
  }
}

// Strided axis: one thread per line, rows kSharedAhead ahead in both sweeps. The right-hand side
// is read once through the read-only path (row i is read before x's row i is written, so x may
// be d); d' is read back with plain loads (this thread wrote it).
template <class CT, int NR>
__global__ void __launch_bounds__(kSharedBlock) shared_stream_kernel(const Args A, const Pair<CT>* __restrict__ sw,
                                                                     const CT* __restrict__ cp) {
  constexpr int K = kSharedAhead;
  const int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= A.lay.n_lines) return;
  const int64_t n = A.lay.n, es = A.lay.es, base = A.lay.off(line);
  const CT* D = (const CT*)A.d + base * NR;
  CT* X = (CT*)A.x + base * NR;
  const int64_t step = es * NR;
  Vals<CT, NR> buf[K];
#pragma unroll
  for (int u = 0; u < K; ++u)
    if (u < n) load_vals<CT, NR, true>(buf[u], D + u * step);
  CT dp[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) dp[q] = CT(0);
  for (int64_t i0 = 0; i0 < n; i0 += K) {
    Vals<CT, NR> nxt[K];
#pragma unroll
    for (int u = 0; u < K; ++u)
      if (i0 + K + u < n) load_vals<CT, NR, true>(nxt[u], D + (i0 + K + u) * step);
#pragma unroll
    for (int u = 0; u < K; ++u) {
      const int64_t i = i0 + u;
      if (i < n) {
        const Pair<CT> f = sw[i];
#pragma unroll
        for (int q = 0; q < NR; ++q) dp[q] = (buf[u].v[q] - f.sub * dp[q]) * f.w;
        store_vals<CT, NR>(X + i * step, dp);
      }
    }
#pragma unroll
    for (int u = 0; u < K; ++u) buf[u] = nxt[u];
  }
  // backward: x_{n-1} = d'_{n-1} (in dp); rows n-2 .. 0
  CT xn[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) xn[q] = dp[q];
#pragma unroll
  for (int u = 0; u < K; ++u)
    if (n - 2 - u >= 0) load_vals<CT, NR, false>(buf[u], X + (n - 2 - u) * step);
  for (int64_t i0 = n - 2; i0 >= 0; i0 -= K) {
    Vals<CT, NR> nxt[K];
#pragma unroll
    for (int u = 0; u < K; ++u)
      if (i0 - K - u >= 0) load_vals<CT, NR, false>(nxt[u], X + (i0 - K - u) * step);
#pragma unroll
    for (int u = 0; u < K; ++u) {
      const int64_t i = i0 - u;
      if (i >= 0) {
        const CT c = cp[i];
#pragma unroll
        for (int q = 0; q < NR; ++q) xn[q] = buf[u].v[q] - c * xn[q];
        store_vals<CT, NR>(X + i * step, xn);
      }
    }
#pragma unroll
    for (int u = 0; u < K; ++u) buf[u] = nxt[u];
  }
  bool ok = true;
#pragma unroll
  for (int q = 0; q < NR; ++q) ok &= finite(xn[q]);
  if (!ok) report_error(A.st, 5);
}

TDMA_DEV void stage_copy(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
TDMA_DEV void stage_copy(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
TDMA_DEV void stage_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> TDMA_DEV void stage_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Unit-stride lines: see the file comment. Chunk c of a line is its elements
// [c * kStageElems, (c + 1) * kStageElems) of the n * NR interleaved values; lane k copies element
// k mod E of the chunk of lines k / E, k / E + 32 / E, ... of its warp, so the same lane writes a
// value of x in the forward sweep and reads it back in the backward sweep.
template <class CT, int NR>
__global__ void __launch_bounds__(kSharedBlock) shared_staged_kernel(const Args A, const Pair<CT>* __restrict__ sw,
                                                                     const CT* __restrict__ cp) {
  constexpr int E = kStageElems, R = E / NR, PT = kStagePitch;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  CT* tile = (CT*)smem_raw + (size_t)warp * 2 * 32 * PT;  // [2 buffers][32 lines][PT]
  int64_t* s_off = (int64_t*)((CT*)smem_raw + (size_t)(kSharedBlock / 32) * 2 * 32 * PT) + warp * 32;
  const int64_t line0 = (int64_t)blockIdx.x * kSharedBlock + warp * 32;
  const int64_t L = A.lay.n_lines, n = A.lay.n;
  if (line0 >= L) return;
  const int lines = L - line0 < 32 ? (int)(L - line0) : 32;
  s_off[lane] = lane < lines ? A.lay.off(line0 + lane) * NR : 0;
  __syncwarp();
  const int64_t total = n * NR;
  const int nc = (int)((total + E - 1) / E);
  const CT* D = (const CT*)A.d;
  CT* X = (CT*)A.x;
  constexpr int LPI = 32 / E;  // lines per copy instruction
  const int e = lane % E, sub = lane / E;
  auto issue = [&](const CT* src, int c, int b) {
    const int64_t k = (int64_t)c * E + e;
    if (k < total) {
      CT* t = tile + (size_t)b * 32 * PT + e;
      for (int j = sub; j < lines; j += LPI) stage_copy(t + j * PT, src + s_off[j] + k);
    }
    stage_commit();
  };
  auto drain = [&](int c, int b) {
    const int64_t k = (int64_t)c * E + e;
    if (k < total) {
      const CT* t = tile + (size_t)b * 32 * PT + e;
      for (int j = sub; j < lines; j += LPI) X[s_off[j] + k] = t[j * PT];
    }
  };
  const bool mine = lane < lines;
  CT dp[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) dp[q] = CT(0);
  // forward sweep, chunks 0 .. nc-1
  issue(D, 0, 0);
  for (int c = 0; c < nc; ++c) {
    const int b = c & 1;
    if (c + 1 < nc) { issue(D, c + 1, b ^ 1); stage_wait<1>(); } else { stage_wait<0>(); }
    __syncwarp();
    if (mine) {
      CT* t = tile + (size_t)b * 32 * PT + lane * PT;
      const int64_t r0 = (int64_t)c * R;
      const int rows = n - r0 < R ? (int)(n - r0) : R;
      for (int r = 0; r < rows; ++r) {
        const Pair<CT> f = sw[r0 + r];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          dp[q] = (t[r * NR + q] - f.sub * dp[q]) * f.w;
          t[r * NR + q] = dp[q];
        }
      }
    }
    __syncwarp();
    drain(c, b);
    __syncwarp();
  }
  // backward sweep, chunks nc-1 .. 0; x_{n-1} = d'_{n-1} is already in place
  CT xn[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) xn[q] = dp[q];
  issue(X, nc - 1, 0);
  for (int c = nc - 1, s = 0; c >= 0; --c, ++s) {
    const int b = s & 1;
    if (c > 0) { issue(X, c - 1, b ^ 1); stage_wait<1>(); } else { stage_wait<0>(); }
    __syncwarp();
    if (mine) {
      CT* t = tile + (size_t)b * 32 * PT + lane * PT;
      const int64_t r0 = (int64_t)c * R;
      const int rows = n - r0 < R ? (int)(n - r0) : R;
      for (int r = rows - 1; r >= 0; --r) {
        const int64_t i = r0 + r;
        if (i == n - 1) continue;
        const CT cc = cp[i];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          xn[q] = t[r * NR + q] - cc * xn[q];
          t[r * NR + q] = xn[q];
        }
      }
    }
    __syncwarp();
    drain(c, b);
    __syncwarp();
  }
  bool ok = true;
#pragma unroll
  for (int q = 0; q < NR; ++q) ok &= finite(xn[q]);
  if (mine && !ok) report_error(A.st, 5);
}

template <class CT, int NR>
inline cudaError_t prepare_shared_kernels() {
  return cudaFuncSetAttribute(shared_staged_kernel<CT, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)shared_staged_smem<CT>());
}

inline cudaError_t prepare_shared(tdma_precision_t p, int nrhs) {
  if (p == TDMA_F64) return nrhs == 1 ? prepare_shared_kernels<double, 1>() : prepare_shared_kernels<double, 2>();
  return nrhs == 1 ? prepare_shared_kernels<float, 1>() : prepare_shared_kernels<float, 2>();
}

template <class CT, int NR, bool TR>
inline cudaError_t launch_shared(const Args& A, cudaStream_t s) {
  Pair<CT>* sw = (Pair<CT>*)A.ws;
  CT* cp = (CT*)(sw + A.lay.n);
  shared_factor_kernel<CT, TR><<<1, kFactorThreads, 0, s>>>(A, sw, cp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((A.lay.n_lines + kSharedBlock - 1) / kSharedBlock);
  if (A.lay.es == 1)
    shared_staged_kernel<CT, NR><<<blocks, kSharedBlock, shared_staged_smem<CT>(), s>>>(A, sw, cp);
  else
    shared_stream_kernel<CT, NR><<<blocks, kSharedBlock, 0, s>>>(A, sw, cp);
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
