// FP32 storage + refinement, block tile staged by TMA, reduced system solved in two levels.
//
// One block owns Lb adjacent lines; each line has P uniform partitions of m rows (thread
// tid = j + Lb k owns partition k of line j). Four TMA tensor copies bring the whole tile of
// a, b, c (float) and d (double) into shared memory in one go: the 4D box
// {Lb lines, 1, P partitions, m rows} lands as element (row t, partition k, line j) at
// t * T + tid, so every thread reads its rows conflict-free. All refinement passes then read
// shared memory: HBM sees one read of the inputs and, through a TMA store, one write of x.
//
// Per pass: Stage A (float modified-Thomas sweep of the partition, factors kept in registers
// after the first pass), Stage B (the 2P-row reduced system, see reduced_two_level), Stage C
// (interior update) and the refinement bookkeeping of kernels_refine_reg.cuh.
//
// Stage B in two levels (the same partition-and-reduce step applied to the reduced system
// itself): the 2P rows of a line are cut into G groups of S rows, thread (j, g) reduces its
// group to two endpoint rows with the modified-Thomas sweep, one thread per line solves the
// resulting 2G-row system, and the groups fill in their interiors. Latency drops from 2P
// dependent rows to about S + 2G; the level factors are kept for later passes.
#pragma once
#include "layout.cuh"
#include "tma.cuh"
#include "kernels_refine.cuh"

namespace tdma {

// shared-memory layout of one line's reduced system (floats)
struct RedLayout {
  int R2, G, S, pitch;
  __host__ __device__ RedLayout(int P, int G_) : R2(2 * P), G(G_), S(2 * P / G_), pitch(0) {
    pitch = 5 * R2 + 2 * G + 8 * G + 1;
  }
  // offsets inside a line block
  __host__ __device__ int sub() const { return 0; }
  __host__ __device__ int sup() const { return R2; }
  __host__ __device__ int rhs() const { return 2 * R2; }
  __host__ __device__ int l1al() const { return 3 * R2; }
  __host__ __device__ int l1ga() const { return 4 * R2; }
  __host__ __device__ int rho() const { return 5 * R2; }
  __host__ __device__ int q() const { return 5 * R2 + G; }
  __host__ __device__ int sub2() const { return 5 * R2 + 2 * G; }
  __host__ __device__ int cp2() const { return 5 * R2 + 4 * G; }
  __host__ __device__ int iw2() const { return 5 * R2 + 6 * G; }
  __host__ __device__ int rhs2() const { return 5 * R2 + 8 * G; }
};

// Solve the reduced systems of the block's lines in place (solution left in rhs). Must be
// called by all threads of the block (contains barriers). `first` selects factor-and-solve.
TDMA_DEV bool reduced_two_level(float* red, const RedLayout& L, int Lb, int tid, bool first, int64_t lines_left) {
  const int j = tid % Lb, g = tid / Lb;
  bool ok = true;
  // ---- level 1: group g of line j reduces its S rows to two endpoint rows
  if (g < L.G && j < lines_left) {
    float* R = red + (size_t)j * L.pitch;
    const int r0 = g * L.S;
    const float sub0 = R[L.sub() + r0], sup0 = R[L.sup() + r0], h0 = R[L.rhs() + r0];
    float alpha = -1.f, gamma = 0.f, delta = 0.f, F = 0.f, Gs = 0.f, Q = 1.f;
    for (int t = 1; t < L.S; ++t) {
      const int i = r0 + t;
      const float s = R[L.sub() + i], h = R[L.rhs() + i];
      const float r = rcp(1.f - s * gamma);
      const float ar = s * r;
      if (first) {
        alpha = -ar * alpha;
        gamma = R[L.sup() + i] * r;
      }
      delta = r * h - ar * delta;
      if (t <= L.S - 2) {
        if (first) {
          R[L.l1al() + i] = alpha;
          R[L.l1ga() + i] = gamma;
          Gs += Q * alpha;
        } else {
          gamma = R[L.l1ga() + i];
        }
        R[L.rhs() + i] = delta;
        F += Q * delta;
        Q = -Q * gamma;
      }
    }
    float rho;
    if (first) {
      rho = rcp(1.f - sup0 * Gs);
      R[L.rho() + g] = rho;
      R[L.q() + g] = Q;
      R[L.sub2() + 2 * g] = rho * sub0;
      R[L.cp2() + 2 * g] = rho * sup0 * Q;
      R[L.sub2() + 2 * g + 1] = alpha;
      R[L.cp2() + 2 * g + 1] = gamma;
    } else {
      rho = R[L.rho() + g];
    }
    R[L.rhs2() + 2 * g] = rho * (h0 - sup0 * F);
    R[L.rhs2() + 2 * g + 1] = delta;
  }
  __syncthreads();
  // ---- level 2: the 2G-row system of each line, one thread per line
  if (g == 0 && j < lines_left) {
    float* R = red + (size_t)j * L.pitch;
    ok = first ? reduced_factor_solve<float>(R + L.sub2(), R + L.cp2(), R + L.iw2(), R + L.rhs2(), 2 * L.G)
               : reduced_resolve<float>(R + L.sub2(), R + L.cp2(), R + L.iw2(), R + L.rhs2(), 2 * L.G);
  }
  __syncthreads();
  // ---- back substitution inside the groups
  if (g < L.G && j < lines_left) {
    float* R = red + (size_t)j * L.pitch;
    const int r0 = g * L.S;
    const float v0 = R[L.rhs2() + 2 * g], vn = R[L.rhs2() + 2 * g + 1];
    R[L.rhs() + r0] = v0;
    R[L.rhs() + r0 + L.S - 1] = vn;
    float v = vn;
    for (int t = L.S - 2; t >= 1; --t) {
      const int i = r0 + t;
      v = R[L.rhs() + i] - R[L.l1al() + i] * v0 - R[L.l1ga() + i] * v;
      R[L.rhs() + i] = v;
    }
  }
  __syncthreads();
  return ok;
}

__host__ __device__ inline size_t refine_tma_smem_bytes(int T, int Lb, int P, int M, int G) {
  const RedLayout L(P, G);
  size_t off = 0;
  off += (size_t)T * M * 8;                       // d tile (x staging at the end)
  off += (size_t)T * M * 4 * 3;                   // a, b, c tiles
  off += (size_t)T * M * 4;                       // low parts of x
  off += (size_t)T * 4 * 4;                       // partition endpoints
  off += (size_t)Lb * L.pitch * 4;                // reduced systems
  off += (size_t)Lb * 4 * 4;                      // per-line norms
  return off + 128;                               // alignment slack
}

constexpr uint32_t kTmaWaitPolls = 1u << 24;

template <int M, int MINB>
__global__ void __launch_bounds__(256, MINB)
    refine_tma_kernel(const Args A, const __grid_constant__ TmaMaps maps, const int G, const int use_tma) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_done;
  const int T = blockDim.x, tid = threadIdx.x;
  const int P = A.P, Lb = A.Lb;
  const int j = tid % Lb, k = tid / Lb;
  const int64_t line0 = (int64_t)blockIdx.x * Lb;
  const int64_t line_raw = line0 + j;
  const int64_t lines_left = A.lay.n_lines - line0;
  const bool active = line_raw < A.lay.n_lines;
  const int m = (int)(A.lay.n / P);  // uniform partitions

  unsigned char* p = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  double* t_d = reinterpret_cast<double*>(p);
  float* t_a = reinterpret_cast<float*>(t_d + (size_t)T * M);
  float* t_b = t_a + (size_t)T * M;
  float* t_c = t_b + (size_t)T * M;
  float* s_xl = t_c + (size_t)T * M;
  float* s_ex = s_xl + (size_t)T * M;
  const RedLayout RL(P, G);
  float* red = s_ex + 4 * (size_t)T;
  unsigned* s_nrm = reinterpret_cast<unsigned*>(red + (size_t)Lb * RL.pitch);
  float* R = red + (size_t)j * RL.pitch;

  // ---------------- tile load: TMA boxes {Lb, 1, P, m}, or plain loads into the same layout
  const int64_t ic = A.lay.ic;
  const int c_in = (int)(line0 % ic), c_out = (int)(line0 / ic);
  if (use_tma) {
    if (tid == 0) {
      mbar_init(&bar, 1);
      mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
      const uint32_t fbytes = (uint32_t)T * m * 4;
      mbar_arrive_expect_tx(&bar, 3 * fbytes + 2 * fbytes);
      tma_load_4d(t_a, &maps.a, &bar, c_in, c_out, 0, 0);
      tma_load_4d(t_b, &maps.b, &bar, c_in, c_out, 0, 0);
      tma_load_4d(t_c, &maps.c, &bar, c_in, c_out, 0, 0);
      tma_load_4d(t_d, &maps.d, &bar, c_in, c_out, 0, 0);
    }
  } else if (active) {
    const int64_t es = A.lay.es;
    const int64_t base = A.lay.off(line_raw) + (int64_t)k * m * es;
#pragma unroll
    for (int t = 0; t < M; ++t) {
      if (t < m) {
        t_a[(size_t)t * T + tid] = ldg((const float*)A.a + base + t * es);
        t_b[(size_t)t * T + tid] = ldg((const float*)A.b + base + t * es);
        t_c[(size_t)t * T + tid] = ldg((const float*)A.c + base + t * es);
        t_d[(size_t)t * T + tid] = ldg((const double*)A.d + base + t * es);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < M; ++t) s_xl[(size_t)t * T + tid] = 0.f;
  if (tid < Lb) { s_nrm[4 * tid] = 0u; s_nrm[4 * tid + 1] = 0u; s_nrm[4 * tid + 2] = 0u; s_nrm[4 * tid + 3] = 0u; }
  if (use_tma) {
    if (!mbar_wait_bounded(&bar, 0, kTmaWaitPolls)) report_error(A.st, 6);
  }
  __syncthreads();

  const bool first_part = (k == 0), last_part = (k == P - 1);
  float al[M], ga[M], de[M], xh[M];
#pragma unroll
  for (int t = 0; t < M; ++t) { al[t] = 0.f; ga[t] = 0.f; de[t] = 0.f; xh[t] = 0.f; }
  float a0 = 0.f, c0 = 0.f, rho = 1.f, prev_dx = 0.f;
  bool line_done = !active;
  const float keep = certify_keep(A.tol);
  float dom = -INFINITY;  // max over this partition's rows of dom_excess
  bool certified = true;  // the block's rows certify the floor

  int it = 0;
  for (;; ++it) {
    // ---------------- Stage A
    float xm_h = 0.f, xm_l = 0.f, xn_h = 0.f, xn_l = 0.f;
    if (it > 0) {
      if (!first_part) { xm_h = s_ex[2 * T + tid - Lb]; xm_l = s_ex[3 * T + tid - Lb]; }
      if (!last_part) { xn_h = s_ex[tid + Lb]; xn_l = s_ex[T + tid + Lb]; }
    }
    float alpha = -1.f, gamma = 0.f, delta = 0.f, F = 0.f, Gs = 0.f, Q = 1.f, rhs0 = 0.f, rhs_last = 0.f;
    float b0 = 1.f, pm_h = xm_h, pm_l = xm_l;
#pragma unroll
    for (int t = 0; t < M; ++t) {
      if (t < m) {
        const size_t o = (size_t)t * T + tid;
        float a = t_a[o], b = t_b[o], c = t_c[o];
        const double dv = t_d[o];
        if (first_part && t == 0) a = 0.f;
        if (last_part && t == m - 1) c = 0.f;
        if (it == 0) dom = fmaxf(dom, dom_excess(a, b, c, keep));
        float rhs;
        if (it == 0) {
          rhs = split_f64(dv).h;
        } else {
          const float x0h = xh[t], x0l = s_xl[o];
          float xph, xpl;
          if (t + 1 < m) { xph = xh[t + 1 < M ? t + 1 : 0]; xpl = s_xl[o + T]; }
          else { xph = xn_h; xpl = xn_l; }
          rhs = residual_ff(a, b, c, split_f64(dv), ff{pm_h, pm_l}, ff{x0h, x0l}, ff{xph, xpl});
          pm_h = x0h; pm_l = x0l;
        }
        if (t == 0) {
          a0 = a; b0 = b; c0 = c; rhs0 = rhs;
        } else {
          const float r = rcp(b - a * gamma);
          const float ar = a * r;
          if (it == 0) {
            alpha = -ar * alpha;
            gamma = c * r;
          } else if (t <= m - 2) {
            gamma = ga[t];
          }
          delta = r * rhs - ar * delta;
          if (t <= m - 2) {
            if (it == 0) { al[t] = alpha; ga[t] = gamma; Gs += Q * alpha; }
            de[t] = delta;
            F += Q * delta;
            Q = -Q * gamma;
          } else {
            rhs_last = delta;
          }
        }
      }
    }
    if (it == 0) {
      rho = rcp(b0 - c0 * Gs);
      if (active) {
        R[RL.sub() + 2 * k] = rho * a0;
        R[RL.sup() + 2 * k] = rho * c0 * Q;
        R[RL.sub() + 2 * k + 1] = alpha;
        R[RL.sup() + 2 * k + 1] = gamma;
      }
    }
    if (active) {
      R[RL.rhs() + 2 * k] = rho * (rhs0 - c0 * F);
      R[RL.rhs() + 2 * k + 1] = rhs_last;
    }
    if (__syncthreads_or(it == 0 && dom > 0.f)) certified = false;
    // ---------------- Stage B (two levels, contains barriers)
    if (!reduced_two_level(red, RL, Lb, tid, it == 0, lines_left)) report_error(A.st, 5);
    // ---------------- Stage C and update
    const float u0 = R[RL.rhs() + 2 * k], un = R[RL.rhs() + 2 * k + 1];
    float mdx = 0.f, mx = 0.f, v = un;
    float first_h = 0.f, first_l = 0.f, last_h = 0.f, last_l = 0.f;
#pragma unroll
    for (int t = M - 1; t >= 0; --t) {
      if (t < m) {
        float xt;
        if (t == m - 1) xt = un;
        else if (t == 0) xt = u0;
        else xt = de[t] - al[t] * u0 - ga[t] * v;
        v = xt;
        mdx = fmaxf(mdx, fabsf(xt));
        float h, l;
        if (it == 0) {
          h = xt; l = 0.f;
        } else {
          const size_t o = (size_t)t * T + tid;
          const ff nx = ff_add(ff{xh[t], s_xl[o]}, xt);
          h = nx.h; l = nx.l;
          s_xl[o] = l;
        }
        xh[t] = h;
        mx = fmaxf(mx, fabsf(h));
        if (t == 0) { first_h = h; first_l = l; }
        if (t == m - 1) { last_h = h; last_l = l; }
      }
    }
    s_ex[tid] = first_h; s_ex[T + tid] = first_l; s_ex[2 * T + tid] = last_h; s_ex[3 * T + tid] = last_l;
    if (Lb < 32) {
      for (int off = Lb; off < 32; off <<= 1) {
        mdx = fmaxf(mdx, __shfl_xor_sync(0xffffffffu, mdx, off));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      }
    }
    const int par = it & 1;
    if (active && ((tid & 31) < Lb || Lb >= 32)) {
      atomicMax(&s_nrm[4 * j + 2 * par], __float_as_uint(mdx));
      atomicMax(&s_nrm[4 * j + 2 * par + 1], __float_as_uint(mx));
    }
    if (tid == 0) s_done = 1;
    __syncthreads();
    if (tid < Lb) {
      const float dxn = __uint_as_float(s_nrm[4 * tid + 2 * par]);
      const float xn = __uint_as_float(s_nrm[4 * tid + 2 * par + 1]);
      s_nrm[4 * tid + 2 * (par ^ 1)] = 0u;
      s_nrm[4 * tid + 2 * (par ^ 1) + 1] = 0u;
      if (tid < lines_left) {
        if (it > 0) {
          line_done = refine_done(dxn, xn, prev_dx, A.tol, certified);
        } else {
          line_done = (xn == 0.f);
        }
        prev_dx = dxn;
        if (!(finite(dxn) && finite(xn))) report_error(A.st, 5);
        if (!line_done) s_done = 0;
      }
    }
    __syncthreads();
    if (s_done || it >= A.max_iters) break;
  }
  if (tid < Lb && tid < lines_left) {
    report_iters(A.st, it);
    if (!line_done) report_error(A.st, 7);
  }
  // ---------------- x in FP64: staged in the d tile, written by one TMA store
#pragma unroll
  for (int t = 0; t < M; ++t) {
    if (t < m) {
      const size_t o = (size_t)t * T + tid;
      t_d[o] = ff_to_f64(ff{xh[t], s_xl[o]});
    }
  }
  if (use_tma) {
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tma_store_4d(&maps.x, t_d, c_in, c_out, 0, 0);
      bulk_commit();
      bulk_wait_read_all();
    }
  } else if (active) {
    const int64_t es = A.lay.es;
    const int64_t base = A.lay.off(line_raw) + (int64_t)k * m * es;
#pragma unroll
    for (int t = 0; t < M; ++t)
      if (t < m) ((double*)A.x)[base + t * es] = t_d[(size_t)t * T + tid];
  }
}


// groups of the two-level reduced solve for P partitions (2P rows): about sqrt(2P) groups
__host__ __device__ constexpr int fixed_groups(int P) { return P >= 64 ? 8 : (P >= 16 ? 4 : (P >= 4 ? 2 : 1)); }

// ---------------------------------------------------------------------------------------
// Fixed-geometry variant: T = 256 threads, P partitions of exactly M rows (n = P M), Lb = 256/P
// lines per block, all known at compile time. Same algorithm as refine_tma_kernel; the row
// loops carry no runtime bounds, shared-memory offsets are immediates, and d is split into its
// float pair once (stored back into its tile slot) instead of once per pass.
template <int M, int P>
__global__ void __launch_bounds__(256, 2)
    refine_tma_fixed_kernel(const Args A, const __grid_constant__ TmaMaps maps, const int use_tma) {
  constexpr int T = 256, Lb = T / P, G = fixed_groups(P);
  static_assert(Lb * P == T && Lb >= 1, "geometry");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_done;
  const int tid = threadIdx.x;
  const int j = tid % Lb, k = tid / Lb;
  const int64_t line0 = (int64_t)blockIdx.x * Lb;
  const int64_t line_raw = line0 + j;
  const int64_t lines_left = A.lay.n_lines - line0;
  const bool active = line_raw < A.lay.n_lines;

  unsigned char* p = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  double* t_d = reinterpret_cast<double*>(p);
  float* t_a = reinterpret_cast<float*>(t_d + T * M);
  float* t_b = t_a + T * M;
  float* t_c = t_b + T * M;
  float* s_xl = t_c + T * M;
  float* s_ex = s_xl + T * M;
  const RedLayout RL(P, G);
  float* red = s_ex + 4 * T;
  unsigned* s_nrm = reinterpret_cast<unsigned*>(red + Lb * RL.pitch);
  float* R = red + j * RL.pitch;
  // this thread's column of each tile
  const float* ca = t_a + tid;
  const float* cb = t_b + tid;
  const float* cc = t_c + tid;
  double* cd = t_d + tid;
  float2* cd2 = reinterpret_cast<float2*>(t_d) + tid;  // (dh, dl) after the first pass
  float* cxl = s_xl + tid;

  const int64_t ic = A.lay.ic;
  const int c_in = (int)(line0 % ic), c_out = (int)(line0 / ic);
  if (use_tma) {
    if (tid == 0) {
      mbar_init(&bar, 1);
      mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
      const uint32_t fbytes = (uint32_t)T * M * 4;
      mbar_arrive_expect_tx(&bar, 5 * fbytes);
      tma_load_4d(t_a, &maps.a, &bar, c_in, c_out, 0, 0);
      tma_load_4d(t_b, &maps.b, &bar, c_in, c_out, 0, 0);
      tma_load_4d(t_c, &maps.c, &bar, c_in, c_out, 0, 0);
      tma_load_4d(t_d, &maps.d, &bar, c_in, c_out, 0, 0);
    }
  } else if (active) {
    const int64_t es = A.lay.es;
    const int64_t base = A.lay.off(line_raw) + (int64_t)k * M * es;
#pragma unroll
    for (int t = 0; t < M; ++t) {
      t_a[t * T + tid] = ldg((const float*)A.a + base + t * es);
      t_b[t * T + tid] = ldg((const float*)A.b + base + t * es);
      t_c[t * T + tid] = ldg((const float*)A.c + base + t * es);
      t_d[t * T + tid] = ldg((const double*)A.d + base + t * es);
    }
  }
#pragma unroll
  for (int t = 0; t < M; ++t) cxl[t * T] = 0.f;
  if (tid < Lb) { s_nrm[4 * tid] = 0u; s_nrm[4 * tid + 1] = 0u; s_nrm[4 * tid + 2] = 0u; s_nrm[4 * tid + 3] = 0u; }
  if (use_tma) {
    if (!mbar_wait_bounded(&bar, 0, kTmaWaitPolls)) report_error(A.st, 6);
  }
  __syncthreads();

  const bool first_part = (k == 0), last_part = (k == P - 1);
  float al[M], ga[M], de[M], xh[M];
  float a0 = 0.f, c0 = 0.f, rho = 1.f, prev_dx = 0.f;
  bool line_done = !active;
  const float keep = certify_keep(A.tol);
  float dom = -INFINITY;  // max over this partition's rows of dom_excess
  bool certified = true;  // the block's rows certify the floor

  int it = 0;
  for (;; ++it) {
    // ---------------- Stage A
    float pm_h = 0.f, pm_l = 0.f, xn_h = 0.f, xn_l = 0.f;
    if (it > 0) {
      if (!first_part) { pm_h = s_ex[2 * T + tid - Lb]; pm_l = s_ex[3 * T + tid - Lb]; }
      if (!last_part) { xn_h = s_ex[tid + Lb]; xn_l = s_ex[T + tid + Lb]; }
    }
    float alpha = -1.f, gamma = 0.f, delta = 0.f, F = 0.f, Gs = 0.f, Q = 1.f, rhs0 = 0.f, b0 = 1.f;
#pragma unroll
    for (int t = 0; t < M; ++t) {
      float a = ca[t * T], b = cb[t * T], c = cc[t * T];
      if (t == 0 && first_part) a = 0.f;
      if (t == M - 1 && last_part) c = 0.f;
      if (it == 0) dom = fmaxf(dom, dom_excess(a, b, c, keep));
      float rhs;
      if (it == 0) {
        const ff dd = split_f64(cd[t * T]);
        cd2[t * T] = make_float2(dd.h, dd.l);
        rhs = dd.h;
      } else {
        const float2 dd = cd2[t * T];
        const float x0h = xh[t], x0l = cxl[t * T];
        const float xph = (t + 1 < M) ? xh[t + 1 < M ? t + 1 : 0] : xn_h;
        const float xpl = (t + 1 < M) ? cxl[(t + 1 < M ? t + 1 : 0) * T] : xn_l;
        rhs = residual_ff(a, b, c, ff{dd.x, dd.y}, ff{pm_h, pm_l}, ff{x0h, x0l}, ff{xph, xpl});
        pm_h = x0h; pm_l = x0l;
      }
      if (t == 0) {
        a0 = a; b0 = b; c0 = c; rhs0 = rhs;
      } else {
        const float r = rcp(b - a * gamma);
        const float ar = a * r;
        if (it == 0) {
          alpha = -ar * alpha;
          gamma = c * r;
        } else if (t <= M - 2) {
          gamma = ga[t];
        }
        delta = r * rhs - ar * delta;
        if (t <= M - 2) {
          if (it == 0) { al[t] = alpha; ga[t] = gamma; Gs += Q * alpha; }
          de[t] = delta;
          F += Q * delta;
          Q = -Q * gamma;
        }
      }
    }
    if (it == 0) {
      rho = rcp(b0 - c0 * Gs);
      if (active) {
        R[RL.sub() + 2 * k] = rho * a0;
        R[RL.sup() + 2 * k] = rho * c0 * Q;
        R[RL.sub() + 2 * k + 1] = alpha;
        R[RL.sup() + 2 * k + 1] = gamma;
      }
    }
    if (active) {
      R[RL.rhs() + 2 * k] = rho * (rhs0 - c0 * F);
      R[RL.rhs() + 2 * k + 1] = delta;
    }
    if (__syncthreads_or(it == 0 && dom > 0.f)) certified = false;
    if (!reduced_two_level(red, RL, Lb, tid, it == 0, lines_left)) report_error(A.st, 5);
    // ---------------- Stage C and update
    const float u0 = R[RL.rhs() + 2 * k], un = R[RL.rhs() + 2 * k + 1];
    float mdx = fmaxf(fabsf(u0), fabsf(un)), mx = 0.f, v = un;
#pragma unroll
    for (int t = M - 1; t >= 0; --t) {
      const float xt = (t == M - 1) ? un : (t == 0 ? u0 : de[t] - al[t] * u0 - ga[t] * v);
      v = xt;
      if (t > 0 && t < M - 1) mdx = fmaxf(mdx, fabsf(xt));
      if (it == 0) {
        xh[t] = xt;
      } else {
        const ff nx = ff_add(ff{xh[t], cxl[t * T]}, xt);
        xh[t] = nx.h;
        cxl[t * T] = nx.l;
      }
      mx = fmaxf(mx, fabsf(xh[t]));
    }
    s_ex[tid] = xh[0];
    s_ex[T + tid] = cxl[0];
    s_ex[2 * T + tid] = xh[M - 1];
    s_ex[3 * T + tid] = cxl[(M - 1) * T];
    if (Lb < 32) {
#pragma unroll
      for (int off = Lb; off < 32; off <<= 1) {
        mdx = fmaxf(mdx, __shfl_xor_sync(0xffffffffu, mdx, off));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      }
    }
    const int par = it & 1;
    if (active && ((tid & 31) < Lb || Lb >= 32)) {
      atomicMax(&s_nrm[4 * j + 2 * par], __float_as_uint(mdx));
      atomicMax(&s_nrm[4 * j + 2 * par + 1], __float_as_uint(mx));
    }
    if (tid == 0) s_done = 1;
    __syncthreads();
    if (tid < Lb) {
      const float dxn = __uint_as_float(s_nrm[4 * tid + 2 * par]);
      const float xn = __uint_as_float(s_nrm[4 * tid + 2 * par + 1]);
      s_nrm[4 * tid + 2 * (par ^ 1)] = 0u;
      s_nrm[4 * tid + 2 * (par ^ 1) + 1] = 0u;
      if (tid < lines_left) {
        if (it > 0) {
          line_done = refine_done(dxn, xn, prev_dx, A.tol, certified);
        } else {
          line_done = (xn == 0.f);
        }
        prev_dx = dxn;
        if (!(finite(dxn) && finite(xn))) report_error(A.st, 5);
        if (!line_done) s_done = 0;
      }
    }
    __syncthreads();
    if (s_done || it >= A.max_iters) break;
  }
  if (tid < Lb && tid < lines_left) {
    report_iters(A.st, it);
    if (!line_done) report_error(A.st, 7);
  }
#pragma unroll
  for (int t = 0; t < M; ++t) cd[t * T] = ff_to_f64(ff{xh[t], cxl[t * T]});
  if (use_tma) {
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tma_store_4d(&maps.x, t_d, c_in, c_out, 0, 0);
      bulk_commit();
      bulk_wait_read_all();
    }
  } else if (active) {
    const int64_t es = A.lay.es;
    const int64_t base = A.lay.off(line_raw) + (int64_t)k * M * es;
#pragma unroll
    for (int t = 0; t < M; ++t) ((double*)A.x)[base + t * es] = cd[t * T];
  }
}

// compile-time geometries of the fixed kernel: (rows per partition, partitions)
#define TDMA_REFINE_FIXED_SHAPES(X) X(16, 64) X(16, 32) X(16, 16) X(8, 32) X(8, 8)

}  // namespace tdma
