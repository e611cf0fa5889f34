// FP32 storage + refinement with the per-row state of every partition held in registers.
//
// Same algorithm as kernels_refine.cuh (Stage A modified-Thomas sweep in float, Stage B reduced
// solve, Stage C interior update; then extra-precise residual and correction until the line
// error estimate is below tolerance), organised for throughput:
//   - a partition has at most M rows (compile-time), so alpha, gamma, delta and the high part
//     of x live in registers, fully unrolled over rows;
//   - the first pass streams a, b, c, d from HBM; later passes read the same addresses again
//     and are served by L1/L2 (the block's lines were read microseconds earlier), so HBM
//     traffic stays one read of the inputs and one write of x;
//   - the Stage A factors (alpha, gamma and the row-0 fix) and the LU factors of the reduced
//     system are computed once and reused by every correction;
//   - only the low parts of x (nonzero after the first correction) and the partition endpoints
//     go through shared memory.
#pragma once
#include "layout.cuh"
#include "kernels_refine.cuh"

namespace tdma {

template <class BT>
__host__ __device__ inline size_t refine_reg_smem_bytes(int T, int Lb, int P, int M) {
  const size_t pitch = (size_t)4 * 2 * P + 1;
  return sizeof(BT) * (size_t)Lb * pitch + sizeof(float) * ((size_t)M * T + 4 * (size_t)T) +
         sizeof(unsigned) * 4 * (size_t)Lb + 16;
}

template <int M, class BT, int MINB>
__global__ void __launch_bounds__(256, MINB) refine_reg_kernel(const Args A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int T = blockDim.x, tid = threadIdx.x;
  const int P = A.P, Lb = A.Lb;
  const int j = tid % Lb, k = tid / Lb;
  const int64_t line_raw = (int64_t)blockIdx.x * Lb + j;
  const bool active = line_raw < A.lay.n_lines;
  const int64_t line = active ? line_raw : A.lay.n_lines - 1;  // inactive threads mirror a valid line
  const int R2 = 2 * P;
  const int pitch = 4 * R2 + 1;
  BT* red = reinterpret_cast<BT*>(smem_raw);
  BT* r_sub = red + (size_t)j * pitch;
  BT* r_cp = r_sub + R2;
  BT* r_rhs = r_cp + 2 * R2;
  float* s_xl = reinterpret_cast<float*>(red + (size_t)Lb * pitch);  // [M][T]
  float* s_ex = s_xl + (size_t)M * T;                                 // first h/l, last h/l: [4][T]
  unsigned* s_nrm = reinterpret_cast<unsigned*>(s_ex + 4 * (size_t)T);  // [Lb][4]
  __shared__ int s_done;

  int64_t start = 0;
  int m = 0;
  partition(A.lay.n, P, k, start, m);
  const int64_t es = A.lay.es;
  const int64_t base = A.lay.off(line) + start * es;
  const float* pa = (const float*)A.a + base;
  const float* pb = (const float*)A.b + base;
  const float* pc = (const float*)A.c + base;
  const double* pd = (const double*)A.d + base;
  const bool first_part = (k == 0), last_part = (k == P - 1);

  float al[M], ga[M], de[M], xh[M];
#pragma unroll
  for (int t = 0; t < M; ++t) { al[t] = 0.f; ga[t] = 0.f; de[t] = 0.f; xh[t] = 0.f; }
  float a0 = 0.f, c0 = 0.f, rho = 1.f, prev_dx = 0.f;
  bool line_done = !active;
  const float keep = certify_keep(A.tol);
  float dom = -INFINITY;  // max over this partition's rows of dom_excess
  bool certified = true;  // the block's rows certify the floor
  if (tid < Lb) { s_nrm[4 * tid] = 0u; s_nrm[4 * tid + 1] = 0u; s_nrm[4 * tid + 2] = 0u; s_nrm[4 * tid + 3] = 0u; }
#pragma unroll
  for (int t = 0; t < M; ++t) s_xl[(size_t)t * T + tid] = 0.f;

  int it = 0;
  for (;; ++it) {
    // ---------------- Stage A
    float xm_h = 0.f, xm_l = 0.f, xn_h = 0.f, xn_l = 0.f;  // x_{-1} and x_m of this partition
    if (it > 0) {
      if (!first_part) { xm_h = s_ex[2 * T + tid - Lb]; xm_l = s_ex[3 * T + tid - Lb]; }
      if (!last_part) { xn_h = s_ex[tid + Lb]; xn_l = s_ex[T + tid + Lb]; }
    }
    float alpha = -1.f, gamma = 0.f, delta = 0.f, F = 0.f, G = 0.f, Q = 1.f, rhs0 = 0.f, rhs_last = 0.f;
    float b0 = 1.f;
    float pm_h = xm_h, pm_l = xm_l;  // x_{t-1} while sweeping
#pragma unroll
    for (int t = 0; t < M; ++t) {
      if (t < m) {
        float a = ldg(pa + t * es), b = ldg(pb + t * es), c = ldg(pc + t * es);
        const double dv = ldg(pd + t * es);
        if (first_part && t == 0) a = 0.f;
        if (last_part && t == m - 1) c = 0.f;
        if (it == 0) dom = fmaxf(dom, dom_excess(a, b, c, keep));
        float rhs;
        if (it == 0) {
          const ff dd = split_f64(dv);
          rhs = dd.h;
        } else {
          const float x0h = xh[t], x0l = s_xl[(size_t)t * T + tid];
          float xph, xpl;
          if (t + 1 < m) { xph = xh[t + 1 < M ? t + 1 : 0]; xpl = s_xl[(size_t)(t + 1 < M ? t + 1 : 0) * T + tid]; }
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
            if (it == 0) { al[t] = alpha; ga[t] = gamma; G += Q * alpha; }
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
      rho = rcp(b0 - c0 * G);
      if (active) {
        r_sub[2 * k] = widen<BT>(rho * a0);
        r_cp[2 * k] = widen<BT>(rho * c0 * Q);
        r_sub[2 * k + 1] = widen<BT>(alpha);
        r_cp[2 * k + 1] = widen<BT>(gamma);
      }
    }
    if (active) {
      r_rhs[2 * k] = widen<BT>(rho * (rhs0 - c0 * F));
      r_rhs[2 * k + 1] = widen<BT>(rhs_last);
    }
    if (__syncthreads_or(it == 0 && dom > 0.f)) certified = false;
    // ---------------- Stage B: one thread per line
    if (tid < Lb && (int64_t)blockIdx.x * Lb + tid < A.lay.n_lines) {
      BT* sub = red + (size_t)tid * pitch;
      const bool ok = (it == 0) ? reduced_factor_solve<BT>(sub, sub + R2, sub + 2 * R2, sub + 3 * R2, R2)
                                : reduced_resolve<BT>(sub, sub + R2, sub + 2 * R2, sub + 3 * R2, R2);
      if (!ok) report_error(A.st, 5);
    }
    __syncthreads();
    // ---------------- Stage C and update
    const float u0 = narrow(r_rhs[2 * k]), un = narrow(r_rhs[2 * k + 1]);
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
          const ff nx = ff_add(ff{xh[t], s_xl[(size_t)t * T + tid]}, xt);
          h = nx.h; l = nx.l;
          s_xl[(size_t)t * T + tid] = l;
        }
        xh[t] = h;
        mx = fmaxf(mx, fabsf(h));
        if (t == 0) { first_h = h; first_l = l; }
        if (t == m - 1) { last_h = h; last_l = l; }
      }
    }
    s_ex[tid] = first_h; s_ex[T + tid] = first_l; s_ex[2 * T + tid] = last_h; s_ex[3 * T + tid] = last_l;
    // per-line maxima: lanes of one line sit Lb apart inside a warp (Lb divides 32) or alone
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
      const bool live = (int64_t)blockIdx.x * Lb + tid < A.lay.n_lines;
      if (live) {
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
  if (tid < Lb && (int64_t)blockIdx.x * Lb + tid < A.lay.n_lines) {
    report_iters(A.st, it);
    if (!line_done) report_error(A.st, 7);
  }
  if (active) {
    double* px = (double*)A.x + base;
#pragma unroll
    for (int t = 0; t < M; ++t)
      if (t < m) px[t * es] = ff_to_f64(ff{xh[t], s_xl[(size_t)t * T + tid]});
  }
}

}  // namespace tdma
