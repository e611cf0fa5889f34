// Ragged batches: thousands of lines of uneven length in one persistent launch.
//
// The paper batches systems of one direction into composite systems and tunes the batch size
// (Sections 4.2.1-4.2.3). Here lines of any length share one launch: at plan time the lines are
// sorted longest first and cut into groups of similar length; group g has P_g partitions per
// line (about 16 rows per partition, at most 256) and up to 256 / P_g lines, so one block of
// 256 threads solves a group with thread (j, k) on partition k of line j. Blocks stay resident
// and pull group indices from a device counter (atomicAdd), longest groups first, which keeps
// the tail of the launch short. Items are independent: no block ever waits on another.
//
// Stage A/B/C follow kernels_dc.cuh (F64, F32) and kernels_refine.cuh (F32 + refinement). Long
// lines do not fit on chip (16384 rows x 24 bytes of Stage A scratch), so the per-row scratch
// (alpha, gamma, delta, and for refinement the two parts of x) lives in the workspace, per line
// in a [row][partition] layout that keeps a warp's accesses contiguous. Line data are packed
// with unit stride at ragged_offsets[l].
#pragma once
#include "tdma.h"
#include "layout.cuh"
#include "kernels_dc.cuh"
#include "kernels_refine.cuh"
#include "kernels_backward.cuh"

namespace tdma {

constexpr int kRaggedThreads = 256;
constexpr int kRaggedRowsPerPart = 16;

struct RaggedGroup {
  int32_t first;  // index of the group's first line in the sorted order
  int32_t count;  // lines in the group
  int32_t P;      // partitions per line
  int32_t pad;
};

// Device tables owned by the plan (built on the host at plan time).
struct RaggedTables {
  const int32_t* order;    // line indices, longest first
  const int64_t* sbase;    // per line: start of its scratch region (elements)
  const RaggedGroup* groups;
  int32_t n_groups;
  int32_t* queue;          // work counter, zeroed before every launch
  int64_t scratch_elems;   // elements of each scratch array
};

template <class CT, bool TR = false>
__global__ void __launch_bounds__(kRaggedThreads, 3) ragged_dc_kernel(const Args A, const RaggedTables RT) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT* red = reinterpret_cast<CT*>(smem_raw);
  __shared__ int s_g;
  const int tid = threadIdx.x;
  CT* s_alpha = (CT*)A.ws;
  CT* s_gamma = s_alpha + RT.scratch_elems;
  CT* s_delta = s_gamma + RT.scratch_elems;
  for (;;) {
    if (tid == 0) s_g = atomicAdd(RT.queue, 1);
    __syncthreads();
    const int g = s_g;
    if (g >= RT.n_groups) break;
    const RaggedGroup G = RT.groups[g];
    const int P = G.P, cnt = G.count, R2 = 2 * P, pitch = 3 * R2 + 1;
    const int j = tid % cnt, k = tid / cnt;
    const bool active = k < P;
    const int32_t li = RT.order[G.first + j];
    const int64_t n = A.rlen[li], base = A.roff[li], sb = RT.sbase[li];
    CT* r_sub = red + (size_t)j * pitch;
    CT* r_sup = r_sub + R2;
    CT* r_rhs = r_sup + R2;
    int64_t start = 0;
    int m = 0;
    partition(n, P, k, start, m);
    if (active && n == 1) {
      const CT v = ldg((const CT*)A.d + base) * rcp(ldg((const CT*)A.b + base));
      if (!finite(v)) report_error(A.st, 5);
      ((CT*)A.x)[base] = v;
    } else if (active) {
      // ---- Stage A
      const CT* pa = (const CT*)A.a + base + start;
      const CT* pb = (const CT*)A.b + base + start;
      const CT* pc = (const CT*)A.c + base + start;
      const CT* pd = (const CT*)A.d + base + start;
      // row t of this partition (with TR: of the transpose, sub c_{i-1}, super a_{i+1})
      auto sub = [&](int t) -> CT {
        if (k == 0 && t == 0) return CT(0);
        return TR ? ldg(pc + t - 1) : ldg(pa + t);
      };
      auto sup = [&](int t) -> CT {
        if (k == P - 1 && t == m - 1) return CT(0);
        return TR ? ldg(pa + t + 1) : ldg(pc + t);
      };
      CT a0 = sub(0), b0 = ldg(pb), c0 = sup(0), d0 = ldg(pd);
      CT alpha = CT(-1), gamma = CT(0), delta = CT(0), Q = CT(1), Gs = CT(0), F = CT(0);
      for (int t = 1; t < m; ++t) {
        const CT a = sub(t), b = ldg(pb + t), d = ldg(pd + t);
        const CT c = sup(t);
        const CT r = rcp(b - a * gamma);
        const CT ar = a * r;
        alpha = -ar * alpha;
        gamma = c * r;
        delta = r * d - ar * delta;
        if (t <= m - 2) {
          const int64_t o = sb + (int64_t)(t - 1) * P + k;
          s_alpha[o] = alpha;
          s_gamma[o] = gamma;
          s_delta[o] = delta;
          F += Q * delta;
          Gs += Q * alpha;
          Q = -Q * gamma;
        }
      }
      const CT rho = rcp(b0 - c0 * Gs);
      r_sub[2 * k] = rho * a0;
      r_sup[2 * k] = rho * c0 * Q;
      r_rhs[2 * k] = rho * (d0 - c0 * F);
      r_sub[2 * k + 1] = alpha;
      r_sup[2 * k + 1] = gamma;
      r_rhs[2 * k + 1] = delta;
    }
    __syncthreads();
    // ---- Stage B: one thread per line, or two levels for long reduced systems (the group's
    // lines all have P > 16 partitions, so n > 1)
    if (R2 > kTwoLevelRows) {
      reduced_two_level<CT, 1>(red, pitch, cnt, cnt, R2, A.st);
    } else if (tid < cnt && n > 1) {
      if (!reduced_solve<CT, 1>(r_sub, r_sup, r_rhs, R2, R2)) report_error(A.st, 5);
    }
    __syncthreads();
    // ---- Stage C
    if (active && n > 1) {
      CT* px = (CT*)A.x + base + start;
      const CT x0 = r_rhs[2 * k];
      CT xn = r_rhs[2 * k + 1];
      px[0] = x0;
      px[m - 1] = xn;
      for (int t = m - 2; t >= 1; --t) {
        const int64_t o = sb + (int64_t)(t - 1) * P + k;
        xn = s_delta[o] - s_alpha[o] * x0 - s_gamma[o] * xn;
        px[t] = xn;
      }
    }
    __syncthreads();  // shared memory is reused by the next group
  }
}

// F32 storage + refinement on ragged groups: same passes as refine_kernel (first pass solves
// fl(d); later passes solve for the correction from the extra-precise residual), with alpha,
// gamma, delta and both parts of x in the workspace. Partition-row scratch index: sb + t P + k.
template <bool TR = false>
__global__ void __launch_bounds__(kRaggedThreads) ragged_refine_kernel(const Args A, const RaggedTables RT) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* red = reinterpret_cast<float*>(smem_raw);
  __shared__ int s_g, s_done;
  __shared__ unsigned s_nrm[2 * kRaggedThreads];
  __shared__ float s_prev[kRaggedThreads];
  const int tid = threadIdx.x;
  const int64_t E = RT.scratch_elems;
  float* s_alpha = (float*)A.ws;
  float* s_gamma = s_alpha + E;
  float* s_delta = s_gamma + E;
  float* s_xh = s_delta + E;
  float* s_xl = s_xh + E;
  for (;;) {
    if (tid == 0) s_g = atomicAdd(RT.queue, 1);
    __syncthreads();
    const int g = s_g;
    if (g >= RT.n_groups) break;
    const RaggedGroup G = RT.groups[g];
    const int P = G.P, cnt = G.count, R2 = 2 * P, pitch = 4 * R2 + 1;
    const int j = tid % cnt, k = tid / cnt;
    const bool active = k < P;
    const int32_t li = RT.order[G.first + j];
    const int64_t n = A.rlen[li], base = A.roff[li], sb = RT.sbase[li];
    float* R = red + (size_t)j * pitch;  // sub, cp, iw, rhs
    int64_t start = 0;
    int m = 0;
    partition(n, P, k, start, m);
    const float* pa = (const float*)A.a + base + start;
    const float* pb = (const float*)A.b + base + start;
    const float* pc = (const float*)A.c + base + start;
    const double* pd = (const double*)A.d + base + start;
    auto xo = [&](int t) { return sb + (int64_t)t * P + k; };  // x parts of row t of this partition
    float rho = 1.f, a0 = 0.f, c0 = 0.f;
    if (tid < cnt) { s_nrm[2 * tid] = 0u; s_nrm[2 * tid + 1] = 0u; }
    int it = 0;
    bool line_done = false;
    const float keep = certify_keep(A.tol);
    float dom = -INFINITY;  // max over this partition's rows of dom_excess
    bool certified = true;  // the group's rows certify the floor
    for (;; ++it) {
      // ---- Stage A
      if (active) {
        float alpha = -1.f, gamma = 0.f, delta = 0.f, Q = 1.f, Gs = 0.f, F = 0.f, rhs0 = 0.f, b0 = 1.f;
        ff pm{0.f, 0.f};
        if (it > 0 && k > 0) {  // x_{-1}: last row of partition k-1 (row m_{k-1}-1 at index (m_{k-1}-1) P + k-1)
          int64_t sp; int mp;
          partition(n, P, k - 1, sp, mp);
          const int64_t o = sb + (int64_t)(mp - 1) * P + (k - 1);
          pm = ff{s_xh[o], s_xl[o]};
        }
        for (int t = 0; t < m; ++t) {
          float a = (k == 0 && t == 0) ? 0.f : (TR ? ldg(pc + t - 1) : ldg(pa + t));
          const float b = ldg(pb + t);
          float c = (k == P - 1 && t == m - 1) ? 0.f : (TR ? ldg(pa + t + 1) : ldg(pc + t));
          if (it == 0) dom = fmaxf(dom, dom_excess(a, b, c, keep));
          const ff dd = split_f64(ldg(pd + t));
          float rhs;
          if (it == 0) {
            rhs = __fadd_rn(dd.h, dd.l);
          } else {
            const ff x0{s_xh[xo(t)], s_xl[xo(t)]};
            ff xp{0.f, 0.f};
            if (t + 1 < m) xp = ff{s_xh[xo(t + 1)], s_xl[xo(t + 1)]};
            else if (k < P - 1) xp = ff{s_xh[sb + (k + 1)], s_xl[sb + (k + 1)]};
            rhs = residual_ff(a, b, c, dd, pm, x0, xp);
            pm = x0;
          }
          if (t == 0) { a0 = a; b0 = b; c0 = c; rhs0 = rhs; continue; }
          const float r = rcp(b - a * gamma);
          const float ar = a * r;
          const int64_t o = sb + (int64_t)(t - 1) * P + k;
          if (it == 0) {
            alpha = -ar * alpha;
            gamma = c * r;
          } else if (t <= m - 2) {
            gamma = s_gamma[o];
          }
          delta = r * rhs - ar * delta;
          if (t <= m - 2) {
            if (it == 0) { s_alpha[o] = alpha; s_gamma[o] = gamma; Gs += Q * alpha; }
            s_delta[o] = delta;
            F += Q * delta;
            Q = -Q * gamma;
          }
        }
        if (n == 1) {
          R[3 * R2] = rhs0 * rcp(b0);  // a single equation: the solution itself
        } else {
          if (it == 0) {
            rho = rcp(b0 - c0 * Gs);
            R[2 * k] = rho * a0;
            R[R2 + 2 * k] = rho * c0 * Q;
            R[2 * k + 1] = alpha;
            R[R2 + 2 * k + 1] = gamma;
          }
          R[3 * R2 + 2 * k] = rho * (rhs0 - c0 * F);
          R[3 * R2 + 2 * k + 1] = delta;
        }
      }
      if (__syncthreads_or(it == 0 && dom > 0.f)) certified = false;
      // ---- Stage B: one thread per line
      if (tid < cnt && n > 1) {
        const bool ok = (it == 0) ? reduced_factor_solve<float>(R, R + R2, R + 2 * R2, R + 3 * R2, R2)
                                  : reduced_resolve<float>(R, R + R2, R + 2 * R2, R + 3 * R2, R2);
        if (!ok) report_error(A.st, 5);
      }
      __syncthreads();
      // ---- Stage C: correction (or first solution) into x, with per-line maxima
      if (active) {
        float mdx = 0.f, mx = 0.f;
        auto upd = [&](int t, float v) {
          const int64_t o = xo(t);
          ff nx{v, 0.f};
          if (it > 0) nx = ff_add(ff{s_xh[o], s_xl[o]}, v);
          s_xh[o] = nx.h;
          s_xl[o] = nx.l;
          mdx = fmaxf(mdx, fabsf(v));
          mx = fmaxf(mx, fabsf(nx.h));
        };
        if (n == 1) {
          upd(0, R[3 * R2]);
        } else {
          const float u0 = R[3 * R2 + 2 * k], un = R[3 * R2 + 2 * k + 1];
          upd(0, u0);
          upd(m - 1, un);
          float v = un;
          for (int t = m - 2; t >= 1; --t) {
            const int64_t o = sb + (int64_t)(t - 1) * P + k;
            v = s_delta[o] - s_alpha[o] * u0 - s_gamma[o] * v;
            upd(t, v);
          }
        }
        atomicMax(&s_nrm[2 * j], __float_as_uint(mdx));
        atomicMax(&s_nrm[2 * j + 1], __float_as_uint(mx));
      }
      if (tid == 0) s_done = 1;
      __syncthreads();
      if (tid < cnt) {
        const float dxn = __uint_as_float(s_nrm[2 * tid]), xn = __uint_as_float(s_nrm[2 * tid + 1]);
        s_nrm[2 * tid] = 0u;
        s_nrm[2 * tid + 1] = 0u;
        if (it > 0) {
          line_done = refine_done(dxn, xn, s_prev[tid], A.tol, certified);
        } else {
          line_done = (xn == 0.f);
        }
        s_prev[tid] = dxn;
        if (!(finite(dxn) && finite(xn))) report_error(A.st, 5);
        if (!line_done) s_done = 0;
      }
      __syncthreads();
      if (s_done || it >= A.max_iters) break;
    }
    if (tid < cnt) {
      report_iters(A.st, it);
      if (!line_done) report_error(A.st, 7);
    }
    // ---- x in FP64
    if (active) {
      double* px = (double*)A.x + base + start;
      for (int t = 0; t < m; ++t) px[t] = ff_to_f64(ff{s_xh[xo(t)], s_xl[xo(t)]});
    }
    __syncthreads();
  }
}

// Gradient epilogue for ragged batches (kRaggedEpiThreads per block): grad_a_i = -lambda_i x_{i-1},
// grad_b_i = -lambda_i x_i, grad_c_i = -lambda_i x_{i+1}, with grad_a = 0 on a line's first row and
// grad_c = 0 on its last. The blocks take lines in turn, a block's warps consecutive windows of 32
// rows of its line: x_{i-1} and x_{i+1} come from the neighbouring lanes, across a window's edges
// by one load each, so that a long line keeps many warps busy.
constexpr int kRaggedEpiThreads = 128;
template <class GT, class XT>
__global__ void __launch_bounds__(kRaggedEpiThreads) ragged_epilogue(const int64_t n_lines,
                                                                     const int64_t* __restrict__ roff,
                                                                     const int32_t* __restrict__ rlen,
                                                                     const XT* __restrict__ x,
                                                                     const XT* __restrict__ lam, GT* __restrict__ ga,
                                                                     GT* __restrict__ gb, GT* __restrict__ gc) {
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t l = blockIdx.x; l < n_lines; l += gridDim.x) {
    const int64_t base = roff[l];
    const int n = rlen[l];
    for (int i0 = wb * 32; i0 < n; i0 += nw * 32) {  // the same for the 32 lanes
      const int i = i0 + lane;
      const bool in = i < n;
      const XT xc = in ? x[base + i] : XT(0);
      const XT lv = in ? lam[base + i] : XT(0);
      XT xp = __shfl_up_sync(~0u, xc, 1), xn = __shfl_down_sync(~0u, xc, 1);
      if (lane == 0) xp = i > 0 ? x[base + i - 1] : XT(0);
      if (lane == 31) xn = i + 1 < n ? x[base + i + 1] : XT(0);
      if (in) {
        const int64_t e = base + i;
        if (gb) gb[e] = neg_prod<GT>(lv, xc);
        if (ga) ga[e] = i > 0 ? neg_prod<GT>(lv, xp) : GT(0);
        if (gc) gc[e] = i + 1 < n ? neg_prod<GT>(lv, xn) : GT(0);
      }
    }
  }
}

inline size_t ragged_smem_bytes(tdma_precision_t p) {
  // reduced systems of one group: sum over lines of (pitch) words, pitch <= 4 * 2P + 1, lines * P <= 256;
  // the two-level solve (P > 16, at most 15 lines) adds 6 ceil(2P / 16) words per line after them,
  // at most 6 (256 / 8 + 15) = 282 words, within the same bound (3 * 2P + 1 pitch: <= 1792 + 282)
  const size_t words = (size_t)kRaggedThreads * 8 + kRaggedThreads;
  return words * (p == TDMA_F64 ? 8 : 4);
}

}  // namespace tdma
