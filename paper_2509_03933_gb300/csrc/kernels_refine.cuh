// Float storage and sweeps, accuracy won back by iterative refinement (mixed-precision
// iterative refinement: Wilkinson 1963, Moler 1967; the paper keeps everything in FP64).
//
// Inputs: a, b, c float; d double. Output: x double. One block holds Lb lines split into P
// partitions each (thread (j, k) = partition k of line j), and runs, without leaving the block:
//   x = solve32(fl(d));  repeat: r = d - A x (extra precise), dx = solve32(r), x += dx
// until the estimated error of every line is below the tolerance. solve32 is the fused
// Stage A / B / C divide-and-conquer solve of kernels_dc.cuh in float; its Stage A factors
// (alpha, gamma) do not depend on the right-hand side and are kept from the first pass, and
// the reduced system's LU factors are kept from the first Stage B.
//
// Arithmetic that must be better than float never touches the FP64 pipe (about 1/60 of the
// FP32 rate on GB300): d is split into a float pair by integer bit operations, x is carried
// as an unevaluated float pair (h + l, about 48 significant bits), and the residual is an
// error-free-transformation dot product (TwoProduct / TwoSum, accurate as if computed with
// twice the float precision; Ogita, Rump and Oishi 2005). Only the final store adds the two
// halves in FP64. Stage B (the reduced endpoint solve) runs in FP64 when SB64 is set.
//
// Convergence (per line, infinity norms): with dx_0 = x_0, rho_t = |dx_t| / |dx_{t-1}| is the
// observed contraction and rho_t |dx_t| estimates the error left after the update. That estimate
// knows nothing of the accuracy floor of the float-pair residual: its rounding errors, about 2^-48
// of the residual's terms, reach x amplified by the condition number, and the refinement cannot
// get below about kappa 2^-52 |x| (measured; kappa 2^-48 in the worst case). A line is therefore
// done once rho_t |dx_t| <= tol |x| only when its floor is certified below tol: every row is
// diagonally dominant with 1 - (|a_i| + |c_i|) / |b_i| >= theta and 2^-51 / theta <= tol, which
// bounds the condition number of the row-scaled matrix by 1 / theta (Varah 1975: a row-diagonally
// dominant matrix has ||A^-1||_inf <= 1 / min_i (|a_ii| - sum_j |a_ij|)). Other lines are done only
// when the last correction itself is below tol |x| (at the floor the corrections stay at its level,
// so such lines end with TDMA_ERR_NOT_CONVERGED instead of a result short of the tolerance). The
// certificate is evaluated per line where the kernel gathers its lines' norms anyway and per block
// elsewhere (a block with one uncertified row applies the strict rule to all of its lines). The
// block stops when all of its lines are done or after max_iters corrections; lines still above the
// tolerance then raise TDMA_ERR_NOT_CONVERGED.
#pragma once
#include "layout.cuh"
#include "kernels_dc.cuh"

namespace tdma {

template <class BT>
__host__ __device__ inline size_t refine_smem_bytes(int T, int Lb, int P, int mmax) {
  const size_t slots = mmax > 2 ? (size_t)(mmax - 2) : 0;
  const size_t per_thread = (3 * slots + 2 * (size_t)mmax) * sizeof(float);
  const size_t pitch = (size_t)4 * 2 * P + 1;  // sub, cp, iw, rhs
  return per_thread * T + sizeof(BT) * (size_t)Lb * pitch + (size_t)Lb * 4 * sizeof(unsigned) + 16;
}

// Reduced system: factor and solve (first pass), keeping cp and 1/w for later passes.
template <class BT>
TDMA_DEV bool reduced_factor_solve(BT* sub, BT* cp, BT* iw, BT* rhs, int rows) {
  BT c = cp[0];  // sup[0] on entry
  BT dp = rhs[0];
  iw[0] = BT(1);
  for (int i = 1; i < rows; ++i) {
    const BT s = sub[i];
    const BT w = rcp(BT(1) - s * c);
    c = cp[i] * w;
    cp[i] = c;
    iw[i] = w;
    dp = (rhs[i] - s * dp) * w;
    rhs[i] = dp;
  }
  BT u = dp;
  bool ok = finite(u);
  for (int i = rows - 2; i >= 0; --i) {
    u = rhs[i] - cp[i] * u;
    rhs[i] = u;
  }
  return ok && finite(u);
}
template <class BT>
TDMA_DEV bool reduced_resolve(const BT* sub, const BT* cp, const BT* iw, BT* rhs, int rows) {
  BT dp = rhs[0];
  for (int i = 1; i < rows; ++i) {
    dp = (rhs[i] - sub[i] * dp) * iw[i];
    rhs[i] = dp;
  }
  BT u = dp;
  bool ok = finite(u);
  for (int i = rows - 2; i >= 0; --i) {
    u = rhs[i] - cp[i] * u;
    rhs[i] = u;
  }
  return ok && finite(u);
}

template <class BT> TDMA_DEV BT widen(float v);
template <> TDMA_DEV float widen<float>(float v) { return v; }
template <> TDMA_DEV double widen<double>(float v) { return f2d(v); }
TDMA_DEV float narrow(float v) { return v; }
TDMA_DEV float narrow(double v) { return __double2float_rn(v); }

struct Coef { float a, b, c; double d; };

// ---- certified stop rule (see the header)
constexpr float kRefineFloor = 4.440892098500626e-16f;  // 2^-51: twice the measured floor per unit condition
// keep = 1 - 2^-51 / tol; a row is certified when |a| + |c| <= keep |b|
TDMA_DEV float certify_keep(float tol) { return 1.f - kRefineFloor / tol; }
// |a| + |c| - keep |b|: positive when the row is not dominant enough to certify the floor
TDMA_DEV float dom_excess(float a, float b, float c, float keep) { return fmaf(-keep, fabsf(b), fabsf(a) + fabsf(c)); }
// Stop rule of a line after a correction: |dx|, |x| and the previous |dx| (|x_0| after the first).
TDMA_DEV bool refine_done(float dxn, float xn, float prev, float tol, bool certified) {
  if (dxn == 0.f) return true;
  if (!certified) return dxn <= tol * xn;
  const float ratio = prev > 0.f ? dxn / prev : 0.f;
  return ratio * dxn <= tol * xn;
}

// Row i (or with TR the transposed row, as load_row) of the float coefficients and double d.
template <bool TR = false>
TDMA_DEV void load_coef(Coef& r, const Args& A, int64_t e, int64_t i) {
  if constexpr (TR) {
    r.a = i > 0 ? ldg((const float*)A.c + e - A.lay.es) : 0.f;
    r.c = i < A.lay.n - 1 ? ldg((const float*)A.a + e + A.lay.es) : 0.f;
  } else {
    r.a = ldg((const float*)A.a + e);
    r.c = ldg((const float*)A.c + e);
  }
  r.b = ldg((const float*)A.b + e);
  r.d = ldg((const double*)A.d + e);
}

// Extra-precise residual d - (a xm + b x0 + c xp) rounded to float.
TDMA_DEV float residual_ff(float a, float b, float c, ff dd, ff xm, ff x0, ff xp) {
  const ff p1 = two_prod(b, x0.h), p2 = two_prod(a, xm.h), p3 = two_prod(c, xp.h);
  const ff s1 = two_sum(dd.h, -p1.h);
  const ff s2 = two_sum(s1.h, -p2.h);
  const ff s3 = two_sum(s2.h, -p3.h);
  float err = dd.l - p1.l - p2.l - p3.l + s1.l + s2.l + s3.l;
  err = __fmaf_rn(-b, x0.l, err);
  err = __fmaf_rn(-a, xm.l, err);
  err = __fmaf_rn(-c, xp.l, err);
  return __fadd_rn(s3.h, err);
}

template <class BT, bool TR = false>
__global__ void __launch_bounds__(512) refine_kernel(const Args A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int T = blockDim.x, tid = threadIdx.x;
  const int P = A.P, Lb = A.Lb;
  const int j = tid % Lb, k = tid / Lb;
  const int64_t line = (int64_t)blockIdx.x * Lb + j;
  const bool active = line < A.lay.n_lines;
  const int mmax = A.mmax;
  const int slots = mmax > 2 ? mmax - 2 : 0;
  float* s_alpha = reinterpret_cast<float*>(smem_raw);
  float* s_gamma = s_alpha + (size_t)slots * T;
  float* s_delta = s_gamma + (size_t)slots * T;
  float* s_xh = s_delta + (size_t)slots * T;
  float* s_xl = s_xh + (size_t)mmax * T;
  const int R2 = 2 * P;
  const int pitch = 4 * R2 + 1;
  BT* red = reinterpret_cast<BT*>(s_xl + (size_t)mmax * T);
  BT* r_sub = red + (size_t)j * pitch;
  BT* r_cp = r_sub + R2;
  BT* r_iw = r_cp + R2;
  BT* r_rhs = r_iw + R2;
  unsigned* s_red = reinterpret_cast<unsigned*>(red + (size_t)Lb * pitch);  // per line: |dx| x2, |x| x2
  __shared__ int s_done;

  int64_t start = 0;
  int m = 0;
  partition(A.lay.n, P, k, start, m);
  const int64_t base = active ? A.lay.off(line) : 0;
  const int64_t es = A.lay.es;
  const bool single = (A.lay.n == 1);

  // neighbours' x slots: last row of partition k-1, first row of partition k+1
  const int prev_tid = tid - Lb, next_tid = tid + Lb;
  int mprev = 0;
  if (k > 0) { int64_t sp; partition(A.lay.n, P, k - 1, sp, mprev); }

  if (tid < Lb) {
    s_red[4 * tid + 0] = 0u; s_red[4 * tid + 1] = 0u; s_red[4 * tid + 2] = 0u; s_red[4 * tid + 3] = 0u;
  }
  // row-0 quantities that do not depend on the right-hand side
  float a0 = 0.f, b0 = 1.f, c0 = 0.f, rho = 1.f;
  float prev_dx = 0.f;  // line owner: |dx_{t-1}|
  bool line_done = !active;
  const float keep = certify_keep(A.tol);
  float dom = -INFINITY;  // max over this partition's rows of dom_excess
  bool certified = true;  // the block's rows certify the floor
  __syncthreads();

  int it = 0;
  for (;; ++it) {
    // ------------- Stage A (it == 0: factor and sweep fl(d); it > 0: sweep the residual)
    float F = 0.f, rhs0 = 0.f, rhs_last = 0.f, vsingle = 0.f;
    float alpha = -1.f, gamma = 0.f, delta = 0.f, G = 0.f, Q = 1.f;
    if (active) {
      ff xm, x0, xp;
      if (it > 0) {
        x0 = {s_xh[tid], s_xl[tid]};
        xm = (k > 0) ? ff{s_xh[(size_t)(mprev - 1) * T + prev_tid], s_xl[(size_t)(mprev - 1) * T + prev_tid]}
                     : ff{0.f, 0.f};
      }
      for (int t = 0; t < m; ++t) {
        Coef cf;
        load_coef<TR>(cf, A, base + (start + t) * es, start + t);
        if (k == 0 && t == 0) cf.a = 0.f;
        if (k == P - 1 && t == m - 1) cf.c = 0.f;
        if (it == 0) dom = fmaxf(dom, dom_excess(cf.a, cf.b, cf.c, keep));
        const ff dd = split_f64(cf.d);
        float rhs;
        if (it == 0) {
          rhs = __fadd_rn(dd.h, dd.l);
        } else {
          if (t + 1 < m) xp = {s_xh[(size_t)(t + 1) * T + tid], s_xl[(size_t)(t + 1) * T + tid]};
          else xp = (k < P - 1) ? ff{s_xh[next_tid], s_xl[next_tid]} : ff{0.f, 0.f};
          rhs = residual_ff(cf.a, cf.b, cf.c, dd, xm, x0, xp);
          xm = x0;
          x0 = xp;
        }
        if (t == 0) {
          a0 = cf.a; b0 = cf.b; c0 = cf.c;
          rhs0 = rhs;
          continue;
        }
        // gamma holds gamma_{t-1} (0 at t = 1); alpha/gamma of rows 1..m-2 come from pass 0
        const float r = rcp(cf.b - cf.a * gamma);
        const float ar = cf.a * r;
        if (it == 0) {
          alpha = -ar * alpha;
          gamma = cf.c * r;
        } else if (t <= m - 2) {
          gamma = s_gamma[(size_t)(t - 1) * T + tid];
        }
        delta = r * rhs - ar * delta;
        if (t <= m - 2) {
          const size_t o = (size_t)(t - 1) * T + tid;
          if (it == 0) {
            s_alpha[o] = alpha;
            s_gamma[o] = gamma;
            G += Q * alpha;
          }
          s_delta[o] = delta;
          F += Q * delta;
          Q = -Q * gamma;
        } else {
          rhs_last = delta;
        }
      }
      if (single) {
        // n == 1: b x = d handled directly
        vsingle = rhs0 * rcp(b0);
        if (it == 0) { s_xh[tid] = vsingle; s_xl[tid] = 0.f; }
        else { const ff nx = ff_add({s_xh[tid], s_xl[tid]}, vsingle); s_xh[tid] = nx.h; s_xl[tid] = nx.l; }
      } else {
        if (it == 0) {
          rho = rcp(b0 - c0 * G);
          r_sub[2 * k] = widen<BT>(rho * a0);
          r_cp[2 * k] = widen<BT>(rho * c0 * Q);
          r_sub[2 * k + 1] = widen<BT>(alpha);
          r_cp[2 * k + 1] = widen<BT>(gamma);
        }
        r_rhs[2 * k] = widen<BT>(rho * (rhs0 - c0 * F));
        r_rhs[2 * k + 1] = widen<BT>(rhs_last);
      }
    }
    if (__syncthreads_or(it == 0 && dom > 0.f)) certified = false;
    // ------------- Stage B
    if (!single && tid < Lb && (int64_t)blockIdx.x * Lb + tid < A.lay.n_lines) {
      BT* sub = red + (size_t)tid * pitch;
      const bool ok = (it == 0) ? reduced_factor_solve<BT>(sub, sub + R2, sub + 2 * R2, sub + 3 * R2, R2)
                                : reduced_resolve<BT>(sub, sub + R2, sub + 2 * R2, sub + 3 * R2, R2);
      if (!ok) report_error(A.st, 5);
    }
    __syncthreads();
    // ------------- Stage C: the correction (or first solution) and the norms of this pass
    if (active && !single) {
      float u0 = narrow(r_rhs[2 * k]), un = narrow(r_rhs[2 * k + 1]);
      float mdx = fmaxf(fabsf(u0), fabsf(un)), mx = 0.f;
      auto update = [&](int t, float v) {
        const size_t o = (size_t)t * T + tid;
        if (it == 0) { s_xh[o] = v; s_xl[o] = 0.f; mx = fmaxf(mx, fabsf(v)); }
        else { const ff nx = ff_add({s_xh[o], s_xl[o]}, v); s_xh[o] = nx.h; s_xl[o] = nx.l; mx = fmaxf(mx, fabsf(nx.h)); }
      };
      update(0, u0);
      update(m - 1, un);
      float v = un;
      for (int t = m - 2; t >= 1; --t) {
        const size_t o = (size_t)(t - 1) * T + tid;
        v = s_delta[o] - s_alpha[o] * u0 - s_gamma[o] * v;
        mdx = fmaxf(mdx, fabsf(v));
        update(t, v);
      }
      const int par = it & 1;
      atomicMax(&s_red[4 * j + 2 * par], __float_as_uint(mdx));
      atomicMax(&s_red[4 * j + 2 * par + 1], __float_as_uint(mx));
    } else if (active && single) {
      const int par = it & 1;
      atomicMax(&s_red[4 * j + 2 * par], __float_as_uint(fabsf(vsingle)));
      atomicMax(&s_red[4 * j + 2 * par + 1], __float_as_uint(fabsf(s_xh[tid])));
    }
    __syncthreads();
    // ------------- convergence test, one thread per line
    if (tid == 0) s_done = 1;
    __syncthreads();
    if (tid < Lb) {
      const int par = it & 1;
      const float mdx = __uint_as_float(s_red[4 * tid + 2 * par]);
      const float mx = __uint_as_float(s_red[4 * tid + 2 * par + 1]);
      s_red[4 * tid + 2 * (par ^ 1)] = 0u;
      s_red[4 * tid + 2 * (par ^ 1) + 1] = 0u;
      const bool live = (int64_t)blockIdx.x * Lb + tid < A.lay.n_lines;
      if (live && it > 0) {
        line_done = refine_done(mdx, mx, prev_dx, A.tol, certified);
      } else if (live) {
        line_done = (mx == 0.f);
      }
      if (live) prev_dx = mdx;
      if (!line_done) s_done = 0;
      if (live && !(finite(mdx) && finite(mx))) report_error(A.st, 5);
    }
    __syncthreads();
    if (s_done || it >= A.max_iters) break;
  }
  if (tid < Lb && (int64_t)blockIdx.x * Lb + tid < A.lay.n_lines) {
    report_iters(A.st, it);
    if (!line_done) report_error(A.st, 7);
  }
  // ------------- store x in FP64
  if (active) {
    for (int t = 0; t < m; ++t) {
      const size_t o = (size_t)t * T + tid;
      ((double*)A.x)[base + (start + t) * es] = ff_to_f64({s_xh[o], s_xl[o]});
    }
  }
}

}  // namespace tdma
