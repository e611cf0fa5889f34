// FP32 storage + refinement for lines spread over a thread-block cluster.
//
// The paper splits each system into slabs held by different GPUs (Section 2.1, Fig. 4): Stage A
// runs on every slab, the slabs' interface rows travel to the reduced solve (A2B), and the
// endpoint values travel back (B2C) for Stage C. Here a slab is one CTA of a cluster of C CTAs
// on C SMs, and the two exchanges are distributed-shared-memory (DSMEM) reads and writes:
//   - the cluster owns Lb = 32 adjacent lines; CTA r owns rows [r n/C, (r+1) n/C) of all of them,
//     split into PC partitions of M rows (thread tid = j + Lb k: line j, local partition k);
//   - one TMA copy per array brings the CTA's tile {32 lines, PC partitions, M rows} into
//     shared memory: 128-byte rows for float arrays, 256-byte rows for d;
//   - Stage B in two levels: each CTA reduces the 2 PC interface rows of each line to two rows
//     (level 1, one thread per line); CTA 0 gathers the 2C rows of each line from the cluster,
//     solves them and writes the endpoint values back (level 2, the A2B/B2C of the paper);
//   - per-line norms for the refinement test are max-reduced into CTA 0 and read back by all.
// Everything else (float modified-Thomas Stage A, extra-precise residual, float-pair x, TMA
// store of x) follows kernels_refine_tma.cuh.
#pragma once
#include <cooperative_groups.h>
#include "layout.cuh"
#include "tma.cuh"
#include "kernels_refine.cuh"

namespace tdma {

namespace cg = cooperative_groups;

template <int PC, int C>
struct ClusterRed {
  // per line (floats): level-1 rows sub/sup/rhs [2PC] and factors al/ga [2PC], row-0 fix rho;
  // published level-1 result (read by every CTA of the cluster): sub/sup [2] and rhs [2][2]
  // (double-buffered by pass parity); this CTA's copy of the level-2 system sub2/cp2/iw2/rhs2 [2C]
  static constexpr int R1 = 2 * PC, R2 = 2 * C;
  static constexpr int SUB = 0, SUP = R1, RHS = 2 * R1, AL = 3 * R1, GA = 4 * R1, RHO = 5 * R1;
  static constexpr int PSUB = 5 * R1 + 1, PSUP = PSUB + 2, PRHS = PSUP + 2;
  static constexpr int SUB2 = PRHS + 4, CP2 = SUB2 + R2, IW2 = CP2 + R2, RHS2 = IW2 + R2;
  static constexpr int GN = RHS2 + R2;  // gathered per-CTA maxima [C][2]
  static constexpr int PITCH = GN + R2 + 1;
};

template <int M, int PC, int C>
__host__ __device__ constexpr size_t refine_cluster_smem_bytes() {
  constexpr int T = 256, Lb = T / PC;
  // d tile (split into float pairs after the first read), a/b/c tiles, first-solution values
  // at partition ends, reduced systems, per-line norms [2][2]
  return (size_t)T * M * 8 + (size_t)T * M * 4 * 3 + (size_t)T * 2 * 4 + (size_t)Lb * ClusterRed<PC, C>::PITCH * 4 +
         (size_t)Lb * 4 * 4 + 128;
}

template <int M, int PC, int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(256, 2)
    refine_cluster_kernel(const Args A, const __grid_constant__ TmaMaps maps) {
  constexpr int T = 256, Lb = T / PC;
  using RL = ClusterRed<PC, C>;
  static_assert(Lb * PC == T, "geometry");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_done;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  const int j = tid % Lb, k = tid / Lb;
  const int64_t line0 = (int64_t)(blockIdx.x / C) * Lb;
  const int64_t lines_left = A.lay.n_lines - line0;
  const bool active = line0 + j < A.lay.n_lines;
  const int kg = rank * PC + k;  // partition index within the line
  const int Ptot = C * PC;

  unsigned char* p = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  double* t_d = reinterpret_cast<double*>(p);
  float* t_a = reinterpret_cast<float*>(t_d + T * M);
  float* t_b = t_a + T * M;
  float* t_c = t_b + T * M;
  float* s_ex = t_c + T * M;  // first solution at partition ends: [first | last] x T
  float* red = s_ex + 2 * T;
  unsigned* s_nrm = reinterpret_cast<unsigned*>(red + Lb * RL::PITCH);
  float* R = red + j * RL::PITCH;
  const float* ca = t_a + tid;
  const float* cb = t_b + tid;
  const float* cc = t_c + tid;
  const double* cd = t_d + tid;
  float2* cd2 = reinterpret_cast<float2*>(t_d) + tid;
  const int64_t es = A.lay.es;
  // this partition's rows of x in global memory (x between corrections after the first)
  double* px = (double*)A.x + A.lay.off(active ? line0 + j : A.lay.n_lines - 1) + (int64_t)kg * M * es;

  const int64_t ic = A.lay.ic;
  const int c_in = (int)(line0 % ic), c_out = (int)(line0 / ic);
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t fbytes = (uint32_t)T * M * 4;
    mbar_arrive_expect_tx(&bar, 5 * fbytes);
    tma_load_4d(t_a, &maps.a, &bar, c_in, c_out, rank * PC, 0);
    tma_load_4d(t_b, &maps.b, &bar, c_in, c_out, rank * PC, 0);
    tma_load_4d(t_c, &maps.c, &bar, c_in, c_out, rank * PC, 0);
    tma_load_4d(t_d, &maps.d, &bar, c_in, c_out, rank * PC, 0);
  }
  if (!mbar_wait_bounded(&bar, 0, kTmaWaitPolls)) report_error(A.st, 6);
  __syncthreads();

  const bool first_part = (kg == 0), last_part = (kg == Ptot - 1);
  float al[M], ga[M], de[M], xh[M];
  float a0 = 0.f, c0 = 0.f, rho = 1.f, prev_dx = 0.f;
  bool line_done = !active;
  const float keep = certify_keep(A.tol);
  float dom = -INFINITY;  // max over this partition's rows of dom_excess
  bool certified = true;  // line owner: every row of the line (all CTAs) certifies the floor
  const float* ex_prev = rank > 0 ? cluster.map_shared_rank(s_ex, rank - 1) : s_ex;
  const float* ex_next = rank < C - 1 ? cluster.map_shared_rank(s_ex, rank + 1) : s_ex;

  int it = 0;
  for (;; ++it) {
    const int par = it & 1;
    // ---------------- Stage A
    // x_{-1} and x_m of this partition: from the partition-end values of the first solution
    // (first correction) or from x in global memory (later corrections)
    ff pm{0.f, 0.f}, xn{0.f, 0.f};
    if (it == 1) {
      if (!first_part) pm.h = (k > 0) ? s_ex[T + tid - Lb] : ex_prev[T + tid + (PC - 1) * Lb];
      if (!last_part) xn.h = (k < PC - 1) ? s_ex[tid + Lb] : ex_next[tid - (PC - 1) * Lb];
    } else if (it > 1) {
      if (!first_part) pm = split_f64(px[-es]);
      if (!last_part) xn = split_f64(px[M * es]);
    }
    // x of this partition during a correction: the first solution in registers for the first
    // correction, x re-read from global memory for later ones
    auto xval = [&](int t) -> ff { return (it == 1) ? ff{xh[t], 0.f} : split_f64(px[t * es]); };
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
        cd2[t * T] = make_float2(dd.h, dd.l);  // same thread, same slot: read before write
        rhs = dd.h;
      } else {
        const float2 dd = cd2[t * T];
        const ff x0 = xval(t);
        const ff xp = (t + 1 < M) ? xval(t + 1 < M ? t + 1 : 0) : xn;
        rhs = residual_ff(a, b, c, ff{dd.x, dd.y}, pm, x0, xp);
        pm = x0;
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
      R[RL::SUB + 2 * k] = rho * a0;
      R[RL::SUP + 2 * k] = rho * c0 * Q;
      R[RL::SUB + 2 * k + 1] = alpha;
      R[RL::SUP + 2 * k + 1] = gamma;
    }
    R[RL::RHS + 2 * k] = rho * (rhs0 - c0 * F);
    R[RL::RHS + 2 * k + 1] = delta;
    __syncthreads();
    // ---------------- Stage B, level 1: the CTA's 2 PC rows of line j -> two published rows
    if (k == 0) {
      const float sub0 = R[RL::SUB], sup0 = R[RL::SUP], h0 = R[RL::RHS];
      float al1 = -1.f, ga1 = 0.f, de1 = 0.f, F1 = 0.f, G1 = 0.f, Q1 = 1.f;
#pragma unroll
      for (int t = 1; t < RL::R1; ++t) {
        const float sv = R[RL::SUB + t], h = R[RL::RHS + t];
        const float r = rcp(1.f - sv * ga1);
        const float ar = sv * r;
        if (it == 0) {
          al1 = -ar * al1;
          ga1 = R[RL::SUP + t] * r;
        }
        de1 = r * h - ar * de1;
        if (t <= RL::R1 - 2) {
          if (it == 0) {
            R[RL::AL + t] = al1;
            R[RL::GA + t] = ga1;
            G1 += Q1 * al1;
          } else {
            ga1 = R[RL::GA + t];
          }
          R[RL::RHS + t] = de1;
          F1 += Q1 * de1;
          Q1 = -Q1 * ga1;
        }
      }
      float rho1;
      if (it == 0) {
        rho1 = rcp(1.f - sup0 * G1);
        R[RL::RHO] = rho1;
        R[RL::PSUB] = rho1 * sub0;
        R[RL::PSUP] = rho1 * sup0 * Q1;
        R[RL::PSUB + 1] = al1;
        R[RL::PSUP + 1] = ga1;
      } else {
        rho1 = R[RL::RHO];
      }
      R[RL::PRHS + 2 * par] = rho1 * (h0 - sup0 * F1);
      R[RL::PRHS + 2 * par + 1] = de1;
    }
    cluster.sync();
    // ---------------- level 2, solved redundantly by every CTA: thread (j, q) fetches CTA q's
    // published rows of line j (one DSMEM read set per thread, all in flight together)
    if (k < C) {
      const float* Rq = cluster.map_shared_rank(red, k) + j * RL::PITCH;
      if (it == 0) {
        const float s0 = Rq[RL::PSUB], s1 = Rq[RL::PSUB + 1], p0 = Rq[RL::PSUP], p1 = Rq[RL::PSUP + 1];
        R[RL::SUB2 + 2 * k] = s0;
        R[RL::SUB2 + 2 * k + 1] = s1;
        R[RL::CP2 + 2 * k] = p0;
        R[RL::CP2 + 2 * k + 1] = p1;
      }
      const float h0 = Rq[RL::PRHS + 2 * par], h1 = Rq[RL::PRHS + 2 * par + 1];
      R[RL::RHS2 + 2 * k] = h0;
      R[RL::RHS2 + 2 * k + 1] = h1;
    }
    __syncthreads();
    if (k == 0 && j < lines_left) {
      const bool ok = (it == 0) ? reduced_factor_solve<float>(R + RL::SUB2, R + RL::CP2, R + RL::IW2, R + RL::RHS2, RL::R2)
                                : reduced_resolve<float>(R + RL::SUB2, R + RL::CP2, R + RL::IW2, R + RL::RHS2, RL::R2);
      if (!ok && rank == 0) report_error(A.st, 5);
      // level-1 back substitution with this CTA's endpoints
      const float v0 = R[RL::RHS2 + 2 * rank], vn = R[RL::RHS2 + 2 * rank + 1];
      R[RL::RHS] = v0;
      R[RL::RHS + RL::R1 - 1] = vn;
      float v = vn;
#pragma unroll
      for (int t = RL::R1 - 2; t >= 1; --t) {
        v = R[RL::RHS + t] - R[RL::AL + t] * v0 - R[RL::GA + t] * v;
        R[RL::RHS + t] = v;
      }
    }
    __syncthreads();
    // ---------------- Stage C and update
    const float u0 = R[RL::RHS + 2 * k], un = R[RL::RHS + 2 * k + 1];
    float mdx = fmaxf(fabsf(u0), fabsf(un)), mx = 0.f, v = un;
#pragma unroll
    for (int t = M - 1; t >= 0; --t) {
      const float xt = (t == M - 1) ? un : (t == 0 ? u0 : de[t] - al[t] * u0 - ga[t] * v);
      v = xt;
      if (t > 0 && t < M - 1) mdx = fmaxf(mdx, fabsf(xt));
      if (it == 0) {
        xh[t] = xt;
      } else {
        // corrected x goes straight to its final place (the answer if this was the last pass)
        const ff nx = ff_add(xval(t), xt);
        xh[t] = nx.h;
        if (active) px[t * es] = ff_to_f64(nx);
      }
      mx = fmaxf(mx, fabsf(xh[t]));
    }
    if (it == 0) {
      s_ex[tid] = xh[0];
      s_ex[T + tid] = xh[M - 1];
    }
    bool stop = (A.max_iters == 0);
    if (it > 0) {
      // per-line maxima of this CTA, published by parity; the decision uses all C CTAs' values
      if (Lb < 32) {
#pragma unroll
        for (int off = Lb; off < 32; off <<= 1) {
          mdx = fmaxf(mdx, __shfl_xor_sync(0xffffffffu, mdx, off));
          mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        }
      }
      if (tid < Lb) { s_nrm[4 * tid + 2 * par] = 0u; s_nrm[4 * tid + 2 * par + 1] = 0u; }
      __syncthreads();
      if ((tid & 31) < Lb || Lb >= 32) {
        atomicMax(&s_nrm[4 * j + 2 * par], __float_as_uint(mdx));
        atomicMax(&s_nrm[4 * j + 2 * par + 1], __float_as_uint(mx));
      }
      if (tid == 0) s_done = 1;
    } else {
      // the first correction always runs; keep |x_0| per line for the contraction estimate, and
      // whether the line's rows in this CTA certify the refinement's floor (word 3: 0 if they do)
      unsigned unc = __float_as_uint(fmaxf(dom, 0.f));
      if (Lb < 32) {
#pragma unroll
        for (int off = Lb; off < 32; off <<= 1) {
          mdx = fmaxf(mdx, __shfl_xor_sync(0xffffffffu, mdx, off));
          unc = max(unc, __shfl_xor_sync(0xffffffffu, unc, off));
        }
      }
      if (tid < Lb) { s_nrm[4 * tid + 2] = 0u; s_nrm[4 * tid + 3] = 0u; }
      __syncthreads();
      if ((tid & 31) < Lb || Lb >= 32) {
        atomicMax(&s_nrm[4 * j + 2], __float_as_uint(mdx));
        atomicMax(&s_nrm[4 * j + 3], unc);
      }
    }
    cluster.sync();  // endpoints and norms of every CTA visible
    // thread (j, q) fetches CTA q's maxima of line j; the line owner reduces them
    float* gn = R + RL::GN;
    if (k < C) {
      const unsigned* nq = cluster.map_shared_rank(s_nrm, k);
      if (it == 0) {
        gn[2 * k] = __uint_as_float(nq[4 * j + 2]);
        gn[2 * k + 1] = __uint_as_float(nq[4 * j + 3]);
      } else {
        const unsigned u0v = nq[4 * j + 2 * par], u1v = nq[4 * j + 2 * par + 1];
        gn[2 * k] = __uint_as_float(u0v);
        gn[2 * k + 1] = __uint_as_float(u1v);
      }
    }
    __syncthreads();
    if (it == 0) {
      if (tid < Lb) {
        float m0 = 0.f;
        unsigned u = 0u;
#pragma unroll
        for (int q = 0; q < C; ++q) {
          m0 = fmaxf(m0, gn[2 * q]);
          u = max(u, __float_as_uint(gn[2 * q + 1]));
        }
        prev_dx = m0;
        certified = (u == 0u);
      }
      if (stop) break;
      continue;
    }
    if (tid < Lb) {
      float dxn = 0.f, xn = 0.f;
#pragma unroll
      for (int q = 0; q < C; ++q) {
        dxn = fmaxf(dxn, gn[2 * q]);
        xn = fmaxf(xn, gn[2 * q + 1]);
      }
      if (tid < lines_left) {
        line_done = refine_done(dxn, xn, prev_dx, A.tol, certified);
        prev_dx = dxn;
        if (rank == 0 && !(finite(dxn) && finite(xn))) report_error(A.st, 5);
        if (!line_done) s_done = 0;
      }
    }
    __syncthreads();
    if (s_done || it >= A.max_iters) break;
  }
  if (rank == 0 && tid < Lb && tid < lines_left) {
    report_iters(A.st, it);
    if (!line_done && A.max_iters > 0) report_error(A.st, 7);
  }
  // without any correction the float solution is the answer (a warp stores 256 contiguous bytes)
  if (it == 0 && active) {
#pragma unroll
    for (int t = 0; t < M; ++t) px[t * es] = f2d(xh[t]);
  }
  cluster.sync();  // no CTA leaves while others may still read its shared memory
}

// compiled cluster geometries: (rows per partition M, partitions per CTA PC, cluster size C);
// one line spans n = C PC M rows.
#define TDMA_REFINE_CLUSTER_SHAPES(X) X(16, 8, 8) X(16, 8, 4) X(16, 8, 2)

}  // namespace tdma
