// FP32 storage + refinement with each line spread over a thread-block cluster; Stage B as a
// log-depth merge tree over warp lanes and then over the cluster's CTAs.
//
// Geometry. A cluster of C CTAs owns 32 adjacent lines. CTA r holds rows [r n/C, (r+1) n/C) of
// all of them as 8 partitions of M rows (n = 8 C M). Warp w holds lines 4w..4w+3 and lane
// 4p + jj holds partition p of line 4w + jj: the 8 partitions of a line sit in 8 lanes of one
// warp, so the CTA-level part of the reduced solve needs shuffles only, no CTA barrier.
// The tile {32 lines, 8 partitions, M rows} of a, b, c (float) and d (double, two boxes of 16
// lines) arrives by TMA with the 128-byte swizzle: for a fixed row, the 32 lanes of a warp then
// read 32 distinct banks.
//
// Stage A (Section 2.1, Algorithm 1) per partition is the modified Thomas sweep used by the other
// kernels; it leaves, for the partition's first and last unknowns x_s and x_e, the two rows
//     x_s + S u + U x_e = H,        alpha x_s + x_e + Gamma v = Delta,
// with u = x_{s-1} and v = x_{e+1} the outside neighbours. Solving the 2 x 2 system gives the
// block form  x_s = p1 + q1 u + r1 v,  x_e = p2 + q2 u + r2 v.  Two adjacent blocks L, R merge
// into one by eliminating the unknowns on either side of their boundary, y = x_{e(L)} and
// z = x_{s(R)}:  y = L.p2 + L.q2 u + L.r2 z,  z = R.p1 + R.q1 y + R.r1 v.  Three merge levels
// over the lanes of a line give the CTA's block (the paper's A2B); each CTA pushes it into the
// shared memory of every CTA of the cluster (DSMEM stores), waits for the others', and every CTA
// merges the C blocks of the line the same way. The line ends have no outside neighbours
// (u = v = 0), so the down-sweep of the two trees hands every partition its own u and v (the
// paper's B2C), and Stage C is x_t = delta_t - alpha_t x_s - gamma_t x_{t+1}.
//
// Refinement (the FP32 + refinement path): pass 0 solves with the float part of d; pass 1
// recomputes the same factors and solves for the extra-precise residual r = d - A x_0 (float
// pairs); x = x_0 + dx goes to global memory in FP64. The stop rule (per line, on the line's
// max norms) compares the line's max |dx| with a bound made of its max |x_0|, which the pass-1
// exchange already brings to every CTA: so each CTA takes the rule on its own rows, and the line
// meets it exactly when every CTA's rows do. Out of place, the per-line flags of a group travel
// with the next group's pass-0 exchange (the cluster's last group has one exchange of its own),
// and a group that needs further corrections (rare) gets them then, from global memory; in place
// (x is d) the rule takes one exchange of the line maxima and the corrections follow at once.
// Later passes re-read x from global memory.
// Exchanges are point to point (st.async into the other CTAs' shared memory, completing on
// their mbarriers): a CTA waits only for the data it needs, never for another CTA's threads, and
// the block exchanges have one mbarrier per warp, so that a warp waits only for its own 4 lines
// (warp w of every CTA of the cluster holds the same lines), not for the CTA's other warps.
#pragma once
#include <cooperative_groups.h>
#include "layout.cuh"
#include "tma.cuh"
#include "kernels_refine.cuh"
#include "kernels_refine_tma.cuh"  // kTmaWaitPolls
#include "merge_tree.cuh"
#include "bits.cuh"

namespace tdma {

constexpr int kTreeLines = 32;               // lines per cluster
constexpr int kTreeParts = 8;                // partitions per CTA
constexpr int kTreeSlotPitch = 32 * 8 + 4;   // per source CTA: 32 lines x 8 floats (+4: banks)
constexpr int kTreeNormPitch = 32 * 2 + 4;   // per source CTA: 32 lines x 2 words
// Polls of an exchange wait (about 6 ms with the back-off of mbar_wait_bounded; a tile's CTAs
// live for tens of microseconds). After one wait gives up the thread stops waiting for the rest
// of the tile, but it still sends everything, so its peers are not held up and no CTA leaves
// while others may still store into its shared memory.
constexpr uint32_t kTreeWaitPolls = 1u << 16;

TDMA_DEV void tree_wait(uint64_t* bar, uint32_t phase, bool& alive, DevStatus* st) {
  if (!alive) return;
  if (!mbar_wait_bounded(bar, phase, kTreeWaitPolls)) {
    alive = false;
    report_error(st, 6);
  }
}

// maximum over the 8 lanes (bits 2..4 of the lane index) that hold one line
TDMA_DEV unsigned line_max(unsigned v) {
#pragma unroll
  for (int l = 0; l < 3; ++l) v = max(v, __shfl_xor_sync(~0u, v, 4 << l));
  return v;
}

template <int M, int C>
__host__ __device__ constexpr size_t refine_tree_smem_bytes() {
  // a, b, c tiles (M x 8 x 32 floats each), d (two M x 8 x 16 double boxes), block slots and
  // norm slots (double-buffered by pass parity), 1 KB for the swizzle alignment
  return 1024 + 5 * (size_t)M * 1024 + 2 * (size_t)C * kTreeSlotPitch * 4 + 2 * (size_t)C * kTreeNormPitch * 4;
}

// Stage B for one pass: CTA tree, exchange of the CTA blocks, cluster tree, down-sweeps.
// The exchange is point to point: lane p sends this CTA's block of line j (and `extra`, a
// per-line norm of this CTA as abs_bits) into slot [rank][j] of CTA p with st.async, which
// completes on CTA p's mbarrier bar[w] of this buffer (w: the warp, whose 4 lines are the same in
// every CTA); warp w waits on its own bar[w] for the C x 4 slots of its lines (phase `phase`), so
// no warp waits for other threads, only for the data of its lines.
// `extra_max` is the maximum of `extra` over the cluster. Returns this partition's (u, v) and
// this CTA's first and last unknowns of the line as the neighbouring CTAs see them (every CTA
// computes the cluster tree from the same data in the same order, so the values agree bit for
// bit).
// `extra2` (with F2) rides in the slot's last word the same way: its maximum over the cluster comes
// back in extra2_max.
template <int C, bool F2 = false>
TDMA_DEV void tree_stage_b(const Blk& b, unsigned extra, float* slots, uint64_t* bar, uint32_t phase, int rank, int p,
                           int jj, int j, float& u, float& v, float& xs_c, float& xe_c, unsigned& extra_max,
                           bool& alive, DevStatus* st, unsigned extra2 = 0u, unsigned* extra2_max = nullptr) {
  constexpr int LC = C == 8 ? 3 : (C == 4 ? 2 : 1);
  Aff kc[3];
  const Blk B = tree_up<3>(b, p, kc);
  bar += threadIdx.x >> 5;  // this warp's barrier: its 4 lines from every CTA
  if ((threadIdx.x & 31) == 0) mbar_arrive_expect_tx(bar, (uint32_t)C * 4u * 32u);
  if (p < C) {
    const uint32_t dst = map_rank(slots + rank * kTreeSlotPitch + j * 8, p), rb = map_rank(bar, p);
    st_async4(dst, B.p1, B.q1, B.r1, B.p2, rb);
    st_async4(dst + 16, B.q2, B.r2, __uint_as_float(extra), __uint_as_float(extra2), rb);
  }
  tree_wait(bar, phase, alive, st);
  const float4* s = reinterpret_cast<const float4*>(slots + (p & (C - 1)) * kTreeSlotPitch + j * 8);
  const float4 s0 = s[0], s1 = s[1];
  extra_max = line_max(__float_as_uint(s1.z));
  if constexpr (F2) *extra2_max = line_max(__float_as_uint(s1.w));
  float uq = 0.f, vq = 0.f, xsq = 0.f, xeq = 0.f;
  {
    Mrg kq[3];
    tree_up_full<LC>(Blk{s0.x, s0.y, s0.z, s0.w, s1.x, s1.y}, p, kq);
    tree_down_full<LC>(uq, vq, xsq, xeq, p, kq);  // the line ends have u = v = 0
  }
  const int src = (rank << 2) | jj;
  u = __shfl_sync(~0u, uq, src);
  v = __shfl_sync(~0u, vq, src);
  xs_c = __shfl_sync(~0u, xsq, src);
  xe_c = __shfl_sync(~0u, xeq, src);
  tree_down<3>(u, v, p, kc);
}

// Per-line maxima over the cluster, in two halves so that work can go between sending and
// waiting: send this CTA's (dx, xm) of line j (already reduced over the line's lanes) to every
// CTA; then wait for the C sources and reduce.
template <int C>
TDMA_DEV void tree_norms_push(unsigned dx, unsigned xm, unsigned* norms, uint64_t* bar, int rank, int p, int j) {
  if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, (uint32_t)C * kTreeLines * 8u);
  if (p < C) st_async2(map_rank(norms + rank * kTreeNormPitch + j * 2, p), dx, xm, map_rank(bar, p));
}
template <int C>
TDMA_DEV void tree_norms_read(unsigned& dx, unsigned& xm, const unsigned* norms, uint64_t* bar, uint32_t phase, int p,
                              int j, bool& alive, DevStatus* st) {
  tree_wait(bar, phase, alive, st);
  const uint2 v = *reinterpret_cast<const uint2*>(norms + (p & (C - 1)) * kTreeNormPitch + j * 2);
  dx = line_max(v.x);
  xm = line_max(v.y);
}

// Stage A state of one partition of M rows (modified Thomas, row-1 relation summed forward).
template <int M>
struct Sweep {
  float al[M], ga[M], de[M];  // rows 1..M-2
  float alpha = -1.f, gamma = 0.f, delta = 0.f, F = 0.f, G = 0.f, Q = 1.f;
  float a0 = 0.f, b0 = 1.f, c0 = 0.f, h0 = 0.f;
  // row t (a compile-time constant after unrolling) with right-hand side rhs
  TDMA_DEV void row(int t, float a, float b, float c, float rhs) {
    if (t == 0) {
      a0 = a; b0 = b; c0 = c; h0 = rhs;
      return;
    }
    const float r = rcp(fmaf(-a, gamma, b));
    const float ar = a * r;
    alpha = -ar * alpha;
    gamma = c * r;
    delta = fmaf(r, rhs, -ar * delta);
    if (t <= M - 2) {
      al[t] = alpha; ga[t] = gamma; de[t] = delta;
      G = fmaf(Q, alpha, G);
      F = fmaf(Q, delta, F);
      Q = -Q * gamma;
    }
  }
  // Row t of a further solve with the same matrix: alpha and gamma of the interior rows (and of
  // the last row, in alpha / gamma) and G stay from the first solve; delta, F and Q are redone.
  TDMA_DEV void row_rhs(int t, float a, float b, float rhs) {
    if (t == 0) {
      h0 = rhs;
      delta = 0.f;
      F = 0.f;
      Q = 1.f;
      return;
    }
    const float r = rcp(fmaf(-a, t >= 2 ? ga[t >= 2 ? t - 1 : 1] : 0.f, b));  // pivot of row t
    delta = fmaf(r, rhs, -(a * r) * delta);
    if (t <= M - 2) {
      de[t] = delta;
      F = fmaf(Q, delta, F);
      Q = -Q * ga[t];
    }
  }
  // row 0 becomes x_s + S u + U x_e = H with x_1 = F - G x_s + Q x_e substituted
  TDMA_DEV Blk block() const {
    const float rho = rcp(fmaf(-c0, G, b0));
    return part_block(rho * a0, rho * (c0 * Q), rho * fmaf(-c0, F, h0), alpha, gamma, delta);
  }
  // the partition's first and last unknowns for its outside neighbours (u, v)
  TDMA_DEV static float first(const Blk& b, float u, float v) { return fmaf(b.q1, u, fmaf(b.r1, v, b.p1)); }
  TDMA_DEV static float last(const Blk& b, float u, float v) { return fmaf(b.q2, u, fmaf(b.r2, v, b.p2)); }
  // Stage C handing each row's value to f(t, x_t), from row M-1 down to row 0
  template <class Fn>
  TDMA_DEV void solve_visit(float xs, float xe, Fn&& f) const {
    f(M - 1, xe);
    float xn = xe;
#pragma unroll
    for (int t = M - 2; t >= 1; --t) {
      xn = fmaf(-ga[t], xn, fmaf(-al[t], xs, de[t]));
      f(t, xn);
    }
    f(0, xs);
  }
  // Stage C from the partition's first and last unknowns
  TDMA_DEV void solve(float xs, float xe, float (&x)[M]) const {
    x[0] = xs;
    x[M - 1] = xe;
    float xn = xe;
#pragma unroll
    for (int t = M - 2; t >= 1; --t) {
      xn = fmaf(-ga[t], xn, fmaf(-al[t], xs, de[t]));
      x[t] = xn;
    }
  }
};

// Per-line stop rule of the refinement (refine_done): for a line whose rows certify the float-pair
// residual's floor, rho |dx|_inf <= tol |x|_inf with the contraction estimate rho = |dx| / |dx_prev|
// (|dx_0| = |x_0|); for another line |dx|_inf <= tol |x|_inf. A non-finite norm ends the line with
// status 5.
TDMA_DEV bool tree_line_done(unsigned gdx, unsigned gxm, unsigned& prev, bool active, float tol, bool certified,
                             bool reporter, DevStatus* st) {
  if (!active) return true;
  if (!(bits_finite(gdx) && bits_finite(gxm))) {
    if (reporter) report_error(st, 5);
    return true;
  }
  const float pv = __uint_as_float(prev);
  prev = gdx;
  return refine_done(__uint_as_float(gdx), __uint_as_float(gxm), pv, tol, certified);
}

// One thread loads a group's tile. Lines along a strided axis: the M rows of a, b, c (float) and d
// (double, two boxes of 16 lines) arrive on bar[0], 5 KB per row, one box per array (a wait part
// way through the row loop, for a second half of the rows, kept the compiler from moving shared
// loads ahead across it and cost more than it overlapped). Unit-stride
// lines (XL): the CTA's 8 M rows of the 32 lines, a, b and c in boxes of 32 rows and d in boxes of
// 16 rows (each box 128 bytes of every line, 4 KB), all on bar[0]; `parts` selects a, b and c (1),
// d (2) or both (3), and `arrive` whether this call also arrives on bar[0] (without it, the copies
// count towards a phase whose arrival comes later).
template <int M, bool XL>
TDMA_DEV void tree_load_tiles(const TmaMaps& maps, float* ta, float* tb, float* tc, double* td, uint64_t* bar, int c_in,
                              int c_out, int c_p, int parts = 3, bool arrive = true) {
  if constexpr (!XL) {
    mbar_arrive_expect_tx(&bar[0], 5u * M * 1024u);
    tma_load_4d(ta, &maps.a, &bar[0], c_in, c_out, c_p, 0);
    tma_load_4d(tb, &maps.b, &bar[0], c_in, c_out, c_p, 0);
    tma_load_4d(tc, &maps.c, &bar[0], c_in, c_out, c_p, 0);
    tma_load_4d(td, &maps.d, &bar[0], c_in, c_out, c_p, 0);
    tma_load_4d(td + M * 128, &maps.d, &bar[0], c_in + 16, c_out, c_p, 0);
  } else {
    const int r0 = c_p * M;  // the CTA's first row (c_p = rank x 8 partitions)
    const uint32_t bytes = ((parts & 1) ? 3u * M * 1024u : 0u) + ((parts & 2) ? 2u * M * 1024u : 0u);
    if (arrive) mbar_arrive_expect_tx(&bar[0], bytes);
    else mbar_expect_tx(&bar[0], bytes);
    if (parts & 1) {
#pragma unroll
      for (int i = 0; i < M / 4; ++i) {
        tma_load_3d(ta + i * 1024, &maps.a, &bar[0], r0 + 32 * i, c_in, c_out);
        tma_load_3d(tb + i * 1024, &maps.b, &bar[0], r0 + 32 * i, c_in, c_out);
        tma_load_3d(tc + i * 1024, &maps.c, &bar[0], r0 + 32 * i, c_in, c_out);
      }
    }
    if (parts & 2) {
#pragma unroll
      for (int i = 0; i < M / 2; ++i) tma_load_3d(td + i * 512, &maps.d, &bar[0], r0 + 16 * i, c_in, c_out);
    }
  }
}

// Persistent: the grid holds the clusters that fit on the GPU at once, and cluster k takes line
// groups k, k + K, k + 2K, ... (K clusters). The next group's tiles are loaded while the current
// group is still in its second half (after the pass-1 exchange: Stage C, the x store, the norm
// exchange and the verdict): x goes from registers to global memory, so the tiles are dead once
// pass 1 has formed its residual, and the rare later corrections read their operands from global
// memory. A solve in place (x is d) cannot read d back from global memory after x went out, so it
// keeps the tiles for the later corrections: x leaves through the a and b tiles by TMA store, the
// next group's tiles load at its top, and a later correction reloads a and b and takes c and the
// d pairs from the tiles.
//
// XL: lines with unit element stride (rows contiguous in memory). The CTA's rows of the 32 lines
// arrive as boxes of 128 bytes per line with the 128-byte swizzle (a, b, c: 32 rows; d: 16 rows),
// so that partition p of line j reads rows 4q..4q+3 of a, b and c as one 16-byte word at chunk
// (4 (p mod 2) + q) XOR (j mod 8) of box p / 2, and rows 2q, 2q + 1 of d at chunk q XOR (j mod 8)
// of box p: the 8 lanes of each quarter-warp access of a, b and c then cover the 32 banks, and d
// costs two wavefronts per quarter. A thread's x rows are contiguous in memory but 8 KB apart from
// its lane neighbours', so x goes out through the d tile (the thread's own d slots) by TMA store;
// the next group's a, b and c tiles load early, its d tile as soon as the store has read it.
template <int M, int C, bool XL>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(256, 2)
    refine_tree_kernel(const Args A, const __grid_constant__ TmaMaps maps) {
  static_assert(C == 2 || C == 4 || C == 8, "cluster size");
  static_assert(M >= 4 && M % 2 == 0, "rows per partition");
  static_assert(!XL || M == 16, "unit-stride tiles: a partition is half of a 32-row box");
  extern __shared__ __align__(16) unsigned char smem_raw[];  // aligned to 1 KB below
  // tile mbarrier: the whole tile of a group arrives on bar[0]
  __shared__ __align__(8) uint64_t bar[1];
  // exchange mbarriers: wbar[q][w] the block slots of warp w's lines in even (q = 0) / odd passes,
  // nbar[q] the norm slots
  __shared__ __align__(8) uint64_t wbar[2][8];
  __shared__ __align__(8) uint64_t nbar[2];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, p = lane >> 2, jj = lane & 3;
  const int j = 4 * w + jj;  // line within the cluster's 32
  const int rank = (int)cluster_rank();
  const int kg = rank * kTreeParts + p;  // partition index within the line
  const bool first_part = kg == 0, last_part = kg == C * kTreeParts - 1;
  const int64_t n_groups = (A.lay.n_lines + kTreeLines - 1) / kTreeLines;
  const int64_t n_clusters = gridDim.x / C;

  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  float* ta = reinterpret_cast<float*>(base);
  float* tb = ta + M * 256;
  float* tc = tb + M * 256;
  double* td = reinterpret_cast<double*>(tc + M * 256);
  float* slots = reinterpret_cast<float*>(td + M * 256);
  unsigned* norms = reinterpret_cast<unsigned*>(slots + 2 * C * kTreeSlotPitch);
  float2* td2 = reinterpret_cast<float2*>(td);  // d as float pairs, written in place by pass 0
  // Element of row t of this thread's partition in the a, b, c tiles (fidx) and in the d tile
  // (didx). Strided lines: the 128-byte swizzle (16-byte chunk index XOR 128-byte row index mod
  // 8, the row index mod 8 being the partition p), row t 1 KB further. XL: see the kernel header.
  const int j7 = j & 7;
  const int fo = XL ? ((p >> 1) << 10) + (j << 5) : p * 32 + (((w ^ p) & 7) << 2) + jj;
  const int fx = ((p & 1) << 2) ^ j7;  // XL: rows 4q..4q+3 of a, b, c are in chunk fx ^ q
  const int dof = XL ? (p << 9) + (j << 4)
                     : (w >> 2) * (M * 128) + p * 16 + ((((w & 3) * 2 + (jj >> 1)) ^ p) << 1) + (jj & 1);
  auto fidx = [&](int t) { return XL ? fo + ((fx ^ (t >> 2)) << 2) + (t & 3) : fo + t * 256; };
  auto didx = [&](int t) { return XL ? dof + (((t >> 1) ^ j7) << 1) + (t & 1) : dof + t * 128; };
  // x leaves from registers to global memory, or by TMA store from the thread's d slots (XL) or,
  // in place, from the a and b tiles (32 KB, the layout of the d tile)
  const bool inplace = A.x == A.d;
  double* const tx = (XL && !inplace) ? td : reinterpret_cast<double*>(ta);
  const int64_t es = A.lay.es, ic = A.lay.ic;
  const float keep = certify_keep(A.tol);

  if (tid == 0) {
    mbar_init(&bar[0], 1);
#pragma unroll
    for (int i = 0; i < 16; ++i) mbar_init(&wbar[i >> 3][i & 7], 1);
    mbar_init(&nbar[0], 1);
    mbar_init(&nbar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // the barriers are initialised and this CTA runs; the matching wait precedes the first
  // store into another CTA's shared memory
  cluster_arrive();
  bool started = false, alive = true;
  uint32_t tph0 = 0, xph0 = 0, xph1 = 0, xph2 = 0, xph3 = 0;  // phases of bar[0], wbar[0..1][w], nbar[0..1]
  // Out of place, the stop rule of a group is settled one group later (see below), from what this
  // thread keeps of its line in the cluster's previous group: this CTA's max |dx| of the line in
  // pndx (bits 0..30; bit 31: the line failed the rule on this CTA's rows), the group's certificate,
  // and the line's flag over the cluster once the next pass-0 exchange has brought it (pfl).
  bool pcert = false;
  unsigned pndx = 0u, pfl = 0u;

  // Further corrections of group gg (rare): a fresh float solve of the residual per pass, operands
  // from global memory (out of place the tiles hold another group's rows by then); in place, a and
  // b reloaded into their tiles (which held the outgoing x) and c and the d pairs from the tiles.
  // Every CTA of the cluster runs the same passes (the decision is the cluster's). prevd is the
  // line's previous max |dx| (the ratio of the rule). Reports the corrections made and, for a line
  // still short of the rule after max_iters, TDMA_ERR_NOT_CONVERGED.
  auto later = [&](int64_t gg, bool cert, unsigned prevd, bool line_done, bool all_done) {
    const int64_t l0 = gg * kTreeLines;
    const bool act = l0 + j < A.lay.n_lines;
    const bool rep = rank == 0 && p == 0 && act;
    const int64_t eo = A.lay.off(act ? l0 + j : 0) + (int64_t)kg * M * es;
    double* pxg = (double*)A.x + eo;
    const int ci = (int)(l0 % ic), co = (int)(l0 / ic), cp = rank * kTreeParts;
    const float* ga = (const float*)A.a + eo;
    const float* gb = (const float*)A.b + eo;
    const float* gc = (const float*)A.c + eo;
    const double* gd = (const double*)A.d + eo;
    int it = 1;
    while (!all_done && it < A.max_iters) {
      ++it;
      if (tid == 0 && (XL || inplace)) {
        bulk_wait_all();  // x of the last pass is in global memory
        fence_proxy_async_global();
      }
      if (inplace) {
        if (tid == 0) {
          mbar_arrive_expect_tx(&bar[0], 2u * M * 1024u);  // a and b again (x went through their tiles)
          if constexpr (XL) {
#pragma unroll
            for (int i = 0; i < M / 4; ++i) {
              tma_load_3d(ta + i * 1024, &maps.a, &bar[0], cp * M + 32 * i, ci, co);
              tma_load_3d(tb + i * 1024, &maps.b, &bar[0], cp * M + 32 * i, ci, co);
            }
          } else {
            tma_load_4d(ta, &maps.a, &bar[0], ci, co, cp, 0);
            tma_load_4d(tb, &maps.b, &bar[0], ci, co, cp, 0);
          }
        }
        if (!mbar_wait_bounded(&bar[0], tph0, kTmaWaitPolls) && alive) {
          alive = false;
          report_error(A.st, 6);
        }
        tph0 ^= 1u;
      }
      cluster_arrive();  // x of the previous pass, written by every CTA, visible to all
      cluster_wait();
      Sweep<M> S;
      ff xm{0.f, 0.f}, xc{0.f, 0.f}, xe{0.f, 0.f};
      if (act) {
        if (!first_part) xm = split_f64(pxg[-es]);
        if (!last_part) xe = split_f64(pxg[M * es]);
        xc = split_f64(pxg[0]);
      }
#pragma unroll
      for (int t = 0; t < M; ++t) {
        float a = 0.f, b = 1.f, c = 0.f;
        ff dd{0.f, 0.f};
        if (inplace) {
          a = ta[fidx(t)];
          b = tb[fidx(t)];
          c = tc[fidx(t)];
          const float2 dp = td2[didx(t)];
          dd = ff{dp.x, dp.y};
        } else if (act) {
          a = ga[t * es];
          b = gb[t * es];
          c = gc[t * es];
          dd = split_f64(gd[t * es]);
        }
        if (t == 0 && first_part) a = 0.f;
        if (t == M - 1 && last_part) c = 0.f;
        const ff xn = t == M - 1 ? xe : (act ? split_f64(pxg[(t + 1) * es]) : ff{0.f, 0.f});
        S.row(t, a, b, c, residual_ff(a, b, c, dd, xm, xc, xn));
        xm = xc;
        xc = xn;
      }
      const Blk blk = S.block();
      float u, v, xs_c, xe_c;
      unsigned unused;
      // pass `it` uses the buffers of its parity; the phase counters follow each mbarrier
      const int q = it & 1;
      tree_stage_b<C>(blk, 0u, slots + q * C * kTreeSlotPitch, wbar[q], (q ? xph1 : xph0) & 1u, rank, p, jj, j, u, v,
                      xs_c, xe_c, unused, alive, A.st);
      if (q) ++xph1; else ++xph0;
      float dx[M];
      S.solve(Sweep<M>::first(blk, u, v), Sweep<M>::last(blk, u, v), dx);
      unsigned ndx = 0u, nxm = 0u;
      if (act) {
#pragma unroll
        for (int t = 0; t < M; ++t) {
          const double xn = pxg[t * es] + f2d(dx[t]);
          pxg[t * es] = xn;
          ndx = max(ndx, abs_bits(dx[t]));
          nxm = max(nxm, abs_bits(__double2float_rn(xn)));
        }
      }
      unsigned* nb = norms + q * C * kTreeNormPitch;
      unsigned gdx, gxm;
      tree_norms_push<C>(line_max(ndx), line_max(nxm), nb, &nbar[q], rank, p, j);
      tree_norms_read<C>(gdx, gxm, nb, &nbar[q], (q ? xph3 : xph2) & 1u, p, j, alive, A.st);
      if (q) ++xph3; else ++xph2;
      line_done = tree_line_done(gdx, gxm, prevd, act, A.tol, cert, rep, A.st);
      all_done = __syncthreads_and(line_done) != 0;
    }
    if (rep) {
      report_iters(A.st, it);
      if (!line_done) report_error(A.st, 7);
    }
  };
  // Out of place: the previous group gg failed the rule on some line (pflag: this thread's line's
  // flag over the cluster). Every CTA of the cluster comes here at the same point.
  auto settle = [&](unsigned pflag, int64_t gg) {
    cluster_arrive();  // every CTA is past its reads of the norm slots
    cluster_wait();
    if (A.max_iters <= 1) {
      if (rank == 0 && p == 0 && pflag != 0u) report_error(A.st, 7);
      return;
    }
    unsigned gdx1, unused;  // the line's max |dx| of pass 1 of group gg
    tree_norms_push<C>(pndx & 0x7FFFFFFFu, 0u, norms + C * kTreeNormPitch, &nbar[1], rank, p, j);
    tree_norms_read<C>(gdx1, unused, norms + C * kTreeNormPitch, &nbar[1], xph3 & 1u, p, j, alive, A.st);
    ++xph3;
    later(gg, pcert, gdx1, pflag == 0u, false);
  };

  for (int64_t g = blockIdx.x / C; g < n_groups; g += n_clusters) {
    const int64_t line0 = g * kTreeLines;
    const bool active = line0 + j < A.lay.n_lines;
    const bool reporter = rank == 0 && p == 0 && active;  // one thread per line reports
    const int64_t eoff = A.lay.off(active ? line0 + j : 0) + (int64_t)kg * M * es;  // this partition's row 0
    double* px = (double*)A.x + eoff;
    const int c_in = (int)(line0 % ic), c_out = (int)(line0 / ic), c_p = rank * kTreeParts;
    // every group after the cluster's first came in during the previous group (XL: its a, b and
    // c), unless in place
    const bool first_group = g == (int64_t)(blockIdx.x / C);
    if (tid == 0 && (inplace || first_group)) {
      bulk_wait_read_all();  // the previous group's x store has read the tile it went through
      tree_load_tiles<M, XL>(maps, ta, tb, tc, td, bar, c_in, c_out, c_p, (inplace || first_group) ? 3 : 2);
    }
    if (!mbar_wait_bounded(&bar[0], tph0, kTmaWaitPolls) && alive) {
      alive = false;
      report_error(A.st, 6);
    }
    tph0 ^= 1u;

    // ---------------- pass 0: float solve with the float part of d
    float x0[M];
    float u0, v0;
    unsigned nx;
    bool certified;  // the line's rows (all CTAs) certify the floor of the float-pair residual
    Sweep<M> S;  // its factors serve pass 1 as well (same matrix)
    {
      float dom = -INFINITY;  // max over this partition's rows of dom_excess
      if constexpr (XL) {
#pragma unroll
        for (int q = 0; q < M / 4; ++q) {  // rows 4q..4q+3
          const int f4 = fo + ((fx ^ q) << 2), d0 = dof + (((2 * q) ^ j7) << 1), d1 = dof + (((2 * q + 1) ^ j7) << 1);
          const float4 a4 = *reinterpret_cast<const float4*>(ta + f4);
          const float4 b4 = *reinterpret_cast<const float4*>(tb + f4);
          const float4 c4 = *reinterpret_cast<const float4*>(tc + f4);
          const double2 e0 = *reinterpret_cast<const double2*>(td + d0);
          const double2 e1 = *reinterpret_cast<const double2*>(td + d1);
          const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
          const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
          const double dv[4] = {e0.x, e0.y, e1.x, e1.y};
          ff sp[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int t = 4 * q + u;
            float a = av[u], c = cv[u];
            if (t == 0 && first_part) a = 0.f;
            if (t == M - 1 && last_part) c = 0.f;
            dom = fmaxf(dom, dom_excess(a, bv[u], c, keep));
            sp[u] = split_f64_fast(dv[u]);
            S.row(t, a, bv[u], c, sp[u].h);
          }
          // same thread, same 16 bytes: read before write
          *reinterpret_cast<float4*>(td + d0) = make_float4(sp[0].h, sp[0].l, sp[1].h, sp[1].l);
          *reinterpret_cast<float4*>(td + d1) = make_float4(sp[2].h, sp[2].l, sp[3].h, sp[3].l);
        }
      } else {
#pragma unroll
        for (int t = 0; t < M; ++t) {
          float a = ta[fidx(t)], b = tb[fidx(t)], c = tc[fidx(t)];
          if (t == 0 && first_part) a = 0.f;
          if (t == M - 1 && last_part) c = 0.f;
          dom = fmaxf(dom, dom_excess(a, b, c, keep));
          const ff dd = split_f64_fast(td[didx(t)]);
          td2[didx(t)] = make_float2(dd.h, dd.l);  // same thread, same 8 bytes: read before write
          S.row(t, a, b, c, dd.h);
        }
      }
      const Blk blk = S.block();
      if (!started) {
        cluster_wait();  // every CTA of the cluster has started
        started = true;
      }
      // rides on the exchange as `extra`: 0 when every row of this CTA's part of the line certifies
      const unsigned unc = line_max(__float_as_uint(fmaxf(dom, 0.f)));
      unsigned unc_line;
      float xs_c, xe_c;
      // the flags of the previous group's lines ride along (out of place)
      tree_stage_b<C, true>(blk, unc, slots, wbar[0], xph0 & 1u, rank, p, jj, j, u0, v0, xs_c, xe_c, unc_line, alive,
                            A.st, pndx >> 31, &pfl);
      ++xph0;
      certified = unc_line == 0u;
      // Boundary unknowns exactly as the neighbours will see them in the residual: at a CTA edge
      // the cluster tree's values, elsewhere the partition's own block form.
      const float xs = (p == 0 && rank > 0) ? xs_c : Sweep<M>::first(blk, u0, v0);
      const float xe = (p == kTreeParts - 1 && rank < C - 1) ? xe_c : Sweep<M>::last(blk, u0, v0);
      S.solve(xs, xe, x0);
      // inside the CTA the neighbours' values come from the neighbouring lanes
      const float from_prev = __shfl_up_sync(~0u, x0[M - 1], 4), from_next = __shfl_down_sync(~0u, x0[0], 4);
      if (p > 0) u0 = from_prev;
      if (p < kTreeParts - 1) v0 = from_next;
      nx = 0u;
#pragma unroll
      for (int t = 0; t < M; ++t) nx = max(nx, abs_bits(x0[t]));
      nx = line_max(nx);  // this CTA's rows of the line
    }
    // at least one correction always runs (the host passes max_iters >= 1)
    {
      // ---------------- pass 1: correction for r = d - A x_0, x = x_0 + dx
      unsigned prev, gdx = 0u, gxm = 0u, ndx_l;
      bool fixup = false;  // out of place: some line of the cluster's previous group failed the rule
      {
        auto row1 = [&](int t, float a, float b, float c, float dh, float dl) {
          if (t == 0 && first_part) a = 0.f;
          if (t == M - 1 && last_part) c = 0.f;
          const float xm = t == 0 ? u0 : x0[t > 0 ? t - 1 : 0];
          const float xp = t == M - 1 ? v0 : x0[t < M - 1 ? t + 1 : 0];
          S.row_rhs(t, a, b, residual_f(a, b, c, dh, dl, xm, x0[t], xp));
        };
        if constexpr (XL) {
#pragma unroll
          for (int q = 0; q < M / 4; ++q) {
            const int f4 = fo + ((fx ^ q) << 2);
            const float4 a4 = *reinterpret_cast<const float4*>(ta + f4);
            const float4 b4 = *reinterpret_cast<const float4*>(tb + f4);
            const float4 c4 = *reinterpret_cast<const float4*>(tc + f4);
            const float4 e0 = *reinterpret_cast<const float4*>(td + dof + (((2 * q) ^ j7) << 1));
            const float4 e1 = *reinterpret_cast<const float4*>(td + dof + (((2 * q + 1) ^ j7) << 1));
            row1(4 * q, a4.x, b4.x, c4.x, e0.x, e0.y);
            row1(4 * q + 1, a4.y, b4.y, c4.y, e0.z, e0.w);
            row1(4 * q + 2, a4.z, b4.z, c4.z, e1.x, e1.y);
            row1(4 * q + 3, a4.w, b4.w, c4.w, e1.z, e1.w);
          }
        } else {
#pragma unroll
          for (int t = 0; t < M; ++t) {
            const float2 dd = td2[didx(t)];
            row1(t, ta[fidx(t)], tb[fidx(t)], tc[fidx(t)], dd.x, dd.y);
          }
        }
        const Blk blk = S.block();
        float u, v, xs_c, xe_c;
        tree_stage_b<C>(blk, nx, slots + C * kTreeSlotPitch, wbar[1], xph1 & 1u, rank, p, jj, j, u, v, xs_c, xe_c,
                        prev, alive, A.st);  // prev: line max |x_0|
        ++xph1;
        // Every thread has finished its pass-1 sweep, the last read of the a, b and c tiles (and,
        // unless x goes through it, of the d tile): the next group's rows may come in. The d pairs
        // written in place by pass 0 are ordered before the copies' writes by each writer's proxy
        // fence. The same barrier gathers the previous group's verdict: every CTA of the cluster
        // holds the same per-line flags (from this group's pass-0 exchange), so all agree.
        if (!inplace) {
          fence_proxy_async_smem();
          fixup = __syncthreads_or(pfl != 0u) != 0;
          if (tid == 0 && g + n_clusters < n_groups) {
            const int64_t l1 = (g + n_clusters) * kTreeLines;
            tree_load_tiles<M, XL>(maps, ta, tb, tc, td, bar, (int)(l1 % ic), (int)(l1 / ic), c_p, XL ? 1 : 3, !XL);
          }
        }
        float dx[M];
        S.solve(Sweep<M>::first(blk, u, v), Sweep<M>::last(blk, u, v), dx);
        unsigned ndx = 0u;
#pragma unroll
        for (int t = 0; t < M; ++t) ndx = max(ndx, abs_bits(dx[t]));
        ndx_l = line_max(ndx);  // this CTA's rows of the line
        if (inplace) tree_norms_push<C>(ndx_l, nx, norms + C * kTreeNormPitch, &nbar[1], rank, p, j);
        // x = x_0 + dx (exact widenings, one FP64 add): straight to global memory (for a fixed
        // row the four lines of a lane quad are 32 contiguous bytes), or by TMA store through the
        // thread's own d slots (XL) or, in place, through the a and b tiles (every thread's pass-1
        // sweep is done: the barrier below)
        if (!XL && !inplace) {
          if (active) {
#pragma unroll
            for (int t = 0; t < M; ++t) px[t * es] = f2d_fast(x0[t]) + f2d_fast(dx[t]);
          }
        } else {
          if (inplace) __syncthreads();
          if constexpr (XL) {
#pragma unroll
            for (int q = 0; q < M / 2; ++q)
              *reinterpret_cast<double2*>(tx + dof + ((q ^ j7) << 1)) =
                  make_double2(f2d_fast(x0[2 * q]) + f2d_fast(dx[2 * q]), f2d_fast(x0[2 * q + 1]) + f2d_fast(dx[2 * q + 1]));
          } else {
#pragma unroll
            for (int t = 0; t < M; ++t) tx[didx(t)] = f2d_fast(x0[t]) + f2d_fast(dx[t]);
          }
          fence_proxy_async_smem();
          __syncthreads();
          if (tid == 0) {  // out-of-range lines of a partial group are not written
            if constexpr (XL) {
#pragma unroll
              for (int i = 0; i < M / 2; ++i) tma_store_3d(&maps.x, tx + i * 512, c_p * M + 16 * i, c_in, c_out);
            } else {
              tma_store_4d(&maps.x, tx, c_in, c_out, c_p, 0);
              tma_store_4d(&maps.x, tx + M * 128, c_in + 16, c_out, c_p, 0);
            }
            bulk_commit();
            if (XL && !inplace && g + n_clusters < n_groups) {  // the next group's d tile, once the store has read it
              bulk_wait_read_all();
              const int64_t l1 = (g + n_clusters) * kTreeLines;
              tree_load_tiles<M, XL>(maps, ta, tb, tc, td, bar, (int)(l1 % ic), (int)(l1 / ic), c_p, 2, true);
            }
          }
        }
        if (inplace) {
          tree_norms_read<C>(gdx, gxm, norms + C * kTreeNormPitch, &nbar[1], xph3 & 1u, p, j, alive, A.st);
          ++xph3;
        }
      }
      if (inplace) {  // the rule on the line maxima now, and this group's further corrections
        bool line_done = tree_line_done(gdx, gxm, prev, active, A.tol, certified, reporter, A.st);
        const bool all_done = __syncthreads_and(line_done) != 0;
        later(g, certified, prev, line_done, all_done);
      } else {
        if (fixup) settle(pfl, g - n_clusters);  // the previous group's further corrections (rare)
        // This group's rule on this CTA's rows of each line. prev is the line's max |x_0| over the
        // cluster and the rule is monotone in max |dx|, so the line meets it exactly when every
        // CTA's rows do: the verdict needs no exchange of |dx| maxima now, only the flags, which
        // ride on the next group's pass-0 exchange.
        const bool fin = bits_finite(ndx_l) && bits_finite(prev);
        if (!fin && active && p == 0) report_error(A.st, 5);
        const bool fail = active && fin &&
                          !refine_done(__uint_as_float(ndx_l), __uint_as_float(prev), __uint_as_float(prev), A.tol,
                                       certified);
        pndx = (ndx_l & 0x7FFFFFFFu) | (fail ? 0x80000000u : 0u);
        pcert = certified;
      }
    }
    // Where x went through the tiles by TMA store, the next TMA load into them waits for the store's
    // read (at the top); the generic-proxy writes to them (d split in place, x) were fenced before
    // the store, and the last barrier above ordered every read.
  }
  if (!started) cluster_wait();  // a CTA without a group still completes the start-up barrier
  const int64_t g_first = blockIdx.x / C;
  if (!inplace && g_first < n_groups) {  // the cluster's last group: one exchange of its per-line flags
    const int64_t g_last = g_first + (n_groups - 1 - g_first) / n_clusters * n_clusters;
    cluster_arrive();  // every CTA is past its reads of the norm slots
    cluster_wait();
    unsigned f, unused;
    tree_norms_push<C>(pndx >> 31, 0u, norms + C * kTreeNormPitch, &nbar[1], rank, p, j);
    tree_norms_read<C>(f, unused, norms + C * kTreeNormPitch, &nbar[1], xph3 & 1u, p, j, alive, A.st);
    ++xph3;
    if (__syncthreads_or(f != 0u)) settle(f, g_last);
    if (rank == 0 && tid == 0) report_iters(A.st, 1);
  }
  if (tid == 0) bulk_wait_all();  // the last x store has been written
  // every store into this CTA's shared memory has arrived: each exchange was waited for
}

// compiled geometries: (rows per partition M, cluster size C); a line spans n = 8 C M rows.
#define TDMA_REFINE_TREE_SHAPES(X) X(16, 8) X(16, 4) X(16, 2)

}  // namespace tdma
