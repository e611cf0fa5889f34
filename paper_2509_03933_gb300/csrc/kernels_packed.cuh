// Packed unit-stride lines (ragged batches) with FP32 storage + refinement: one chunk of whole
// lines per thread-block cluster, Stage B as merge trees over lanes, warps and cluster ranks.
//
// Lines packed one after another with unit stride form one long tridiagonal system whose
// coupling across a line boundary is zero (a_0 = c_{n-1} = 0 of every line). A divide-and-conquer
// solve of that long system is therefore exactly the set of per-line solves: when the merge of
// two blocks meets a line boundary, the terms that couple them vanish and the merge only copies.
// At plan time the lines, in memory order, are cut into chunks of whole, contiguous lines of at
// most kPackChunk rows; chunk g is solved by one cluster of kPackC CTAs with 224 partitions each
// of M rows (M odd, the smallest with 896 M >= rows), the rows past the chunk's end being
// identity rows (a = c = d = 0, b = 1: decoupled unknowns equal to 0), so that every partition is
// full and the row loops are straight-line code compiled for each M. The paper batches lines of
// one direction into composite systems (Section 4.2.1); here the batch is a chunk and the
// composite system is the chunk's rows.
//
// Data path per chunk: every CTA's segment of a, b, c (float) and d (double) is one contiguous
// run of rows in memory and lands in shared memory in the same order, partition k's rows at
// [k M, (k + 1) M): the 16-byte-aligned interior of each array by one bulk copy (cp.async.bulk,
// completing on the CTA's tile mbarrier), the few elements before and after it by plain loads.
// With M odd the 32 lanes of a warp, k M + t apart, read 32 distinct banks (4-byte words) or the
// 32 banks in each half-warp (8-byte words), with no padding. Pass 0 solves with the float part of
// d; pass 1 solves for the extra-precise residual (float pairs) and corrects; x = x_0 + dx in FP64
// goes over the thread's own d slots (with x over d, into the space of a and b), and each warp
// copies its own 32 M contiguous rows out, coalesced. The next chunk's a, b and c copies go out
// as soon as pass 1's Stage B has passed its last read of them, its d copies once every warp's x
// has left. Per-line maxima of |x_0| and |dx| go to a per-line table by atomics; after a cluster
// barrier every CTA applies the stop rule of the other refinement kernels to the chunk's lines.
// Lines that need more corrections (rare) take further passes that read x back from global
// memory.
#pragma once
#include <cooperative_groups.h>
#include "layout.cuh"
#include "tma.cuh"
#include "kernels_refine.cuh"
#include "merge_tree.cuh"
#include "bits.cuh"
#include "kernels_refine_tree.cuh"

namespace tdma {

constexpr int kPackC = 4;                    // CTAs per cluster
constexpr int kPackW = 7;                    // compute warps per CTA
constexpr int kPackT = 32 * kPackW;          // compute threads (partitions) per CTA
constexpr int kPackThreads = kPackT + 32;    // + one coordinator warp
constexpr int kPackM = 21;                   // rows per partition at most (odd)
constexpr int kPackRowBits = 21;             // metadata bits of the row starts (bit 21: line end after)
constexpr int kPackTile = kPackT * kPackM + 8;  // tile elements: a segment and its alignment shift
constexpr int kPackChunk = kPackC * kPackT * kPackM;  // rows per chunk at most (18816)
constexpr uint32_t kPackWaitPolls = 1u << 16;
// Per-line words of the norm table (float bits of non-negative values): [0] max |dx| and [1] max
// |x_0| of the first correction (zero at launch, written once); [2] max |dx|, [3] max |x| of a
// further correction and [4] the previous max |dx| (reset by the line's owner after each use).
constexpr int kPackNormWords = 6;

struct PackedChunk {
  int64_t base;   // element index of the chunk's first row
  int32_t rows;   // rows in the chunk (1..kPackChunk)
  int32_t M;      // rows per partition: partition k holds rows [k M, min((k + 1) M, rows))
  int32_t line0;  // position, in memory order, of the chunk's first line (its norm slot)
  int32_t nlines; // lines in the chunk
  int32_t meta;   // block of the partition metadata (chunks of the same structure share one)
  int32_t pad;
};

// Partition metadata (one pair of words per partition of every distinct chunk structure):
//   x bits 0..20  bit t: row t of the partition starts a line
//   x bit 21      the row after the partition's last row starts a line or lies past the chunk
//   y             line of the partition's first row, counted from the chunk's first line
struct PackedTables {
  const PackedChunk* chunks;
  const uint2* meta;      // kPackC * kPackT pairs per distinct chunk structure
  uint32_t* norms;        // kPackNormWords per line in memory order (see packed_first_verdict)
  uint32_t* fix;          // [0]: chunks listed for further corrections, [1..]: their indices (out of place)
  int32_t n_chunks;
};

// L2 prefetch of the 16-byte-aligned part of [p, p + bytes)
TDMA_DEV void prefetch_l2_range(const void* p, int64_t bytes) {
  const uint64_t s = ((uint64_t)p + 15) & ~(uint64_t)15, e = ((uint64_t)p + bytes) & ~(uint64_t)15;
  if (e > s)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(s), "r"((uint32_t)(e - s)) : "memory");
}
TDMA_DEV uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
TDMA_DEV void st_cluster_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Stage A of one partition of m <= MM rows (runtime m, rows unrolled): the modified Thomas sweep
// of the merge-tree kernel with the row-1 relation summed in the forward pass.
template <int MM>
struct SweepR {
  float al[MM], ga[MM], de[MM];  // rows 1..m-2
  float alpha = -1.f, gamma = 0.f, delta = 0.f, F = 0.f, G = 0.f, Q = 1.f;
  float a0 = 0.f, b0 = 1.f, c0 = 0.f, h0 = 0.f;
  TDMA_DEV void row(int t, int m, float a, float b, float c, float rhs) {
    if (t == 0) {
      a0 = a; b0 = b; c0 = c; h0 = rhs;
      return;
    }
    if (t >= m) return;
    const float r = rcp(fmaf(-a, gamma, b));
    const float ar = a * r;
    alpha = -ar * alpha;
    gamma = c * r;
    delta = fmaf(r, rhs, -ar * delta);
    if (t <= m - 2) {
      al[t] = alpha; ga[t] = gamma; de[t] = delta;
      G = fmaf(Q, alpha, G);
      F = fmaf(Q, delta, F);
      Q = -Q * gamma;
    }
  }
  // Block form of the partition (all zero for an empty one: a decoupled unknown x = 0, which
  // merges with its neighbours without changing them).
  TDMA_DEV Blk block(int m) const {
    if (m <= 0) return Blk{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (m == 1) {
      const float ib = rcp(b0);
      return Blk{h0 * ib, -a0 * ib, -c0 * ib, h0 * ib, -a0 * ib, -c0 * ib};
    }
    const float rho = rcp(fmaf(-c0, G, b0));
    return part_block(rho * a0, rho * (c0 * Q), rho * fmaf(-c0, F, h0), alpha, gamma, delta);
  }
  TDMA_DEV static float first(const Blk& b, float u, float v) { return fmaf(b.q1, u, fmaf(b.r1, v, b.p1)); }
  TDMA_DEV static float last(const Blk& b, float u, float v) { return fmaf(b.q2, u, fmaf(b.r2, v, b.p2)); }
  // Stage C from the partition's first and last unknowns, handing each row's value to f(t, x_t)
  // from row m-1 down to row 0 (x_0 = xs; x_{m-1} = xe for m >= 2).
  template <class Fn>
  TDMA_DEV void solve_visit(int m, float xs, float xe, Fn&& f) const {
    float xn = xe;
#pragma unroll
    for (int t = MM - 1; t >= 0; --t) {
      if (t < m) {
        float v;
        if (t == 0) v = xs;
        else if (t == m - 1) v = xe;
        else v = fmaf(-ga[t > 0 ? t : 1], xn, fmaf(-al[t > 0 ? t : 1], xs, de[t > 0 ? t : 1]));
        xn = v;
        f(t, v);
      }
    }
  }
};

// Stage B of one pass, split between the compute warps and the coordinator warp of the CTA.
//   1. compute warps: 5-level merge tree over each warp's 32 partitions (shuffles); lane 0 puts
//      the warp's block into shared memory and arrives on named barrier 1;
//   2. coordinator: merges the 7 warp blocks, sends the CTA block into the shared memory of
//      every CTA of the cluster (st.async completing on the receiver's mbarrier), merges the C
//      CTA blocks (every CTA computes the same values in the same order), walks both trees back
//      down and leaves, per warp, its outside neighbours (u, v) and its first and last unknowns
//      exactly as the neighbouring warp or CTA sees them; arrives on named barrier 2;
//   3. compute warps: the warp's values, then the lane tree back down to the partition.
// tree_up_full over the 8 slots g = 0..7 of the coordinator's lanes, where slot 7 holds no
// rows (the CTA has 7 compute warps): it is the identity of the merge, so the level-0 merge of
// slots 6 and 7 copies block 6, and the down-sweep stops above level 0 for that pair.
TDMA_DEV Blk tree_up_full_ident7(Blk b, int g, Mrg (&keep)[3]) {
  // level 0 by hand
  {
    const Blk o = shfl_xor_blk(b, 1);
    const bool in_right = g & 1;
    const Blk& L = in_right ? o : b;
    const Blk& R = in_right ? b : o;
    const float D = rcp(fmaf(-L.r2, R.q1, 1.f));
    Aff y, z;
    y.p = D * fmaf(L.r2, R.p1, L.p2);
    y.q = D * L.q2;
    y.r = D * (L.r2 * R.r1);
    z.p = fmaf(R.q1, y.p, R.p1);
    z.q = R.q1 * y.q;
    z.r = fmaf(R.q1, y.r, R.r1);
    Blk nb{fmaf(L.r1, z.p, L.p1), fmaf(L.r1, z.q, L.q1), L.r1 * z.r, fmaf(R.q2, y.p, R.p2), R.q2 * y.q,
           fmaf(R.q2, y.r, R.r2)};
    if ((g >> 1) == 3) nb = L;  // slots 6 and 7: the pair is block 6 alone (no level-0 descent)
    keep[0] = Mrg{y, z};
    b = nb;
  }
  Mrg k2[3];
  const Blk B = tree_up_full<2, 1>(b, g >> 1, k2);
  keep[1] = k2[0];
  keep[2] = k2[1];
  return B;
}

TDMA_DEV void named_arrive(int id) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(kPackThreads) : "memory"); }
TDMA_DEV void named_sync(int id) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kPackThreads) : "memory"); }

struct WarpEdge { float u, v, xs, xe; };

TDMA_DEV WarpEdge packed_compute_b(const Blk& blk, float* wsl, const float4* dsl, int w, int lane, float& u,
                                   float& v) {
  Aff kl[5];
  const Blk W = tree_up<5, 0, 5>(blk, lane, kl);
  if (lane == 0) {
    float4* s = reinterpret_cast<float4*>(wsl + w * 8);
    s[0] = make_float4(W.p1, W.q1, W.r1, W.p2);
    s[1] = make_float4(W.q2, W.r2, 0.f, 0.f);
  }
  named_arrive(1);
  named_sync(2);
  const float4 e = dsl[w];
  u = e.x;
  v = e.y;
  tree_down<5, 5>(u, v, lane, kl);
  return WarpEdge{e.x, e.y, e.z, e.w};
}

template <int C>
TDMA_DEV void packed_coord_b(const float* wsl, float4* dsl, float* csl, uint64_t* bar, uint32_t phase, int rank,
                             int lane, bool& alive, DevStatus* st) {
  constexpr int LC = C == 8 ? 3 : (C == 4 ? 2 : 1);
  named_sync(1);
  const float4* sw = reinterpret_cast<const float4*>(wsl + (lane & 7) * 8);
  const float4 w0 = sw[0], w1 = sw[1];
  Mrg kw[3];
  const Blk B = tree_up_full_ident7(Blk{w0.x, w0.y, w0.z, w0.w, w1.x, w1.y}, lane & 7, kw);
  if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)C * 32u);
  if (lane < C) {  // the CTA block to every CTA of the cluster (slot `rank` there)
    const uint32_t dst = map_rank(csl + rank * 8, lane), rb = map_rank(bar, lane);
    st_async4(dst, B.p1, B.q1, B.r1, B.p2, rb);
    st_async4(dst + 16, B.q2, B.r2, 0.f, 0.f, rb);
  }
  if (alive && !mbar_wait_bounded(bar, phase, kPackWaitPolls)) {
    alive = false;
    report_error(st, 6);
  }
  const float4* sc = reinterpret_cast<const float4*>(csl + (lane & (C - 1)) * 8);
  const float4 c0 = sc[0], c1 = sc[1];
  float uq = 0.f, vq = 0.f, xsq = 0.f, xeq = 0.f;
  {
    Mrg kc[3];
    tree_up_full<LC, 0>(Blk{c0.x, c0.y, c0.z, c0.w, c1.x, c1.y}, lane & (C - 1), kc);
    tree_down_full<LC>(uq, vq, xsq, xeq, lane & (C - 1), kc);  // the chunk ends have u = v = 0
  }
  float uc = __shfl_sync(~0u, uq, rank), vc = __shfl_sync(~0u, vq, rank);
  float xsc = __shfl_sync(~0u, xsq, rank), xec = __shfl_sync(~0u, xeq, rank);
  // down the warp tree; the pair (6, 7) is block 6 alone, so level 0 leaves its values as they
  // are, and warp 6 keeps the CTA's last unknown exactly as the cluster tree gave it
  const int g = lane & 7;
#pragma unroll
  for (int l = 2; l >= 0; --l) {
    if (l == 0 && (g >> 1) == 3) break;
    const float y = fmaf(kw[l].y.q, uc, fmaf(kw[l].y.r, vc, kw[l].y.p));
    const float z = fmaf(kw[l].z.q, uc, fmaf(kw[l].z.r, vc, kw[l].z.p));
    if ((g >> l) & 1) { uc = y; xsc = z; } else { vc = z; xec = y; }
  }
  if (lane < kPackW) dsl[lane] = make_float4(uc, vc, xsc, xec);
  named_arrive(2);
}

// Segmented maxima of one partition's rows into the per-line table, fed from the last row down:
// rows of one line form a piece, flushed by an atomic pair when the walk passes the row that
// starts its line; a warp whose rows all belong to one line reduces first and makes one pair.
struct LineMax {
  unsigned pdx, px;
  unsigned unc;  // first correction: nonzero if this partition's rows do not certify the floor
  int cur;   // line of the rows being accumulated
  int slot;  // first of the two words written (0: first correction, 2: further ones)
  TDMA_DEV void init(uint32_t mask, int m, int line, int slot_, unsigned unc_ = 0u) {
    pdx = px = 0u;
    unc = unc_;
    slot = slot_;
    cur = line + __popc(mask & ~1u & ((1u << m) - 1u));
  }
  TDMA_DEV void add(int t, uint32_t mask, float dxv, float xv, uint32_t* norms) {
    pdx = max(pdx, abs_bits(dxv));
    px = max(px, abs_bits(xv));
    if (t > 0 && ((mask >> t) & 1u)) {  // row t starts line `cur`: its piece is complete
      atomicMax(&norms[kPackNormWords * cur + slot], pdx);
      atomicMax(&norms[kPackNormWords * cur + slot + 1], px);
      if (unc) atomicMax(&norms[kPackNormWords * cur + 5], unc);
      pdx = px = 0u;
      --cur;
    }
  }
  // the piece of row 0 (line `cur`), warp-reduced when the whole warp lies in one line
  TDMA_DEV void finish(uint32_t mask, int m, int lane, uint32_t* norms) {
    const bool one_line = __all_sync(~0u, (mask & ~1u) == 0u && (lane == 0 || (mask & 1u) == 0u));
    if (one_line) {
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        pdx = max(pdx, __shfl_xor_sync(~0u, pdx, o));
        px = max(px, __shfl_xor_sync(~0u, px, o));
        unc = max(unc, __shfl_xor_sync(~0u, unc, o));
      }
      const int l0 = __shfl_sync(~0u, cur, 0);
      if (lane == 0) {
        atomicMax(&norms[kPackNormWords * l0 + slot], pdx);
        atomicMax(&norms[kPackNormWords * l0 + slot + 1], px);
        if (unc) atomicMax(&norms[kPackNormWords * l0 + 5], unc);
      }
    } else if (m > 0) {
      atomicMax(&norms[kPackNormWords * cur + slot], pdx);
      atomicMax(&norms[kPackNormWords * cur + slot + 1], px);
      if (unc) atomicMax(&norms[kPackNormWords * cur + 5], unc);
    }
  }
};

// Stop rule of the refinement, as in the other refinement kernels (refine_done): a line whose
// rows certify the float-pair residual's floor (word 5 of its table entry is 0) is done when its
// estimated error rho |dx| <= tol |x| with rho = |dx| / |dx_prev| (|dx_prev| = |x_0| after the first
// correction); another line when |dx| <= tol |x|. A non-finite norm ends the line with status 5.
TDMA_DEV bool line_rule(uint32_t gdx, uint32_t gx, uint32_t prev, float tol, bool certified, bool& bad) {
  bad = !(bits_finite(gdx) && bits_finite(gx));
  if (bad) return true;
  return refine_done(__uint_as_float(gdx), __uint_as_float(gx), __uint_as_float(prev), tol, certified);
}

// After the first correction: every CTA of the cluster reads the norms of all lines of the chunk
// (complete after the cluster barrier, written by no one afterwards) and so reaches the same
// verdict without another exchange. Returns true when some line needs a further correction; with
// `last_pass` such a line reports status 7 instead. Statuses are reported by CTA rank 0.
TDMA_DEV bool packed_first_verdict(const PackedChunk& ch, const uint32_t* norms, float tol, bool last_pass,
                                   bool reporter, DevStatus* st) {
  bool more = false;
  for (int l = threadIdx.x; l < ch.nlines; l += blockDim.x) {
    const uint32_t* nl = norms + (int64_t)kPackNormWords * (ch.line0 + l);
    const uint32_t gdx = ld_relaxed_u32(nl), gx = ld_relaxed_u32(nl + 1), unc = ld_relaxed_u32(nl + 5);
    bool bad;
    const bool done = line_rule(gdx, gx, gx, tol, unc == 0u, bad);
    if (bad && reporter) report_error(st, 5);
    if (!done) {
      if (last_pass) { if (reporter) report_error(st, 7); }
      else more = true;
    }
  }
  return more;
}

// After a further correction: the thread holding each line's first row applies the rule to words
// 2 and 3 (previous |dx| in word 4, or word 0 after the first correction) and resets them.
TDMA_DEV bool packed_later_verdict(uint32_t mask, int m, int line, uint32_t* norms, bool first_later, float tol,
                                   bool last_pass, DevStatus* st) {
  bool more = false;
  uint32_t own = m > 0 ? (mask & ((m >= 32 ? 0u : (1u << m)) - 1u)) : 0u;
  while (own) {
    const int t = __ffs(own) - 1;
    own &= own - 1u;
    const int L = line + __popc(mask & ~1u & ((2u << t) - 1u));
    uint32_t* nl = norms + (int64_t)kPackNormWords * L;
    const uint32_t gdx = ld_relaxed_u32(nl + 2), gx = ld_relaxed_u32(nl + 3);
    const uint32_t prev = ld_relaxed_u32(nl + (first_later ? 0 : 4));
    const uint32_t unc = ld_relaxed_u32(nl + 5);
    nl[2] = 0u;
    nl[3] = 0u;
    nl[4] = gdx;
    bool bad;
    const bool done = line_rule(gdx, gx, prev, tol, unc == 0u, bad);
    if (bad) report_error(st, 5);
    if (!done) {
      if (last_pass) report_error(st, 7);
      else more = true;
    }
  }
  return more;
}

// One further correction of a partition (rare): the coefficients read from global memory (with
// TR those of the transposed rows), d from the shared-memory float pairs when they are still there
// (sd: the partition's first row, else null) or from global memory, x of the partition and its neighbours read back from
// global memory; residual in float pairs, Stage A/B/C, x += dx written back. Kept out of line so
// that its registers do not weigh on the two main passes.
template <bool TR>
__device__ __noinline__ void packed_later_pass(const PackedTables& PT, const float* fa, const float* fb,
                                               const float* fc, const double* gd, const float2* sd, float* wslq,
                                               const float4* dslq, double* gx, int64_t prow, int w, int lane,
                                               int kp, int m, uint32_t mask, uint32_t endmask, int line, int row0,
                                               int rows) {
  SweepR<kPackM> S;
  ff xm{0.f, 0.f}, xc{0.f, 0.f};
  if (m > 0) {
    if (kp > 0) xm = split_f64(__ldcg(gx + prow - 1));
    xc = split_f64(__ldcg(gx + prow));
  }
#pragma unroll
  for (int t = 0; t < kPackM; ++t) {
    if (t < m) {
      const int64_t gi = prow + t;
      const float a = ((mask >> t) & 1u) ? 0.f : (TR ? fc[gi - 1] : fa[gi]);
      const float c = ((endmask >> t) & 1u) ? 0.f : (TR ? fa[gi + 1] : fc[gi]);
      const float b = fb[gi];
      ff dd;
      if (sd) {
        const float2 v = sd[t];
        dd = ff{v.x, v.y};
      } else {
        dd = split_f64(gd[gi]);
      }
      const bool has_next = t + 1 < m || row0 + t + 1 < rows;
      const ff xn = has_next ? split_f64(__ldcg(gx + gi + 1)) : ff{0.f, 0.f};
      S.row(t, m, a, b, c, residual_ff(a, b, c, dd, xm, xc, xn));
      xm = xc;
      xc = xn;
    }
  }
  const Blk blk = S.block(m);
  float u, v;
  packed_compute_b(blk, wslq, dslq, w, lane, u, v);
  // Every read of x above happened before its warp arrived on named barrier 1; another warp
  // writes only after barrier 2, and another CTA only after receiving this CTA's block, which
  // left after barrier 1.
  LineMax nm;
  nm.init(mask, m, line, 2);
  S.solve_visit(m, SweepR<kPackM>::first(blk, u, v), SweepR<kPackM>::last(blk, u, v), [&](int t, float dxv) {
    const double xv = __ldcg(gx + prow + t) + f2d(dxv);
    gx[prow + t] = xv;
    nm.add(t, mask, dxv, __double2float_rn(xv), PT.norms);
  });
  nm.finish(mask, m, lane, PT.norms);
}

// Passes 0 and 1 of one compute thread for chunks of MM rows per partition (every partition
// full; a and c already zero where lines start and end); ra, rb, rc, rd: the partition's first row
// in the tiles. Pass 0 solves with the float part of d (split in place into float pairs), pass 1
// solves for the extra-precise residual with the same factors, and x = x_0 + dx (exact widenings,
// one FP64 add) goes to rx: over the thread's own d pairs (read by its pass-1 sweep), or, when x is
// written over d, into the a and b space (named barrier 2 of pass 1 completes only after every
// compute warp has arrived on barrier 1, after its last read of the tiles). The per-line maxima of
// |dx| and |x_0| go to the line table.
template <int MM>
TDMA_DEV void packed_passes(const float* ra, const float* rb, const float* rc, const double* rd, float2* rd2,
                            double* rx, float* wsl0, const float4* dsl0, float* wsl1, const float4* dsl1, int w,
                            int lane, bool edge_s, bool edge_e, uint32_t mask, int line, uint32_t* norms,
                            float keep) {
  Sweep<MM> S;
  float x0[MM];
  float u0, v0;
  float dom = -INFINITY;  // max over this partition's rows of dom_excess
  {
#pragma unroll
    for (int t = 0; t < MM; ++t) {
      const ff dd = split_f64_fast(rd[t]);
      rd2[t] = make_float2(dd.h, dd.l);  // same thread, same 8 bytes
      const float a = ra[t], b = rb[t], c = rc[t];
      dom = fmaxf(dom, dom_excess(a, b, c, keep));
      S.row(t, a, b, c, dd.h);
    }
    const Blk blk = S.block();
    float u, v;
    const WarpEdge e = packed_compute_b(blk, wsl0, dsl0, w, lane, u, v);
    // unknowns at warp and CTA edges exactly as the neighbouring warp computes them
    const float xs = edge_s ? e.xs : Sweep<MM>::first(blk, u, v);
    const float xe = edge_e ? e.xe : Sweep<MM>::last(blk, u, v);
    S.solve(xs, xe, x0);
    const float from_prev = __shfl_up_sync(~0u, x0[MM - 1], 1), from_next = __shfl_down_sync(~0u, x0[0], 1);
    u0 = lane == 0 ? e.u : from_prev;
    v0 = lane == 31 ? e.v : from_next;
  }
  {
#pragma unroll
    for (int t = 0; t < MM; ++t) {
      const float a = ra[t], b = rb[t], c = rc[t];
      const float2 dd = rd2[t];
      const float xm = t == 0 ? u0 : x0[t > 0 ? t - 1 : 0];
      const float xp = t == MM - 1 ? v0 : x0[t < MM - 1 ? t + 1 : 0];
      S.row_rhs(t, a, b, residual_f(a, b, c, dd.x, dd.y, xm, x0[t], xp));
    }
    const Blk blk = S.block();
    float u, v;
    const WarpEdge e = packed_compute_b(blk, wsl1, dsl1, w, lane, u, v);
    const float xs = edge_s ? e.xs : Sweep<MM>::first(blk, u, v);
    const float xe = edge_e ? e.xe : Sweep<MM>::last(blk, u, v);
    LineMax nm;
    nm.init(mask, MM, line, 0, __float_as_uint(fmaxf(dom, 0.f)));
    S.solve_visit(xs, xe, [&](int t, float dxv) {
      rx[t] = f2d_fast(x0[t]) + f2d_fast(dxv);
      nm.add(t, mask, dxv, x0[t], norms);
    });
    nm.finish(mask, MM, lane, norms);
  }
}

// compiled rows per partition (the plan rounds M up to one of these)
#define TDMA_PACKED_M(X) X(3) X(5) X(7) X(9) X(11) X(13) X(15) X(17) X(19) X(21)

// Chunk g's segment for this CTA: rows [seg0, seg0 + segn) of the chunk, starting at element gbase.
struct PackedSeg {
  int64_t gbase;
  int M, seg0, segn, rows;
};
TDMA_DEV PackedSeg packed_seg(const PackedTables& PT, int g, int rank) {
  const PackedChunk ch = PT.chunks[g];
  PackedSeg q;
  q.M = ch.M;
  q.seg0 = rank * kPackT * ch.M;
  q.segn = max(0, min(ch.rows - q.seg0, kPackT * ch.M));
  q.gbase = ch.base + q.seg0;
  q.rows = ch.rows;
  return q;
}

// One array's copy into its tile. Tile element sh + i holds segment row i, read from src[i]
// (src: the global element of segment row 0; for the transposed rows of TR shifted by one) for
// the rows i in [lo, hi); sh is src's position within its 16-byte word (0..3 floats, 0..1
// doubles), so that the bulk copy of the interior [a0, a1), 16-byte aligned at both ends in global
// memory, lands 16-byte aligned in the tile too. Rows outside [lo, hi) lie past a line's end
// (zero) or past the chunk (identity rows).
struct PackedArr {
  const char* src;  // global address of segment row 0 (one before the array when lo >= 1)
  char* tile;       // tile base (16-byte aligned)
  int es, sh, lo, hi, a0, a1;
};
TDMA_DEV PackedArr packed_arr(const void* base, int64_t s, void* tile, int es, int lo, int hi) {
  PackedArr r;
  r.es = es;
  r.src = reinterpret_cast<const char*>(base) + s * es;
  r.tile = reinterpret_cast<char*>(tile);
  const int k = 16 / es;
  r.sh = (int)((reinterpret_cast<uintptr_t>(r.src) / (uintptr_t)es) & (uintptr_t)(k - 1));
  r.lo = lo;
  r.hi = max(lo, hi);
  r.a0 = min(r.hi, lo + ((k - ((r.sh + lo) & (k - 1))) & (k - 1)));
  r.a1 = max(r.a0, r.hi - ((r.sh + r.hi) & (k - 1)));
  return r;
}
// The four tiles' copies of segment q: (a, b, c, d), or with TR the transposed rows
// (c_{i-1}, b, a_{i+1}, d), whose first and last elements would come from outside the chunk and
// are not read (they fall on a line start and a line end, where they are zero).
template <bool TR>
TDMA_DEV void packed_arrs(const Args& A, const PackedSeg& q, float* ta, float* tb, float* tc, double* td,
                          PackedArr (&r)[4]) {
  if (!TR) {
    r[0] = packed_arr(A.a, q.gbase, ta, 4, 0, q.segn);
    r[2] = packed_arr(A.c, q.gbase, tc, 4, 0, q.segn);
  } else {
    r[0] = packed_arr(A.c, q.gbase - 1, ta, 4, q.seg0 == 0 ? 1 : 0, q.segn);
    r[2] = packed_arr(A.a, q.gbase + 1, tc, 4, 0, min(q.segn, q.rows - q.seg0 - 1));
  }
  r[1] = packed_arr(A.b, q.gbase, tb, 4, 0, q.segn);
  r[3] = packed_arr(A.d, q.gbase, td, 8, 0, q.segn);
}
// One thread: the bulk copies of the tiles in `parts` (bit j: tile j of a, b, c, d) of segment q,
// counted on the tile mbarrier (with `arrive` this call also arrives on it; without, the copies
// count towards a phase whose arrival comes later).
template <bool TR>
TDMA_DEV void packed_bulk(const Args& A, const PackedSeg& q, float* ta, float* tb, float* tc, double* td,
                          uint64_t* bar, int parts, bool arrive) {
  PackedArr r[4];
  packed_arrs<TR>(A, q, ta, tb, tc, td, r);
  uint32_t bytes = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if ((parts >> j) & 1) bytes += (uint32_t)(r[j].a1 - r[j].a0) * (uint32_t)r[j].es;
  if (arrive) mbar_arrive_expect_tx(bar, bytes);
  else mbar_expect_tx(bar, bytes);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (!((parts >> j) & 1) || r[j].a1 <= r[j].a0) continue;
    const int es = r[j].es;
    bulk_load_1d(r[j].tile + (size_t)(r[j].sh + r[j].a0) * es, r[j].src + (size_t)r[j].a0 * es,
                 (uint32_t)(r[j].a1 - r[j].a0) * (uint32_t)es, bar);
  }
}
// Every thread of the CTA: the tile elements of segment q that the bulk copies do not bring: rows
// [lo, a0) and [a1, hi) by plain loads (at most three of each per array), zeros at [0, lo) and
// [hi, segn), and identity rows past the chunk's end.
template <bool TR>
TDMA_DEV void packed_fill(const Args& A, const PackedSeg& q, float* ta, float* tb, float* tc, double* td, int tid) {
  PackedArr r[4];
  packed_arrs<TR>(A, q, ta, tb, tc, td, r);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const PackedArr& x = r[j];
    const int head = x.a0, tail = x.hi - x.a1;  // rows [0, a0) then [a1, hi), then [hi, segn)
    for (int i = tid; i < head + tail + (q.segn - x.hi); i += kPackThreads) {
      const int row = i < head ? i : (i < head + tail ? x.a1 + (i - head) : x.hi + (i - head - tail));
      const bool load = row >= x.lo && row < x.hi;
      if (x.es == 4) {
        const float v = load ? __ldg(reinterpret_cast<const float*>(x.src) + row) : 0.f;
        reinterpret_cast<float*>(x.tile)[x.sh + row] = v;
      } else {
        const double v = load ? __ldg(reinterpret_cast<const double*>(x.src) + row) : 0.0;
        reinterpret_cast<double*>(x.tile)[x.sh + row] = v;
      }
    }
  }
  // identity rows past the chunk's end: a = c = d = 0, b = 1
  for (int i = q.segn + tid; i < kPackT * q.M; i += kPackThreads) {
    ta[r[0].sh + i] = 0.f;
    tb[r[1].sh + i] = 1.f;
    tc[r[2].sh + i] = 0.f;
    td[r[3].sh + i] = 0.0;
  }
}

// L2 prefetch of chunk g's segment for this CTA (one thread)
TDMA_DEV void packed_prefetch(const PackedTables& PT, const Args& A, int g, int rank) {
  const PackedChunk nx = PT.chunks[g];
  const int s1 = rank * kPackT * nx.M;
  const int n1 = max(0, min(nx.rows - s1, kPackT * nx.M));
  if (n1 <= 0) return;
  const int64_t b1 = nx.base + s1;
  prefetch_l2_range((const float*)A.a + b1 - 1, 4ll * (n1 + 2));
  prefetch_l2_range((const float*)A.b + b1, 4ll * n1);
  prefetch_l2_range((const float*)A.c + b1 - 1, 4ll * (n1 + 2));
  prefetch_l2_range((const double*)A.d + b1, 8ll * n1);
}

// Shared memory of the Stage B hand-offs and of the per-chunk verdict (both kernels below).
template <int C>
struct PackedXchg {
  uint64_t xbar[2];      // exchange mbarriers, by pass parity
  float wsl[2][8 * 8];   // warp blocks (slot 7 unused), by pass parity
  float4 dsl[2][8];      // per warp: u, v, first and last unknowns
  float csl[2][C * 8];   // CTA blocks of the cluster, by pass parity
  uint32_t s_more;       // epoch stamp: some line of the chunk needs more
};
// One thread: the barriers and the empty warp slot 7 (before the CTA's first barrier).
template <int C>
TDMA_DEV void packed_xchg_init(PackedXchg<C>& X) {
  mbar_init(&X.xbar[0], 1);
  mbar_init(&X.xbar[1], 1);
  X.s_more = 0u;
  for (int i = 0; i < 8; ++i) X.wsl[i / 4][7 * 8 + (i & 3)] = 0.f;
  mbar_fence_init();
}

// Where this thread stands in chunk g: its rows (m of M, from segment row tid M), the line starts
// among them (mask), the line ends (endmask, c = 0 there) and the line of its first row.
struct PackedPart {
  PackedChunk ch;
  PackedSeg q;
  int m;
  uint32_t mask, endmask;
  int line;
};
template <int C>
TDMA_DEV PackedPart packed_part(const PackedTables& PT, int g, int rank, int tid, int kp, bool coord) {
  PackedPart r;
  r.ch = PT.chunks[g];
  r.q = packed_seg(PT, g, rank);
  const int M = r.q.M;
  r.m = coord ? 0 : max(0, min(M, r.q.segn - tid * M));
  const uint2 meta = coord ? make_uint2(0u, 0u) : PT.meta[(int64_t)r.ch.meta * (C * kPackT) + kp];
  r.mask = meta.x & ((1u << kPackRowBits) - 1u);
  r.line = r.ch.line0 + (int)meta.y;
  // c = 0 on rows that end a line: row t ends one when row t + 1 starts one
  r.endmask = r.m > 0 ? ((r.mask >> 1) | (((meta.x >> kPackRowBits) & 1u) << (r.m - 1))) : 0u;
  return r;
}

// Further corrections of a chunk some of whose lines failed the stop rule after the first one
// (rare): passes that read the coefficients and x from global memory (d too, unless sd holds the
// chunk's d pairs), every CTA of the cluster the same number of times (the cluster's verdict),
// until every line meets the rule or max_iters corrections. Returns the corrections made.
template <int C, bool TR>
TDMA_DEV int packed_more_passes(const Args& A, const PackedTables& PT, const PackedPart& P, const float2* sd,
                                PackedXchg<C>& X, uint32_t (&xph)[2], uint32_t& epoch, bool& alive, int tid, int w,
                                int lane, int rank, int kp, bool coord) {
  const int M = P.q.M;
  int it = 1;
  bool again = true;
  cluster_arrive();  // x of every CTA went out before this arrival
  cluster_wait();
  while (again && it < A.max_iters) {
    ++it;
    const int qp = it & 1;
    if (coord) {
      packed_coord_b<C>(X.wsl[qp], X.dsl[qp], X.csl[qp], &X.xbar[qp], xph[qp] & 1u, rank, lane, alive, A.st);
      ++xph[qp];
    } else {
      packed_later_pass<TR>(PT, (const float*)A.a, (const float*)A.b, (const float*)A.c, (const double*)A.d, sd,
                            X.wsl[qp], X.dsl[qp], (double*)A.x, P.q.gbase + (int64_t)tid * M, w, lane, kp, P.m, P.mask,
                            P.endmask, P.line, P.q.seg0 + tid * M, P.ch.rows);
    }
    __syncthreads();
    ++epoch;
    cluster_arrive();
    cluster_wait();
    bool more = !coord && packed_later_verdict(P.mask, P.m, P.line, PT.norms, it == 2, A.tol, it >= A.max_iters, A.st);
    more = __syncthreads_or(more) != 0;
    if (more && tid < C) st_cluster_u32(map_rank(&X.s_more, tid), epoch);
    cluster_arrive();
    cluster_wait();
    again = X.s_more == epoch;
  }
  return it;
}

// Persistent: the grid holds the clusters that fit on the GPU at once; cluster q takes chunks
// q, q + Q, q + 2Q, ... (Q clusters, chunks sorted longest first at plan time). Warps 0..6 of a
// CTA compute (one partition per thread), warp 7 coordinates Stage B. Out of place (IP false), the
// next chunk's a, b and c copies go out (from the coordinator) as soon as pass 1's Stage B has
// passed the compute warps' last read of them, and its d copies once every warp's x has left the
// d tile, so that they overlap Stage C, the x copy-out and the per-line stop rule; a chunk with a
// line that needs further corrections (rare) is listed for packed_fixup_kernel, launched after
// this kernel, which reads the coefficients, d and x from global memory. (Kept out of this kernel,
// whose call into the further passes cost spills on the main path: 0.75 -> 0.69 ms on the
// 20000-line batch without it.) In place (IP true, x is d), d stays in shared memory until its
// chunk is done, every copy of the next chunk goes out after it, and the further corrections run
// here, with d from the shared-memory float pairs.
template <int C, bool TR, bool IP>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(kPackThreads, 2)
    packed_refine_kernel(const Args A, const PackedTables PT) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) PackedXchg<C> X;
  __shared__ __align__(8) uint64_t tbar;  // tile copies of a chunk
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const float keep = certify_keep(A.tol);
  const bool coord = w == kPackW;
  const int rank = (int)cluster_rank();
  const int kp = rank * kPackT + tid;  // partition index within the chunk (compute threads)
  float* ta = reinterpret_cast<float*>(smem_raw);
  float* tb = ta + kPackTile;
  float* tc = tb + kPackTile;
  double* td = reinterpret_cast<double*>(tc + kPackTile);
  float2* td2 = reinterpret_cast<float2*>(td);
  double* tx_ab = reinterpret_cast<double*>(ta);  // with x over d, x leaves through the a and b space
  double* gx = (double*)A.x;
  constexpr bool overlap = !IP;  // with x over d, d must stay in shared memory until done

  if (tid == 0) {
    packed_xchg_init<C>(X);
    mbar_init(&tbar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  cluster_arrive();  // barriers initialised; the matching wait precedes the first remote store
  bool started = false, alive = true;
  uint32_t xph[2] = {0u, 0u}, tph = 0u;
  uint32_t epoch = 0u;
  const int n_clusters = (int)(gridDim.x / C);
  const int g0 = (int)(blockIdx.x / C);
  if (g0 < PT.n_chunks) {
    if (tid == 0) packed_bulk<TR>(A, packed_seg(PT, g0, rank), ta, tb, tc, td, &tbar, 15, true);
    if (coord && lane == 0 && g0 + n_clusters < PT.n_chunks) packed_prefetch(PT, A, g0 + n_clusters, rank);
  }

  for (int g = g0; g < PT.n_chunks; g += n_clusters) {
    const PackedPart P = packed_part<C>(PT, g, rank, tid, kp, coord);
    const PackedSeg& q = P.q;
    const int M = q.M;
    const bool has_next = g + n_clusters < PT.n_chunks;
    PackedArr r[4];
    packed_arrs<TR>(A, q, ta, tb, tc, td, r);

    // with x over d, this chunk's copies go out now (the previous chunk is done with the tiles)
    if (!overlap && g != g0 && tid == 0) packed_bulk<TR>(A, q, ta, tb, tc, td, &tbar, 15, true);
    packed_fill<TR>(A, q, ta, tb, tc, td, tid);
    if (!mbar_wait_bounded(&tbar, tph, kPackWaitPolls) && alive) {
      alive = false;
      report_error(A.st, 6);
    }
    tph ^= 1u;
    __syncthreads();
    if (!started) {
      cluster_wait();  // every CTA of the cluster has started: remote stores may begin
      started = true;
    }
    // a = 0 where a line starts, c = 0 where one ends (each thread its own rows)
    for (uint32_t bm = P.mask; bm; bm &= bm - 1u) ta[r[0].sh + tid * M + (__ffs(bm) - 1)] = 0.f;
    for (uint32_t bm = P.endmask; bm; bm &= bm - 1u) tc[r[2].sh + tid * M + (__ffs(bm) - 1)] = 0.f;
    // this chunk's generic-proxy writes to the tiles come before the next chunk's copies into them
    fence_proxy_async_smem();
    const bool edge_s = lane == 0 && kp > 0, edge_e = lane == 31 && kp + 1 < C * kPackT;

    if (coord) {
      packed_coord_b<C>(X.wsl[0], X.dsl[0], X.csl[0], &X.xbar[0], xph[0] & 1u, rank, lane, alive, A.st);
      packed_coord_b<C>(X.wsl[1], X.dsl[1], X.csl[1], &X.xbar[1], xph[1] & 1u, rank, lane, alive, A.st);
      ++xph[0];
      ++xph[1];
      // pass 1's barrier 1 is behind: every compute warp has made its last read of a, b and c
      if (overlap && has_next && lane == 0) {
        packed_bulk<TR>(A, packed_seg(PT, g + n_clusters, rank), ta, tb, tc, td, &tbar, 7, false);
        if (g + 2 * n_clusters < PT.n_chunks) packed_prefetch(PT, A, g + 2 * n_clusters, rank);
      }
    } else {
      const int o = tid * M;
      double* rx = overlap ? td + r[3].sh + o : tx_ab + o;
      switch (M) {
#define TDMA_PASSES(MM)                                                                                      \
  case MM:                                                                                                    \
    packed_passes<MM>(ta + r[0].sh + o, tb + r[1].sh + o, tc + r[2].sh + o, td + r[3].sh + o, td2 + r[3].sh + o, \
                      rx, X.wsl[0], X.dsl[0], X.wsl[1], X.dsl[1], w, lane, edge_s, edge_e, P.mask, P.line,      \
                      PT.norms, keep);                                                                        \
    break;
        TDMA_PACKED_M(TDMA_PASSES)
#undef TDMA_PASSES
        default: {  // not a compiled M (the plan never makes one): report; the barriers still run
          if (tid == 0) report_error(A.st, 2);
          float du, dv;
          packed_compute_b(Blk{0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, X.wsl[0], X.dsl[0], w, lane, du, dv);
          packed_compute_b(Blk{0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, X.wsl[1], X.dsl[1], w, lane, du, dv);
        }
      }
      fence_proxy_async_smem();  // the d pairs and x come before the next chunk's copies
      // x in FP64: the warp's own 32 M rows, contiguous in memory, coalesced
      __syncwarp();
      const double* xs = overlap ? td + r[3].sh : tx_ab;
      const int w0 = w * 32 * M, w1 = min(w0 + 32 * M, q.segn);
      for (int i = w0 + lane; i < w1; i += 32) gx[q.gbase + i] = xs[i];
    }
    __syncthreads();  // every warp's x has left the d tile; the line maxima of this CTA are in
    // arrive on the cluster barrier now and wait only after the next chunk's d copies are out
    ++epoch;
    cluster_arrive();
    if (overlap && has_next && tid == 0)
      packed_bulk<TR>(A, packed_seg(PT, g + n_clusters, rank), ta, tb, tc, td, &tbar, 8, true);
    cluster_wait();  // the atomics of every CTA are complete and visible
    // ---------------- stop rule per line: every CTA evaluates all lines of the chunk
    const bool again =
        __syncthreads_or(packed_first_verdict(P.ch, PT.norms, A.tol, A.max_iters <= 1, rank == 0, A.st)) != 0;
    int it = 1;
    if (again && A.max_iters > 1) {
      if constexpr (IP) {  // further corrections here, d from the shared-memory pairs
        it = packed_more_passes<C, TR>(A, PT, P, coord ? nullptr : td2 + r[3].sh + tid * M, X, xph, epoch, alive,
                                       tid, w, lane, rank, kp, coord);
      } else if (rank == 0 && tid == 0) {  // listed for packed_fixup_kernel (every CTA reached the same verdict)
        PT.fix[1 + atomicAdd(PT.fix, 1u)] = (uint32_t)g;
      }
    }
    if (rank == 0 && tid == 0) report_iters(A.st, it);
  }
  if (!started) cluster_wait();  // a cluster without a chunk still completes the start-up barrier
}

// Further corrections of the chunks that packed_refine_kernel (out of place) listed, launched
// after it on the same stream: cluster k takes listed chunks k, k + K, ... with the same thread
// geometry (the partitions of a chunk, warp 7 coordinating Stage B). x, the coefficients and d
// come from global memory; the per-line table holds the first correction's maxima.
template <int C, bool TR>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(kPackThreads, 2)
    packed_fixup_kernel(const Args A, const PackedTables PT) {
  __shared__ __align__(16) PackedXchg<C> X;
  const int n_fix = (int)ld_relaxed_u32(PT.fix);  // written by the previous launch
  if ((int)(blockIdx.x / C) >= n_fix) return;       // the whole cluster leaves together
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const bool coord = w == kPackW;
  const int rank = (int)cluster_rank();
  const int kp = rank * kPackT + tid;
  if (tid == 0) packed_xchg_init<C>(X);
  __syncthreads();
  cluster_arrive();  // every CTA's barriers are initialised before the first remote store
  cluster_wait();
  bool alive = true;
  uint32_t xph[2] = {0u, 0u}, epoch = 0u;
  for (int k = (int)(blockIdx.x / C); k < n_fix; k += (int)(gridDim.x / C)) {
    const PackedPart P = packed_part<C>(PT, (int)PT.fix[1 + k], rank, tid, kp, coord);
    const int it = packed_more_passes<C, TR>(A, PT, P, nullptr, X, xph, epoch, alive, tid, w, lane, rank, kp, coord);
    if (rank == 0 && tid == 0) report_iters(A.st, it);
  }
}

}  // namespace tdma
