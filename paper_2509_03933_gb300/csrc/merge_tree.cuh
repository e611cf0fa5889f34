// Merge trees over partition blocks (Stage B of the divide-and-conquer solve), cluster
// exchange helpers and the extra-precise float residual, shared by the cluster kernels.
//
// A run of rows [s, e] of a tridiagonal system, solved for its own right-hand side, leaves its
// first and last unknowns as affine functions of the two unknowns just outside it,
// u = x_{s-1} and v = x_{e+1} (the block form below). Two adjacent blocks merge into the block
// of their union by eliminating the two unknowns on either side of their boundary; a tree of
// merges over all partitions of a line reduces the line to one block, and since the line ends
// have no outside neighbours (u = v = 0) the tree walked back down hands every partition its
// own u and v (Section 2.1: the reduced solve of Stage B, exact like the paper's x = x~ - Y y).
#pragma once
#include "common.cuh"
#include "tma.cuh"

namespace tdma {

// x_s = p1 + q1 u + r1 v and x_e = p2 + q2 u + r2 v for a row range [s, e] of a line.
struct Blk { float p1, q1, r1, p2, q2, r2; };
// one interior unknown of a merge as an affine function of the merged block's (u, v)
struct Aff { float p, q, r; };

TDMA_DEV Blk shfl_xor_blk(const Blk& b, int m) {
  return {__shfl_xor_sync(~0u, b.p1, m), __shfl_xor_sync(~0u, b.q1, m), __shfl_xor_sync(~0u, b.r1, m),
          __shfl_xor_sync(~0u, b.p2, m), __shfl_xor_sync(~0u, b.q2, m), __shfl_xor_sync(~0u, b.r2, m)};
}

// Block form of one partition from its two Stage A rows (see the header).
TDMA_DEV Blk part_block(float S, float U, float H, float al, float Ga, float De) {
  const float id = rcp(fmaf(-U, al, 1.f));
  return {id * fmaf(-U, De, H), -S * id, id * (U * Ga), id * fmaf(-al, H, De), id * (al * S), -Ga * id};
}

// Merge L = [s1, e1] and R = [e1 + 1, e2]. From y = L.p2 + L.q2 u + L.r2 z and
// z = R.p1 + R.q1 y + R.r1 v: y (1 - L.r2 R.q1) = L.p2 + L.r2 R.p1 + L.q2 u + L.r2 R.r1 v, then
// z from y; the merged rows are L's first row with z and R's last row with y substituted.
// `keep` receives the unknown that becomes this lane's neighbour on the way down: y for a lane
// inside R (its u), z for a lane inside L (its v).
TDMA_DEV Blk merge(const Blk& L, const Blk& R, bool in_right, Aff& keep) {
  const float D = rcp(fmaf(-L.r2, R.q1, 1.f));
  const float py = D * fmaf(L.r2, R.p1, L.p2);
  const float qy = D * L.q2;
  const float ry = D * (L.r2 * R.r1);
  const float pz = fmaf(R.q1, py, R.p1);
  const float qz = R.q1 * qy;
  const float rz = fmaf(R.q1, ry, R.r1);
  keep = in_right ? Aff{py, qy, ry} : Aff{pz, qz, rz};
  return {fmaf(L.r1, pz, L.p1), fmaf(L.r1, qz, L.q1), L.r1 * rz, fmaf(R.q2, py, R.p2), R.q2 * qy, fmaf(R.q2, ry, R.r2)};
}

// Up-sweep over 2^LV consecutive blocks held by lanes whose index bits SH.. carry the block
// number g; every lane of a group ends with the group's merged block.
template <int LV, int SH = 2, int NK = 3>
TDMA_DEV Blk tree_up(Blk b, int g, Aff (&keep)[NK]) {
#pragma unroll
  for (int l = 0; l < LV; ++l) {
    const Blk o = shfl_xor_blk(b, 1 << (SH + l));
    const bool in_right = (g >> l) & 1;
    b = merge(in_right ? o : b, in_right ? b : o, in_right, keep[l]);
  }
  return b;
}
// Down-sweep: (u, v) of the whole group in, (u, v) of this lane's block out.
template <int LV, int NK = 3>
TDMA_DEV void tree_down(float& u, float& v, int g, const Aff (&keep)[NK]) {
#pragma unroll
  for (int l = LV - 1; l >= 0; --l) {
    const float val = fmaf(keep[l].q, u, fmaf(keep[l].r, v, keep[l].p));
    if ((g >> l) & 1) u = val; else v = val;
  }
}

// Cluster level: the merges keep both interior unknowns, so that the down-sweep also gives each
// block the values of its own first and last unknowns exactly as its neighbours see them (the
// lowest level that sets u = y also gives x_s = z; the one that sets v = z gives x_e = y).
struct Mrg { Aff y, z; };
template <int LV, int SH = 2>
TDMA_DEV Blk tree_up_full(Blk b, int g, Mrg (&keep)[3]) {
#pragma unroll
  for (int l = 0; l < LV; ++l) {
    const Blk o = shfl_xor_blk(b, 1 << (SH + l));
    const bool in_right = (g >> l) & 1;
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
    keep[l] = Mrg{y, z};
    b = Blk{fmaf(L.r1, z.p, L.p1), fmaf(L.r1, z.q, L.q1), L.r1 * z.r, fmaf(R.q2, y.p, R.p2), R.q2 * y.q, fmaf(R.q2, y.r, R.r2)};
  }
  return b;
}
template <int LV>
TDMA_DEV void tree_down_full(float& u, float& v, float& xs, float& xe, int g, const Mrg (&keep)[3]) {
#pragma unroll
  for (int l = LV - 1; l >= 0; --l) {
    const float y = fmaf(keep[l].y.q, u, fmaf(keep[l].y.r, v, keep[l].y.p));
    const float z = fmaf(keep[l].z.q, u, fmaf(keep[l].z.r, v, keep[l].z.p));
    if ((g >> l) & 1) { u = y; xs = z; } else { v = z; xe = y; }
  }
}

// ---- cluster helpers (inline PTX) ------------------------------------------------------
TDMA_DEV uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
TDMA_DEV void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
TDMA_DEV void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
// shared::cluster address of `p` in the shared memory of CTA `rank`
TDMA_DEV uint32_t map_rank(const void* p, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
// Asynchronous stores into another CTA's shared memory; each completes `bytes` of the
// transaction count of the mbarrier at `bar` in that CTA (st.async, sm_90+).
TDMA_DEV void st_async4(uint32_t addr, float a, float b, float c, float d, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(addr),
               "f"(a), "f"(b), "f"(c), "f"(d), "r"(bar)
               : "memory");
}
TDMA_DEV void st_async2(uint32_t addr, unsigned a, unsigned b, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.u32 [%0], {%1, %2}, [%3];" ::"r"(addr), "r"(a),
               "r"(b), "r"(bar)
               : "memory");
}

// Norms travel as the bit patterns of |v|: for non-negative floats the unsigned order is the
// numeric order, and NaN (above +inf) survives a max reduction, so one test after the reduction
// (bits >= 0x7f800000) finds any non-finite value.
TDMA_DEV unsigned abs_bits(float v) { return __float_as_uint(v) & 0x7fffffffu; }
TDMA_DEV bool bits_finite(unsigned b) { return b < 0x7f800000u; }
// r = d - (a xm + b x + c xp) for float x values and d = dh + dl, as if in twice the float
// precision: FMA TwoProduct of the three products and TwoSum of the first two subtractions,
// whose results are of the size of x. The last subtraction is either exact (Sterbenz: both
// operands within a factor two) or already of the size of the residual, so it is rounded once.
TDMA_DEV float residual_f(float a, float b, float c, float dh, float dl, float xm, float x, float xp) {
  const ff p1 = two_prod(b, x), p2 = two_prod(a, xm), p3 = two_prod(c, xp);
  const ff s1 = two_sum(dh, -p1.h);
  const ff s2 = two_sum(s1.h, -p2.h);
  const float s3 = __fsub_rn(s2.h, p3.h);
  const float err = __fsub_rn(__fadd_rn(__fadd_rn(dl, s1.l), s2.l), __fadd_rn(__fadd_rn(p1.l, p2.l), p3.l));
  return __fadd_rn(s3, err);
}

}  // namespace tdma
