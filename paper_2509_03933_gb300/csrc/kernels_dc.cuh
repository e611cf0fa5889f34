// Fused divide-and-conquer solve of uniform lines: Stage A, Stage B and Stage C in one block.
//
// Section 2.1 splits each system into p partitions: Stage A solves the decoupled partitions,
// Stage B the reduced interface system (size 2p - 2, Section 2.2), Stage C corrects every
// unknown (about 4 L / p flops). On one GPU a partition is one thread: thread (j, k) of a
// block owns partition k of line j, adjacent threads own adjacent lines, so on strided axes
// a warp's loads of one row are contiguous. The paper's A2B/B2C messages become shared
// memory traffic inside the block.
//
// Stage A here is the modified Thomas sweep (each partition reduced to relations between
// its two endpoint unknowns and the neighbouring partitions' endpoints):
//   row 0:           a_0 x_{-1} + b_0 x_0 + c_0 x_1 = d_0             (kept in registers)
//   rows t = 1..m-1: alpha_t x_0 + x_t + gamma_t x_{t+1} = delta_t, with
//     r = 1 / (b_t - a_t gamma_{t-1}), alpha_t = -r a_t alpha_{t-1}, gamma_t = r c_t,
//     delta_t = r (d_t - a_t delta_{t-1}), starting from (alpha, gamma, delta) = (-1, 0, 0).
//   Row m-1 is then a reduced row. Row 1 expressed through x_0 and x_{m-1} is accumulated
//   in the same forward pass (x_1 = F - G x_0 + Q x_{m-1}, F = sum Q_t delta_t,
//   G = sum Q_t alpha_t, Q_{t+1} = -Q_t gamma_t over t = 1..m-2), so row 0 becomes the
//   other reduced row without a backward elimination pass:
//     rho = 1 / (b_0 - c_0 G): rho a_0 x_{-1} + x_0 + rho c_0 Q x_{m-1} = rho (d_0 - c_0 F).
// Stage B solves the 2P-row unit-diagonal tridiagonal system of every line by Thomas, one
// thread per line. Stage C walks back: x_t = delta_t - alpha_t x_0 - gamma_t x_{t+1}.
#pragma once
#include "layout.cuh"

namespace tdma {

template <class CT, int NR> struct Row {
  CT a, b, c;
  CT d[NR];
};

// Row i of the system, or with TR of its transpose A^T (sub-diagonal c_{i-1}, super-diagonal
// a_{i+1}; the adjoint solve of the backward pass). Reads stay inside the line.
template <class CT, int NR, bool TR = false>
TDMA_DEV void load_row(Row<CT, NR>& r, const Args& A, int64_t e, int64_t i, CT shift) {
  const int64_t ci = A.bcast ? i : e;
  if constexpr (TR) {
    const int64_t st = A.bcast ? 1 : A.lay.es;
    r.a = i > 0 ? ldg((const CT*)A.c + ci - st) : CT(0);
    r.c = i < A.lay.n - 1 ? ldg((const CT*)A.a + ci + st) : CT(0);
  } else {
    r.a = ldg((const CT*)A.a + ci);
    r.c = ldg((const CT*)A.c + ci);
  }
  r.b = ldg((const CT*)A.b + ci) + shift;
  if constexpr (NR == 1) {
    r.d[0] = ldg((const CT*)A.d + e);
  } else if constexpr (sizeof(CT) == 8) {
    const double2 v = ldg((const double2*)A.d + e);
    r.d[0] = v.x;
    r.d[1] = v.y;
  } else {
    const float2 v = ldg((const float2*)A.d + e);
    r.d[0] = v.x;
    r.d[1] = v.y;
  }
}

template <class CT, int NR> TDMA_DEV void store_x(const Args& A, int64_t e, const CT* v) {
  if constexpr (NR == 1) {
    ((CT*)A.x)[e] = v[0];
  } else if constexpr (sizeof(CT) == 8) {
    ((double2*)A.x)[e] = make_double2(v[0], v[1]);
  } else {
    ((float2*)A.x)[e] = make_float2(v[0], v[1]);
  }
}

// In-place Thomas on a unit-diagonal tridiagonal system of `rows` rows held in shared memory.
// On return rhs[r][*] holds the solution. Returns false on a non-finite result.
template <class AT, int NR>
TDMA_DEV bool reduced_solve(AT* sub, AT* sup, AT* rhs, int rows, int rhs_pitch) {
  AT cp = sup[0];
  AT dp[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) dp[r] = rhs[r * rhs_pitch];
  for (int i = 1; i < rows; ++i) {
    const AT s = sub[i];
    const AT iw = rcp(AT(1) - s * cp);
    cp = sup[i] * iw;
    sup[i] = cp;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      dp[r] = (rhs[r * rhs_pitch + i] - s * dp[r]) * iw;
      rhs[r * rhs_pitch + i] = dp[r];
    }
  }
  bool ok = true;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    AT u = dp[r];
    ok &= finite(u);
    for (int i = rows - 2; i >= 0; --i) {
      u = rhs[r * rhs_pitch + i] - sup[i] * u;
      rhs[r * rhs_pitch + i] = u;
    }
    ok &= finite(u);
  }
  return ok;
}

// Reduced systems longer than this many rows are solved in two levels (below).
constexpr int kTwoLevelRows = 32;
constexpr int kTwoLevelSeg = 16;
__host__ __device__ inline int two_level_groups(int R2) {
  return R2 > kTwoLevelRows ? (R2 + kTwoLevelSeg - 1) / kTwoLevelSeg : 0;
}

// Two-level solve of the unit-diagonal reduced systems (R2 = 2P rows, NR right-hand sides) of the
// lines of a block, in place: the solution replaces the right-hand sides. Line j's system sits at
// red + j * pitch as sub[R2], sup[R2], rhs[NR][R2]. One thread per line over 2P rows is a chain
// of 2P dependent reciprocals, and a dependent FP64 operation of one thread takes about 85 cycles
// on GB300 (a 512-row system: about 150 us). Level 1: the rows are cut into G segments of
// kTwoLevelSeg rows, one thread per segment, each reduced to its two end rows by the modified
// Thomas sweep of Stage A (unit diagonal); level 2: one thread per line solves the 2G end rows
// (kept after the Lr line regions); level 1 back: each segment's interior from its two end
// values. Thread q * Lr + j works on segment q of line j; lines j >= lines_valid are skipped;
// every thread of the block must call this.
template <class CT, int NR>
TDMA_DEV void reduced_two_level(CT* red, int pitch, int Lr, int lines_valid, int R2, DevStatus* st) {
  constexpr int S = kTwoLevelSeg;
  const int G = (R2 + S - 1) / S, tid = threadIdx.x;
  const int j = tid % Lr, q = tid / Lr;
  const bool act = q < G && j < lines_valid;
  CT* r_sub = red + (size_t)j * pitch;
  CT* r_sup = r_sub + R2;
  CT* r_rhs = r_sup + R2;
  CT* s2 = red + (size_t)Lr * pitch + (size_t)j * (2 + NR) * 2 * G;  // level-2 rows of line j
  CT* c2 = s2 + 2 * G;
  CT* h2 = c2 + 2 * G;  // NR blocks of 2G
  const int r0 = q * S, len = R2 - r0 < S ? R2 - r0 : S;
  bool ok = true;
  if (act) {
    const CT sub0 = r_sub[r0], sup0 = r_sup[r0];
    CT h0[NR], delta[NR], F[NR];
    CT alpha = CT(-1), gamma = CT(0), Gs = CT(0), Q = CT(1);
#pragma unroll
    for (int e = 0; e < NR; ++e) { h0[e] = r_rhs[e * R2 + r0]; delta[e] = CT(0); F[e] = CT(0); }
    for (int t = 1; t < len; ++t) {
      const int i = r0 + t;
      const CT sb = r_sub[i], c = r_sup[i];
      const CT r = rcp(CT(1) - sb * gamma);
      ok &= finite(r);
      const CT ar = sb * r;
      alpha = -ar * alpha;
      gamma = c * r;
#pragma unroll
      for (int e = 0; e < NR; ++e) delta[e] = r * r_rhs[e * R2 + i] - ar * delta[e];
      if (t <= len - 2) {
        r_sub[i] = alpha;
        r_sup[i] = gamma;
#pragma unroll
        for (int e = 0; e < NR; ++e) {
          r_rhs[e * R2 + i] = delta[e];
          F[e] += Q * delta[e];
        }
        Gs += Q * alpha;
        Q = -Q * gamma;
      }
    }
    const CT rho = rcp(CT(1) - sup0 * Gs);
    ok &= finite(rho);
    s2[2 * q] = rho * sub0;
    c2[2 * q] = rho * sup0 * Q;
    s2[2 * q + 1] = alpha;
    c2[2 * q + 1] = gamma;
#pragma unroll
    for (int e = 0; e < NR; ++e) {
      h2[e * 2 * G + 2 * q] = rho * (h0[e] - sup0 * F[e]);
      h2[e * 2 * G + 2 * q + 1] = delta[e];
    }
  }
  __syncthreads();
  if (tid < lines_valid) ok &= reduced_solve<CT, NR>(s2, c2, h2, 2 * G, 2 * G);
  __syncthreads();
  if (act) {
#pragma unroll
    for (int e = 0; e < NR; ++e) {
      const CT xf = h2[e * 2 * G + 2 * q];
      CT xn = h2[e * 2 * G + 2 * q + 1];
      r_rhs[e * R2 + r0] = xf;
      r_rhs[e * R2 + r0 + len - 1] = xn;
      for (int t = len - 2; t >= 1; --t) {
        const int i = r0 + t;
        xn = r_rhs[e * R2 + i] - r_sub[i] * xf - r_sup[i] * xn;
        r_rhs[e * R2 + i] = xn;
      }
    }
  }
  if (!ok) report_error(st, 5);
}

// Parallel diagonally dominant (PDD) reduced solve for partition k of P. Stage A left partition
// j's end rows as the unit-diagonal pair
//     sub[2j] x_{j-1,last} + x_{j,0} + sup[2j] x_{j,last} = rhs[2j],
//     sub[2j+1] x_{j,0} + x_{j,last} + sup[2j+1] x_{j+1,0} = rhs[2j+1],
// which solved for the ends give the spike form x_{j,0} = t0 - v0 y_L - w0 y_R and
// x_{j,last} = tL - vL y_L - wL y_R in the neighbours' end values y_L = x_{j-1,last},
// y_R = x_{j+1,0}. At the interface of partitions j and j+1 the method drops v_j(last) y_L and
// w_{j+1}(0) y_R, leaving the 2x2 system
//     y1 + wL_j y2 = tL_j,    v0_{j+1} y1 + y2 = t0_{j+1}
// for y1 = x_{j,last}, y2 = x_{j+1,0}. Partition k takes y_L from its left interface, y_R from
// its right one (0 at the ends of the line) and returns its end values from the spike form;
// nothing is written, so every partition reads its neighbours' rows directly.
template <class CT, int NR> struct PddEnds {
  CT v0, w0, vL, wL, t0[NR], tL[NR];
};
template <class CT, int NR>
TDMA_DEV PddEnds<CT, NR> pdd_spikes(const CT* sub, const CT* sup, const CT* rhs, int R2, int j) {
  const CT A0 = sub[2 * j], C0 = sup[2 * j], A1 = sub[2 * j + 1], C1 = sup[2 * j + 1];
  const CT id = rcp(CT(1) - C0 * A1);
  PddEnds<CT, NR> e;
  e.v0 = A0 * id;
  e.w0 = -C0 * C1 * id;
  e.vL = -A1 * A0 * id;
  e.wL = C1 * id;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    const CT D0 = rhs[q * R2 + 2 * j], D1 = rhs[q * R2 + 2 * j + 1];
    e.t0[q] = (D0 - C0 * D1) * id;
    e.tL[q] = (D1 - A1 * D0) * id;
  }
  return e;
}
template <class CT, int NR>
TDMA_DEV void pdd_ends(const CT* sub, const CT* sup, const CT* rhs, int R2, int k, int P, CT* x0, CT* xn) {
  const PddEnds<CT, NR> e = pdd_spikes<CT, NR>(sub, sup, rhs, R2, k);
  CT yl[NR], yr[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) { yl[q] = CT(0); yr[q] = CT(0); }
  if (k > 0) {  // left interface: y1 = x_{k-1,last}
    const PddEnds<CT, NR> l = pdd_spikes<CT, NR>(sub, sup, rhs, R2, k - 1);
    const CT id = rcp(CT(1) - l.wL * e.v0);
#pragma unroll
    for (int q = 0; q < NR; ++q) yl[q] = (l.tL[q] - l.wL * e.t0[q]) * id;
  }
  if (k < P - 1) {  // right interface: y2 = x_{k+1,0}
    const PddEnds<CT, NR> r = pdd_spikes<CT, NR>(sub, sup, rhs, R2, k + 1);
    const CT id = rcp(CT(1) - e.wL * r.v0);
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const CT y1 = (e.tL[q] - e.wL * r.t0[q]) * id;
      yr[q] = r.t0[q] - r.v0 * y1;
    }
  }
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    x0[q] = e.t0[q] - e.v0 * yl[q] - e.w0 * yr[q];
    xn[q] = e.tL[q] - e.vL * yl[q] - e.wL * yr[q];
  }
}

// Shared-memory plan of the fused kernel (all in units of CT):
//   scratch  alpha, gamma, delta[NR]: (mmax - 2) slots x T threads each, slot-major
//   reduced  per line: sub[2P], sup[2P], rhs[NR][2P], line pitch (2 + NR) 2P + 1
template <class CT, int NR>
__host__ __device__ inline size_t dc_smem_bytes(int T, int Lb, int P, int mmax) {
  const size_t slots = mmax > 2 ? (size_t)(mmax - 2) : 0;
  const size_t pitch = (size_t)(2 + NR) * 2 * P + 1;
  const size_t level2 = (size_t)Lb * (2 + NR) * 2 * two_level_groups(2 * P);  // two-level Stage B
  return sizeof(CT) * ((2 + NR) * slots * T + (size_t)Lb * pitch + level2);
}

constexpr int kChunk = 2;  // rows loaded ahead of the forward sweep

// GS: the per-row Stage A scratch lives in the workspace (a [slot][thread] region per block)
// instead of shared memory, for partitions too long to keep enough threads per SM on chip.
template <class CT, int NR, bool TR = false, bool GS = false>
__global__ void __launch_bounds__(512) dc_kernel(const Args A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT* sm = reinterpret_cast<CT*>(smem_raw);
  const int T = blockDim.x, tid = threadIdx.x;
  const int P = A.P, Lb = A.Lb;
  const int j = tid % Lb, k = tid / Lb;
  const int64_t line = (int64_t)blockIdx.x * Lb + j;
  const bool active = line < A.lay.n_lines;
  const int slots = A.mmax > 2 ? A.mmax - 2 : 0;
  CT* s_alpha = GS ? (CT*)A.ws + (size_t)blockIdx.x * (2 + NR) * slots * T : sm;
  CT* s_gamma = s_alpha + (size_t)slots * T;
  CT* s_delta = s_gamma + (size_t)slots * T;  // NR blocks
  CT* red = GS ? sm : s_delta + (size_t)NR * slots * T;
  const int R2 = 2 * P;
  const int pitch = (2 + NR) * R2 + 1;
  CT* r_sub = red + (size_t)j * pitch;
  CT* r_sup = r_sub + R2;
  CT* r_rhs = r_sup + R2;

  int64_t start = 0;
  int m = 0;
  partition(A.lay.n, P, k, start, m);
  const int64_t base = active ? A.lay.off(line) : 0;
  const int64_t es = A.lay.es;
  const CT shift = (active && A.shift) ? ldg((const CT*)A.shift + line) : CT(0);

  // ---------------- Stage A: forward modified-Thomas sweep
  if (active) {
    Row<CT, NR> r0;
    load_row<CT, NR, TR>(r0, A, base + start * es, start, shift);
    if (k == 0) r0.a = CT(0);                      // a_0 of the line is ignored
    if (m == 1) {                                  // n == 1: a single equation b x = d
      CT v[NR];
      const CT ib = rcp(r0.b);
#pragma unroll
      for (int q = 0; q < NR; ++q) v[q] = r0.d[q] * ib;
      bool ok = true;
#pragma unroll
      for (int q = 0; q < NR; ++q) ok &= finite(v[q]);
      if (!ok) report_error(A.st, 5);
      store_x<CT, NR>(A, base + start * es, v);
    } else {
      CT alpha = CT(-1), gamma = CT(0), delta[NR];
      CT Q = CT(1), G = CT(0), F[NR];
#pragma unroll
      for (int q = 0; q < NR; ++q) { delta[q] = CT(0); F[q] = CT(0); }

      Row<CT, NR> buf[kChunk];
#pragma unroll
      for (int u = 0; u < kChunk; ++u)
        if (1 + u < m) load_row<CT, NR, TR>(buf[u], A, base + (start + 1 + u) * es, start + 1 + u, shift);
      for (int t0 = 1; t0 < m; t0 += kChunk) {
        Row<CT, NR> nxt[kChunk];
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
          const int t = t0 + kChunk + u;
          if (t < m) load_row<CT, NR, TR>(nxt[u], A, base + (start + t) * es, start + t, shift);
        }
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
          const int t = t0 + u;
          if (t < m) {
            Row<CT, NR>& rw = buf[u];
            if (k == P - 1 && t == m - 1) rw.c = CT(0);  // c_{n-1} of the line is ignored
            const CT r = rcp(rw.b - rw.a * gamma);
            const CT ar = rw.a * r;
            alpha = -ar * alpha;
            gamma = rw.c * r;
#pragma unroll
            for (int q = 0; q < NR; ++q) delta[q] = r * rw.d[q] - ar * delta[q];
            if (t <= m - 2) {
              const size_t o = (size_t)(t - 1) * T + tid;
              s_alpha[o] = alpha;
              s_gamma[o] = gamma;
#pragma unroll
              for (int q = 0; q < NR; ++q) {
                s_delta[(size_t)q * slots * T + o] = delta[q];
                F[q] += Q * delta[q];
              }
              G += Q * alpha;
              Q = -Q * gamma;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < kChunk; ++u) buf[u] = nxt[u];
      }
      // reduced rows 2k (row 0 after the fix) and 2k+1 (row m-1)
      const CT rho = rcp(r0.b - r0.c * G);
      r_sub[2 * k] = rho * r0.a;
      r_sup[2 * k] = rho * r0.c * Q;
      r_sub[2 * k + 1] = alpha;
      r_sup[2 * k + 1] = gamma;
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        r_rhs[q * R2 + 2 * k] = rho * (r0.d[q] - r0.c * F[q]);
        r_rhs[q * R2 + 2 * k + 1] = delta[q];
      }
    }
  }
  if (A.lay.n == 1) return;  // no Stage B / C for single-unknown lines
  __syncthreads();

  // ---------------- Stage B: reduced 2P-row system per line, one thread per line or in two
  // levels above 32 rows (exact), or the PDD interface systems, each partition's thread on its
  // own (approximate)
  if (!A.pdd && R2 > kTwoLevelRows) {
    const int64_t left = A.lay.n_lines - (int64_t)blockIdx.x * Lb;
    reduced_two_level<CT, NR>(red, pitch, Lb, left < Lb ? (int)left : Lb, R2, A.st);
    __syncthreads();
  } else if (!A.pdd) {
    if (tid < Lb) {
      const int64_t l2 = (int64_t)blockIdx.x * Lb + tid;
      if (l2 < A.lay.n_lines) {
        CT* sub = red + (size_t)tid * pitch;
        if (!reduced_solve<CT, NR>(sub, sub + R2, sub + 2 * R2, R2, R2)) report_error(A.st, 5);
      }
    }
    __syncthreads();
  }

  // ---------------- Stage C: endpoint values from Stage B, interior by back substitution
  if (active) {
    CT x0[NR], xn[NR];
    if (A.pdd) {
      pdd_ends<CT, NR>(r_sub, r_sup, r_rhs, R2, k, P, x0, xn);
      bool ok = true;
#pragma unroll
      for (int q = 0; q < NR; ++q) ok &= finite(x0[q]) && finite(xn[q]);
      if (!ok) report_error(A.st, 5);
    } else {
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        x0[q] = r_rhs[q * R2 + 2 * k];
        xn[q] = r_rhs[q * R2 + 2 * k + 1];
      }
    }
    store_x<CT, NR>(A, base + start * es, x0);
    store_x<CT, NR>(A, base + (start + m - 1) * es, xn);
    for (int t = m - 2; t >= 1; --t) {
      const size_t o = (size_t)(t - 1) * T + tid;
      const CT al = s_alpha[o], ga = s_gamma[o];
#pragma unroll
      for (int q = 0; q < NR; ++q) xn[q] = s_delta[(size_t)q * slots * T + o] - al * x0[q] - ga * xn[q];
      store_x<CT, NR>(A, base + (start + t) * es, xn);
    }
  }
}

}  // namespace tdma
