// Exact residual of one tridiagonal row for FP64 operands, on the integer pipes (host and device
// code, so that a host program can check it against exact rational arithmetic).
#pragma once
#include <cstdint>
#include "bits.cuh"

namespace tdma {

// ---- exact residual of one row, r = d - a xm - b x - c xp, for FP64 operands ----------------
// The three products of 53-bit significands are exact 106-bit integers; they and d are placed in
// one 128-bit two's-complement fixed-point accumulator whose unit is 2^(E - 106), E bounding the
// exponent of the largest term (the sum, below 2^(E + 2), cannot overflow). Bits of a term below
// that unit are dropped (in all under 2^-104 of the largest term, far below a residual of an FP64
// solution); everything else is exact integer arithmetic. The result is returned as a float
// truncated to 24 significant bits (0 below the float range); non-finite operands give NaN.
// Integer pipes only, and no branch depends on the operands.
struct U128 { uint64_t lo, hi; };

TDMA_HD U128 mul_u64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return U128{a * b, __umul64hi(a, b)};
#else
  const unsigned __int128 p = (unsigned __int128)a * b;
  return U128{(uint64_t)p, (uint64_t)(p >> 64)};
#endif
}
TDMA_HD U128 add_u128(U128 a, U128 b) {
  const uint64_t lo = a.lo + b.lo;
  return U128{lo, a.hi + b.hi + (lo < a.lo ? 1ull : 0ull)};
}
TDMA_HD U128 neg_u128(U128 a) { return add_u128(U128{~a.lo, ~a.hi}, U128{1ull, 0ull}); }

// v = (-1)^neg * m * 2^e with m < 2^53; false for infinities and NaN
TDMA_HD bool decode_f64(double v, uint64_t& m, int& e, bool& neg) {
  const uint64_t u = dbits(v);
  neg = (u >> 63) != 0;
  const int ef = (int)((u >> 52) & 0x7FF);
  const uint64_t f = u & ((1ull << 52) - 1ull);
  if (ef == 0x7FF) return false;
  if (ef == 0) { m = f; e = -1074; }
  else { m = f | (1ull << 52); e = ef - 1075; }
  return true;
}

// an FP64 operand decoded once: (-1)^neg * m * 2^e, ok = finite
struct DecF64 {
  uint64_t m;
  int e;
  bool neg, ok;
};
TDMA_HD DecF64 dec_f64(double v) {
  DecF64 r;
  r.ok = decode_f64(v, r.m, r.e, r.neg);
  return r;
}

// v >> s for s >= 0 (0 for s >= 128), without branches: both 64-bit halves computed, then selected
TDMA_HD U128 shr_u128_bf(U128 v, uint32_t s) {
  const uint32_t sm = s & 63u;
  const uint64_t lo_a = (v.lo >> sm) | ((v.hi << 1) << (63u - sm));  // (hi << (64 - sm)) for sm in 0..63
  const uint64_t hi_a = v.hi >> sm;
  const bool big = s >= 64u, gone = s >= 128u;
  return U128{gone ? 0ull : (big ? hi_a : lo_a), big ? 0ull : hi_a};
}
// m << s for m < 2^53 and 0 <= s <= 71, without branches
TDMA_HD U128 shl_u53_bf(uint64_t m, uint32_t s) {
  const uint32_t sm = s & 63u;
  const uint64_t lo_a = m << sm, hi_a = (m >> 1) >> (63u - sm);  // (m >> (64 - sm)) for sm in 0..63
  const bool big = s >= 64u;
  return U128{big ? 0ull : lo_a, big ? lo_a : hi_a};
}

// residual_exact on decoded operands (a kernel decodes shared coefficients once). The fixed-point
// unit is 2^(E - 106), E bounding the largest term, so every product term is shifted right (its
// bits below the unit dropped: under 2^-104 of the largest term in all) and only d may move left;
// the sum stays below 2^(E + 2), well inside 128 bits. No branches depend on the operands.
TDMA_HD float residual_exact_dec(const DecF64& dd, const DecF64& da, const DecF64& dxm, const DecF64& db,
                                 const DecF64& dx, const DecF64& dc, const DecF64& dxp) {
  const bool finite_all = dd.ok && da.ok && dxm.ok && db.ok && dx.ok && dc.ok && dxp.ok;
  const U128 p1 = mul_u64(da.m, dxm.m), p2 = mul_u64(db.m, dx.m), p3 = mul_u64(dc.m, dxp.m);
  const int e1 = da.e + dxm.e, e2 = db.e + dx.e, e3 = dc.e + dxp.e;
  const bool z1 = (p1.lo | p1.hi) == 0ull, z2 = (p2.lo | p2.hi) == 0ull, z3 = (p3.lo | p3.hi) == 0ull;
  const bool z0 = dd.m == 0ull;
  const int lowest = -100000;
  int top = z0 ? lowest : dd.e + 53;
  top = max(top, z1 ? lowest : e1 + 106);
  top = max(top, z2 ? lowest : e2 + 106);
  top = max(top, z3 ? lowest : e3 + 106);
  const int unit = top - 106;
  // product terms: shifted right by top - (e + 106) >= 0; zero terms contribute nothing
  const U128 t1 = shr_u128_bf(p1, z1 ? 128u : (uint32_t)(top - (e1 + 106)));
  const U128 t2 = shr_u128_bf(p2, z2 ? 128u : (uint32_t)(top - (e2 + 106)));
  const U128 t3 = shr_u128_bf(p3, z3 ? 128u : (uint32_t)(top - (e3 + 106)));
  // d: shifted by dd.e - unit, which is at most 53
  const int sd = dd.e - unit;
  U128 t0 = sd >= 0 ? shl_u53_bf(dd.m, (uint32_t)min(sd, 71)) : shr_u128_bf(U128{dd.m, 0ull}, (uint32_t)min(-sd, 128));
  if (z0) t0 = U128{0ull, 0ull};
  // acc = d - a xm - b x - c xp (two's complement)
  const bool n1 = da.neg == dxm.neg, n2 = db.neg == dx.neg, n3 = dc.neg == dxp.neg;  // the term is -(product)
  U128 acc = dd.neg ? neg_u128(t0) : t0;
  acc = add_u128(acc, n1 ? neg_u128(t1) : t1);
  acc = add_u128(acc, n2 ? neg_u128(t2) : t2);
  acc = add_u128(acc, n3 ? neg_u128(t3) : t3);
  const bool rneg = (acc.hi >> 63) != 0ull;
  if (rneg) acc = neg_u128(acc);
  const bool zero = (acc.lo | acc.hi) == 0ull;
  int lz;
#ifdef __CUDA_ARCH__
  lz = acc.hi ? __clzll((long long)acc.hi) : 64 + __clzll((long long)acc.lo);
#else
  lz = acc.hi ? __builtin_clzll(acc.hi) : (acc.lo ? 64 + __builtin_clzll(acc.lo) : 128);
#endif
  const int p = 127 - lz;  // leading bit of the magnitude
  const uint64_t top24 = p >= 23 ? shr_u128_bf(acc, (uint32_t)(p - 23)).lo : (acc.lo << (uint32_t)max(23 - p, 0));
  const int be = unit + p + 127;  // biased float exponent of the result
  const uint32_t sign = rneg ? 0x80000000u : 0u;
  uint32_t bits = sign | ((uint32_t)max(min(be, 254), 1) << 23) | ((uint32_t)top24 & 0x7FFFFFu);
  if (be <= 0 || zero || top == lowest) bits = sign;    // below the float range (or exactly zero)
  if (be >= 255) bits = sign | 0x7F800000u;
  if (!finite_all) bits = 0x7FC00000u;
  return bitsf(bits);
}

TDMA_HD float residual_exact(double d, double a, double xm, double b, double x, double c, double xp) {
  return residual_exact_dec(dec_f64(d), dec_f64(a), dec_f64(xm), dec_f64(b), dec_f64(x), dec_f64(c), dec_f64(xp));
}

// Float with the leading 24 significant bits of a double (truncated), on the integer pipe for
// normal magnitudes (the plain conversion otherwise).
TDMA_HD float f64_to_f32_trunc(double v) {
  float h, l;
  if (split_normal(v, h, l)) return h;
  return (float)v;
}

}  // namespace tdma
