// Exact residual of one tridiagonal row for FP64 operands, on the integer pipes (host and device
// code, so that a host program can check it against exact rational arithmetic).
#pragma once
#include <cstdint>
#include "bits.cuh"

namespace tdma {

// ---- exact residual of one row, r = d - a xm - b x - c xp, for FP64 operands ----------------
// The three products of 53-bit significands are exact 106-bit integers; they and d are placed in
// one 128-bit two's-complement fixed-point accumulator whose unit is 2^(E - 124), E bounding the
// exponent of the largest term (so the sum, below 2^(E + 2), cannot overflow). Bits of a term
// below that unit are dropped (an error under 2^-122 of the largest term); everything else is
// exact integer arithmetic. The result is returned as a float truncated to 24 significant bits
// (0 below the float range); non-finite operands give NaN. Integer pipes only: no FP64 arithmetic.
struct U128 { uint64_t lo, hi; };

TDMA_HD U128 mul_u64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return U128{a * b, __umul64hi(a, b)};
#else
  const unsigned __int128 p = (unsigned __int128)a * b;
  return U128{(uint64_t)p, (uint64_t)(p >> 64)};
#endif
}
TDMA_HD U128 shl_u128(U128 v, int s) {  // 0 <= s < 128
  if (s == 0) return v;
  if (s < 64) return U128{v.lo << s, (v.hi << s) | (v.lo >> (64 - s))};
  return U128{0ull, v.lo << (s - 64)};
}
TDMA_HD U128 shr_u128(U128 v, int s) {  // s >= 0
  if (s == 0) return v;
  if (s >= 128) return U128{0ull, 0ull};
  if (s < 64) return U128{(v.lo >> s) | (v.hi << (64 - s)), v.hi >> s};
  return U128{v.hi >> (s - 64), 0ull};
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

// residual_exact on decoded operands (a kernel decodes shared coefficients once)
TDMA_HD float residual_exact_dec(const DecF64& dd, const DecF64& da, const DecF64& dxm, const DecF64& db,
                                 const DecF64& dx, const DecF64& dc, const DecF64& dxp) {
  uint64_t mv[7];
  int ev[7];
  bool sv[7];
  const DecF64* in[7] = {&dd, &da, &dxm, &db, &dx, &dc, &dxp};
  bool finite_all = true;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    mv[k] = in[k]->m;
    ev[k] = in[k]->e;
    sv[k] = in[k]->neg;
    finite_all &= in[k]->ok;
  }
  if (!finite_all) return bitsf(0x7FC00000u);
  // terms: d, and -a xm, -b x, -c xp as significand products
  U128 tm[4];
  int te[4], tw[4];
  bool tn[4];
  tm[0] = U128{mv[0], 0ull};
  te[0] = ev[0];
  tw[0] = 53;
  tn[0] = sv[0];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    tm[k + 1] = mul_u64(mv[1 + 2 * k], mv[2 + 2 * k]);
    te[k + 1] = ev[1 + 2 * k] + ev[2 + 2 * k];
    tw[k + 1] = 106;
    tn[k + 1] = !(sv[1 + 2 * k] != sv[2 + 2 * k]);  // the minus sign of the product term
  }
  int top = -100000;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if ((tm[k].lo | tm[k].hi) != 0ull && te[k] + tw[k] > top) top = te[k] + tw[k];
  if (top == -100000) return 0.f;
  const int unit = top - 124;
  U128 acc{0ull, 0ull};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if ((tm[k].lo | tm[k].hi) == 0ull) continue;  // zero terms (their exponent field means nothing)
    const int sh = te[k] - unit;  // at most 71 for d and 18 for a product: the sum stays below 2^126
    U128 t = sh >= 0 ? shl_u128(tm[k], sh) : shr_u128(tm[k], -sh);
    acc = add_u128(acc, tn[k] ? neg_u128(t) : t);
  }
  const bool rneg = (acc.hi >> 63) != 0;
  if (rneg) acc = neg_u128(acc);
  if ((acc.lo | acc.hi) == 0ull) return 0.f;
  int lz;
#ifdef __CUDA_ARCH__
  lz = acc.hi ? __clzll((long long)acc.hi) : 64 + __clzll((long long)acc.lo);
#else
  lz = acc.hi ? __builtin_clzll(acc.hi) : 64 + __builtin_clzll(acc.lo);
#endif
  const int p = 127 - lz;  // leading bit of the magnitude
  const U128 top24 = p >= 23 ? shr_u128(acc, p - 23) : shl_u128(acc, 23 - p);
  const int be = unit + p + 127;  // biased float exponent of the result
  if (be <= 0) return rneg ? -0.f : 0.f;
  if (be >= 255) return bitsf((rneg ? 0x80000000u : 0u) | 0x7F800000u);
  return bitsf((rneg ? 0x80000000u : 0u) | ((uint32_t)be << 23) | ((uint32_t)top24.lo & 0x7FFFFFu));
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
