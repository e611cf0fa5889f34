// Device helpers shared by the solver kernels.
//
// GB300 runs FP64 arithmetic, and every conversion to or from FP64, on a narrow pipe
// (about 1/60 of the FP32 rate), while the MUFU unit gives a 20-bit reciprocal seed for
// free. The helpers below therefore (1) build an FP64 reciprocal from that seed with two
// Newton-Raphson steps, (2) move data between FP64 and pairs of floats with integer bit
// operations instead of conversion instructions, and (3) provide the error-free float
// transformations (Knuth's TwoSum, FMA-based TwoProduct; Dekker 1971, Ogita-Rump-Oishi
// 2005) used by the extra-precise residual of the refinement path.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define TDMA_DEV __device__ __forceinline__

namespace tdma {

// ---- status block -------------------------------------------------------------------
// word 0: first error code (0 = none), word 1: max refinement corrections used.
struct DevStatus { int32_t err; int32_t iters; int32_t pad[2]; };

TDMA_DEV void report_error(DevStatus* st, int32_t code) {
  if (st) atomicCAS(&st->err, 0, code);
}
TDMA_DEV void report_iters(DevStatus* st, int32_t it) {
  if (st) atomicMax(&st->iters, it);
}

// ---- reciprocals ----------------------------------------------------------------------
// FP64: MUFU seed y (relative error below 2^-20) refined by the series 1/w = y / (1 - e) with
// e = 1 - w y, truncated after the quadratic term: y (1 + e + e^2) = (1/w) (1 - e^3), a relative
// error below 2^-60 before the final rounding; three dependent FMAs (two Newton-Raphson steps
// take four). The seed flushes subnormals to zero, in its input (w subnormal) and in its output
// (|w| >= 2^1022, whose reciprocal lies below the normal range), so those w, and zeros,
// infinities and NaN, take the IEEE division instead: a pivot beyond the normal range then gives
// its correctly rounded reciprocal, a zero or subnormal pivot an infinite one, and an infinite or
// NaN pivot NaN, so that the callers' finiteness checks see them. The test is on the exponent
// bits (integer pipe); no normal pivot below 2^1022 takes the division.
TDMA_DEV double rcp(double w) {
  const unsigned ex = ((unsigned)__double2hiint(w) >> 20) & 0x7FFu;
  if (ex - 1u >= 0x7FCu) return ex == 0x7FFu ? w - w : 1.0 / w;
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(w));
  const double e = fma(-w, y, 1.0);
  return fma(y, fma(e, e, e), y);
}
// FP32: the MUFU reciprocal (about one ulp).
TDMA_DEV float rcp(float w) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(w));
  return y;
}

template <class T> TDMA_DEV bool finite(T v) { return isfinite(v); }

// ---- float pairs (unevaluated sums h + l) --------------------------------------------
struct ff { float h, l; };

// s + e = a + b exactly (Knuth's TwoSum, no ordering assumption).
TDMA_DEV ff two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// s + e = a + b exactly when |a| >= |b| (Dekker's Fast2Sum).
TDMA_DEV ff fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// p + e = a * b exactly (barring underflow), using the fused multiply-add.
TDMA_DEV ff two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
// (h, l) + v, renormalised.
TDMA_DEV ff ff_add(ff x, float v) {
  ff s = two_sum(x.h, v);
  return fast_two_sum(s.h, __fadd_rn(s.l, x.l));
}

// ---- FP64 <-> float pairs by bit manipulation ----------------------------------------
// Split a double into h + l with h carrying the leading 24 significant bits (truncated) and
// l the next 24 (rounded); about 5 low bits are dropped (relative 2^-48). Exact bit work on
// the integer pipe; out-of-float-range magnitudes fall back to a rounding conversion.
TDMA_DEV ff split_f64(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FF);
  if (e >= 897 && e <= 1150) {  // normal float exponent range
    const unsigned hb = sign | ((unsigned)(e - 896) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const float h = __uint_as_float(hb);
    const unsigned rem = lo & 0x1FFFFFFFu;  // remaining 29 significand bits, weight 2^(e-1075)
    // rem * 2^(e-1075) = (rem * 2^-52) * 2^(e-1023); both factors are normal floats.
    float l = __fmul_rn(__uint2float_rn(rem), 2.220446049250313e-16f /* 2^-52 */);
    l = __fmul_rn(l, __uint_as_float((unsigned)(e - 1023 + 127) << 23));
    return {h, sign ? -l : l};
  }
  if (e == 0 && (hi & 0xFFFFFu) == 0 && lo == 0) return {__uint_as_float(sign), 0.0f};  // +-0
  return {__double2float_rn(v), 0.0f};
}

// Exact float -> double by bit manipulation (normal floats and zeros; others converted).
TDMA_DEV double f2d(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xFF;
  if (e != 0 && e != 0xFF) {
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    const unsigned long long bits = sign | ((unsigned long long)(e + 896) << 52) |
                                    ((unsigned long long)(b & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)bits);
  }
  if ((b & 0x7FFFFFFFu) == 0) return __longlong_as_double((long long)((unsigned long long)(b) << 32));
  return (double)f;
}

// h + l rounded to double: two exact widenings and one FP64 add.
TDMA_DEV double ff_to_f64(ff x) { return f2d(x.h) + f2d(x.l); }

// ---- vector helpers -------------------------------------------------------------------
template <int NR, class T> struct Vec { T v[NR]; };

}  // namespace tdma
