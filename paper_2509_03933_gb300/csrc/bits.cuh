// Short integer-pipe paths between FP64 values and float pairs, for the kernels where they run
// once per unknown. They compute what split_f64 and f2d in common.cuh compute, with fewer
// instructions on the common path (normal magnitudes) and those functions as the fallback.
// Host and device both compile them, so that a host program can check them bit for bit.
#pragma once
#include <cstdint>
#include <cstring>
#include "common.cuh"

namespace tdma {

#ifdef __CUDACC__
#define TDMA_HD __host__ __device__ __forceinline__
#else
#define TDMA_HD inline
#endif

TDMA_HD uint32_t fbits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
#endif
}
TDMA_HD float bitsf(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}
TDMA_HD uint64_t dbits(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t u;
  std::memcpy(&u, &d, 8);
  return u;
#endif
}
TDMA_HD double bitsd(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  std::memcpy(&d, &u, 8);
  return d;
#endif
}

// Normal-range part of the split: for a double v of biased exponent e in [949, 1150]
// (2^-74 <= |v| < 2^128), h = v truncated to its leading 24 significant bits and
// l = the remaining 29 bits rounded to 24 (|v - h - l| <= 2^-48 |v|). Returns false outside the
// range (then nothing is written).
//   h: the high word shifted left by 3 takes in the next 3 significand bits (bits 29..31 of the
//      low word); its 9 exponent bits left at 23..31 are e mod 512, and e - 896 (the float
//      exponent, 1..254) is (e mod 512) - 384 modulo 512, so one subtraction and a mask give
//      the float's exponent and fraction; the sign comes from the high word.
//   l: the low 29 bits as an integer, converted with rounding, times 2^(e - 1075) (a normal
//      float: e - 1075 >= -126), with the sign of v.
TDMA_HD bool split_normal(double v, float& h, float& l) {
  const uint64_t u = dbits(v);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const uint32_t e = (hi >> 20) & 0x7FFu;
  if (e - 949u >= 202u) return false;
  const uint32_t sign = hi & 0x80000000u;
#ifdef __CUDA_ARCH__
  const uint32_t t = __funnelshift_l(lo, hi, 3);
#else
  const uint32_t t = (hi << 3) | (lo >> 29);
#endif
  h = bitsf(((t - (384u << 23)) & 0x7FFFFFFFu) | sign);
  const float scale = bitsf((e - 948u) << 23);  // 2^(e - 1075)
#ifdef __CUDA_ARCH__
  const float m = __fmul_rn(__uint2float_rn(lo & 0x1FFFFFFFu), scale);
#else
  const float m = (float)(lo & 0x1FFFFFFFu) * scale;
#endif
  l = bitsf(fbits(m) | sign);
  return true;
}

// Normal or zero float -> the same value as a double: the exponent rebased by 1023 - 127 = 896
// and the 23 fraction bits moved to the top of the 52. Returns false for subnormals, infinities
// and NaN.
TDMA_HD bool widen_normal(float f, double& d) {
  const uint32_t b = fbits(f), a = b & 0x7FFFFFFFu;
  if (a == 0u) {
    d = bitsd((uint64_t)b << 32);
    return true;
  }
  if (a - 0x00800000u >= 0x7F000000u) return false;
  const uint32_t hi = ((a >> 3) + (896u << 20)) | (b & 0x80000000u);
  d = bitsd(((uint64_t)hi << 32) | (uint64_t)(b << 29));
  return true;
}

// Double -> float rounded to nearest, ties to even, for the doubles whose float lies in the
// normal range: biased exponent e in [897, 1150] (2^-126 <= |v| < 2^128). The float keeps the
// sign, the exponent rebased by 896 and the top 23 of the 52 fraction bits; the other 29 bits
// decide the rounding (up above half, or at half when the kept bits are odd); a carry out of the
// fraction moves to the exponent, up to infinity for the largest values, as the rounding rule
// gives. Returns false outside the range (then nothing is written).
TDMA_HD bool narrow_normal(double v, float& f) {
  const uint64_t u = dbits(v);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const uint32_t e = (hi >> 20) & 0x7FFu;
  if (e - 897u >= 254u) return false;
#ifdef __CUDA_ARCH__
  const uint32_t keep = __funnelshift_l(lo, hi, 3) & 0x7FFFFFu;
#else
  const uint32_t keep = ((hi << 3) | (lo >> 29)) & 0x7FFFFFu;
#endif
  const uint32_t rest = lo & 0x1FFFFFFFu, half = 1u << 28;
  const uint32_t up = (rest > half || (rest == half && (keep & 1u))) ? 1u : 0u;
  f = bitsf((((e - 896u) << 23) | keep) + up | (hi & 0x80000000u));
  return true;
}

#ifdef __CUDACC__
// Device entry points with the general routines as the (rare) fallback.
TDMA_DEV ff split_f64_fast(double v) {
  ff r;
  if (split_normal(v, r.h, r.l)) return r;
  return split_f64(v);
}
TDMA_DEV double f2d_fast(float f) {
  double d;
  if (widen_normal(f, d)) return d;
  return f2d(f);
}
TDMA_DEV float d2f_fast(double v) {
  float f;
  if (narrow_normal(v, f)) return f;
  return __double2float_rn(v);
}
#endif

}  // namespace tdma
