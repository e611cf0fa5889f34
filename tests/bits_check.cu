// Host check of the FP64 <-> float-pair bit paths in paper_2509_03933_gb300/csrc/bits.cuh:
//   split_normal(v): h = v truncated to 24 significant bits, l = (float)(v - h) (v - h is exact
//   in double), l carries the sign of v; false exactly outside 949 <= biased exponent <= 1150.
//   widen_normal(f) == (double)f for every normal float and for +-0; false otherwise.
//   narrow_normal(v) == (float)v (round to nearest, ties to even) for every double whose biased
//   exponent is in [897, 1150]; false otherwise.
// Prints "OK <cases>" or the first mismatch.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include "bits.cuh"

using namespace tdma;

static uint64_t s = 0x9E3779B97F4A7C15ull;
static uint64_t next() {  // splitmix64
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int main() {
  long cases = 0;
  for (int i = 0; i < 4000000; ++i) {
    const uint64_t r = next();
    const uint32_t e = 900 + (uint32_t)(next() % 300);  // around and inside the range
    const uint64_t u = (r & 0x800FFFFFFFFFFFFFull) | ((uint64_t)e << 52);
    const double v = bitsd(u);
    float h = 0.f, l = 0.f;
    const bool ok = split_normal(v, h, l);
    const bool in = e >= 949 && e <= 1150;
    if (ok != in) { std::printf("range mismatch e=%u\n", e); return 1; }
    ++cases;
    if (!ok) continue;
    const double ht = bitsd(u & ~((1ull << 29) - 1));  // truncation to 24 significant bits
    if ((double)h != ht) { std::printf("h mismatch %a %a\n", v, (double)h); return 1; }
    const double rem = v - ht;  // exact
    if (l != (float)rem) { std::printf("l mismatch %a %a %a\n", v, (double)l, rem); return 1; }
    if (std::fabs(v - (double)h - (double)l) > std::ldexp(std::fabs(v), -48)) { std::printf("bound %a\n", v); return 1; }
  }
  for (uint64_t k = 0; k < 6000000; ++k) {
    const uint32_t b = k < 4 ? (uint32_t[]){0u, 0x80000000u, 0x00800000u, 0x7F7FFFFFu}[k] : (uint32_t)next();
    const float f = bitsf(b);
    double d = 0.0;
    const bool ok = widen_normal(f, d);
    const bool normal = std::isnormal(f) || f == 0.f;
    if (ok != normal) { std::printf("class mismatch %08x\n", b); return 1; }
    ++cases;
    if (ok && (dbits(d) != dbits((double)f))) { std::printf("widen mismatch %08x\n", b); return 1; }
  }
  for (uint64_t k = 0; k < 6000000; ++k) {
    // doubles of every exponent near the float range, with fractions that are ties, just below
    // and just above them, or random; and the largest values, which round up to infinity
    const uint64_t r = next();
    const uint32_t e = k < 6 ? (uint32_t[]){896u, 897u, 1150u, 1150u, 1151u, 0u}[k] : 880 + (uint32_t)(next() % 290);
    uint64_t frac = r & 0xFFFFFFFFFFFFFull;
    const int kind = (int)(k % 4);
    if (kind == 1) frac = (frac & ~0x1FFFFFFFull) | 0x10000000ull;        // exactly half
    if (kind == 2) frac = (frac & ~0x1FFFFFFFull) | 0x0FFFFFFFull;        // just below half
    if (kind == 3) frac = (frac & ~0x1FFFFFFFull) | 0x10000001ull;        // just above half
    if (k == 3) frac = 0xFFFFFFFFFFFFFull;                                // rounds up to infinity
    const uint64_t u = (r & 0x8000000000000000ull) | ((uint64_t)e << 52) | frac;
    const double v = bitsd(u);
    float f = 0.f;
    const bool ok = narrow_normal(v, f);
    const bool in = e >= 897 && e <= 1150;
    if (ok != in) { std::printf("narrow range mismatch e=%u\n", e); return 1; }
    ++cases;
    if (ok && fbits(f) != fbits((float)v)) { std::printf("narrow mismatch %a %a %a\n", v, (double)f, (double)(float)v); return 1; }
  }
  std::printf("OK %ld\n", cases);
  return 0;
}
