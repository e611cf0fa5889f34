// Host driver for tests/test_bits_host.py: reads lines of 7 hexadecimal doubles
// (d a xm b x c xp) from stdin and prints residual_exact(...) of each as a 32-bit hex pattern.
#include <cstdio>
#include <cstdint>
#include <cstring>
#include "exact_residual.cuh"

int main() {
  unsigned long long u[7];
  while (std::scanf("%llx %llx %llx %llx %llx %llx %llx", &u[0], &u[1], &u[2], &u[3], &u[4], &u[5], &u[6]) == 7) {
    double v[7];
    for (int k = 0; k < 7; ++k) std::memcpy(&v[k], &u[k], 8);
    const float r = tdma::residual_exact(v[0], v[1], v[2], v[3], v[4], v[5], v[6]);
    std::printf("%08x\n", tdma::fbits(r));
  }
  return 0;
}
