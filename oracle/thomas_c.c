/*
 * Plain C FP64 Thomas algorithm over a batch of lines: the oracle's reference solve, used to time
 * the CPU baseline on the host's cores.
 *
 * TEST INFRASTRUCTURE ONLY: built by oracle/c_thomas.py (gcc) and loaded by tests/ and by the CPU
 * baseline leg and reference arm of bench.py; shares no code with the CUDA library.
 *
 * Thomas algorithm (Section 1; no pivoting):
 *   c'_0 = c_0 / b_0, d'_0 = d_0 / b_0;
 *   for i >= 1: w = b_i - a_i c'_{i-1}, c'_i = c_i / w (0 for i = n-1), d'_i = (d_i - a_i d'_{i-1}) / w;
 *   x_{n-1} = d'_{n-1}; x_i = d'_i - c'_i x_{i+1}.
 * a_0 and c_{n-1} of every line are ignored. Compiled with -ffp-contract=off, so that every
 * operation is one IEEE rounding, in the order written (the numpy oracle does the same).
 *
 * Layout: unknown i of line l is element l * line_stride + i * row_stride of a, b, c, d and x.
 * Lines are taken in blocks of up to 8 (the rows of a block of adjacent lines share cache lines);
 * blocks are spread over `threads` OpenMP threads. x may alias d.
 */
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define BLOCK 8

int oracle_thomas(int64_t n, int64_t n_lines, int64_t row_stride, int64_t line_stride, const double* a,
                  const double* b, const double* c, const double* d, double* x, int threads) {
  if (n < 1 || n_lines < 0 || threads < 1) return 1;
  const int64_t n_blocks = (n_lines + BLOCK - 1) / BLOCK;
  int failed = 0;
#pragma omp parallel num_threads(threads) reduction(| : failed)
  {
    double* cp = (double*)malloc(sizeof(double) * (size_t)n * BLOCK);
    if (!cp) {
      failed = 1;
    } else {
#pragma omp for schedule(static)
      for (int64_t blk = 0; blk < n_blocks; ++blk) {
        const int64_t l0 = blk * BLOCK;
        const int nb = (int)(n_lines - l0 < BLOCK ? n_lines - l0 : BLOCK);
        /* forward elimination: c' in the scratch, d' in x */
        for (int j = 0; j < nb; ++j) {
          const int64_t e = (l0 + j) * line_stride;
          cp[j] = n > 1 ? c[e] / b[e] : 0.0;
          x[e] = d[e] / b[e];
        }
        for (int64_t i = 1; i < n; ++i) {
          for (int j = 0; j < nb; ++j) {
            const int64_t e = (l0 + j) * line_stride + i * row_stride;
            const double ai = a[e];
            const double w = b[e] - ai * cp[(i - 1) * BLOCK + j];
            cp[i * BLOCK + j] = i < n - 1 ? c[e] / w : 0.0;
            x[e] = (d[e] - ai * x[e - row_stride]) / w;
          }
        }
        /* back substitution */
        for (int64_t i = n - 2; i >= 0; --i) {
          for (int j = 0; j < nb; ++j) {
            const int64_t e = (l0 + j) * line_stride + i * row_stride;
            x[e] = x[e] - cp[i * BLOCK + j] * x[e + row_stride];
          }
        }
      }
      free(cp);
    }
  }
  return failed;
}

/* OpenMP threads available to this process (1 without OpenMP). */
int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
