// Line addressing and partitioning shared by the kernels.
#pragma once
#include "common.cuh"

namespace tdma {

// Element j of line l sits at off(l) + j * es, off(l) = (l / ic) * os + (l % ic) * is.
struct Layout {
  int64_t n, n_lines, es, ic, is, os;
  TDMA_DEV int64_t off(int64_t l) const { return (l / ic) * os + (l % ic) * is; }
};

// Partition k of P over n rows: the first n mod P partitions take one extra row.
TDMA_DEV void partition(int64_t n, int P, int k, int64_t& start, int& m) {
  const int64_t q = n / P, r = n % P;
  m = (int)(q + (k < r ? 1 : 0));
  start = (int64_t)k * q + (k < r ? k : r);
}

// Arguments of the uniform-line kernels (passed by value).
struct Args {
  const void* a;
  const void* b;
  const void* c;
  const void* d;
  void* x;
  const void* shift;   // per-line diagonal shift or nullptr
  Layout lay;
  int P;               // partitions per line
  int Lb;              // lines per block
  int mmax;            // rows of the largest partition
  int bcast;           // coefficients are 1D arrays of length n
  int pdd;             // approximate reduced solve (parallel diagonally dominant)
  DevStatus* st;
  // refinement
  int max_iters;
  float tol;
  // ragged batches
  const int64_t* roff;
  const int32_t* rlen;
  void* ws;            // workspace (variant dependent)
};

template <class T> TDMA_DEV T ldg(const T* p) { return __ldg(p); }

}  // namespace tdma
