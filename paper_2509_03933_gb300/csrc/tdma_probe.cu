// Measurement probe: FP64 fused multiply-add throughput of the current GPU, the second roofline
// of the FP64 solve paths (their sweeps are chains of FP64 fused multiply-adds, multiplies and
// reciprocal refinements, all on the FP64 pipe).
#include <cuda_runtime.h>
#include <cstdint>
#include "tdma.h"

namespace {

constexpr int kChains = 8;  // independent dependency chains per thread

// Every thread runs kChains independent chains x <- x * y + z for `iters` steps. With y < 1 and
// z > 0 the values stay finite and positive, so the host's sentinel (negative) is never met; the
// compiler cannot know that, so no chain is dead code.
__global__ void fp64_fma_kernel(double* out, int64_t iters, double y, double z, double sentinel) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1.0 + 1e-3 * (double)(threadIdx.x + k);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], y, z);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == sentinel) out[blockIdx.x] = s;
}

}  // namespace

extern "C" tdma_status_t tdma_probe_fp64_fma(int32_t blocks, int32_t threads, int64_t iters, double* out,
                                             int64_t* fma_count, void* stream) {
  if (blocks < 1 || threads < 32 || threads > 1024 || threads % 32 != 0 || iters < 1 || out == nullptr)
    return TDMA_ERR_INVALID_ARG;
  fp64_fma_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(out, iters, 0.999999, 1e-6, -1.0);
  if (cudaGetLastError() != cudaSuccess) return TDMA_ERR_CUDA;
  if (fma_count) *fma_count = (int64_t)blocks * threads * iters * kChains;
  return TDMA_OK;
}
