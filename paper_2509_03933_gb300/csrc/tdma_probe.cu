// Measurement and diagnostic probes: FP64 fused multiply-add throughput of the current GPU (the
// second roofline of the FP64 solve paths, whose sweeps are chains of FP64 fused multiply-adds,
// multiplies and reciprocal refinements, all on the FP64 pipe), and the bounded wait of the solver
// kernels made to run out.
#include <cuda_runtime.h>
#include <cstdint>
#include "tdma.h"
#include "tma.cuh"

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

// The bounded mbarrier wait every TMA and cluster exchange of the solver kernels uses
// (mbar_wait_bounded), on a barrier that expects one arrival which never comes: no copy and no peer
// store is pending on it, so giving up leaves nothing in flight. Each thread polls `polls` times,
// gives up, and records TDMA_ERR_TIMEOUT in *status as the solver kernels do.
__global__ void bounded_wait_kernel(uint32_t polls, int32_t* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tdma::mbar_init(&bar, 1);
    tdma::mbar_fence_init();
  }
  __syncthreads();
  if (!tdma::mbar_wait_bounded(&bar, 0, polls)) atomicCAS(status, 0, (int32_t)TDMA_ERR_TIMEOUT);
}

}  // namespace

extern "C" tdma_status_t tdma_probe_bounded_wait(uint32_t polls, int32_t* status, void* stream) {
  if (status == nullptr || polls < 1 || polls > (1u << 20)) return TDMA_ERR_INVALID_ARG;
  bounded_wait_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(polls, status);
  return cudaGetLastError() == cudaSuccess ? TDMA_OK : TDMA_ERR_CUDA;
}

extern "C" tdma_status_t tdma_probe_fp64_fma(int32_t blocks, int32_t threads, int64_t iters, double* out,
                                             int64_t* fma_count, void* stream) {
  if (blocks < 1 || threads < 32 || threads > 1024 || threads % 32 != 0 || iters < 1 || out == nullptr)
    return TDMA_ERR_INVALID_ARG;
  fp64_fma_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(out, iters, 0.999999, 1e-6, -1.0);
  if (cudaGetLastError() != cudaSuccess) return TDMA_ERR_CUDA;
  if (fma_count) *fma_count = (int64_t)blocks * threads * iters * kChains;
  return TDMA_OK;
}
