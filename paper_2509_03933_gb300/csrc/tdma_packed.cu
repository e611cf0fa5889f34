// Launch side of the chunk kernel: every instantiation of packed_refine_kernel and
// packed_fixup_kernel is made here (declarations in packed_launch.h).
#include <mutex>
#include "packed_launch.h"

namespace tdma {

namespace {

template <class K> cudaError_t raise_smem(K kernel, size_t bytes) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// The chunk kernel, then, out of place, the further corrections of the chunks it listed (that
// launch leaves at once when none is listed). In place (x is d) the chunk kernel makes them
// itself, from the d pairs it still holds.
template <bool TR>
cudaError_t launch(const PackedTables& pk, const tdma_config_t& c, const Args& A, cudaStream_t s) {
  const size_t sm = (size_t)c.smem_bytes;
  if (A.x == A.d) {
    packed_refine_kernel<kPackC, TR, true><<<c.blocks, c.threads_per_block, sm, s>>>(A, pk);
    return cudaGetLastError();
  }
  packed_refine_kernel<kPackC, TR, false><<<c.blocks, c.threads_per_block, sm, s>>>(A, pk);
  if (A.max_iters > 1) packed_fixup_kernel<kPackC, TR><<<c.blocks, c.threads_per_block, 0, s>>>(A, pk);
  return cudaGetLastError();
}

}  // namespace

cudaError_t packed_prepare(size_t bytes) {
  cudaError_t e = raise_smem(packed_refine_kernel<kPackC, false, false>, bytes);
  if (e == cudaSuccess) e = raise_smem(packed_refine_kernel<kPackC, false, true>, bytes);
  if (e == cudaSuccess) e = raise_smem(packed_refine_kernel<kPackC, true, false>, bytes);
  if (e == cudaSuccess) e = raise_smem(packed_refine_kernel<kPackC, true, true>, bytes);
  return e;
}

int packed_resident_clusters(size_t bytes) {
  cudaLaunchConfig_t lc{};
  lc.gridDim = dim3(kPackC);
  lc.blockDim = dim3(kPackThreads);
  lc.dynamicSmemBytes = bytes;
  int resident = 0;
  if (cudaOccupancyMaxActiveClusters(&resident, packed_refine_kernel<kPackC, false, false>, &lc) != cudaSuccess)
    resident = 0;
  (void)cudaGetLastError();
  return resident;
}

cudaError_t packed_launch(bool tr, const PackedTables& pk, const tdma_config_t& c, int64_t n_lines, const Args& A,
                          cudaStream_t s) {
  const cudaError_t e = cudaMemsetAsync(pk.norms, 0, sizeof(uint32_t) * (kPackNormWords * (size_t)n_lines + 1), s);
  if (e != cudaSuccess) return e;
  return tr ? launch<true>(pk, c, A, s) : launch<false>(pk, c, A, s);
}

}  // namespace tdma
