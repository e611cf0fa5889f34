// Ragged batches (filled in below).
#pragma once
#include "tdma.h"
#include "layout.cuh"

namespace tdma {
inline void ragged_config(const tdma_desc_t&, tdma_config_t& c) { c = tdma_config_t{}; c.variant = TDMA_VARIANT_RAGGED; }
inline cudaError_t launch_ragged(tdma_precision_t, const Args&, const tdma_config_t&, cudaStream_t) {
  return cudaErrorNotSupported;
}
inline cudaError_t prepare_ragged(tdma_precision_t, size_t) { return cudaSuccess; }
inline size_t ragged_workspace(const tdma_desc_t&, const tdma_config_t&) { return 0; }
}  // namespace tdma
