// P = 1 Thomas sweep with the elimination factors kept in the workspace (filled in below).
#pragma once
#include "tdma.h"
#include "layout.cuh"

namespace tdma {
inline bool use_thomas_variant(const tdma_desc_t&) { return false; }
inline void thomas_config(const tdma_desc_t&, tdma_config_t&) {}
inline cudaError_t launch_thomas(tdma_precision_t, int, const Args&, const tdma_config_t&, cudaStream_t) {
  return cudaErrorNotSupported;
}
inline cudaError_t prepare_thomas(tdma_precision_t, int, size_t) { return cudaSuccess; }
}  // namespace tdma
