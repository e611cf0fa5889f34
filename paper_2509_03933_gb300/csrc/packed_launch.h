// Launch side of the chunk kernel (kernels_packed.cuh). Its template instantiations live in their
// own translation unit (tdma_packed.cu), which compiles in parallel with the rest of the library.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include "tdma.h"
#include "kernels_packed.cuh"

namespace tdma {

// Raise (never lower) the dynamic shared-memory limit of every chunk-kernel instantiation.
cudaError_t packed_prepare(size_t bytes);
// Clusters of the chunk kernel resident on the device at once with `bytes` of dynamic shared
// memory per CTA (0 when the query fails).
int packed_resident_clusters(size_t bytes);
// Zero the per-line maxima and the count of listed chunks, launch the chunk kernel with config c
// (tr: on the transposed rows of the adjoint) and, out of place, the kernel that takes the listed
// chunks' further corrections.
cudaError_t packed_launch(bool tr, const PackedTables& pk, const tdma_config_t& c, int64_t n_lines, const Args& A,
                          cudaStream_t s);

}  // namespace tdma
