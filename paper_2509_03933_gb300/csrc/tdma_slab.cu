// C ABI of the split-line stages (lines divided into slabs of rows held by different ranks):
// Stage A over a slab, Stage B over the gathered slab pairs, Stage C over a slab. The exchange
// between them belongs to the caller (an all-to-all between ranks).
#include "tdma.h"
#include "common.cuh"
#include "kernels_slab.cuh"

using namespace tdma;

namespace {

bool slab_desc_ok(const tdma_slab_desc_t* d) {
  return d && d->n_local >= 2 && d->n_lines >= 0 && d->inner_count >= 1 && d->elem_stride >= 0 &&
         d->inner_stride >= 0 && d->outer_stride >= 0 && (d->nrhs == 1 || d->nrhs == 2) &&
         (d->first == 0 || d->first == 1) && (d->last == 0 || d->last == 1);
}

SlabArgs slab_args(const tdma_slab_desc_t* d, int64_t line0, int64_t count) {
  SlabArgs S{};
  S.lay = Layout{d->n_local, d->n_lines, d->elem_stride, d->inner_count, d->inner_stride, d->outer_stride};
  S.first = d->first;
  S.last = d->last;
  S.line0 = line0;
  S.count = count;
  return S;
}

unsigned blocks_for(int64_t count) { return (unsigned)((count + 127) / 128); }

}  // namespace

extern "C" {

size_t tdma_slab_scratch_bytes(const tdma_slab_desc_t* d, int64_t count) {
  if (!slab_desc_ok(d) || count < 0) return 0;
  return (size_t)(d->n_local - 2) * (size_t)(2 + d->nrhs) * (size_t)count * sizeof(double);
}

size_t tdma_slab_pairs_work_bytes(int32_t n_slabs, int64_t count, int32_t nrhs) {
  if (n_slabs < 1 || count < 0 || (nrhs != 1 && nrhs != 2)) return 0;
  return (size_t)2 * n_slabs * (size_t)count * (size_t)(1 + nrhs) * sizeof(double);
}

tdma_status_t tdma_slab_reduce(const tdma_slab_desc_t* desc, const double* a, const double* b, const double* c,
                               const double* d, int64_t line0, int64_t count, double* reduced, double* scratch,
                               int32_t* status, void* stream) {
  if (!slab_desc_ok(desc) || line0 < 0 || count < 0 || line0 + count > desc->n_lines) return TDMA_ERR_INVALID_ARG;
  if (count == 0) return TDMA_OK;
  if (!a || !b || !c || !d || !reduced || (desc->n_local > 2 && !scratch)) return TDMA_ERR_INVALID_ARG;
  SlabArgs S = slab_args(desc, line0, count);
  S.a = a; S.b = b; S.c = c; S.d = d;
  S.red = reduced;
  S.scratch = scratch;
  S.st = (DevStatus*)status;
  cudaStream_t s = (cudaStream_t)stream;
  if (desc->nrhs == 1) slab_reduce_kernel<1><<<blocks_for(count), 128, 0, s>>>(S);
  else slab_reduce_kernel<2><<<blocks_for(count), 128, 0, s>>>(S);
  return cudaGetLastError() == cudaSuccess ? TDMA_OK : TDMA_ERR_CUDA;
}

tdma_status_t tdma_slab_pairs_solve(int32_t n_slabs, int64_t count, int32_t nrhs, const double* gathered,
                                    double* ends, double* work, int32_t* status, void* stream) {
  if (n_slabs < 1 || count < 0 || (nrhs != 1 && nrhs != 2)) return TDMA_ERR_INVALID_ARG;
  if (count == 0) return TDMA_OK;
  if (!gathered || !ends || !work) return TDMA_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (nrhs == 1)
    pairs_solve_kernel<1><<<blocks_for(count), 128, 0, s>>>(n_slabs, count, gathered, ends, work, (DevStatus*)status);
  else
    pairs_solve_kernel<2><<<blocks_for(count), 128, 0, s>>>(n_slabs, count, gathered, ends, work, (DevStatus*)status);
  return cudaGetLastError() == cudaSuccess ? TDMA_OK : TDMA_ERR_CUDA;
}

tdma_status_t tdma_slab_finish(const tdma_slab_desc_t* desc, int64_t line0, int64_t count, const double* ends,
                               const double* scratch, double* x, void* stream) {
  if (!slab_desc_ok(desc) || line0 < 0 || count < 0 || line0 + count > desc->n_lines) return TDMA_ERR_INVALID_ARG;
  if (count == 0) return TDMA_OK;
  if (!ends || !x || (desc->n_local > 2 && !scratch)) return TDMA_ERR_INVALID_ARG;
  SlabArgs S = slab_args(desc, line0, count);
  S.x = x;
  S.ends = ends;
  S.scratch = const_cast<double*>(scratch);
  cudaStream_t s = (cudaStream_t)stream;
  if (desc->nrhs == 1) slab_finish_kernel<1><<<blocks_for(count), 128, 0, s>>>(S);
  else slab_finish_kernel<2><<<blocks_for(count), 128, 0, s>>>(S);
  return cudaGetLastError() == cudaSuccess ? TDMA_OK : TDMA_ERR_CUDA;
}

}  // extern "C"
