// C ABI of the batched tridiagonal solver (declarations and contract in include/tdma.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>

#include "tdma.h"
#include "kernels_dc.cuh"
#include "kernels_refine.cuh"
#include "kernels_thomas.cuh"
#include "kernels_ragged.cuh"
#include "kernels_backward.cuh"

using namespace tdma;

struct tdma_plan_s {
  tdma_desc_t desc;
  tdma_config_t cfg;
  DevStatus* status = nullptr;  // device
  int device = 0;
  bool refine_sb64 = true;
  size_t workspace = 0;
};

namespace {

constexpr int kMaxSmem = 227 * 1024;

bool is_uniform(const tdma_desc_t& d) { return d.n > 0; }

size_t elem_bytes_coef(tdma_precision_t p) { return p == TDMA_F64 ? 8 : 4; }

// smem of the fused kernel for a given shape
size_t dc_bytes(const tdma_desc_t& d, int T, int Lb, int P, int mmax) {
  if (d.precision == TDMA_F64)
    return d.nrhs == 2 ? dc_smem_bytes<double, 2>(T, Lb, P, mmax) : dc_smem_bytes<double, 1>(T, Lb, P, mmax);
  if (d.precision == TDMA_F32)
    return d.nrhs == 2 ? dc_smem_bytes<float, 2>(T, Lb, P, mmax) : dc_smem_bytes<float, 1>(T, Lb, P, mmax);
  return refine_smem_bytes<double>(T, Lb, P, mmax);
}

// Pick lines-per-block for partitions P: a warp should cover >= 8 adjacent lines on strided
// axes (contiguous 64/32 byte segments per row), blocks up to 256 threads, smem within limits.
bool choose_block(const tdma_desc_t& d, int P, tdma_config_t& c) {
  const int64_t n = d.n;
  const int mmax = (int)((n + P - 1) / P);
  int Lb = std::max(1, 256 / P);
  Lb = (int)std::min<int64_t>(Lb, std::max<int64_t>(1, d.n_lines));
  if (Lb > 32) Lb = 32 * (Lb / 32);
  while (Lb > 1 && dc_bytes(d, Lb * P, Lb, P, mmax) > (size_t)kMaxSmem) Lb /= 2;
  const int T = Lb * P;
  if (T > 512) return false;
  const size_t smem = dc_bytes(d, T, Lb, P, mmax);
  if (smem > (size_t)kMaxSmem) return false;
  c.partitions = P;
  c.rows_per_thread = mmax;
  c.lines_per_block = Lb;
  c.threads_per_block = T;
  c.smem_bytes = (int64_t)smem;
  c.blocks = (int32_t)((d.n_lines + Lb - 1) / Lb);
  c.variant = d.precision == TDMA_F32_REFINE ? TDMA_VARIANT_REFINE : TDMA_VARIANT_DC;
  return true;
}

int default_partitions(const tdma_desc_t& d) {
  // rows per thread near 16 for long lines; short lines keep P small
  const int64_t n = d.n;
  if (n < 32) return 1;
  int P = (int)std::min<int64_t>(64, (n + 15) / 16);
  while (P > 1 && n / P < 2) --P;
  return std::max(1, P);
}

tdma_status_t validate(const tdma_desc_t& d) {
  if (d.n < 0 || d.n_lines < 0) return TDMA_ERR_INVALID_ARG;
  if (d.nrhs != 1 && d.nrhs != 2) return TDMA_ERR_INVALID_ARG;
  if (d.precision != TDMA_F64 && d.precision != TDMA_F32 && d.precision != TDMA_F32_REFINE)
    return TDMA_ERR_INVALID_ARG;
  if (d.partitions < 0) return TDMA_ERR_INVALID_ARG;
  if (d.n == 0) {  // ragged
    if (d.n_lines > 0 && (!d.ragged_offsets || !d.ragged_lengths || d.ragged_max_n < 1))
      return TDMA_ERR_INVALID_ARG;
    if (d.coef_broadcast || d.diag_shift) return TDMA_ERR_UNSUPPORTED;
  } else {
    if (d.inner_count < 1 || d.elem_stride < 0 || d.inner_stride < 0 || d.outer_stride < 0)
      return TDMA_ERR_INVALID_ARG;
    if (d.partitions > 1 && d.n / d.partitions < 2) return TDMA_ERR_INVALID_ARG;
    if (d.partitions > 1024) return TDMA_ERR_INVALID_ARG;
  }
  if (d.precision == TDMA_F32_REFINE) {
    if (d.nrhs != 1 || d.coef_broadcast || d.diag_shift) return TDMA_ERR_UNSUPPORTED;
    if (d.max_refine_iters < 0) return TDMA_ERR_INVALID_ARG;
  }
  return TDMA_OK;
}

Args make_args(const tdma_plan_s* p, const void* a, const void* b, const void* c, const void* d, void* x,
               void* ws) {
  Args A{};
  A.a = a; A.b = b; A.c = c; A.d = d; A.x = x;
  A.shift = p->desc.diag_shift;
  A.lay = Layout{p->desc.n, p->desc.n_lines, p->desc.elem_stride, p->desc.inner_count, p->desc.inner_stride,
                 p->desc.outer_stride};
  A.P = p->cfg.partitions;
  A.Lb = p->cfg.lines_per_block;
  A.mmax = p->cfg.rows_per_thread;
  A.bcast = p->desc.coef_broadcast;
  A.st = p->status;
  A.max_iters = p->desc.max_refine_iters > 0 ? p->desc.max_refine_iters : 4;
  A.tol = (float)(p->desc.refine_tol > 0 ? p->desc.refine_tol : 1e-13);
  A.roff = p->desc.ragged_offsets;
  A.rlen = p->desc.ragged_lengths;
  A.ws = ws;
  return A;
}

template <class K> cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_forward(const tdma_plan_s* p, const Args& A, cudaStream_t s) {
  const tdma_config_t& c = p->cfg;
  if (p->desc.n_lines == 0) return cudaSuccess;
  const dim3 grid(c.blocks), block(c.threads_per_block);
  const size_t sm = (size_t)c.smem_bytes;
  switch (c.variant) {
    case TDMA_VARIANT_DC:
      if (p->desc.precision == TDMA_F64) {
        if (p->desc.nrhs == 1) dc_kernel<double, 1><<<grid, block, sm, s>>>(A);
        else dc_kernel<double, 2><<<grid, block, sm, s>>>(A);
      } else {
        if (p->desc.nrhs == 1) dc_kernel<float, 1><<<grid, block, sm, s>>>(A);
        else dc_kernel<float, 2><<<grid, block, sm, s>>>(A);
      }
      break;
    case TDMA_VARIANT_REFINE:
      if (p->refine_sb64) refine_kernel<double><<<grid, block, sm, s>>>(A);
      else refine_kernel<float><<<grid, block, sm, s>>>(A);
      break;
    case TDMA_VARIANT_THOMAS:
      return launch_thomas(p->desc.precision, p->desc.nrhs, A, c, s);
    case TDMA_VARIANT_RAGGED:
      return launch_ragged(p->desc.precision, A, c, s);
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t prepare_kernel(const tdma_plan_s* p) {
  const size_t sm = (size_t)p->cfg.smem_bytes;
  switch (p->cfg.variant) {
    case TDMA_VARIANT_DC:
      if (p->desc.precision == TDMA_F64)
        return p->desc.nrhs == 1 ? set_smem(dc_kernel<double, 1>, sm) : set_smem(dc_kernel<double, 2>, sm);
      return p->desc.nrhs == 1 ? set_smem(dc_kernel<float, 1>, sm) : set_smem(dc_kernel<float, 2>, sm);
    case TDMA_VARIANT_REFINE:
      return p->refine_sb64 ? set_smem(refine_kernel<double>, sm) : set_smem(refine_kernel<float>, sm);
    case TDMA_VARIANT_THOMAS:
      return prepare_thomas(p->desc.precision, p->desc.nrhs, sm);
    case TDMA_VARIANT_RAGGED:
      return prepare_ragged(p->desc.precision, sm);
  }
  return cudaSuccess;
}

bool aligned(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

}  // namespace

extern "C" {

const char* tdma_status_string(tdma_status_t s) {
  switch (s) {
    case TDMA_OK: return "ok";
    case TDMA_ERR_INVALID_ARG: return "invalid argument";
    case TDMA_ERR_UNSUPPORTED: return "unsupported configuration";
    case TDMA_ERR_WORKSPACE: return "workspace too small";
    case TDMA_ERR_CUDA: return "CUDA runtime error";
    case TDMA_ERR_NONFINITE: return "zero or non-finite pivot";
    case TDMA_ERR_TIMEOUT: return "bounded wait timed out";
    case TDMA_ERR_NOT_CONVERGED: return "refinement did not converge";
  }
  return "unknown status";
}

tdma_status_t tdma_plan_create(tdma_plan_t* plan, const tdma_desc_t* desc, size_t* workspace_bytes) {
  if (!plan || !desc) return TDMA_ERR_INVALID_ARG;
  *plan = nullptr;
  const tdma_status_t v = validate(*desc);
  if (v != TDMA_OK) return v;
  tdma_plan_s* p = new (std::nothrow) tdma_plan_s();
  if (!p) return TDMA_ERR_INVALID_ARG;
  p->desc = *desc;
  if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return TDMA_ERR_CUDA; }
  tdma_config_t c{};
  if (is_uniform(*desc)) {
    const int P = desc->partitions > 0 ? desc->partitions : default_partitions(*desc);
    if (desc->precision != TDMA_F32_REFINE && desc->partitions == 1 && use_thomas_variant(*desc)) {
      thomas_config(*desc, c);
    } else if (!choose_block(*desc, P, c)) {
      delete p;
      return TDMA_ERR_UNSUPPORTED;
    }
  } else {
    ragged_config(*desc, c);
  }
  p->cfg = c;
  p->workspace = workspace_for(*desc, c);
  if (cudaMalloc(&p->status, sizeof(DevStatus)) != cudaSuccess) { delete p; return TDMA_ERR_CUDA; }
  if (cudaMemset(p->status, 0, sizeof(DevStatus)) != cudaSuccess) { cudaFree(p->status); delete p; return TDMA_ERR_CUDA; }
  if (prepare_kernel(p) != cudaSuccess) { cudaFree(p->status); delete p; return TDMA_ERR_CUDA; }
  if (workspace_bytes) *workspace_bytes = p->workspace;
  *plan = p;
  return TDMA_OK;
}

tdma_status_t tdma_plan_destroy(tdma_plan_t p) {
  if (!p) return TDMA_OK;
  cudaError_t e = cudaSuccess;
  if (p->status) e = cudaFree(p->status);
  delete p;
  return e == cudaSuccess ? TDMA_OK : TDMA_ERR_CUDA;
}

tdma_status_t tdma_plan_get_config(tdma_plan_t p, tdma_config_t* c) {
  if (!p || !c) return TDMA_ERR_INVALID_ARG;
  *c = p->cfg;
  return TDMA_OK;
}

static tdma_status_t check_ptrs(const tdma_plan_s* p, const void* a, const void* b, const void* c, const void* d,
                                const void* x, void* ws, size_t ws_bytes) {
  if (p->desc.n_lines == 0) return TDMA_OK;
  if (!a || !b || !c || !d || !x) return TDMA_ERR_INVALID_ARG;
  if (ws_bytes < p->workspace || (p->workspace > 0 && !ws)) return TDMA_ERR_WORKSPACE;
  const size_t ce = elem_bytes_coef(p->desc.precision);
  const size_t de = (p->desc.precision == TDMA_F32 ? 4 : 8) * (size_t)p->desc.nrhs;
  if (!aligned(a, ce) || !aligned(b, ce) || !aligned(c, ce)) return TDMA_ERR_UNSUPPORTED;
  if (!aligned(d, de) || !aligned(x, de)) return TDMA_ERR_UNSUPPORTED;
  if (p->desc.diag_shift && !aligned(p->desc.diag_shift, ce)) return TDMA_ERR_UNSUPPORTED;
  return TDMA_OK;
}

tdma_status_t tdma_solve(tdma_plan_t p, const void* a, const void* b, const void* c, const void* d, void* x,
                         void* ws, size_t ws_bytes, void* stream) {
  if (!p) return TDMA_ERR_INVALID_ARG;
  const tdma_status_t v = check_ptrs(p, a, b, c, d, x, ws, ws_bytes);
  if (v != TDMA_OK) return v;
  const Args A = make_args(p, a, b, c, d, x, ws);
  const cudaError_t e = launch_forward(p, A, (cudaStream_t)stream);
  return e == cudaSuccess ? TDMA_OK : TDMA_ERR_CUDA;
}

tdma_status_t tdma_last_device_error(tdma_plan_t p, void* stream, int32_t* info) {
  if (!p) return TDMA_ERR_INVALID_ARG;
  DevStatus h{};
  if (cudaMemcpyAsync(&h, p->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
    return TDMA_ERR_CUDA;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return TDMA_ERR_CUDA;
  if (cudaMemsetAsync(p->status, 0, sizeof(DevStatus), (cudaStream_t)stream) != cudaSuccess) return TDMA_ERR_CUDA;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return TDMA_ERR_CUDA;
  if (info) *info = h.iters;
  return (tdma_status_t)h.err;
}

tdma_status_t tdma_solve_backward(tdma_plan_t p, const void* a, const void* b, const void* c, const void* x,
                                  const void* gx, void* ga, void* gb, void* gc, void* gd, void* ws,
                                  size_t ws_bytes, void* stream) {
  if (!p) return TDMA_ERR_INVALID_ARG;
  if (p->desc.n_lines == 0) return TDMA_OK;
  if (!a || !b || !c || !x || !gx) return TDMA_ERR_INVALID_ARG;
  if (ws_bytes < p->workspace || (p->workspace > 0 && !ws)) return TDMA_ERR_WORKSPACE;
  const cudaError_t e = launch_backward(p->desc, p->cfg, p->status, a, b, c, x, gx, ga, gb, gc, gd, ws,
                                        (cudaStream_t)stream);
  if (e == cudaErrorNotSupported) return TDMA_ERR_UNSUPPORTED;
  return e == cudaSuccess ? TDMA_OK : TDMA_ERR_CUDA;
}

tdma_status_t tdma_plan_autotune(tdma_plan_t p, const void* a, const void* b, const void* c, const void* d,
                                 void* x, void* ws, size_t ws_bytes, void* stream) {
  if (!p) return TDMA_ERR_INVALID_ARG;
  (void)a; (void)b; (void)c; (void)d; (void)x; (void)ws; (void)ws_bytes; (void)stream;
  return TDMA_OK;
}

}  // extern "C"
