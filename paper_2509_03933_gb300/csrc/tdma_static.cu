// Allocation-free Thomas solve: tdma_solve_thomas_static (declared in include/tdma.h).
//
// Some callers cannot allocate device memory once they are running: a time-stepping loop of
// a flow solver that sized all of its GPU memory at start-up and treats any later
// cudaMalloc as a fault, or a host program that owns the device heap through its own pool
// and does not let libraries allocate behind its back. tdma_plan_create allocates a status
// block and tdma_solve wants a caller-provided workspace, so neither suits them. This entry
// point runs the P = 1 Thomas kernel with its elimination factors in a fixed array compiled
// into the library, and calls no cudaMalloc, cudaFree or any other allocating routine.
//
// The array lives in device memory of every GPU that loads the library, for as long as the
// process runs; its size limits the problem (kStaticScratchBytes). All calls share it and it
// keeps whatever the last call left there. Nothing in it has to start at zero: each call
// writes every factor before reading it. Calls whose kernels overlap on the GPU (different
// streams, or different host threads) race on the array and must not be issued.
#include <cstdint>
#include <mutex>

#include <cuda.h>

#include "tdma.h"
#include "kernels_thomas.cuh"

namespace {

constexpr size_t kStaticScratchBytes = 32u << 20;  // 32 MiB: 4 Mi FP64 or 8 Mi FP32 factors
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_thomas_scratch[kStaticScratchBytes];

// Device address of g_thomas_scratch, looked up with the device current, once per device and
// context: the address belongs to the module loaded into a context, so a new primary context (after
// cudaDeviceReset) gets its own lookup. cudaGetSymbolAddress allocates nothing.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(ptr);
  });
  return fn;
}

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const CtxGetCurrentFn get = ctx_get_current();
  CUcontext ctx = nullptr;
  // a context not yet current on this thread reads as null: the lookup below makes it current
  const bool have_ctx = get && get(&ctx) == CUDA_SUCCESS && ctx != nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!have_ctx || !g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_thomas_scratch);
    if (e != cudaSuccess) return e;
    if (!have_ctx && get && get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    g_scratch_addr[dev] = ptr;
    g_scratch_ctx[dev] = ctx;  // null: not known, looked up again next time
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

bool aligned_to(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

extern "C" tdma_status_t tdma_solve_thomas_static(const tdma_desc_t* desc, const void* a, const void* b,
                                                  const void* c, const void* d, void* x, void* stream) {
  if (!desc) return TDMA_ERR_INVALID_ARG;
  const tdma_desc_t& dd = *desc;
  if (dd.n < 1 || dd.n_lines < 0 || (dd.nrhs != 1 && dd.nrhs != 2)) return TDMA_ERR_INVALID_ARG;
  if (dd.precision == TDMA_F32_REFINE || dd.precision == TDMA_F64_REFINE) return TDMA_ERR_UNSUPPORTED;
  if (dd.precision != TDMA_F64 && dd.precision != TDMA_F32) return TDMA_ERR_INVALID_ARG;
  if (dd.partitions < 0) return TDMA_ERR_INVALID_ARG;
  if (dd.inner_count < 1 || dd.elem_stride < 0 || dd.inner_stride < 0 || dd.outer_stride < 0)
    return TDMA_ERR_INVALID_ARG;
  if (dd.partitions > 1) return TDMA_ERR_UNSUPPORTED;  // the Thomas form has one partition
  if (dd.pdd != 0) return TDMA_ERR_UNSUPPORTED;
  if (dd.n_lines == 0) return TDMA_OK;
  if (!a || !b || !c || !d || !x) return TDMA_ERR_INVALID_ARG;
  const size_t eb = dd.precision == TDMA_F64 ? 8 : 4;
  if (!aligned_to(a, eb) || !aligned_to(b, eb) || !aligned_to(c, eb) || !aligned_to(d, eb * dd.nrhs) ||
      !aligned_to(x, eb * dd.nrhs) || (dd.diag_shift && !aligned_to(dd.diag_shift, eb)))
    return TDMA_ERR_UNSUPPORTED;
  // one factor per unknown; larger problems do not fit the fixed array
  if ((uint64_t)dd.n > kStaticScratchBytes / eb / (uint64_t)dd.n_lines) return TDMA_ERR_WORKSPACE;

  void* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return TDMA_ERR_CUDA;

  tdma::Args A{};
  A.a = a; A.b = b; A.c = c; A.d = d; A.x = x;
  A.shift = dd.diag_shift;
  A.lay = tdma::Layout{dd.n, dd.n_lines, dd.elem_stride, dd.inner_count, dd.inner_stride, dd.outer_stride};
  A.P = 1;
  A.Lb = tdma::kThomasBlock;
  A.mmax = (int)dd.n;
  A.bcast = dd.coef_broadcast;
  A.st = nullptr;  // no status block: a zero pivot shows up as non-finite values in x
  A.ws = scratch;
  tdma_config_t cfg{};
  tdma::thomas_config(dd, cfg);
  const cudaError_t e = tdma::launch_thomas(dd.precision, dd.nrhs, A, cfg, (cudaStream_t)stream);
  return e == cudaSuccess ? TDMA_OK : TDMA_ERR_CUDA;
}
