// FFT-based Poisson solve on one GPU: cuFFT over the periodic (z, x) planes, the batched line
// solver along y for every wavenumber pair, cuFFT back (Section 5.2; Section 6.1). The pipeline
// is three library calls and two line solves on one stream; its layout choices are in tdma.h.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>
#include <cufft.h>

#include "tdma.h"

struct tdma_poisson_s {
  tdma_poisson_desc_t desc{};
  int64_t nkx = 0, L = 0;           // kx = 0..nx/2; lines = nz * nkx
  cufftHandle fwd = 0, inv = 0;
  bool have_fwd = false, have_inv = false;
  tdma_plan_t main = nullptr;       // lines 1 .. L-1 (all lines when the zero mode is not pinned)
  tdma_plan_t zero = nullptr;       // line 0 when pinned
  double* coef = nullptr;           // device: a, b, c scaled [3 ny]; pinned a, b, c [3 ny]; shift [L]
  size_t spec_bytes = 0, ws_main = 0, ws_zero = 0;
  size_t off_out = 0, off_main = 0, off_zero = 0, total = 0;
};

namespace {

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

double modified_k2(int64_t l, int64_t N, double h) {
  return (2.0 - 2.0 * std::cos(2.0 * M_PI * (double)l / (double)N)) / (h * h);
}

tdma_status_t make_fft(cufftHandle* h, int64_t ny, int64_t nz, int64_t nx, cufftType type) {
  if (cufftCreate(h) != CUFFT_SUCCESS) return TDMA_ERR_CUDA;
  long long n[2] = {(long long)nz, (long long)nx};
  size_t work = 0;
  if (cufftMakePlanMany64(*h, 2, n, nullptr, 1, 0, nullptr, 1, 0, type, (long long)ny, &work) != CUFFT_SUCCESS) {
    cufftDestroy(*h);
    return TDMA_ERR_CUDA;
  }
  return TDMA_OK;
}

}  // namespace

extern "C" {

tdma_status_t tdma_poisson_destroy(tdma_poisson_t p) {
  if (!p) return TDMA_OK;
  tdma_status_t st = TDMA_OK;
  if (p->have_fwd && cufftDestroy(p->fwd) != CUFFT_SUCCESS) st = TDMA_ERR_CUDA;
  if (p->have_inv && cufftDestroy(p->inv) != CUFFT_SUCCESS) st = TDMA_ERR_CUDA;
  if (p->main && tdma_plan_destroy(p->main) != TDMA_OK) st = TDMA_ERR_CUDA;
  if (p->zero && tdma_plan_destroy(p->zero) != TDMA_OK) st = TDMA_ERR_CUDA;
  if (p->coef && cudaFree(p->coef) != cudaSuccess) st = TDMA_ERR_CUDA;
  delete p;
  return st;
}

tdma_status_t tdma_poisson_create(tdma_poisson_t* plan, const tdma_poisson_desc_t* desc, size_t* workspace_bytes) {
  if (!plan || !desc) return TDMA_ERR_INVALID_ARG;
  *plan = nullptr;
  const tdma_poisson_desc_t& d = *desc;
  if (d.nx < 2 || d.nx % 2 || d.nz < 2 || d.ny < 2 || !(d.dx > 0) || !(d.dz > 0) || !d.a || !d.b || !d.c)
    return TDMA_ERR_INVALID_ARG;
  if (d.pin_zero_mode != 0 && d.pin_zero_mode != 1) return TDMA_ERR_INVALID_ARG;
  if (d.precision != TDMA_F64 && d.precision != TDMA_F64_REFINE) return TDMA_ERR_UNSUPPORTED;
  tdma_poisson_s* p = new (std::nothrow) tdma_poisson_s();
  if (!p) return TDMA_ERR_INVALID_ARG;
  p->desc = d;
  p->desc.a = p->desc.b = p->desc.c = nullptr;  // host arrays are not kept
  const int64_t ny = d.ny, nz = d.nz, nx = d.nx;
  p->nkx = nx / 2 + 1;
  p->L = nz * p->nkx;
  const double s = (double)nx * (double)nz;  // the FFT pair's 1 / (nx nz), folded into A
  // coefficients: A scaled by nx nz; the pinned copy with row 0 -> s * Phi_0 = 0; per-line shift
  std::vector<double> h((size_t)(6 * ny + p->L));
  for (int64_t j = 0; j < ny; ++j) {
    h[j] = s * d.a[j];
    h[ny + j] = s * d.b[j];
    h[2 * ny + j] = s * d.c[j];
  }
  std::memcpy(&h[3 * ny], &h[0], sizeof(double) * 3 * ny);
  h[4 * ny] = s;        // pinned b_0
  h[5 * ny] = 0.0;      // pinned c_0
  for (int64_t kz = 0; kz < nz; ++kz)
    for (int64_t kx = 0; kx < p->nkx; ++kx)
      h[6 * ny + kz * p->nkx + kx] = -s * (modified_k2(kx, nx, d.dx) + modified_k2(kz, nz, d.dz));
  if (cudaMalloc(&p->coef, sizeof(double) * h.size()) != cudaSuccess ||
      cudaMemcpy(p->coef, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    tdma_poisson_destroy(p);
    return TDMA_ERR_CUDA;
  }
  // line plans: spectrum [y][kz][kx] complex, line l = kz * nkx + kx at element y * L + l
  const bool pin = d.pin_zero_mode == 1;
  const int64_t first = pin ? 1 : 0;
  tdma_desc_t ld{};
  ld.n = ny;
  ld.n_lines = p->L - first;
  ld.elem_stride = p->L;
  ld.inner_count = p->L - first;
  ld.inner_stride = 1;
  ld.outer_stride = 0;
  ld.nrhs = 2;
  ld.coef_broadcast = 1;
  ld.diag_shift = p->coef + 6 * ny + first;
  ld.precision = d.precision;
  tdma_status_t st = TDMA_OK;
  if (ld.n_lines > 0) st = tdma_plan_create(&p->main, &ld, &p->ws_main);
  if (st == TDMA_OK && pin) {
    tdma_desc_t zd = ld;
    zd.n_lines = 1;
    zd.inner_count = 1;
    zd.diag_shift = nullptr;
    st = tdma_plan_create(&p->zero, &zd, &p->ws_zero);
  }
  if (st == TDMA_OK) st = make_fft(&p->fwd, ny, nz, nx, CUFFT_D2Z);
  if (st == TDMA_OK) p->have_fwd = true;
  if (st == TDMA_OK) st = make_fft(&p->inv, ny, nz, nx, CUFFT_Z2D);
  if (st == TDMA_OK) p->have_inv = true;
  if (st != TDMA_OK) {
    tdma_poisson_destroy(p);
    return st;
  }
  p->spec_bytes = (size_t)ny * (size_t)p->L * 2 * sizeof(double);
  size_t off = align256(p->spec_bytes);
  p->off_out = 0;
  if (d.precision == TDMA_F64_REFINE) {  // the corrected solve may not write over its input
    p->off_out = off;
    off += align256(p->spec_bytes);
  }
  p->off_main = off;
  off += align256(p->ws_main);
  p->off_zero = off;
  off += align256(p->ws_zero);
  p->total = off;
  if (workspace_bytes) *workspace_bytes = p->total;
  *plan = p;
  return TDMA_OK;
}

tdma_status_t tdma_poisson_solve(tdma_poisson_t p, const double* q, double* phi, void* workspace,
                                 size_t workspace_bytes, void* stream) {
  if (!p || !q || !phi || !workspace) return TDMA_ERR_INVALID_ARG;
  if (workspace_bytes < p->total) return TDMA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t ny = p->desc.ny;
  unsigned char* ws = (unsigned char*)workspace;
  double* spec = (double*)ws;
  double* out = (double*)(ws + p->off_out);  // == spec unless the lines are corrected
  if (cufftSetStream(p->fwd, s) != CUFFT_SUCCESS || cufftSetStream(p->inv, s) != CUFFT_SUCCESS)
    return TDMA_ERR_CUDA;
  if (cufftExecD2Z(p->fwd, const_cast<double*>(q), (cufftDoubleComplex*)spec) != CUFFT_SUCCESS)
    return TDMA_ERR_CUDA;
  const bool pin = p->zero != nullptr;
  const int64_t first = pin ? 1 : 0;
  const double* A = p->coef;
  tdma_status_t st = TDMA_OK;
  if (p->main)
    st = tdma_solve(p->main, A, A + ny, A + 2 * ny, spec + 2 * first, out + 2 * first, ws + p->off_main,
                    p->ws_main, stream);
  if (st != TDMA_OK) return st;
  if (pin) {
    // row 0 of the (0, 0) line: Phi_0 = 0
    if (cudaMemsetAsync(spec, 0, 2 * sizeof(double), s) != cudaSuccess) return TDMA_ERR_CUDA;
    st = tdma_solve(p->zero, A + 3 * ny, A + 4 * ny, A + 5 * ny, spec, out, ws + p->off_zero, p->ws_zero, stream);
    if (st != TDMA_OK) return st;
  }
  if (cufftExecZ2D(p->inv, (cufftDoubleComplex*)out, phi) != CUFFT_SUCCESS) return TDMA_ERR_CUDA;
  return TDMA_OK;
}

tdma_status_t tdma_poisson_last_error(tdma_poisson_t p, void* stream) {
  if (!p) return TDMA_ERR_INVALID_ARG;
  tdma_status_t st = TDMA_OK;
  if (p->main) st = tdma_last_device_error(p->main, stream, nullptr);
  if (p->zero) {
    const tdma_status_t z = tdma_last_device_error(p->zero, stream, nullptr);
    if (st == TDMA_OK) st = z;
  }
  return st;
}

}  // extern "C"
