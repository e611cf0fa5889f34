/*
 * tdma.h -- C ABI of a batched divide-and-conquer tridiagonal solver for one GB300 (sm_103a).
 *
 * Problem (Algorithm 1: "Ax = d, N times; input a, b, c, d; output x"; Section 3.2.1: a, b
 * and c are the sub-, main and super-diagonal of A). For every line l = 0..n_lines-1:
 *
 *     a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i,      i = 0..n-1,
 *
 * with a_0 and c_{n-1} of every line ignored (treated as 0: no coupling outside the line).
 * Lines run along one axis of a strided grid (Section 4.2.1 groups the systems of one
 * direction of a 3D field into batches). Each line is split into P contiguous partitions
 * (Section 2.1: Stage A decoupled solve, Stage B reduced solve, Stage C correction; Section
 * 2.2: the reduced system grows with P); on one GPU the partitions are threads and the
 * paper's A2B/B2C exchanges become on-chip data movement.
 *
 * Memory and ownership
 *   - Every array argument is a DEVICE pointer owned by the caller and must stay valid until
 *     the work queued on `stream` has finished. The library never frees caller memory.
 *   - `workspace` is caller-owned device scratch of at least the size reported by
 *     tdma_plan_create (may be 0 bytes, then NULL is accepted).
 *   - A plan owns host state plus one small device status block, allocated in
 *     tdma_plan_create and freed in tdma_plan_destroy. tdma_solve and tdma_solve_backward
 *     allocate nothing.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *
 * Element layout
 *   An "element" is one unknown of one line. Line l starts at element
 *       off(l) = (l / inner_count) * outer_stride + (l % inner_count) * inner_stride
 *   and its unknown i sits at element off(l) + i * elem_stride (strides in elements, may be
 *   any non-negative values; lines must not overlap when x is written). d and x hold nrhs
 *   consecutive values per element (nrhs = 2: interleaved real/imaginary parts of a complex
 *   right-hand side sharing real coefficients). a, b, c hold one value per element, or, with
 *   coef_broadcast = 1, are 1D arrays of length n shared by all lines.
 *   Ragged batches (n = 0): line l has ragged_lengths[l] unknowns starting at element
 *   ragged_offsets[l], unit stride (packed lines); both arrays are device pointers.
 *
 * Precision (`precision`)
 *   TDMA_F64         a, b, c, d, x, diag_shift double; arithmetic double.
 *   TDMA_F32         all float; arithmetic float.
 *   TDMA_F32_REFINE  a, b, c float; d, x, diag_shift double. Sweeps in float, then
 *                    iterative refinement with an extra-precise residual r = d - A x
 *                    until the estimated error is below refine_tol (relative, per line).
 *   TDMA_F64_REFINE  as TDMA_F64, followed by max_refine_iters (default 1) corrections, for
 *                    badly conditioned lines where plain FP64 elimination stops a few 1e-12
 *                    short: the residual r = d - A x is formed in fixed point to within
 *                    2^-104 of its largest term (integer arithmetic on the 53-bit significands)
 *                    and the correction A dx = r is solved in FP32.
 *                    With coef_broadcast, only the lines that need it are corrected: a line whose
 *                    condition-number bound ||A||_inf / delta is below refine_kappa keeps the plain
 *                    FP64 result (delta: the smallest diagonal-dominance margin of a row,
 *                    |b_i| - |a_i| - |c_i|, which bounds ||A^-1||_inf by 1 / delta for a diagonally
 *                    dominant A; a line without a positive margin is always corrected). The lines
 *                    are picked on the device at every solve (tdma_plan_corrected_lines reports how
 *                    many). Per-element coefficients: every line is corrected.
 *                    Lines whose residuals fall below the float range (right-hand sides under
 *                    about 1e-22) keep the plain FP64 accuracy. x must not alias d; the
 *                    workspace holds the FP32 correction's factors (4 (1 + nrhs) bytes per
 *                    unknown) and the list of corrected lines.
 *
 * Approximate reduced solve (`pdd` = 1)
 *   The parallel diagonally dominant (PDD) method the paper's momentum solver applies to its
 *   diagonally dominant ADI systems (Section 5.1; Section 6.2.2). Each partition k of m rows is
 *   solved on its own, x_k = xt_k - v_k x_{k-1,m-1} - w_k x_{k+1,0} (xt: the partition's solution
 *   without its outer couplings; v, w: its responses to the couplings a_{k,0} and c_{k,m-1});
 *   at every interface between partitions k and k+1 the two end unknowns then follow from a 2x2
 *   system that drops the couplings v_k(m-1) x_{k-1,m-1} and w_{k+1}(0) x_{k+2,0}, which decay
 *   geometrically with m on diagonally dominant lines; finally every partition is updated with
 *   its neighbours' interface values. Exact for P = 1; otherwise an approximation whose error
 *   the caller accepts. Uniform lines, TDMA_F64 or TDMA_F32, partitions >= 1 given explicitly;
 *   no backward pass (tdma_solve_backward returns TDMA_ERR_UNSUPPORTED), autotune keeps the
 *   configuration.
 *
 * Errors
 *   Every call validates its arguments synchronously and returns a status; nothing aborts.
 *   Numerical faults found on the device (a zero or non-finite pivot, refinement that did
 *   not converge, a bounded wait that ran out) are recorded in the plan's device status
 *   block and read back by tdma_last_device_error.
 */
#ifndef TDMA_H_
#define TDMA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TDMA_OK = 0,
  TDMA_ERR_INVALID_ARG = 1,   /* bad descriptor or pointer, detected on the host          */
  TDMA_ERR_UNSUPPORTED = 2,   /* valid but not supported (e.g. misaligned vector access)  */
  TDMA_ERR_WORKSPACE = 3,     /* workspace smaller than tdma_plan_create reported         */
  TDMA_ERR_CUDA = 4,          /* a CUDA runtime call failed                               */
  TDMA_ERR_NONFINITE = 5,     /* device: zero or non-finite pivot / result                */
  TDMA_ERR_TIMEOUT = 6,       /* device: a bounded wait gave up                           */
  TDMA_ERR_NOT_CONVERGED = 7  /* device: refinement hit max_refine_iters                  */
} tdma_status_t;

typedef enum { TDMA_F64 = 0, TDMA_F32 = 1, TDMA_F32_REFINE = 2, TDMA_F64_REFINE = 3 } tdma_precision_t;

typedef struct tdma_plan_s* tdma_plan_t;

typedef struct {
  int64_t n;             /* unknowns per line (uniform lines, >= 1); 0 selects a ragged batch */
  int64_t n_lines;       /* number of lines (>= 0)                                            */
  int64_t elem_stride;   /* element stride between consecutive unknowns of a line             */
  int64_t inner_count;   /* line addressing, see off(l) above (>= 1)                          */
  int64_t inner_stride;
  int64_t outer_stride;
  const int64_t* ragged_offsets; /* device, n_lines entries (n == 0 only)                     */
  const int32_t* ragged_lengths; /* device, n_lines entries, each >= 1 (n == 0 only)          */
  int64_t ragged_max_n;  /* host-known upper bound of ragged_lengths (n == 0 only)            */
  int64_t ragged_total;  /* host-known sum of ragged_lengths (n == 0 only)                    */
  int32_t nrhs;          /* 1, or 2 (interleaved complex right-hand side)                     */
  int32_t coef_broadcast;/* 0: per-element a, b, c; 1: 1D a, b, c of length n for all lines   */
  const void* diag_shift;/* optional device array, one value per line, added to b (may be NULL)*/
  tdma_precision_t precision;
  int32_t partitions;    /* P partitions per line; 0 = choose automatically                   */
  int32_t max_refine_iters; /* TDMA_F32_REFINE: correction steps at most (0 = default 4)     */
  double refine_tol;     /* TDMA_F32_REFINE: target relative error per line (<= 0: 2.5e-13) */
  int32_t pdd;           /* 0: exact; 1: parallel diagonally dominant approximation, see below */
  double refine_kappa;   /* TDMA_F64_REFINE with coef_broadcast: lines whose condition-number bound
                            is below this keep the plain FP64 result (0: 1e5; < 0: correct all)  */
} tdma_desc_t;

/* Launch configuration a plan has settled on (reported for benchmarks and tests). */
typedef struct {
  int32_t partitions;      /* P                                                        */
  int32_t rows_per_thread; /* ceil(n / P) for uniform lines                            */
  int32_t lines_per_block; /* lines handled by one thread block                        */
  int32_t threads_per_block;
  int32_t variant;         /* kernel family, see TDMA_VARIANT_*                        */
  int32_t blocks;          /* grid size of the main launch                             */
  int64_t smem_bytes;      /* dynamic shared memory of the main launch                 */
  int64_t workspace_bytes; /* workspace tdma_solve needs with this configuration        */
} tdma_config_t;

enum {
  TDMA_VARIANT_DC = 0,       /* fused Stage A/B/C, one block per group of lines          */
  TDMA_VARIANT_THOMAS = 1,   /* P = 1 Thomas sweep, elimination factors in the workspace */
  TDMA_VARIANT_REFINE = 2,   /* fused float sweeps with on-chip refinement               */
  TDMA_VARIANT_RAGGED = 3,   /* persistent launch over a device queue of ragged lines    */
  TDMA_VARIANT_REFINE_REG = 4, /* refinement with per-row state in registers             */
  TDMA_VARIANT_REFINE_TMA = 5, /* refinement on a TMA-staged shared-memory tile          */
  TDMA_VARIANT_REFINE_CLUSTER = 6, /* refinement with each line spread over a CTA cluster */
  TDMA_VARIANT_DC_GLOBAL = 7, /* fused Stage A/B/C, Stage A scratch in the workspace        */
  TDMA_VARIANT_REFINE_TREE = 8, /* refinement over a CTA cluster, Stage B as a merge tree    */
  TDMA_VARIANT_PACKED = 9,    /* ragged refinement: chunks of packed lines per CTA cluster */
  TDMA_VARIANT_SHARED = 10,   /* shared coefficients (broadcast, no shift): factorised once  */
  TDMA_VARIANT_REFINE_TREE_X = 11 /* the merge-tree cluster refinement on unit-stride lines  */
};

/* Validate `desc`, choose a launch configuration and report the workspace it needs.
 * Allocates the plan's host state and its small device status block (cudaMalloc on the
 * current device). Returns TDMA_ERR_INVALID_ARG for a bad descriptor (n < 0, n_lines < 0,
 * nrhs not 1 or 2, P larger than n/2 for P > 1, ragged fields missing, ...). */
tdma_status_t tdma_plan_create(tdma_plan_t* plan, const tdma_desc_t* desc, size_t* workspace_bytes);

/* Release a plan (synchronises its device status block first). NULL is accepted. */
tdma_status_t tdma_plan_destroy(tdma_plan_t plan);

/* Solve A x = d for every line (forward pass). x may alias d. Enqueues kernels on `stream`
 * and returns without waiting; allocates nothing. Arrays must be aligned to their element size
 * (both values of a pair with nrhs = 2); the cluster variants (TDMA_VARIANT_REFINE_CLUSTER,
 * _REFINE_TREE, _REFINE_TREE_X) move tiles by TMA and need every array 16-byte aligned.
 * Otherwise TDMA_ERR_UNSUPPORTED, before anything is enqueued. */
tdma_status_t tdma_solve(tdma_plan_t plan, const void* a, const void* b, const void* c,
                         const void* d, void* x, void* workspace, size_t workspace_bytes,
                         void* stream);

/* Backward pass of x = A^{-1} d for a scalar loss with dL/dx = grad_x (adjoint method; the
 * paper has no backward pass): solves A^T lambda = grad_x with the same divide-and-conquer
 * kernels on the transposed diagonals, then writes
 *   grad_d = lambda, grad_b_i = -lambda_i x_i, grad_a_i = -lambda_i x_{i-1} (0 at i = 0),
 *   grad_c_i = -lambda_i x_{i+1} (0 at i = n-1).
 * x is the forward solution. grad_d is required (it holds lambda); grad_a, grad_b and grad_c
 * may be NULL to skip them. With coef_broadcast = 1 the coefficient gradients are sums over
 * lines, ADDED to the length-n arrays given (zero them first). Types follow `precision`
 * (F32_REFINE: grad_a/b/c float, grad_d double). Ragged batches are supported (per-line arrays). */
tdma_status_t tdma_solve_backward(tdma_plan_t plan, const void* a, const void* b, const void* c,
                                  const void* x, const void* grad_x, void* grad_a, void* grad_b,
                                  void* grad_c, void* grad_d, void* workspace,
                                  size_t workspace_bytes, void* stream);

/* Autotune (the on-device analogue of the batch-size estimator of Section 4.2.3): time the
 * launch configurations valid for the plan's lines (partitions per line, lines per block,
 * kernel family) on the caller's data with CUDA events on `stream`, each run several times,
 * overwriting x, and keep the fastest. Only candidates whose workspace fits `workspace_bytes`
 * are tried; afterwards tdma_plan_get_config reports the choice and the workspace it needs.
 * Synchronises `stream`. Choices are cached per process by problem class (precision, n, line
 * count bucket, unit or strided axis, nrhs, broadcast) and, when the environment variable
 * TDMA_AUTOTUNE_CACHE names a file, read from and appended to that file; a plan created with
 * partitions == 0 starts from a cached choice when there is one. Ragged plans keep their
 * configuration (returns TDMA_OK). */
tdma_status_t tdma_plan_autotune(tdma_plan_t plan, const void* a, const void* b, const void* c,
                                 const void* d, void* x, void* workspace, size_t workspace_bytes,
                                 void* stream);

/* Report the launch configuration in use. */
tdma_status_t tdma_plan_get_config(tdma_plan_t plan, tdma_config_t* config);

/* Synchronise `stream`, read and clear the plan's device status block. Returns TDMA_OK or
 * the first device-side error recorded since the last call. If `info` is not NULL it
 * receives the largest number of refinement corrections any line used. */
tdma_status_t tdma_last_device_error(tdma_plan_t plan, void* stream, int32_t* info);

/* Synchronise `stream` and report in *lines how many lines the last TDMA_F64_REFINE solve of the plan
 * corrected (the rest kept the plain FP64 result); 0 for other precisions. Does not clear the plan's
 * status block. */
tdma_status_t tdma_plan_corrected_lines(tdma_plan_t plan, void* stream, int64_t* lines);

/* Static, human-readable name of a status code. */
const char* tdma_status_string(tdma_status_t status);

/* Layout of a batch of lines in HOST memory for tdma_solve_host: n unknowns per line, n_lines
 * lines; unknown i of line l is element l * line_stride + i * row_stride of each array. Two forms
 * are accepted: adjacent lines (line_stride = 1, row_stride >= n_lines; e.g. a C-order grid
 * solved along its slowest axis) and contiguous lines (row_stride = 1, line_stride >= n). */
typedef struct {
  int64_t n;
  int64_t n_lines;
  int64_t line_stride;
  int64_t row_stride;
} tdma_host_layout_t;

/* Solve lines held in HOST memory (page-locked for full copy speed) as a pipeline of slices
 * (Section 4.2: batches of systems in flight; on one GPU, slices of lines in flight on CUDA
 * streams): the host lines are cut into consecutive slices of plan->n_lines lines; slice s goes
 * to staging slot s mod n_slots, whose stream copies the slice's a, b, c, d to the slot's device
 * buffers, solves it with `plan` and copies x back, so that the copies of one slice overlap the
 * solve of another (host-to-device, device-to-host and kernels run concurrently).
 *   plan          created for ONE slice in the slot buffers' compact layout: n as the host
 *                 layout, n_lines = slice lines, and either elem_stride = inner_count = slice
 *                 lines, inner_stride = 1 (adjacent lines) or elem_stride = 1, inner_stride = n,
 *                 inner_count = slice lines (contiguous lines); nrhs = 1, no broadcast, no shift.
 *   layout        the host layout (above); layout->n_lines must be a multiple of the slice lines.
 *   a, b, c, d, x host arrays in the plan's element types; x may not alias d.
 *   slot_buffers  n_slots x 5 device pointers (a, b, c, d, x of slot k at [5k .. 5k+4]), each
 *                 holding one slice; slot_workspaces: n_slots device pointers of workspace_bytes
 *                 each (the plan's workspace; NULL entries allowed when it needs none).
 *   streams       n_slots cudaStream_t (as void*), one per slot.
 * Enqueues everything and returns without waiting; allocates nothing. Errors: TDMA_ERR_INVALID_ARG
 * (layouts that do not match, n_slots < 1, a slice count that does not divide the lines),
 * TDMA_ERR_UNSUPPORTED (nrhs, broadcast or shift), TDMA_ERR_WORKSPACE, TDMA_ERR_CUDA. */
tdma_status_t tdma_solve_host(tdma_plan_t plan, const tdma_host_layout_t* layout, const void* a, const void* b,
                              const void* c, const void* d, void* x, int32_t n_slots,
                              void* const* slot_buffers, void* const* slot_workspaces,
                              size_t workspace_bytes, void* const* streams);

/* Solve A x = d with the one-partition Thomas kernel without allocating anything (the paper has
 * no counterpart; this serves callers that must not allocate device memory while they run, e.g.
 * a solver loop that fixed its GPU memory at start-up, or a host program whose own memory pool
 * owns the device heap). No plan and no workspace: the elimination factors go to a fixed
 * 32 MiB array compiled into the library, present on every GPU that loads it until the
 * process exits. Takes the same descriptor fields as tdma_plan_create for uniform lines
 * (n >= 1; precision TDMA_F64 or TDMA_F32; nrhs, coef_broadcast and diag_shift as there;
 * partitions 0 or 1) and the same device arrays as tdma_solve; x may alias d; enqueues on
 * `stream`. Returns TDMA_ERR_WORKSPACE when n * n_lines factors (8 bytes each in FP64, 4 in FP32)
 * exceed the array; TDMA_ERR_INVALID_ARG for a bad descriptor (n < 1, negative counts or strides,
 * partitions < 0, nrhs not 1 or 2, an unknown precision, a NULL array); TDMA_ERR_UNSUPPORTED for
 * what the plan-based solve supports but this entry does not (TDMA_F32_REFINE, TDMA_F64_REFINE,
 * partitions > 1, pdd, misaligned arrays). Device-side numerical faults are not recorded (no
 * status block): a zero pivot leaves non-finite values in x. The first call on a device, and the
 * first after that device's context was replaced (cudaDeviceReset), looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first call before any stream
 * capture. All calls share the array: calls that could run at the same time on the GPU (other
 * streams, other host threads) race on it and must not be issued. */
tdma_status_t tdma_solve_thomas_static(const tdma_desc_t* desc, const void* a, const void* b,
                                       const void* c, const void* d, void* x, void* stream);

/* ---- FFT-based Poisson solve on one GPU (Section 5.2; Section 6.1, Poisson-v1) ---------------
 * Solves the discrete Poisson equation  D_xx phi + D_yy phi + D_zz phi = q  on a grid periodic in
 * x and z, with the wall-normal operator D_yy given as a tridiagonal matrix (a, b, c along y):
 * a 2D real FFT of every (z, x) plane turns it into one tridiagonal system along y per wavenumber
 * pair, (D_yy - k'_x^2 - k'_z^2) Phi = Q with the modified wavenumbers of the second-order periodic
 * differences k'^2(l) = (2 - 2 cos(2 pi l / N)) / h^2; those lines are solved by the batched
 * solver (broadcast a, b, c with a per-line diagonal shift, complex right-hand side as two
 * interleaved real ones); an inverse FFT returns phi.
 *   Layout: q and phi are DEVICE arrays of ny x nz x nx doubles, x fastest (phi[y][z][x]). The
 *   plane transforms then leave the spectrum as [y][kz][kx] (kx = 0..nx/2), so the lines along y
 *   are adjacent in memory and strided by one plane: no transpose, no 2D-into-3D insertion (the
 *   non-coalesced copy Poisson-v1 works around). phi may alias q.
 *   Scaling: the FFT pair's 1 / (nx nz) is folded into the line coefficients (no extra pass).
 *   Zero mode: with pin_zero_mode = 1 the (kx, kz) = (0, 0) line's row 0 is replaced by Phi_0 = 0
 *   (the Neumann-ended D_yy makes that line singular); solved by its own one-line plan.
 *   FFTs: cuFFT (D2Z / Z2D, batched over y); its plans and work areas are created in
 *   tdma_poisson_create. tdma_poisson_solve allocates nothing. */
typedef struct tdma_poisson_s* tdma_poisson_t;

typedef struct {
  int64_t nx, ny, nz;     /* grid points (nx even, nx, nz >= 2, ny >= 2)                      */
  double dx, dz;          /* periodic spacings (> 0)                                          */
  const double* a;        /* HOST, ny values: D_yy's sub-diagonal (a[0] ignored)              */
  const double* b;        /* HOST, ny values: its diagonal                                    */
  const double* c;        /* HOST, ny values: its super-diagonal (c[ny-1] ignored)            */
  int32_t pin_zero_mode;  /* 1: pin the (0, 0) line as above; 0: solve it as given            */
  tdma_precision_t precision; /* TDMA_F64, or TDMA_F64_REFINE for the wavenumber lines        */
} tdma_poisson_desc_t;

/* Copies the coefficients to the device, creates the cuFFT plans and the line plans, and reports
 * the workspace tdma_poisson_solve needs (the spectrum, twice with TDMA_F64_REFINE, plus the line
 * plans' workspaces). TDMA_ERR_INVALID_ARG for a bad descriptor, TDMA_ERR_UNSUPPORTED for another
 * precision, TDMA_ERR_CUDA when cuFFT or CUDA fails. */
tdma_status_t tdma_poisson_create(tdma_poisson_t* plan, const tdma_poisson_desc_t* desc, size_t* workspace_bytes);

/* phi = the solution for right-hand side q (device arrays as above); enqueued on `stream`.
 * Device-side numerical faults of the line solves are read by tdma_poisson_last_error. */
tdma_status_t tdma_poisson_solve(tdma_poisson_t plan, const double* q, double* phi, void* workspace,
                                 size_t workspace_bytes, void* stream);

/* Synchronise `stream` and read (and clear) the line plans' device status. */
tdma_status_t tdma_poisson_last_error(tdma_poisson_t plan, void* stream);

tdma_status_t tdma_poisson_destroy(tdma_poisson_t plan);

/* ---- Lines split across ranks (Section 2.1; Algorithm 2) --------------------------------------
 * Every rank holds a slab of consecutive rows of every line (the paper's 1D decomposition along
 * the solve axis). Per batch of lines [line0, line0 + count):
 *   1. tdma_slab_reduce on every rank: Stage A over its slab (the slab is one partition). Writes,
 *      per line, the slab's first and last rows as a unit-diagonal pair in the neighbouring slabs'
 *      end unknowns: K = 4 + 2 nrhs doubles [sub0, sup0, sub1, sup1, rhs0[nrhs], rhs1[nrhs]] to
 *      `reduced` ([count][K]), and the interior relations to `scratch`
 *      (tdma_slab_scratch_bytes(desc, count) bytes, [array][row][line]; kept for step 4).
 *   2. an all-to-all (the caller's; the paper's A2B): the rank that solves Stage B for a line
 *      gathers the line's pairs from all W slabs, slab-major: gathered[W][lines][K].
 *   3. tdma_slab_pairs_solve on that rank: the 2W-row unit-diagonal system of every gathered line
 *      by Thomas in FP64; writes every slab's first and last values, ends[W][lines][2 nrhs]
 *      (`work`: tdma_slab_pairs_work_bytes bytes of device scratch).
 *   4. an all-to-all back (B2C), then tdma_slab_finish on every rank: Stage C over its slab from
 *      its own two end values, ends[count][2 nrhs].
 * All arrays are FP64 DEVICE arrays owned by the caller; the slab's a, b, c, d, x use the element
 * addressing of tdma_desc_t with n = n_local rows (d, x with nrhs interleaved values). first /
 * last mark the slab that holds the line's first / last row (its a_0 / c_{n-1} are ignored).
 * n_local >= 2. Zero or non-finite pivots set *status to TDMA_ERR_NONFINITE (status: a device
 * int32, may be NULL). The calls enqueue on `stream` and allocate nothing. */
typedef struct {
  int64_t n_local;        /* rows of this rank's slab (>= 2)                          */
  int64_t n_lines;        /* lines in the local arrays                                */
  int64_t elem_stride;    /* addressing as in tdma_desc_t, with n = n_local           */
  int64_t inner_count;
  int64_t inner_stride;
  int64_t outer_stride;
  int32_t nrhs;           /* 1 or 2                                                   */
  int32_t first;          /* 1: this slab holds row 0 of every line                   */
  int32_t last;           /* 1: this slab holds row n-1 of every line                 */
} tdma_slab_desc_t;

size_t tdma_slab_scratch_bytes(const tdma_slab_desc_t* desc, int64_t count);
size_t tdma_slab_pairs_work_bytes(int32_t n_slabs, int64_t count, int32_t nrhs);
tdma_status_t tdma_slab_reduce(const tdma_slab_desc_t* desc, const double* a, const double* b, const double* c,
                               const double* d, int64_t line0, int64_t count, double* reduced, double* scratch,
                               int32_t* status, void* stream);
tdma_status_t tdma_slab_pairs_solve(int32_t n_slabs, int64_t count, int32_t nrhs, const double* gathered,
                                    double* ends, double* work, int32_t* status, void* stream);
tdma_status_t tdma_slab_finish(const tdma_slab_desc_t* desc, int64_t line0, int64_t count, const double* ends,
                               const double* scratch, double* x, void* stream);

/* ---- Measurement --------------------------------------------------------------------------------
 * FP64 fused multiply-add throughput of the current GPU (the paper has no counterpart; it serves the
 * FP64 roofline of the solve kernels, whose sweeps run on the FP64 pipe). Launches `blocks` blocks of
 * `threads` threads (a multiple of 32, at most 1024); every thread runs 8 independent chains of `iters`
 * FP64 FMAs. The caller times the launch on `stream` (e.g. with CUDA events) and divides *fma_count
 * (set on success to blocks * threads * iters * 8) by the time. `out`: a device array of `blocks`
 * doubles, written only in the impossible case that keeps the chains from being optimised away.
 * TDMA_ERR_INVALID_ARG for bad sizes, TDMA_ERR_CUDA when the launch fails. */
tdma_status_t tdma_probe_fp64_fma(int32_t blocks, int32_t threads, int64_t iters, double* out, int64_t* fma_count,
                                  void* stream);

/* Failure detection without a fault (the paper has no counterpart): every wait of the solver kernels
 * on an mbarrier (TMA tile arrivals, cluster exchanges) polls a bounded number of times and then gives
 * up with TDMA_ERR_TIMEOUT in the plan's status block instead of hanging. This launches one warp that
 * runs that same bounded wait, `polls` polls (1 .. 2^20; about 64 ns each after the first 64), on an
 * mbarrier nothing arrives on and nothing is in flight for, then writes TDMA_ERR_TIMEOUT into *status
 * (a device int32 the caller zeroes first; written only if still 0). The GPU context stays usable.
 * TDMA_ERR_INVALID_ARG for a NULL status or polls out of range. */
tdma_status_t tdma_probe_bounded_wait(uint32_t polls, int32_t* status, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TDMA_H_ */
