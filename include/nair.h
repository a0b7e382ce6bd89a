/*
 * nair.h -- C ABI of the GB300 block-nAIR library (libnair.so).
 *
 * nAIR is the reduction-based algebraic multigrid of Manteuffel, Muenzenmaier,
 * Ruge and Southworth, "Nonsymmetric reduction-based algebraic multigrid"
 * (arXiv 1704.05001).  The library solves a sparse, nonsymmetric, block
 * (near-)triangular system A x = b, such as an upwind DG discretisation of
 * steady transport (Sec. 2.1 and Eq. transport, Sec. 6.1), with flexible
 * GMRES preconditioned by one nAIR V-cycle (Sec. 5 and 6).
 *
 * Conventions for every entry point:
 *   - Matrices are block CSR (BSR) with square b x b blocks, b in 1..32, each
 *     block stored row-major; column indices are sorted and unique within a
 *     row and every block row holds its diagonal block.
 *   - "device" pointers are CUDA global-memory addresses on the current device;
 *     "host" pointers are ordinary CPU memory.  The caller owns every pointer
 *     it passes; the library copies what it keeps and retains no caller
 *     pointer after a call returns.  The device vectors of the solves and
 *     cycles (b, x, w, lambda, f) must start on a 16-byte boundary (as every
 *     cudaMalloc'd or torch-allocated buffer does); a misaligned vector is
 *     rejected with NAIR_ERR_INVALID_ARG before any work is queued.
 *   - Work is ordered on the stream given in nair_params (NULL = the legacy
 *     default stream).  Calls that return sizes or statuses synchronise that
 *     stream.
 *   - Every call returns a nair_status; on failure nair_last_error() returns a
 *     message for the calling thread.  A handle must not be used by two
 *     threads at once.
 */
#ifndef NAIR_H
#define NAIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NAIR_OK = 0,
  NAIR_ERR_INVALID_ARG = 1,    /* bad sizes, pointers, structure or parameters */
  NAIR_ERR_SINGULAR_BLOCK = 2, /* a diagonal block (or the coarsest matrix) is singular */
  NAIR_ERR_NOT_CONVERGED = 3,  /* GMRES reached maxiter above the tolerance */
  NAIR_ERR_BREAKDOWN = 4,      /* non-finite value inside the Krylov iteration */
  NAIR_ERR_OOM = 5,            /* device allocation failed */
  NAIR_ERR_CUDA = 6,           /* any other CUDA runtime error */
  NAIR_ERR_UNSUPPORTED = 7     /* shape outside what the kernels handle */
} nair_status;

typedef enum { NAIR_FP64 = 0, NAIR_MIXED = 1 } nair_precision;

/* How nair_adjoint_solve preconditions A^T.
 *   NAIR_ADJOINT_TRANSPOSED: the transpose of the forward V-cycle, from the
 *     forward hierarchy (R^T interpolates, P^T restricts, C then F block-Jacobi
 *     sweeps on A^T before the coarse-grid correction; Sec. 2, Corollary on
 *     ideal interpolation, and the Remark on pre-F-relaxation).  The first
 *     call only transposes the stored level operators.
 *   NAIR_ADJOINT_REBUILD: a second nAIR hierarchy built for A^T with the same
 *     parameters (its levels are exported with adjoint = 1). */
typedef enum { NAIR_ADJOINT_TRANSPOSED = 0, NAIR_ADJOINT_REBUILD = 1 } nair_adjoint_mode;

/* Cycle of the forward preconditioner (Sec. 5; the F-cycle of the scaling
 * study of Sec. 6).  Both have no pre-relaxation and the same post-relaxation.
 *   NAIR_CYCLE_V: the coarse problem gets one V-cycle from zero.
 *   NAIR_CYCLE_F: the coarse problem gets one F-cycle from zero, then one
 *     V-cycle from that result (which restricts the coarse residual). */
typedef enum { NAIR_CYCLE_V = 0, NAIR_CYCLE_F = 1 } nair_cycle;

/* A block-CSR matrix in device memory (caller-owned, read-only during a call). */
typedef struct {
  int32_t nb_rows;        /* number of block rows = number of elements E */
  int32_t block_size;     /* b, 1..32 */
  int64_t nnzb;           /* number of stored blocks */
  const int32_t *row_ptr; /* device, nb_rows + 1 entries, row_ptr[0] = 0 */
  const int32_t *col_idx; /* device, nnzb block-column indices */
  const double *vals;     /* device, nnzb * b * b doubles */
} nair_bsr;

/* Method parameters (Sec. 5).  nair_default_params fills the defaults given here. */
typedef struct {
  double strength_theta;  /* 0.1: j in S_i iff ||A_ij||_F >= theta max_{k!=i} ||A_ik||_F (Sec. 4.3) */
  double filter_tol;      /* 1e-4: drop X_ij when ||X_ij||_F <= tol ||X_ii||_F (Sec. 5.2) */
  int32_t filter_targets; /* bit 0: filter each Neumann iterate; bit 1: filter coarse operators; 3 */
  int32_t neumann_degree; /* k of Delta^(k) (Eq. neumann); 1 */
  int32_t f_sweeps;       /* F-Jacobi sweeps; <= 0 means k + 1 (Sec. 5.1) */
  int32_t c_sweeps;       /* C-Jacobi sweeps after the F sweeps; 1 */
  int32_t max_levels;     /* 25 */
  int32_t max_coarse;     /* coarsest level when E <= max_coarse; <= 0 means max(2, 192 / b) */
  int32_t max_dense;      /* largest coarsest-level size E*b accepted for the dense solve; 4096 */
  uint64_t cf_seed;       /* seed of the C/F tie-break hash; 0 */
  int32_t precision;      /* nair_precision; NAIR_FP64 */
  int32_t gmres_restart;  /* 50 */
  int32_t maxiter;        /* total preconditioner applications allowed; 500 */
  double tol;             /* relative residual target ||b - A x|| / ||b||; 1e-10 */
  void *stream;           /* cudaStream_t for all work; NULL */
  int32_t keep_setup_data;/* keep strength, L and Delta for nair_get_level; 0 */
  int32_t use_graphs;     /* replay the V-cycle as a CUDA graph; 1 */
  int32_t sweep_timing;   /* stamp every block-Jacobi sweep with the device clock; 0 */
  int32_t adjoint_mode;   /* nair_adjoint_mode; NAIR_ADJOINT_TRANSPOSED */
  int32_t cycle_type;     /* nair_cycle of nair_solve and nair_vcycle; NAIR_CYCLE_V.  The
                             transposed adjoint always uses the transposed V-cycle. */
  int32_t scalar;         /* 0: block nAIR (element blocks on every level); 1: scalar nAIR
                             (Sec. 5.2, the paper's default): the hierarchy is built, degree of
                             freedom by degree of freedom, for D^{-1} A (D the block diagonal,
                             D_ii^{-1} A_ii set to I, zeros not stored) and the preconditioner is
                             the cycle applied to D^{-1} v; GMRES still solves A x = b.  The
                             exported levels then have block size 1.  0 */
} nair_params;

/* Solve report.  history is an optional host buffer owned by the caller. */
typedef struct {
  int32_t iterations;      /* preconditioner applications */
  int32_t levels;          /* hierarchy levels */
  double rel_res;          /* true residual ||b - A x|| / ||b|| at exit (FP64) */
  double setup_ms;         /* last setup time (device events) */
  double solve_ms;         /* this solve (device events) */
  double op_complexity;    /* sum of stored scalars over levels / level 0 (Sec. 6) */
  double cycle_complexity; /* work units per V-cycle, one WU = one SpMV with A (Sec. 6) */
  double *history;         /* host, history_cap doubles: [0] initial, then one per iteration */
  int32_t history_cap;
  int32_t history_len;
} nair_info;

typedef struct nair_handle nair_handle;

/* Fill p with the defaults listed in nair_params. */
void nair_default_params(nair_params *p);

/* Build the nAIR hierarchy of A (Sec. 5): diagonal-block inverses, strength,
 * C/F splitting, truncated Neumann Delta (Eq. neumann), R = [-A_cf Delta  I],
 * one-point P and the filtered coarse operator K = R A P (Eq. rap), level by
 * level, then the inverse of the coarsest operator.  A is validated (row
 * pointers, sorted columns, diagonal blocks) and copied; *out receives a new
 * handle that owns all hierarchy memory until nair_free.  Synchronises the
 * stream.  Errors: INVALID_ARG, SINGULAR_BLOCK, OOM, CUDA, UNSUPPORTED. */
nair_status nair_setup(const nair_bsr *A, const nair_params *p, nair_handle **out);

/* Solve A x = b with FGMRES(m) preconditioned by one V-cycle (no
 * pre-relaxation, F-F-...-C post-relaxation, Sec. 5).  b, x: device, n = E*b
 * doubles; x holds the initial guess on entry and the solution on return.
 * info may be NULL.  Returns NOT_CONVERGED if the tolerance was not met
 * within maxiter (x then holds the last iterate). */
nair_status nair_solve(nair_handle *h, const double *b, double *x, nair_info *info);

/* Solve A^T lambda = w (the adjoint of nair_solve) with FGMRES on A^T.  The
 * preconditioner follows adjoint_mode: the transposed V-cycle of the forward
 * hierarchy (the first call forms A_l^T, R_cf^T, the P^T lists and the
 * transposed diagonal and coarsest inverses, on the device), or a second
 * hierarchy built for A^T on the first call.  Later calls reuse what the
 * first built.  info->setup_ms reports that build.  w, lambda: device, n
 * doubles; lambda holds the initial guess on entry.  Errors as nair_solve. */
nair_status nair_adjoint_solve(nair_handle *h, const double *w, double *lambda, nair_info *info);

/* Apply one cycle (cycle_type) to f with zero initial guess: x = M^{-1} f
 * (device, n doubles). */
nair_status nair_vcycle(nair_handle *h, const double *f, double *x);

/* Apply the transposed cycle of the forward hierarchy to f with zero initial
 * guess: x = M^{-T} f, the preconditioner of NAIR_ADJOINT_TRANSPOSED (device,
 * n doubles).  Forms the transposed operators on first use, whatever
 * adjoint_mode says.  Synchronises the stream. */
nair_status nair_adjoint_vcycle(nair_handle *h, const double *f, double *x);

/* Release every device allocation of the handle (NULL is ignored). */
void nair_free(nair_handle *h);

/* Batches of independent systems (for example the directions of a discrete-
 * ordinates sweep, one A_k per direction).  Each system's work is issued by
 * its own host thread on the stream of its own parameters, so give every
 * system a distinct stream: the launch- and latency-bound parts of the systems
 * (coarse levels, setup, Krylov read-backs) then overlap on the GPU.  count
 * lies in 1..256.  Each call returns once every system is done; the status is
 * NAIR_OK if all succeeded, else the first failing system's status (by index)
 * with a message naming it.  Results are identical to separate calls.
 * Profiling (nair_profile) must be off during batch calls. */

/* Set up count systems: A[k] with parameters p[k]; out[k] receives the handles.
 * On failure every handle of the batch is freed and out[] is all NULL. */
nair_status nair_setup_batch(const nair_bsr *A, const nair_params *p, int32_t count, nair_handle **out);

/* nair_solve(h[k], b[k], x[k], info + k) for every k (distinct handles); info may be NULL. */
nair_status nair_solve_batch(nair_handle *const *h, int32_t count, const double *const *b, double *const *x,
                             nair_info *info);

/* nair_adjoint_solve(h[k], w[k], lambda[k], info + k) for every k (distinct handles). */
nair_status nair_adjoint_solve_batch(nair_handle *const *h, int32_t count, const double *const *w,
                                     double *const *lambda, nair_info *info);

/* Number of levels of the hierarchy: the forward hierarchy when adjoint == 0,
 * the A^T hierarchy of NAIR_ADJOINT_REBUILD when adjoint == 1 (INVALID_ARG
 * before the first adjoint solve or in NAIR_ADJOINT_TRANSPOSED mode). */
nair_status nair_num_levels(const nair_handle *h, int32_t adjoint, int32_t *levels);

/* Relaxation form of each level (a diagnostic for checks and measurement):
 * forms[l] for l < min(cap, levels) of the forward hierarchy's cycle
 * (transposed == 0) or of its transposed cycle (transposed == 1, available
 * after the first adjoint solve in NAIR_ADJOINT_TRANSPOSED mode; INVALID_ARG
 * before).  Values: -1 the coarsest level (direct solve), 0 block-row kernel,
 * 1 level-0 column-compressed coupling blocks, 2 packed scalar rows, 3 packed
 * scalar rows with the F sweeps iterating on y_F = D_FF x_F (transposed:
 * D_FF^T x_F), which apply D^{-1} once per cycle instead of once per sweep.
 * `levels` is nair_num_levels(h, 0); forms must hold cap int32 values. */
nair_status nair_sweep_forms(const nair_handle *h, int32_t transposed, int32_t cap, int32_t *forms);

/* Sizes of one level, 10 int64 values:
 *   E, nnzb(A), nC, nF, nnzb(L), nnzb(Delta), nnzb(R_cf), nnzb(AP), coarsest flag, setup rounds of C/F. */
nair_status nair_level_sizes(const nair_handle *h, int32_t adjoint, int32_t level, int64_t *sizes);

/* Copy one array of a level to host memory.  `which` is a nair_level_array;
 * integer arrays are int32 (CF: int8), value arrays are returned as doubles in
 * block row-major order whatever the storage precision.  *need receives the
 * byte size; nothing is copied when cap < *need (returns INVALID_ARG).  L,
 * Delta and the strength flags exist only when keep_setup_data was set. */
typedef enum {
  NAIR_A_ROWPTR = 0, NAIR_A_COL = 1, NAIR_A_VALS = 2, NAIR_DINV = 3, NAIR_CF = 4,
  NAIR_P_MAP = 5, /* per element: coarse index it interpolates from (C: itself), -1 if none */
  NAIR_DELTA_ROWPTR = 6, NAIR_DELTA_COL = 7, NAIR_DELTA_VALS = 8,
  NAIR_R_ROWPTR = 9, NAIR_R_COL = 10, /* R_cf columns as F indices (position among F elements) */
  NAIR_R_VALS = 11, NAIR_STRONG = 12, /* uint8 per block of A */
  NAIR_LAMBDA = 13, NAIR_L_ROWPTR = 14, NAIR_L_COL = 15, NAIR_L_VALS = 16
} nair_level_array;
nair_status nair_get_level(const nair_handle *h, int32_t adjoint, int32_t level, int32_t which,
                           void *host_out, size_t cap, size_t *need);

/* Batched inverses of nblk b x b blocks (step a1 alone, Sec. 5.2 block
 * scaling): in-place Gauss-Jordan with partial pivoting in FP64.  A, Ainv:
 * device, nblk*b*b doubles.  Returns SINGULAR_BLOCK if any pivot is zero. */
nair_status nair_block_inverse(int32_t nblk, int32_t b, const double *A, double *Ainv, void *stream);

/* Same batched inverses as nair_block_inverse, for callers that cannot allocate
 * device memory (a caching allocator that owns the device, applications that
 * forbid cudaMalloc after start-up, code that must not synchronise the device
 * the way cudaMalloc/cudaFree can).  The paper has no counterpart: this is a
 * deployment variant.  The entry point allocates nothing; its status words live
 * in a 32 KB array in the library's device code, which CUDA sets up on a GPU
 * when it loads that code there (under lazy module loading, the default, at the
 * library's first kernel call on that GPU; with CUDA_MODULE_LOADING=EAGER at
 * start-up) and keeps until the process exits: make one warm-up call before a
 * caching allocator takes the whole device.  One call handles at most 8192 thread
 * blocks of max(1, 256 / b) matrix blocks each (for example 344064 blocks of
 * size 6, 73728 of size 28); larger calls return INVALID_ARG and launch
 * nothing.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, so make that first call
 * before any stream capture.  All calls share the array: calls whose work
 * overlaps on the GPU (other streams, other host threads) race on it, so order
 * them on one stream.  The call synchronises the stream to read the status.
 * Returns SINGULAR_BLOCK, naming the range of blocks, if a pivot is zero. */
nair_status nair_block_inverse_noalloc(int32_t nblk, int32_t b, const double *A, double *Ainv,
                                       void *stream);

/* Parameter-dependent assembly for the transport problem (Eq. transport):
 * vals = vals0 with diagonal blocks vals0[diag_pos[e]] + sigma[e] * M[e]
 * (sigma_t piecewise constant per element, M the element mass matrices).
 * vals0, vals: device nnzb*b*b; diag_pos: device E; M: device E*b*b; sigma: device E. */
nair_status nair_assemble_sigma(int32_t E, int32_t b, int64_t nnzb, const int32_t *diag_pos,
                                const double *vals0, const double *M, const double *sigma,
                                double *vals, void *stream);

/* rhs_e = M_e q_e for every element (device, E*b doubles each). */
nair_status nair_mass_apply(int32_t E, int32_t b, const double *M, const double *q, double *rhs,
                            void *stream);

/* Gradients of J = w . x for A(sigma) x = M q given the adjoint solution
 * lambda = A^{-T} w: gsigma_e = -lambda_e^T M_e x_e (device, E doubles) and
 * gq_e = M_e^T lambda_e (device, E*b doubles). */
nair_status nair_gradients(int32_t E, int32_t b, const double *M, const double *lambda,
                           const double *x, double *gsigma, double *gq, void *stream);

/* Total number of kernels this library has launched in the process so far
 * (a diagnostic counter; every launch site increments it). */
nair_status nair_kernel_launches(int64_t *count);

/* Measured FP64 throughput of the current GPU, in TFLOP/s (two flops per fused
 * multiply-add), written to *tflops.  A diagnostic with no counterpart in the
 * paper: the denominator of the roofline of the FP64-bound kernels.  It
 * launches eight 256-thread blocks per SM on `stream` and reports the best of
 * three timed launches after one warm-up (CUDA events).  mode 0: each thread
 * runs sixteen independent fma chains of `iters` steps (1..1000000); mode 1:
 * each warp runs four independent chains of FP64 tensor-core products
 * (mma.sync m8n8k4); mode 2: both in one loop.  *sm_mhz (may be NULL)
 * receives the SM clock during that launch, from one block's clock64() cycles
 * over its %globaltimer nanoseconds.  Synchronises the stream. */
nair_status nair_fp64_peak(int32_t mode, int32_t iters, double *tflops, double *sm_mhz, void *stream);

/* Device time of the block-Jacobi sweeps of the forward hierarchy, recorded
 * when the handle was set up with sweep_timing = 1: for level `level` and class
 * `cls` (0 = F sweeps, 1 = C sweeps), the number of sweeps run so far and their
 * summed duration in ms, each sweep timed from its first thread block passing
 * the dependency wait to its last thread block finishing (%globaltimer).  The
 * stamps ride inside the kernels, so the CUDA graph and the overlap of
 * consecutive launches are kept.  cls = 2 + k selects sweep k of the cycle
 * alone (k = 0 .. f_sweeps + c_sweeps - 1; the F sweeps come first).  A sweep
 * with no rows to update or copy is not launched and not counted.
 * INVALID_ARG for a level or cls out of range. */
nair_status nair_sweep_timing(const nair_handle *h, int32_t level, int32_t cls, int64_t *sweeps,
                              double *total_ms);

/* Per-kernel timing (diagnostic).  nair_profile(1) clears the counters and
 * starts recording a CUDA event pair around each timed launch site (the
 * V-cycle then runs launch by launch instead of as a graph); nair_profile(0)
 * stops.  nair_profile_entry reads entry idx = 0, 1, ... : its name (copied
 * into name, at most cap bytes with the terminating 0), the number of timed
 * scopes and their total device time in ms; INVALID_ARG past the last entry.
 * Reading entry 0 waits for the recorded events. */
nair_status nair_profile(int32_t enable);
nair_status nair_profile_entry(int32_t idx, char *name, size_t cap, int64_t *launches, double *total_ms);

/* Message describing the last failure on the calling thread ("" if none). */
const char *nair_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NAIR_H */
