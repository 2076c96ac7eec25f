/*
 * pbicgstab.h -- C ABI of libpbicgstab, a GB300 (sm_103a) implementation of the
 * preconditioned pipelined BiCGStab method (p-BiCGStab) analysed in
 * S. Cools, "Analyzing and improving maximal attainable accuracy in the
 * communication hiding pipelined BiCGStab method", arXiv 1809.01948.
 *
 * Problem statement (Section 1): solve A x = b for a sparse, non-singular
 * N x N matrix A, given b and an initial guess x0, with a preconditioner
 * M^{-1} (the four inputs of Algorithm 2), a tolerance on the
 * recursively computed residual norm (Section 3.5) and a residual replacement
 * policy (Section 3.6, Eq. rr).
 *
 * Conventions for every entry point:
 *  - Every function returns a pbcg_status; PBCG_OK (0) on success.
 *  - The library never aborts and never prints.  On failure the thread-local
 *    message pbicgstab_last_error() describes the cause.
 *  - "device" pointers are CUDA global-memory pointers of the current device;
 *    "host" pointers are ordinary CPU memory.  Streams are cudaStream_t passed
 *    as void* (NULL = the legacy default stream).
 *  - Sizes: 1 <= n <= PBCG_MAX_ROWS = 2^30 rows per system, nnz < 2^31 - 1 stored
 *    entries (int32 indices).  The row limit keeps every 32-bit row index the kernels
 *    form (a row plus the grid's thread count, a row plus a diagonal offset) in range.
 *  - A context is bound to the stream given at creation; contexts are not
 *    thread-safe.  Work is stream-ordered; a call blocks the host only when it
 *    returns results in host memory (pbcg_result, host vectors).
 */
#ifndef PBICGSTAB_H
#define PBICGSTAB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PBCG_MAX_ROWS 1073741824

typedef enum pbcg_status {
  PBCG_OK = 0,             /* converged: ||r_i|| <= tol ||b|| and the true residual too   */
  PBCG_INVALID_ARG = 1,    /* bad pointer, size, matrix structure or option; nothing ran  */
  PBCG_CUDA_ERROR = 2,     /* a CUDA call failed; see pbicgstab_last_error()             */
  PBCG_OUT_OF_MEMORY = 3,  /* device allocation failed                                   */
  PBCG_NOT_CONVERGED = 4,  /* max_it iterations done without meeting the tolerance       */
  PBCG_BREAKDOWN = 5,      /* a zero or non-finite alpha denominator, omega, (r0,r_i)    */
  PBCG_STAGNATED = 6,      /* recursive residual met tol, true residual did not, no replacement
                              or restart policy; or no progress (options.stag_window)     */
  PBCG_TIMEOUT = 7         /* a grid-wide wait inside a kernel exceeded timeout_ms       */
} pbcg_status;

typedef enum pbcg_format { PBCG_FMT_CSR = 0, PBCG_FMT_DIA = 1 } pbcg_format;
typedef enum pbcg_dtype { PBCG_F64 = 0, PBCG_F32 = 1 } pbcg_dtype;
typedef enum pbcg_precond_kind {
  PBCG_PREC_NONE = 0,      /* M^{-1} = I (the paper's timing runs, Section 4.1)          */
  PBCG_PREC_JACOBI = 1,    /* M^{-1} = D^{-1}, D = diag(A).  When every diagonal entry is
                              the same d (detected at create) and the automated policy is
                              off, the preconditioned vectors are kept multiplied by d and
                              1/d enters only the x update and the replacement's s = A g:
                              the same iteration in exact arithmetic, fewer FP64 products */
  PBCG_PREC_NEUMANN = 2    /* M^{-1} = sum_{j=0..d} (I - D^{-1}A)^j D^{-1}, degree d >= 1 */
} pbcg_precond_kind;
typedef enum pbcg_precision {
  PBCG_FP64 = 0,           /* every vector, value and operation in FP64                  */
  PBCG_MIXED = 1           /* FP32 values, SpMV, preconditioner and recurrences; FP64 x,
                              b, dot-product results, alpha/beta/omega and replacement
                              residual r = b - A x (FP64 values)                          */
} pbcg_precision;
typedef enum pbcg_storage {
  PBCG_STORAGE_AUTO = 0,    /* option: keep a constant-coefficient stencil as one value per
                               offset plus a 16-bit presence mask per row (see
                               pbicgstab_operator_storage), other matrices as given      */
  PBCG_STORAGE_GENERAL = 1, /* option and query: the CSR / DIA values as given          */
  PBCG_STORAGE_STENCIL = 2  /* query only: the context uses the stencil form             */
} pbcg_storage;
typedef enum pbcg_method {
  PBCG_PIPELINED = 0,      /* Algorithm 2 (p-BiCGStab), two grid-wide reduction phases per
                              iteration, with the replacement policies of the options    */
  PBCG_CLASSIC = 1         /* Algorithm 1 (BiCGStab), the paper's reference method: three
                              reduction phases per iteration (Alg. 1's three GLREDs),
                              stop rule as for Algorithm 2 without replacement          */
} pbcg_method;

/* Sparse matrix description.  All arrays are read once by pbicgstab_create,
 * which keeps its own copies; the caller may free them afterwards.
 *  CSR: row_ptr[n+1], col[nnz] (int32, device), val[nnz] (device, val_dtype).
 *       Column indices within a row must be strictly increasing.
 *  DIA: ndiag (1..16) diagonals, offsets[ndiag] (HOST, strictly increasing,
 *       containing 0), val[ndiag*n] (device, val_dtype) with
 *       val[d*n + i] = A[i, i + offsets[d]] (entries outside 0..n-1 ignored). */
typedef struct pbcg_matrix {
  int32_t format;          /* pbcg_format */
  int32_t val_dtype;       /* pbcg_dtype  */
  int64_t n;
  int64_t nnz;             /* CSR only */
  const int32_t* row_ptr;  /* CSR only, device */
  const int32_t* col;      /* CSR only, device */
  const void* val;         /* device */
  int32_t ndiag;           /* DIA only */
  int32_t reserved0;
  const int32_t* offsets;  /* DIA only, host */
} pbcg_matrix;

typedef struct pbcg_precond {
  int32_t kind;            /* pbcg_precond_kind */
  int32_t degree;          /* Neumann degree d (1..8); ignored otherwise */
} pbcg_precond;

/* Number of doubles per iteration in the optional scalar history:
 * [alpha_i, omega_i, beta_{i+1} (NaN on the last iteration), ||r_{i+1}|| / ||b||,
 *  1.0 if a replacement (Eq. rr) happened in iteration i else 0.0, reserved...] */
#define PBCG_HIST_STRIDE 8

typedef struct pbcg_options {
  int32_t precision;       /* pbcg_precision */
  int32_t max_it;          /* >= 0.  The solve returns INVALID_ARG when
                              (max_it + 1)(8 + 4d) + (4 + 2d)(max_restarts + 1), times the
                              blocks that share a barrier, reaches 2^31 (d = Neumann
                              degree; the grid barrier's 32-bit arrival count must not
                              wrap): about 1.77M iterations for a 152-block launch
                              without Neumann, 294k for 456 blocks with d = 2 */
  double tol;              /* stop when ||r_i|| <= tol ||b|| (recursive, then verified) */
  int32_t rr_period;       /* periodic replacement every P iterations while
                              ||r_i|| >= sqrt(2^-52) ||r_0|| (Section 3.6); 0 = off    */
  int32_t rr_auto;         /* 1: automated replacement, Eq. (criterion): replace when the
                              run-time gap bound f^r of Eq. (DDr_bound) crosses
                              rr_tau * ||r_i||; needs no or Jacobi preconditioning */
  double rr_theta;         /* relative trigger: replace when ||r_i|| <= theta * (residual
                              norm after the previous replacement); 0 = off            */
  double timeout_ms;       /* limit of every grid-wide wait in the kernels; <= 0: 2000 */
  int32_t record_iterates; /* K >= 0: write x_{i+1} to hist_x[i*n .. ] for i < K      */
  int32_t hist_len;        /* capacity of hist_scalars, in iterations (0 = none)      */
  double* hist_x;          /* device, K*n doubles, or NULL when K == 0                */
  double* hist_scalars;    /* device, hist_len*PBCG_HIST_STRIDE doubles, or NULL      */
  int32_t grid_blocks;     /* persistent grid size; 0 = automatic                     */
  int32_t block_threads;   /* threads per block, a multiple of 32 up to 1024, or up to
                              512 for a mixed solve whose working set exceeds L2
                              (INVALID_ARG above); 0 = that maximum.  A system in stencil
                              storage whose row count is a multiple of 4, solved with
                              16-byte aligned b and x (and hist_x) by Algorithm 2 without
                              rr_auto, runs kernels that take four rows per thread in the
                              hot passes when block_threads is 0 or at most their block
                              size: 512, or 768 for a mixed solve whose working set
                              exceeds L2 (0 selects that size)                           */
  int32_t max_restarts;    /* after a breakdown (zero or non-finite omega, (r0,r_i),
                              beta or alpha denominator) restart Algorithm 2 from the
                              current iterate with a new shadow vector, at most this many
                              times (0, the default, = the paper's algorithm: report
                              PBCG_BREAKDOWN)                                          */
  int32_t method;          /* pbcg_method: PBCG_PIPELINED (default, Algorithm 2) or
                              PBCG_CLASSIC (Algorithm 1: FP64 only, no or Jacobi
                              preconditioning, no replacement, no restarts)             */
  double rr_tau;           /* tau of Eq. (criterion); <= 0: sqrt(2^-52)               */
  int32_t operator_storage;/* pbcg_storage: PBCG_STORAGE_AUTO (default) or _GENERAL; fixed
                              at create                                                 */
  int32_t cluster_blocks;  /* batched solver only: thread blocks per system, 1 (one block),
                              2, 4 or 8 (a thread-block cluster); 0 = autotune          */
  int32_t lanes_per_row;   /* batched solver only: threads per matrix row in the SpMVs of
                              the two passes, 1, 2, 4 or 8; 0 = autotune                 */
  int32_t batch_build;     /* batched solver only: 0 = autotune over both builds (a
                              caller-fixed shape runs the 64-register one), 1 = the
                              64-register kernels, 2 = the streaming cluster kernel (40
                              registers, up to six 256-thread or three 512-thread blocks
                              per SM; mixed precision, cluster_blocks 0, 2, 4 or 8,
                              block_threads 0 or <= 512); other values: INVALID_ARG     */
  int32_t restart_period;  /* > 0: restart Algorithm 2 from the current iterate after every P
                              iterations since the last (re)start -- r = b - A x in FP64, the
                              new r as shadow vector, beta = 0 (not in the paper: an FP64
                              outer correction that bounds how long the rounding errors of
                              the auxiliary recurrences can grow, for mixed precision); a
                              failed verification of the stop test then restarts instead of
                              returning STAGNATED.  0 = off                              */
  int32_t stag_window;     /* > 0: return PBCG_STAGNATED when the FP64 true residual, taken
                              at every (re)start, has not halved for this many iterations;
                              x is then the (re)start iterate with the smallest true
                              residual (also at NOT_CONVERGED when it beats the last
                              iterate).  Single-system solves keep that iterate; multi-RHS
                              and batched solves return the last one.  0 = off           */
  double rr_cutoff;        /* periodic replacement stops once ||r_i|| < rr_cutoff ||r_0||
                              (Section 3.6); <= 0: sqrt(2^-52)                          */
  int32_t prefetch_trips;  /* single-system solver: how many grid-wide row sweeps ahead each
                              thread asks L2 for its operands (prefetch.global.L2, which
                              holds no registers); 0 = automatic (1 for the one-row kernels
                              of a stencil system whose working set exceeds L2, else off),
                              < 0 = off, at most 16                                      */
  int32_t barrier_overlap; /* single-system solver: 0 = automatic (on where it applies), < 0
                              = off.  Each block arrives at the grid barrier that ends a
                              reduction phase, computes the next SPMV for the rows of its
                              chunk whose operands are all its own rows, then waits: the
                              on-chip form of overlapping a global reduction with the SPMV
                              (Section 1).  Applies with the chunked row order (matrix
                              bandwidth below half a chunk), no or Jacobi preconditioning,
                              Algorithm 2 without rr_auto                               */
  int32_t staged_sweeps;   /* single-system mixed solve with the four-row kernels and a
                              Neumann preconditioner on stencil storage: the Jacobi sweeps
                              of the preconditioner read their operands from shared-memory
                              stages that bulk copies (TMA) fill a trip ahead, instead of
                              from registers (same products in the same order).  0 =
                              automatic (on when a sweep's operands, 14 bytes per row,
                              exceed L2), > 0 = on, < 0 = off.  Ignored where it does not
                              apply (block_threads a multiple of 32; offsets beyond 8 x
                              block_threads rows multiples of 4; two stages must fit the
                              block's shared memory)                                    */
} pbcg_options;

typedef struct pbcg_result {
  int32_t status;          /* pbcg_status of the solve */
  int32_t iterations;      /* completed iterations of Algorithm 2 (or 1) */
  int32_t n_replacements;  /* executed Eq. (rr) steps (periodic, relative and forced) */
  int32_t n_restarts;      /* restarts after breakdowns (options.max_restarts) */
  double rel_res_recursive;/* ||r_last|| / ||b|| (recursively computed residual) */
  double rel_res_true;     /* ||b - A x|| / ||b||, FP64 */
  double time_ms;          /* device time of the persistent solver kernel (CUDA events
                              recorded on the context's stream around its launch) */
} pbcg_result;

typedef struct pbcg_ctx pbcg_ctx;

/* Fill *opt with defaults: FP64, max_it 10000, tol 1e-10, no replacement, no
 * restarts, no stagnation window, replacement cutoff sqrt(2^-52), timeout 2000 ms, no
 * history, automatic launch shape.  opt: host, non-NULL. */
pbcg_status pbicgstab_default_options(pbcg_options* opt);

/* Create a solver context for A and M^{-1} (Algorithm 2's inputs other than b,
 * x0).  Validates the matrix on the device (monotone row_ptr, columns in range
 * and increasing, finite values, non-zero diagonal when M needs it), copies and
 * converts it (FP32 copy in mixed mode, D^{-1}, the operator A D^{-1} used by the
 * hot loop) and allocates the workspace.  out, A, M, opt: host, non-NULL.
 * Errors: INVALID_ARG (bad arguments or matrix), OUT_OF_MEMORY, CUDA_ERROR. */
pbcg_status pbicgstab_create(pbcg_ctx** out, const pbcg_matrix* A, const pbcg_precond* M,
                             const pbcg_options* opt, void* stream);

/* Replace the solve options (tolerance, iteration limit, replacement policy,
 * history buffers, launch shape) of an existing context.  The precision and the
 * operator storage cannot change.  ctx, opt: host, non-NULL; opt is copied.
 * Errors: INVALID_ARG (NULL, an option out of range, a precision or storage
 * change, a method or policy the preconditioner does not allow); the context
 * keeps its previous options then. */
pbcg_status pbicgstab_set_options(pbcg_ctx* ctx, const pbcg_options* opt);

/* Solve A x = b with p-BiCGStab (Algorithm 2 with Eq. rr replacements per the
 * options), or with classic BiCGStab (Algorithm 1) when options.method is
 * PBCG_CLASSIC.  b: device, n doubles, read only.  x: device, n doubles, read as
 * x0 and overwritten with the last iterate (the solution on PBCG_OK).  res: host
 * or NULL; when non-NULL the call waits for the solve and fills it, otherwise it
 * only enqueues the work.  The caller keeps ownership of b and x and must keep
 * them alive until the stream has passed the solve.  The returned status is the
 * solve's status when res is given (OK, NOT_CONVERGED, BREAKDOWN, STAGNATED,
 * TIMEOUT), else PBCG_OK once the launch succeeded; INVALID_ARG for NULL
 * arguments or a launch shape the device cannot co-schedule, CUDA_ERROR when a
 * launch or copy fails. */
pbcg_status pbicgstab_solve(pbcg_ctx* ctx, const double* b, double* x, pbcg_result* res);

/* Same as pbicgstab_solve with b and x in HOST memory (pinned or pageable): the
 * host-to-device copy of b and x0, the solve and the device-to-host copy of x are
 * enqueued on the context's stream and waited for.  res: host, non-NULL.  The
 * device copies are stream-ordered allocations of this call, freed before it
 * returns on every path.  Errors: as pbicgstab_solve, plus OUT_OF_MEMORY /
 * CUDA_ERROR from the staging allocations and copies. */
pbcg_status pbicgstab_solve_host(pbcg_ctx* ctx, const double* b_host, double* x_host,
                                 pbcg_result* res);

/* Solve A X = B for nrhs right-hand sides with one matrix (Algorithm 2 + Eq. rr for
 * each column independently: its own alpha, beta, omega, replacements and stop).
 * B, X: device, column-major n x nrhs (column c at offset c*n); X is read as the
 * initial guesses and overwritten.  The grid is split into teams of blocks, one
 * team per right-hand side, each with its own barrier and reductions; more than
 * (co-resident blocks) right-hand sides run in waves.  res: host array of nrhs
 * results or NULL; time_ms of every entry is the total kernel time.  Waits.
 * The context keeps the multi-RHS workspace (15 n-vectors per team) until it is
 * destroyed.  Returns PBCG_OK when every column converged, else the first failing
 * status; INVALID_ARG for NULL arguments, nrhs < 1, options.rr_auto or
 * PBCG_CLASSIC; TIMEOUT when a team barrier gave up. */
pbcg_status pbicgstab_solve_multi(pbcg_ctx* ctx, int32_t nrhs, const double* B, double* X,
                                  pbcg_result* res);

/* Create a context for the transposed matrix A^T (CSR only) with the same
 * preconditioner kind and options: the adjoint solve A^T lambda = dL/dx of a
 * differentiable solve.  A^T is built on the device (column counts, scan,
 * scatter, and a per-row sort that makes it independent of atomic order).  *out
 * is a new, independent context (release it with pbicgstab_destroy); src is not
 * modified.  Errors: INVALID_ARG (NULL, or src not CSR), OUT_OF_MEMORY,
 * CUDA_ERROR, or any error of pbicgstab_create for A^T (e.g. a zero diagonal). */
pbcg_status pbicgstab_create_transpose(pbcg_ctx** out, const pbcg_ctx* src);

/* Replace the values of the context's matrix, keeping its sparsity pattern (CSR: the
 * row pointers and columns given at create; DIA: the offsets) and its options and
 * workspace: everything derived from the values is rebuilt (validation, FP64 and FP32
 * copies, D^{-1}, A D^{-1}, the stencil detection and the bound constants) -- what a
 * differentiable solve needs when only the values change between calls.  val: device,
 * nnz (CSR) or ndiag*n (DIA) values of val_dtype, read only.  Waits for the context's
 * stream first.  Errors: INVALID_ARG (NULL, bad dtype, an invalid matrix: the context then
 * refuses to solve until a later update succeeds), OUT_OF_MEMORY, CUDA_ERROR. */
pbcg_status pbicgstab_update_values(pbcg_ctx* ctx, const void* val, int32_t val_dtype);

/* Refresh a transposed context (made by pbicgstab_create_transpose from src) after src's
 * values changed (pbicgstab_update_values on src): A^T's values are gathered from src's
 * through the permutation kept at create_transpose.  Errors: INVALID_ARG (t not a
 * transpose context, or src's pattern differs), OUT_OF_MEMORY, CUDA_ERROR. */
pbcg_status pbicgstab_update_transpose(pbcg_ctx* t, const pbcg_ctx* src);

/* Gradient of a loss with respect to the stored CSR values of the context's
 * matrix, given the adjoint solutions Lam (A^T Lam = dL/dX) and the solutions X
 * (device, column-major n x nrhs):  grad[e] = - sum_c Lam[row_e, c] X[col_e, c]
 * for every stored entry e in CSR order (device, nnz doubles).  Stream-ordered.
 * Errors: INVALID_ARG (NULL, nrhs < 1, or a DIA context), CUDA_ERROR. */
pbcg_status pbicgstab_csr_value_grad(pbcg_ctx* ctx, int32_t nrhs, const double* Lam, const double* X,
                                     double* grad);

/* y = A x with the context's FP64 matrix (the SPMV of Algorithm 2; x, y: device,
 * n doubles, must not overlap).  Stream-ordered.  Errors: INVALID_ARG (NULL),
 * CUDA_ERROR. */
pbcg_status pbicgstab_spmv(pbcg_ctx* ctx, const double* x, double* y);

/* Work vectors of Algorithm 2 as the context's last single-system solve left them
 * (pbicgstab_solve / pbicgstab_solve_host), for checking the state after a step: after
 * an iteration i that ended with an Eq. (rr) replacement these are the replaced
 * r_{i+1}, k_{i+1}, w_{i+1} and s_i, l_i, z_i (Section 3.6), with g_i and the shadow
 * vector r0.  `which` selects one: */
typedef enum pbcg_vector {
  PBCG_VEC_R = 0, PBCG_VEC_RHAT = 1, PBCG_VEC_K = 2, PBCG_VEC_W = 3, PBCG_VEC_G = 4,
  PBCG_VEC_S = 5, PBCG_VEC_L = 6, PBCG_VEC_Z = 7
} pbcg_vector;
/* dst: device, n doubles (the stored vector widened to FP64; with the scaled-form
 * Jacobi of a constant diagonal, k, g and l are returned unscaled, i.e. as M^{-1} r,
 * M^{-1} p and M^{-1} s).  Stream-ordered.  Errors: INVALID_ARG (NULL, unknown
 * `which`), CUDA_ERROR. */
pbcg_status pbicgstab_get_vector(pbcg_ctx* ctx, int32_t which, double* dst);

/* The launch of the context's last single-system solve: info[0] grid blocks, info[1]
 * threads per block, info[2] rows per thread in the hot passes (1, or 4 for the four-row
 * kernels of the stencil storage), info[3] the L2 prefetch distance in row sweeps (0 =
 * off) plus 256 when the barriers overlap the interior SPMV rows (options.barrier_overlap)
 * plus 512 when the Neumann sweeps are staged in shared memory (options.staged_sweeps).
 * All zero before the first solve.  ctx, info: host, non-NULL.  Errors:
 * INVALID_ARG (NULL). */
pbcg_status pbicgstab_launch_info(const pbcg_ctx* ctx, int32_t info[4]);

/* *rel = ||b - A x|| / ||b|| in FP64, the true relative residual whose gap to the
 * recursive residual Section 3 analyses (b, x: device; rel: host).  Waits.
 * Errors: INVALID_ARG (NULL), CUDA_ERROR. */
pbcg_status pbicgstab_true_residual(pbcg_ctx* ctx, const double* b, const double* x, double* rel);

/* Release everything the context owns after waiting for its stream.  NULL is
 * accepted.  Always returns PBCG_OK. */
pbcg_status pbicgstab_destroy(pbcg_ctx* ctx);

/* Thread-local description of the last failure in this thread ("" if none). */
const char* pbicgstab_last_error(void);

/* ---------------------------------------------------------------------------
 * Batched solves: many independent systems A_k x_k = b_k of different sizes,
 * solved by one persistent kernel launch (replayed from a CUDA graph).  Each
 * system is solved by one thread block, or one thread-block cluster of 2, 4 or 8
 * blocks, running Algorithm 2 with Eq. (rr) replacements; blocks (clusters) take
 * systems from a device queue, largest first.
 *
 * Storage: the systems' CSR matrices are concatenated.  For system k (0-based):
 *   rows       row_off[k] .. row_off[k+1]-1 of the concatenated b and x,
 *   row_ptr    row_ptr[row_off[k] + k .. row_off[k+1] + k] (n_k + 1 entries,
 *              local: starting at 0),
 *   col / val  col[nnz_off[k] + e], val[nnz_off[k] + e] with LOCAL column
 *              indices 0 .. n_k-1.
 * row_off and nnz_off (n_sys + 1 int64 each) are HOST arrays; row_ptr, col, val
 * are device arrays.  Preconditioner (per system, Section 2 of the paper): NONE, JACOBI,
 * or NEUMANN of `degree` 1..8 (the Jacobi sweeps of the single-system solver). */
typedef struct pbcg_batch {
  int32_t n_sys;
  int32_t val_dtype;        /* pbcg_dtype */
  const int64_t* row_off;   /* host, n_sys + 1 */
  const int64_t* nnz_off;   /* host, n_sys + 1 */
  const int32_t* row_ptr;   /* device */
  const int32_t* col;       /* device */
  const void* val;          /* device */
  int32_t precond;          /* PBCG_PREC_NONE, PBCG_PREC_JACOBI or PBCG_PREC_NEUMANN */
  int32_t degree;           /* Neumann degree 1..8 (ignored for NONE and JACOBI) */
} pbcg_batch;

/* Per-system outputs, HOST arrays of n_sys entries (any may be NULL). */
typedef struct pbcg_batch_result {
  int32_t* status;
  int32_t* iterations;
  int32_t* n_replacements;
  double* rel_res_true;     /* ||b_k - A_k x_k|| / ||b_k||, FP64 */
  double time_ms;           /* device time of the batched solve kernel */
  int32_t n_ok;             /* systems with status PBCG_OK */
  int32_t block_threads;    /* launch shape used (autotuned when the options ask for 0) */
  int32_t grid_blocks;
  int32_t cluster_blocks;   /* blocks per system (1: one block, else a cluster) */
  int32_t lanes_per_row;    /* threads per row in the SpMVs */
  int32_t batch_build;      /* the kernel build that ran: 1 (64 registers) or 2 (streaming) */
} pbcg_batch_result;

typedef struct pbcg_batch_ctx pbcg_batch_ctx;

/* Validate and prepare a batch (copies of the matrices, D^{-1}, A D^{-1}, FP32
 * copies in mixed mode, workspace, queue order).  The library copies everything it
 * needs: the caller may free its arrays once the call returns.  opt: precision,
 * tol, max_it, replacement policy (periodic / relative; not rr_auto), method
 * PBCG_PIPELINED only, cluster_blocks, lanes_per_row, batch_build; grid_blocks /
 * block_threads = 0 request the autotuner (it times the candidate launch shapes on
 * the first solve and keeps the fastest).  History options are ignored.  Errors:
 * INVALID_ARG (NULL, n_sys < 1, a system of size 0 or above PBCG_MAX_ROWS, decreasing
 * offsets, an invalid matrix found by the device validation, an option out of
 * range), OUT_OF_MEMORY, CUDA_ERROR; *out is NULL then. */
pbcg_status pbicgstab_batch_create(pbcg_batch_ctx** out, const pbcg_batch* batch,
                                   const pbcg_options* opt, void* stream);

/* Solve all systems: b (device, sum n_k doubles), x (device, read as x0 and
 * overwritten).  res: host or NULL (NULL: enqueue only).  The launch is a CUDA
 * graph replay after the first call with the same b and x pointers.  Returns
 * PBCG_OK when every system converged, else the first failing status found
 * (per-system statuses in res->status); INVALID_ARG for NULL arguments or a
 * caller-fixed shape that does not fit, CUDA_ERROR when a launch fails. */
pbcg_status pbicgstab_batch_solve(pbcg_batch_ctx* ctx, const double* b, double* x,
                                  pbcg_batch_result* res);

/* Release everything the batch context owns (after waiting for its stream),
 * including its CUDA graph.  NULL is accepted.  Always returns PBCG_OK. */
pbcg_status pbicgstab_batch_destroy(pbcg_batch_ctx* ctx);

/* One-shot convenience: create, solve (waits when res is NULL too), destroy.
 * Errors: those of pbicgstab_batch_create and pbicgstab_batch_solve. */
pbcg_status pbicgstab_solve_batched(const pbcg_batch* batch, const pbcg_options* opt, void* stream,
                                    const double* b, double* x, pbcg_batch_result* res);

/* ---------------------------------------------------------------------------
 * Allocation-free solve.  The paper has no counterpart: this entry point exists
 * for callers that must not allocate GPU memory -- for example an application
 * whose own allocator has reserved the device memory up front (a cudaMalloc from
 * this library would then fail), or a latency-critical loop that cannot afford
 * the implicit device synchronisation of cudaMalloc/cudaFree.
 *
 * It runs the same persistent FP64 solver kernel as pbicgstab_solve (Algorithm 2
 * with the Eq. (rr) policies of *opt), but every scratch buffer (15 work vectors,
 * D^{-1}, the operator A D^{-1}, reduction partials, barrier and result state)
 * lives in one fixed array of device memory that the library declares
 * statically.  That array is reserved on every GPU that loads the library, for
 * as long as the process runs: 9,044,224 bytes (8.6 MiB).  The call allocates nothing (no
 * cudaMalloc, cudaFree or allocating library routine) and keeps no reference to
 * the caller's arrays after it returns.
 *
 * Limits: n <= PBCG_NOALLOC_MAX_N rows and at most PBCG_NOALLOC_MAX_VALUES stored
 * values (CSR nnz, or ndiag * n for DIA); FP64 values (val_dtype PBCG_F64) and
 * opt->precision == PBCG_FP64; preconditioner NONE or JACOBI.  Larger systems or
 * other settings return PBCG_INVALID_ARG with a message naming the limit.
 *
 * A: device CSR or DIA matrix (DIA offsets on the host), used in place.
 * b: device, read.  x: device, read as x0 and overwritten.  res: host, filled
 * (time_ms is -1: no events are created).  The call waits for the solve.
 *
 * Every call looks up the array's device address (cudaGetSymbolAddress, which
 * allocates nothing) in the current context; the call then validates A on the
 * device and waits for that result, and waits for the solve at the end, so it
 * synchronises `stream` twice.  With default options (block_threads and
 * grid_blocks 0) it uses the launch shape pbicgstab_solve chooses for a context that
 * keeps A as given (options.operator_storage PBCG_STORAGE_GENERAL).  All calls
 * on a device share the one array and it keeps the last call's contents (the
 * solver re-initialises what must start at zero): calls that overlap on the GPU --
 * from several host threads or streams at once -- race on it and must be
 * serialised by the caller. */
#define PBCG_NOALLOC_MAX_N 32768
#define PBCG_NOALLOC_MAX_VALUES 524288
pbcg_status pbicgstab_solve_noalloc(const pbcg_matrix* A, const pbcg_precond* M, const pbcg_options* opt,
                                    const double* b, double* x, pbcg_result* res, void* stream);

/* How the context stores A: PBCG_STORAGE_STENCIL when options.operator_storage was
 * PBCG_STORAGE_AUTO and A is a constant-coefficient stencil -- at most 16 distinct
 * offsets col - row among its non-zero entries, one value per offset and, with a
 * preconditioner, a constant diagonal -- else PBCG_STORAGE_GENERAL.  The stencil form
 * computes the same products in the same order (every SpMV sums in ascending column
 * order).  ctx, storage: host, non-NULL. */
pbcg_status pbicgstab_operator_storage(const pbcg_ctx* ctx, int32_t* storage);

/* Error propagation diagnostics (Section 2.4): column max-norms of the nine products
 * of Eq. (all_error_matrices), U, OU, BA, UEA, BAEA, BPA, UC, BAC, BD, formed from the
 * propagation matrices of Eq. (all_matrices) for the scalars of `iters` iterations of
 * Algorithm 2 (the curves the paper plots against the iteration index).
 *
 * hist: device, iters rows of `stride` doubles (stride >= 3); row i holds alpha_i at
 *   [0], omega_i at [1] and beta_{i+1} at [2] -- exactly the rows a solve writes to
 *   options.hist_scalars (stride PBCG_HIST_STRIDE).  May be NULL when iters == 0.
 * norms: device, 9 * (iters + 1) doubles, written: product p (in the order above) at
 *   norms[p * (iters + 1) + j] for column j = 0 .. iters.  Column j depends on rows
 *   0 .. j-1 only.  A non-finite scalar makes the columns it reaches NaN or Inf.
 * iters: 0 .. 65536 (the work is O(iters^2)).  stream: as elsewhere.  Enqueues only.
 * Errors: INVALID_ARG (NULL pointer, stride < 3, iters out of range), CUDA_ERROR. */
pbcg_status pbicgstab_propagation_norms(const double* hist, int32_t stride, int32_t iters, double* norms,
                                        void* stream);

/* Test hook for the fault-detection path: launches a cooperative grid whose
 * blocks wait at a barrier for `extra_arrivals` more blocks than exist, so the
 * wait can only end by its timeout.  Returns PBCG_OK when the kernel gave up
 * after about timeout_ms and reported PBCG_TIMEOUT in *kernel_status (host).
 * Nothing faults or hangs: every wait has an iteration limit. */
pbcg_status pbicgstab_test_barrier_timeout(double timeout_ms, int32_t extra_arrivals,
                                           int32_t* kernel_status);

#ifdef __cplusplus
}
#endif
#endif /* PBICGSTAB_H */
