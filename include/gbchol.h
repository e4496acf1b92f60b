/*
 * gbchol.h -- C ABI of the GB300 (sm_103a) blocked Cholesky / pivot-free LU
 * library.
 *
 * The method is that of Camarero, "Simple, Fast and Practicable Algorithms
 * for Cholesky, LU and QR Decomposition Using Fast Rectangular Matrix
 * Multiplication" (arXiv:1812.02056), Sec. 2:
 *
 *  - Algorithm 1 (Cholesky): columns are finished one at a time, each from
 *    the columns since the last checkpoint z; every s columns the trailing
 *    matrix receives the delayed rank-s update A[c.., c..] -= R R^T with
 *    R = L[c.., z..c-1], and z moves to c.
 *  - Algorithm 2 (LU, no pivoting, Crout form): the same schedule with
 *    A[c.., c..] -= R_L R_U, L lower triangular, U upper unitriangular.
 *
 * Conventions shared by every call
 *  - Matrices are row-major (the order PyTorch uses): element (i, j) of X is
 *    X[i * ldx + j]; every leading dimension must be >= the row length.
 *  - Pointers may be device memory (cudaMalloc / PyTorch CUDA tensors) or
 *    host memory, unless a call says otherwise.  The library detects which
 *    with cudaPointerGetAttributes; host buffers are staged through the
 *    handle's device workspace and the call then waits for its stream, so a
 *    call on host buffers returns with its outputs in place.  Calls on device
 *    buffers are asynchronous on `stream`.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).
 *  - The caller owns every buffer it passes; the library never frees caller
 *    memory.  The handle owns its workspace (grown on demand, released by
 *    gb_destroy).
 *  - `info` is an int that receives 0 on success or c > 0, the 1-based
 *    column at which the factorization broke down (Cholesky: the value under
 *    the square root was not positive or was NaN; LU: the pivot L_cc was
 *    zero or NaN).  It may be a device or a host pointer.  On breakdown the
 *    contents of the output past column c-1 are unspecified.
 *  - Return values report host-side problems only (see gb_status below).
 *    Nothing traps on the device: device-side errors are reported through
 *    `info` and the handle's error word.
 *
 * Thread safety and ordering: a handle may be used from one host thread at a
 * time, and its calls must be ordered on one stream (its workspace and
 * device flags are shared by all its calls).  Use one handle per stream for
 * concurrent work.
 */
#ifndef GBCHOL_H
#define GBCHOL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
typedef int gb_status;
#define GB_OK 0
/* -k (k = 1, 2, ...): the k-th argument of the call is invalid */
#define GB_ERR_NOMEM (-1001)         /* device or host allocation failed            */
#define GB_ERR_CUDA (-1002)          /* a CUDA runtime call failed                  */
#define GB_ERR_TIMEOUT (-1003)       /* a bounded device-side wait expired          */
#define GB_ERR_NOT_CONVERGED (-1004) /* refinement reached max_iter above tol      */
#define GB_ERR_REJECTED (-1005)      /* server: request larger than the budget      */
#define GB_ERR_UNSUPPORTED (-1006)   /* combination of options not implemented      */
#define GB_ERR_BREAKDOWN (-1007)     /* solve: the factor has a zero/NaN pivot      */
#define GB_ERR_STATE (-1008)         /* object used in the wrong state              */

/* Short English description of a status code (static storage). */
const char *gb_status_string(gb_status st);

/* ------------------------------------------------------------------ dtypes */
/*
 * Arithmetic of a factorization.
 *  GB_F64      A and L/U are double; every step in FP64.
 *  GB_F32      A and L/U are float;  every step in FP32.
 *  GB_MIX_BF16 A is double, L/U are float.  The working matrix is FP32;
 *              Cholesky's pivots (square root and its reciprocal) are the
 *              FP64 operations rounded to FP32, computed as the identical
 *              correctly rounded FP32 operations (double rounding is
 *              innocuous for sqrt and division from 53 to 24 bits); LU's
 *              diagonal blocks run in FP64; the panel rows in FP32; the
 *              delayed rank-s update runs on the tensor cores with BF16
 *              operands and FP32 accumulation.
 *  GB_MIX_F16  as GB_MIX_BF16 with FP16 operands.
 *  GB_MIX_BF16X3  as GB_MIX_BF16, but each operand of the update is split
 *              into three BF16 planes (x = p0 + p1 + p2, each the rounding of
 *              the remainder) and the six leading plane products are
 *              accumulated: the update is accurate to about FP32 at one
 *              sixth of the BF16 tensor rate.
 * Mixed factors are meant to be refined back to FP64 accuracy by
 * gb_chol_solve / gb_lu_solve given the original FP64 matrix.
 */
typedef enum gb_dtype {
  GB_F64 = 0,
  GB_F32 = 1,
  GB_MIX_BF16 = 2,
  GB_MIX_F16 = 3,
  GB_MIX_BF16X3 = 4
} gb_dtype;

/* ------------------------------------------------------------------ handle */
typedef struct gb_handle gb_handle;

/* Create a handle bound to CUDA device `device` (made current by every call
 * that takes the handle).  Returns GB_ERR_CUDA if the device is absent.
 * The handle owns its workspaces and a device memory pool for the copies of
 * host buffers; the pool keeps its memory between calls (a host-buffer call
 * at order n holds on to about its own n x n copies) until gb_destroy. */
gb_status gb_create(gb_handle **h, int device);

/* Wait for the handle's work, release its workspace and free it. */
gb_status gb_destroy(gb_handle *h);

/* Library version, major * 10000 + minor * 100 + patch. */
int gb_version(void);

/* Text of the last CUDA error recorded by this thread (static storage). */
const char *gb_last_error(void);

/* Options set on a handle (all have defaults). */
typedef enum gb_option {
  GB_OPT_INNER_STEP = 1,    /* width of the column steps inside one s-block
                               (default 64, range 1..64).  s <= this value is
                               Algorithm 1/2 exactly as written; larger s
                               factors each block of s columns with this
                               inner step (the paper's remark that s may vary
                               during the execution, Sec. 2, last paragraph). */
  GB_OPT_USE_GRAPHS = 2,    /* 1: replay a captured CUDA graph of the whole
                               block loop for repeated (n, s, dtype, ld)
                               calls on device buffers (default 1).          */
  GB_OPT_TC_UPDATE = 3,     /* mixed dtypes' update: 2 (default) the
                               tcgen05 tensor-core kernel on CTA pairs (two
                               SMs) computing 256 x 256 tiles with pair MMAs;
                               1 the same kernel with one CTA per 128 x 256
                               tile; 0 the SIMT FP32 update.  Other values:
                               error -3.                                     */
  GB_OPT_SPIN_LIMIT = 4,    /* limit of bounded device waits, in units of
                               100 ns of %globaltimer (default 2^26, ~6.7 s). */
  GB_OPT_PROFILE = 5,       /* 1: record CUDA events around every launch of
                               the factorizations (read with
                               gb_profile_read); default 0.                 */
  GB_OPT_BATCHED_EXACT = 6, /* 1: the batched kernel rounds every product and
                               every subtraction separately (no FMA), as the
                               FP64 oracle does; default 0.                  */
  GB_OPT_LOOKAHEAD = 7,     /* 1 (default): each delayed update first updates
                               the next s-block's columns, and the rest of it
                               runs on a second stream while the next block's
                               column steps proceed; 0: one stream.          */
  GB_OPT_STRASSEN = 8,      /* 1: the FP64/FP32 delayed updates use one level
                               of Strassen's multiplication (7 half-size
                               products; the paper's practical variant, Sec. 2
                               timing paragraph): LU's update, and the
                               off-diagonal block of Cholesky's square update
                               (its diagonal halves stay classical); also
                               gb_rank_update without the lower mask.
                               Default 0.                                    */
  GB_OPT_QR_INNER_STEP = 9, /* gb_qr_factor: columns per panel launch, each
                               orthogonalised against the earlier ones of its
                               inner block one at a time (default 16, range
                               1..256; capped by s and by the panel's shared
                               memory, 200 KiB per CTA for ceil(n/8) rows).  */
  GB_OPT_LEFT_LOOKING = 10, /* 1: gb_chol_factor with GB_MIX_BF16 / GB_MIX_F16
                               (tensor-core update on, s a multiple of 64,
                               s < n, n a multiple of 8) accumulates the
                               update of each s-block column from all earlier
                               columns in one tensor-core product (K = z, the
                               columns done) read from a resident 16-bit copy
                               of L, instead of updating the trailing matrix
                               every s columns: the same sums, grouped by
                               tile; FP32 traffic of the working matrix once
                               per block column.  Default 0.                 */
  GB_OPT_TEST_WITHHOLD = 11, /* failure-detection test hook, 0 (default) off:
                               v >= 1 makes block v - 1 (in sweep order) of
                               the forward triangular sweep of gb_chol_solve
                               and gb_lu_solve skip publishing its
                               completion, so the block after it waits until
                               GB_OPT_SPIN_LIMIT runs out, raises the timeout
                               word and returns; the call then reports
                               GB_ERR_TIMEOUT and clears the word.  Nothing
                               faults or hangs; the next call on the handle
                               starts from fresh sync words.                  */
  GB_OPT_INNER_CUDA_CORES = 12, /* 1: gb_chol_factor with a mixed dtype runs
                               the updates inside each s-block (K <= inner
                               step) in FP32 on the CUDA cores instead of the
                               tensor cores; the delayed rank-s updates stay
                               on the tensor cores.  Default 0.              */
  GB_OPT_INNER_RECURSIVE = 13, /* 1: inside each s-block of gb_chol_factor,
                               a column range wider than two inner steps is
                               split in halves (multiples of the inner step):
                               the left half is finished first, the right
                               half then receives the whole left half in one
                               product, then is finished the same way; 0: each
                               inner block updates all the s-block's remaining
                               columns.  The same sums, fewer and larger
                               products.  2 (default): 1 for GB_F64 and the
                               mixed dtypes, 0 for GB_F32.                   */
  GB_OPT_INNER_LOOKAHEAD = 14, /* 1: inside each s-block of gb_chol_factor,
                               each inner product goes first to the next
                               inner block's columns (on the stream of the
                               column steps) and to the rest of the range on
                               a third stream, alongside the next column
                               steps.  The same sums in the same order per
                               element.  0 off, 2 (default): 1 for GB_F64
                               only.                                         */
  GB_OPT_EARLY_REST = 15,     /* 1: with look-ahead, the rest of each s-block's
                               delayed update (the columns after the next
                               s-block) starts as soon as the s-block is
                               factored, alongside the update of the next
                               s-block's columns; 0: after that update.  The
                               same sums.  2 (default): 1 for GB_F64 only.   */
  GB_OPT_RESIDUAL = 16,       /* method of the FP64 residual r = B - A X of
                               refinement and gb_residual.  0: FP64
                               multiply-adds on the CUDA cores.  1: exact
                               digit products on the tensor cores: each row
                               of A and column of X is scaled by a power of
                               two and cut into 11 digits of 5 bits (BF16
                               planes; a truncation below 2^-55 of the row's
                               or column's largest magnitude), the 76 digit
                               pairs that matter are multiplied with exact
                               FP32 accumulation, and the pair sums are
                               combined in FP64; per term the error is below
                               one FP64 rounding of the row's largest
                               product.  Needs 22 n^2 bytes of workspace (the
                               digits of A, made once per solve call); 0 is
                               used when that cannot be had.  2 (default): 1
                               for n >= 2048, else 0.                        */
  GB_OPT_F64_UPDATE = 17      /* GB_F64 delayed and inner updates (C -= R R^T
                               of gb_chol_factor, C -= R_L R_U of
                               gb_lu_factor, and gb_rank_update).  0 (default):
                               FP64 multiply-adds on the CUDA cores.  1: FP64
                               accuracy from exact digit products on the
                               tensor cores: each row of R (column of R_U)
                               is scaled by a power of two and cut into 11
                               digits of 5 bits (BF16 planes), the 76 digit
                               pairs of the 12
                               scales that matter are multiplied with exact
                               FP32 accumulation (K taken in pieces of at
                               most 1024), the scales are combined exactly in
                               integers and the result is subtracted from C
                               in FP64.  Per term the error is below one FP64
                               rounding of the row scales' product; the
                               FP64 multiply-add update rounds at every
                               term.  Workspace 22 n s bytes per stream.     */
} gb_option;

gb_status gb_set_option(gb_handle *h, gb_option opt, int64_t value);
gb_status gb_get_option(gb_handle *h, gb_option opt, int64_t *value);

/* ---------------------------------------------------------------- Cholesky */
/*
 * gb_chol_factor -- Algorithm 1 (fast Cholesky with step s), arXiv:1812.02056
 * Sec. 2.
 *
 *  n     order of A (n >= 0).
 *  s     step: the delayed rank-s update is applied every s columns.  s >= 1;
 *        s >= n means no update (Cholesky-Crout); s = 1 is the recursive
 *        right-looking algorithm (Sec. 2, after Algorithm 3).  s = 0 picks
 *        the tuned step for (n, dt).
 *  dt    arithmetic, see gb_dtype.  A is double for GB_F64 and the mixed
 *        dtypes, float for GB_F32; L is double for GB_F64, float otherwise.
 *  A     n x n symmetric positive-definite matrix, leading dimension lda.
 *        Only the lower triangle (with the diagonal) is read.
 *  L     n x n output, leading dimension ldl.  Receives the lower-triangular
 *        factor with A = L L^T; its strict upper triangle is set to zero.
 *        L may alias A when both have the same element type (in place).
 *  info  see the conventions above.
 */
gb_status gb_chol_factor(gb_handle *h, int64_t n, int64_t s, gb_dtype dt, const void *A,
                         int64_t lda, void *L, int64_t ldl, int *info, void *stream);

/* ---------------------------------------------------------------------- LU */
/*
 * gb_lu_factor -- Algorithm 2 (fast LU with step s, no pivoting),
 * arXiv:1812.02056 Sec. 2.  A must have nonzero leading principal minors.
 *
 *  A     n x n, leading dimension lda, read in full.  Element types as for
 *        gb_chol_factor.
 *  LU    n x n output in compact form, leading dimension ldlu: the lower
 *        triangle with the diagonal holds L, the strict upper triangle holds
 *        the strict upper part of the unit upper triangular U (its diagonal
 *        of ones is implied, not stored).  LU may alias A when both have the
 *        same element type.
 *  s, dt, info, stream as for gb_chol_factor.
 */
gb_status gb_lu_factor(gb_handle *h, int64_t n, int64_t s, gb_dtype dt, const void *A,
                       int64_t lda, void *LU, int64_t ldlu, int *info, void *stream);

/* ---------------------------------------------------------------------- QR */
/*
 * gb_qr_factor -- Algorithm 3 (fast QR with step s), arXiv:1812.02056
 * Sec. 2: A = Q R with Q orthogonal and R upper triangular with a positive
 * diagonal.  Column c of Q is column c of the working matrix made
 * orthogonal to the columns of Q since the last checkpoint, one after the
 * other, and normalised; every s columns the trailing columns lose their
 * components along the last s columns of Q at once (C = B_Q^T B_M,
 * M -= B_Q C); at the end R = Q^T A.  Inside a block of s columns the
 * column steps run in inner blocks of b = min(s, GB_OPT_QR_INNER_STEP, the
 * shared-memory limit of the panel kernel) columns (the paper's remark that
 * s may vary, Sec. 2).
 *
 *  dt    GB_F64 (A, Q, R double) or GB_F32 (float); other dtypes:
 *        GB_ERR_UNSUPPORTED.
 *  A     n x n, leading dimension lda, read in full; must have full rank.
 *  Q     n x n output, leading dimension ldq: the orthonormal columns.
 *  R     n x n output, leading dimension ldr: Q^T A on and above the
 *        diagonal, zeros below.
 *  Q and R must not overlap A or each other (error -7 / -9): A is read
 *  again for R after Q is complete.  Host or device pointers, as for
 *  gb_chol_factor.
 *  s     step (s >= 1; s >= n: no delayed projection; s = 0: 64).
 *  info  0, or c + 1 (1-based) when the projected column c has zero (or
 *        NaN) norm, i.e. A is rank deficient there; Q and R are then
 *        unspecified from that column on.  -1: a bounded wait of the
 *        column-step kernel expired (its cluster-wide sums did not arrive
 *        within GB_OPT_SPIN_LIMIT, clamped to [10 ms, 1 s]); Q and R are
 *        not valid.
 */
gb_status gb_qr_factor(gb_handle *h, int64_t n, int64_t s, gb_dtype dt, const void *A,
                       int64_t lda, void *Q, int64_t ldq, void *R, int64_t ldr, int *info,
                       void *stream);

/* ------------------------------------------------------------------ solves */
typedef struct gb_refine_opts {
  double tol;     /* stop when max_r eta_r <= tol (default 1e-14)           */
  int max_iter;   /* maximum number of corrections (default 30)             */
} gb_refine_opts;

typedef struct gb_solve_stats {
  int iterations; /* corrections applied                                    */
  int converged;  /* 1 if eta <= tol was reached (always 1 without A)       */
  double eta;     /* final max over right-hand sides of
                     ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf);
                     0 when A was not given                                  */
} gb_solve_stats;

/*
 * gb_chol_solve -- solve A X = B from a factor made by gb_chol_factor:
 * L Y = B then L^T X = Y (forward and back substitution).  Not part of the
 * paper, which stops at the factor; it is the use the factor is made for
 * (Sec. 1: "used everywhere to solve linear systems").
 *
 *  factor_dt  the dtype the factor was made with (L is double for GB_F64,
 *             float otherwise).
 *  L, ldl     the factor.
 *  A, lda     NULL for a plain solve in the factor's precision (FP64 for
 *             GB_F64, FP32 otherwise, result stored as double).  Non-NULL:
 *             the original FP64 matrix (full square, symmetric); the call
 *             then refines X in FP64: r = B - A X (FP64), d = solve(L, r)
 *             (factor precision), X += d (FP64), until opts->tol.
 *  B, ldb     n x nrhs right-hand sides (double), row-major.
 *  X, ldx     n x nrhs solution (double); may alias B only when A is NULL.
 *  opts       NULL for defaults.    stats  may be NULL.
 * With A given the call waits for its stream once per correction to read
 * eta.  Returns GB_ERR_NOT_CONVERGED if max_iter corrections left
 * eta > tol (X holds the last iterate), GB_ERR_BREAKDOWN if a diagonal
 * entry of L is zero or not finite.
 */
gb_status gb_chol_solve(gb_handle *h, int64_t n, int64_t nrhs, gb_dtype factor_dt, const void *L,
                        int64_t ldl, const double *A, int64_t lda, const double *B, int64_t ldb,
                        double *X, int64_t ldx, const gb_refine_opts *opts,
                        gb_solve_stats *stats, void *stream);

/*
 * gb_lu_solve -- solve A X = B from a compact factor made by gb_lu_factor:
 * L Y = B, then U X = Y with U unit upper.  Arguments as gb_chol_solve; A,
 * when given, is the original FP64 matrix in full.
 */
gb_status gb_lu_solve(gb_handle *h, int64_t n, int64_t nrhs, gb_dtype factor_dt, const void *LU,
                      int64_t ldlu, const double *A, int64_t lda, const double *B, int64_t ldb,
                      double *X, int64_t ldx, const gb_refine_opts *opts, gb_solve_stats *stats,
                      void *stream);

/*
 * gb_residual -- R = B - A X in FP64 accuracy, the residual step of
 * iterative refinement that gb_chol_solve and gb_lu_solve run when given
 * A, by the method GB_OPT_RESIDUAL selects.  A n x n (lda), X and B
 * n x nrhs (ldx, ldb), R n x nrhs (ldr); all double, row-major, device
 * pointers; nrhs <= 1365.  With `eta` non-NULL writes
 * max_c ||r_c||_inf / (||A||_inf ||x_c||_inf + ||b_c||_inf) there (Inf when
 * anything is not finite).  Waits for the stream.  Returns GB_ERR_TIMEOUT
 * if a bounded device wait of the tensor-core method expired.
 */
gb_status gb_residual(gb_handle *h, int64_t n, int64_t nrhs, const double *A, int64_t lda,
                      const double *X, int64_t ldx, const double *B, int64_t ldb, double *R,
                      int64_t ldr, double *eta, void *stream);

/* --------------------------------------------------- the rank-s update */
/*
 * gb_rank_update -- the delayed update of Algorithms 1 and 2
 * (arXiv:1812.02056 Sec. 2): S := X op(Y) "using a fast rectangular matrix
 * multiplication", then C -= S, with S never stored.
 *
 *  dt       GB_F64: C, X, Y double, FP64 arithmetic (CUDA cores);
 *           GB_F32: float, FP32 arithmetic (CUDA cores);
 *           GB_MIX_BF16 / GB_MIX_F16: C, X, Y float; X and Y are rounded to
 *           BF16 / FP16 and multiplied on the tensor cores (tcgen05) with FP32
 *           accumulation; C stays FP32.  GB_MIX_BF16X3: three-plane BF16
 *           split of X and Y, six tensor-core products (about FP32 accuracy).
 *  lower    1: update only C[i][j] with i >= j (Cholesky, op(Y) = Y^T, M = N
 *           and X = Y allowed); 0: every element.
 *  y_is_kxn 0: op(Y) = Y^T with Y stored N x K (row j of Y is column j of
 *           op(Y)); 1: op(Y) = Y stored K x N (LU's R_U).
 *  C        M x N (ldc); X M x K (ldx); Y as above (ldy).  Device pointers.
 * Asynchronous on `stream`.  Workspace: the mixed dtypes pack X and Y into
 * the handle's workspace.
 */
gb_status gb_rank_update(gb_handle *h, gb_dtype dt, int lower, int y_is_kxn, int64_t M,
                         int64_t N, int64_t K, void *C, int64_t ldc, const void *X, int64_t ldx,
                         const void *Y, int64_t ldy, void *stream);

/*
 * gb_chol_solve_noalloc -- X = (L L^T)^{-1} B by forward and back
 * substitution with a factor from gb_chol_factor, for callers that cannot
 * allocate device memory.  The paper has no counterpart: it is a plain
 * solve (no refinement) that needs no handle.
 *
 * Who needs it: callers that may not call cudaMalloc -- code working inside
 * a memory budget it does not own (a fixed arena handed over by the host
 * application, a pool that is already fully reserved), a latency-critical
 * section where an allocation (which can synchronize the device) is not
 * allowed, or a plugin that must not touch its host program's allocator.
 * gb_create allocates a handle's scratch; this call takes no handle.  Its
 * scratch (the ticket and per-block flags that order the single-launch
 * solve, an error word and a breakdown word) is a file-scope __device__
 * array of 4099 ints that every GPU loading the library holds until exit.
 *
 *  n <= 131072 (larger n returns GB_ERR_UNSUPPORTED); nrhs >= 0.
 *  L, B, X     device pointers on the current device (host pointers and
 *              other GPUs' memory are rejected with -4, -6 or -8: staging
 *              would allocate); layouts as gb_chol_solve; X may alias B.
 *  factor_dt   as gb_chol_solve (L double for GB_F64, float otherwise).
 * Runs on the current device and waits for `stream`: the breakdown and
 * error words are read on the host.  Every call shares the one array and
 * leaves its contents behind; each call clears what must start at zero.
 * Calls that overlap on the GPU race on the array: do not issue them
 * concurrently.  The first call on a device looks up the array's address
 * with that device current (set-up done once per device); make that first
 * call before any stream capture.
 * Returns GB_ERR_BREAKDOWN for a zero or non-finite diagonal entry of L and
 * GB_ERR_TIMEOUT if a bounded device wait expired.
 */
gb_status gb_chol_solve_noalloc(int64_t n, int64_t nrhs, gb_dtype factor_dt, const void *L,
                                int64_t ldl, const double *B, int64_t ldb, double *X,
                                int64_t ldx, void *stream);

/* ---------------------------------------------------------------- served */
/*
 * A continuous-batching request server (no counterpart in the paper, which
 * factors one matrix at a time): factor-and-solve jobs of mixed sizes are
 * submitted at any time; a scheduler thread admits the oldest job as soon as
 * a slot is free and its device-memory footprint fits the budget; each slot
 * owns a handle, a stream and a worker thread, so admitted jobs overlap on
 * the device.  A job runs gb_chol_factor with a step chosen from (n, dtype)
 * alone -- never from the load -- and gb_chol_solve, refined in FP64 for the
 * reduced-precision dtypes, so its result is the same bits alone or among
 * other jobs.
 */
typedef struct gb_server gb_server;

typedef struct gb_request {
  int64_t n, nrhs;     /* order and number of right-hand sides (>= 1)       */
  gb_dtype dtype;      /* factor arithmetic                                  */
  int64_t s;           /* step, or 0 for the served default for (n, dtype)   */
  const double *A;     /* n x n SPD, full symmetric square, host or device   */
  int64_t lda;
  const double *B;     /* n x nrhs right-hand sides, host or device          */
  int64_t ldb;
  double *X;           /* n x nrhs solution, host or device                  */
  int64_t ldx;
  double tol;          /* refinement target (0: 1e-14)                      */
  int max_iter;        /* refinement limit (0: 30)                          */
} gb_request;

typedef struct gb_result {
  gb_status status;    /* GB_OK, GB_ERR_NOT_CONVERGED, GB_ERR_NOMEM, ...     */
  int info;            /* factorization breakdown column (0 = none)          */
  int iterations;      /* refinement corrections                             */
  double eta;          /* final normwise backward error                      */
  double queue_ms;     /* submit -> admission                                */
  double compute_ms;   /* admission -> completion                            */
  double total_ms;     /* submit -> completion                               */
} gb_result;

typedef struct gb_server_stats {
  uint64_t completed, rejected, queued;
  int running, max_running;      /* jobs on the device now / at most so far   */
  double p50_ms, p99_ms, max_ms;  /* total latency of completed jobs            */
  double solves_per_s;            /* completed / (last completion - 1st submit) */
  size_t budget_bytes, bytes_in_use;
} gb_server_stats;

/* Create a server on `device` with `max_slots` (1..64) concurrent jobs and
 * a device-memory budget in bytes (0: 80% of the currently free memory). */
gb_status gb_server_create(int device, size_t hbm_budget, int max_slots, gb_server **out);

/* Queue a job.  The caller's buffers must stay valid until the job is
 * waited for; nothing is copied at submission.  Returns GB_ERR_REJECTED if
 * the job's footprint exceeds the whole budget. */
gb_status gb_server_submit(gb_server *srv, const gb_request *req, uint64_t *ticket);

/* Wait up to timeout_s seconds (< 0: forever) for a job; on success fills
 * *out and forgets the ticket; GB_ERR_TIMEOUT if it is still running. */
gb_status gb_server_wait(gb_server *srv, uint64_t ticket, double timeout_s, gb_result *out);

/* Non-blocking wait: GB_ERR_STATE while the job is pending. */
gb_status gb_server_poll(gb_server *srv, uint64_t ticket, gb_result *out);

gb_status gb_server_get_stats(gb_server *srv, gb_server_stats *out);
gb_status gb_server_reset_stats(gb_server *srv);

/* Finish the queued and running jobs, then stop the threads and free. */
gb_status gb_server_destroy(gb_server *srv);

/* ---------------------------------------------------------- diagnostics */
/* Phases of a factorization, as timed under GB_OPT_PROFILE. */
typedef enum gb_phase {
  GB_PHASE_COPY = 0,   /* A -> working matrix (cast, zero the upper part)  */
  GB_PHASE_DIAG = 1,   /* column steps of the diagonal blocks              */
  GB_PHASE_PANEL = 2,  /* rows (and, for LU, columns of U) of the panel    */
  GB_PHASE_INNER = 3,  /* updates inside an s-block (inner step < s)       */
  GB_PHASE_UPDATE = 4, /* the delayed rank-s update of the trailing matrix */
  GB_NUM_PHASES = 5
} gb_phase;

typedef struct gb_profile {
  int64_t launches[GB_NUM_PHASES]; /* kernel launches per phase              */
  double ms[GB_NUM_PHASES];        /* summed device time per phase (events)  */
  double flops[GB_NUM_PHASES];     /* algorithmic flops per phase            */
  double bytes[GB_NUM_PHASES];     /* algorithmic DRAM bytes per phase       */
} gb_profile;

/* Wait for the events recorded since the last read (or reset), add their
 * times into *out (which the caller zero-initialises once) and forget them.
 * Flops count one multiply-add as 2; bytes count each element of the
 * working matrix read or written once per launch. */
gb_status gb_profile_read(gb_handle *h, gb_profile *out);

/* Total number of kernels this library has launched in the process (all
 * handles).  Callers difference two readings. */
uint64_t gb_kernel_launches(void);

/*
 * gb_measure_fma_peak -- run a register-only fused-multiply-add loop on
 * every SM of the handle's device (dt = GB_F64 for DFMA, GB_F32 for FFMA)
 * and report the achieved rate in flop/s (2 per FMA).  Synchronous.
 */
gb_status gb_measure_fma_peak(gb_handle *h, gb_dtype dt, double *flops_per_s);

/*
 * gb_measure_peak -- the arithmetic rooflines of this GPU's pipes, measured
 * by register- or shared-memory-only loops over every SM of the handle's
 * device, in flop/s (no counterpart in the paper: they are the denominators
 * of the roofline fractions the benchmark reports).  Synchronous.
 *   GB_PEAK_DFMA, GB_PEAK_FFMA  as gb_measure_fma_peak (FP64 / FP32 FMA)
 *   GB_PEAK_DMMA     f64 tensor MMA, mma.sync m8n8k4 (512 flop per warp op)
 *   GB_PEAK_TC_BF16  tcgen05.mma kind::f16, BF16 operands, FP32 accumulate,
 *                    M = 128, N = 256, one CTA per SM, operands in shared
 *                    memory (no memory traffic): dense tensor-pipe peak
 *   GB_PEAK_TC_F16   the same with FP16 operands
 *   GB_PEAK_TC_TF32  tcgen05.mma kind::tf32 (K = 8 per instruction)
 *   GB_PEAK_DFMA_DMMA  FP64 FMAs and f64 MMAs interleaved in one loop, equal
 *                    flops of each: above both single rates only if the
 *                    two run on separate units
 * Returns GB_ERR_UNSUPPORTED for the tcgen05 kinds on a device without
 * them, and GB_ERR_TIMEOUT if the loop's bounded completion wait ran out.
 */
typedef enum gb_peak {
  GB_PEAK_DFMA = 0,
  GB_PEAK_FFMA = 1,
  GB_PEAK_DMMA = 2,
  GB_PEAK_TC_BF16 = 3,
  GB_PEAK_TC_F16 = 4,
  GB_PEAK_TC_TF32 = 5,
  GB_PEAK_DFMA_DMMA = 6
} gb_peak;
gb_status gb_measure_peak(gb_handle *h, gb_peak kind, double *flops_per_s);

/*
 * gb_backward_error -- ||A - L L^T||_F / ||A||_F (is_lu = 0) or
 * ||A - L U||_F / ||A||_F (is_lu = 1, compact factor, unit U), computed on
 * the device in FP64.  A is double (full square); the factor is double for
 * GB_F64 and float otherwise.  Device pointers only.  Writes the result to
 * *out (host) and waits for the stream.
 */
gb_status gb_backward_error(gb_handle *h, int is_lu, int64_t n, gb_dtype factor_dt,
                            const double *A, int64_t lda, const void *F, int64_t ldf,
                            double *out, void *stream);

/* ---------------------------------------------------------------- batched */
/*
 * gb_chol_factor_batched -- Algorithm 1 applied independently to `count`
 * matrices of possibly different orders, in ONE persistent launch: CTAs
 * take matrices longest first (LPT on n^3) from a device ticket.  A matrix
 * whose packed lower triangle fits in shared memory (S = 14080 FP64 or
 * 28160 FP32 elements per CTA: FP64 n <= 167, FP32 n <= 236) runs all of
 * Algorithm 1 in shared memory; a larger one is first copied to L, keeps its
 * panel in shared memory -- so its step is min(s, floor(S / n)) -- and
 * receives the delayed update in place in L.
 *
 *  n[count]    orders (host array), 0 <= n[i] <= 1024.
 *  A[count]    device pointers (host array of pointers) to the inputs; only
 *              the lower triangles are read.
 *  lda[count]  leading dimensions (host array), lda[i] >= n[i].
 *  L[count]    device pointers to the outputs (L[i] may equal A[i]): the
 *              lower triangle receives the factor, the strict upper
 *              triangle is zeroed.
 *  ldl[count]  leading dimensions of the outputs.
 *  dt          GB_F64 (double matrices) or GB_F32 (float matrices).
 *  s           step for every matrix (s >= 1), or 0 for the tuned step of
 *              each matrix's order (gb_batched_tune; a default rule before).
 *  info        count ints (device or host), per-matrix status as above.
 * Uploads the plan (waits for `stream` once), then launches; with a device
 * `info` the launch itself is asynchronous.
 */
gb_status gb_chol_factor_batched(gb_handle *h, int64_t count, const int64_t *n, void *const *A,
                                 const int64_t *lda, void *const *L, const int64_t *ldl,
                                 gb_dtype dt, int64_t s, int *info, void *stream);

/*
 * gb_batched_plan / gb_batched_run -- the two halves of
 * gb_chol_factor_batched.  gb_batched_plan validates the arrays, orders the
 * matrices and uploads the plan into the handle (synchronous; arguments as
 * above).  gb_batched_run(h, info, stream) launches the persistent kernel
 * over the last plan: a ticket reset and one kernel, nothing else, so a
 * caller can capture it into a CUDA graph and replay it (out of place, the
 * inputs stay intact).  info: device array of the plan's count ints.
 */
gb_status gb_batched_plan(gb_handle *h, int64_t count, const int64_t *n, void *const *A,
                          const int64_t *lda, void *const *L, const int64_t *ldl, gb_dtype dt,
                          int64_t s, void *stream);
gb_status gb_batched_run(gb_handle *h, int *info, void *stream);

/*
 * gb_lu_factor_batched -- Algorithm 2 (pivot-free Crout LU with step s,
 * arXiv:1812.02056 Sec. 2) applied independently to `count` matrices of
 * possibly different orders, in ONE persistent launch, like
 * gb_chol_factor_batched.  A matrix held whole in shared memory
 * (n * ld <= S, ld = n rounded up to odd; S as above: FP64 n <= 118, FP32
 * n <= 167) runs all of Algorithm 2 there; a larger one is first copied to
 * LU and keeps an L panel (rows z..n-1) and a U panel (columns z..n-1) of the
 * block in shared memory -- so its step is min(s, floor(S / (2 n))) -- and
 * receives the delayed update of the trailing square in place in LU.
 *
 *  A[count]     device pointers to the inputs, read in full; each must have
 *               nonzero leading principal minors.
 *  LU[count]    device pointers to the outputs (LU[i] may equal A[i]), in
 *               the compact form of gb_lu_factor.
 *  ldlu[count]  leading dimensions of the outputs.
 *  n, lda, dt, info, stream as for gb_chol_factor_batched; s >= 1, or 0 for
 *  min(n, 32).  info[i] = c + 1 when L_cc of matrix i is zero or NaN.
 */
gb_status gb_lu_factor_batched(gb_handle *h, int64_t count, const int64_t *n, void *const *A,
                               const int64_t *lda, void *const *LU, const int64_t *ldlu,
                               gb_dtype dt, int64_t s, int *info, void *stream);

/*
 * gb_lu_batched_plan -- gb_batched_plan for Algorithm 2: the plan that the
 * next gb_batched_run launches is the batched LU of gb_lu_factor_batched.
 */
gb_status gb_lu_batched_plan(gb_handle *h, int64_t count, const int64_t *n, void *const *A,
                             const int64_t *lda, void *const *LU, const int64_t *ldlu,
                             gb_dtype dt, int64_t s, void *stream);

/*
 * gb_batched_tune -- the autotuner of the batched call: for every bucket of
 * 32 orders up to n_max it times the persistent kernel on two waves of
 * synthetic SPD matrices (n I + ones) for steps s in {8, 16, 32, 48, 64, 96,
 * 128} and keeps the fastest in the handle (used when s = 0).  steps_out
 * (optional) receives ceil(n_max / 32) steps.  Allocates and frees its own
 * test matrices; synchronous.
 */
gb_status gb_batched_tune(gb_handle *h, gb_dtype dt, int64_t n_max, int *steps_out, void *stream);

/*
 * gb_tune_step -- the autotuner of the step for gb_chol_factor (kind 0),
 * gb_lu_factor (kind 1) and gb_qr_factor (kind 2) called with s = 0: times
 * the factorization of the n x n test matrix n I + ones in dtype dt for
 * s in {32, 64, 128, 256, 512, 1024} (below n) and inner steps {16, 32, 64}
 * (QR: {8, 16, 32}, the column-step width GB_OPT_QR_INNER_STEP), and keeps
 * the fastest pair (a larger step replaces a smaller one only when it is at
 * least 3% faster: the smaller step is at least as accurate) in the handle
 * for every order in [2^k, 2^(k+1)) with
 * k = floor(log2 n).  Later calls with s = 0 in that range use the pair (the
 * inner step for that call only); without a tuned entry s = 0 keeps its
 * fixed default.  s_out and b_out (optional) receive the pair.  This is the
 * paper's remark that s may be chosen per problem (Sec. 2, last
 * paragraph) made empirical.  Allocates and frees its test matrices;
 * synchronous.  Errors: -2 kind, -3 dtype, -4 n outside [2, 65536],
 * GB_ERR_UNSUPPORTED for a QR dtype other than GB_F64/GB_F32.
 */
gb_status gb_tune_step(gb_handle *h, int kind, gb_dtype dt, int64_t n, int64_t *s_out,
                       int64_t *b_out, void *stream);

#ifdef __cplusplus
} /* extern "C" */
#endif

#endif /* GBCHOL_H */
