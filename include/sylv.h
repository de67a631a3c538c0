/*
 * sylv.h -- C ABI of the GB300 (sm_103a) solver for the triangular Sylvester
 * equation
 *
 *        op(A) * Y + Y * op(B) = alpha * C,      op(X) = X or X^T,
 *
 * with A (m x m) and B (n x n) upper quasi-triangular (real Schur form: upper
 * triangular except for 2x2 diagonal blocks, each marked by a nonzero entry on
 * the first subdiagonal; Schwarz & Kjelgaard Mikkelsen 2019, Sec. 1, eq. (4)).
 * The method is the paper's tiled robust solver (Algorithm 4, "drsylv"): tiles of
 * Y carry local power-of-two scale factors (augmented tiles, Sec. 2.2, Def. 1),
 * diagonal tiles are solved by the robust scalar algorithm (Algorithm 2, with the
 * 1x1/2x2 block solves of Sec. 2.1), off-diagonal tiles are updated with the
 * robust tile update (Algorithm 3), and a final consistency scaling brings every
 * tile to the global factor alpha = min alpha_kl.  alpha is in (0, 1] and is an
 * exact power of two; no entry of Y ever exceeds the overflow threshold Omega.
 *
 * Conventions for every entry point:
 *   - Matrices are column-major with the given leading dimensions (>= max(1, rows)).
 *   - Matrix pointers are DEVICE pointers (cudaMalloc'd or torch CUDA memory) on
 *     the current CUDA device; they stay owned by the caller.  C is overwritten by
 *     Y (the LAPACK convention).
 *   - Only the upper triangle and the first subdiagonal of A and B are read.  Two
 *     consecutive nonzero subdiagonal entries make the input invalid
 *     (SYLV_ERR_STRUCTURE_A / _B).
 *   - Inputs must be finite; every tile of A, B, C must have infinity norm
 *     <= Omega (the precondition of Algorithms 2-4).
 *   - The solve runs on opts->stream (the legacy default stream when NULL).  With
 *     opts->sync != 0 the call waits for the GPU and fills a HOST sylv_result;
 *     with opts->sync == 0 it only enqueues work and writes the sylv_result to the
 *     DEVICE address given, so the call can be captured in a CUDA graph (pass a
 *     caller-owned workspace in that case).
 *   - Return value: a SYLV_* code below.  Negative values -i name the invalid
 *     argument i (1-based, LAPACK style); such calls enqueue no GPU work.
 */
#ifndef SYLV_H
#define SYLV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes (return values and sylv_result.info) ------------------ */
#define SYLV_OK 0
#define SYLV_NEAR_SINGULAR 1   /* a 1x1/2x2 block system was near singular (lambda_i(A) +
                                  lambda_j(B) ~ 0, eq. (1)'s uniqueness condition);
                                  its pivot was raised to smin and the solve went on */
#define SYLV_SCALE_UNDERFLOW 2 /* alpha < 2^-1074: the double `scale` is 0, use log2scale */
#define SYLV_NOT_CONVERGED 3   /* FP32 + refinement did not reach opts->tol */
#define SYLV_OVERFLOWED 4      /* Inf/NaN in an output: the non-robust mode overflowed (Algorithm 1), or a
                                  gradient of the adjoint lies beyond the binary64 range; or
                                  FP32 + refinement (which returns alpha = 1) met a solution beyond
                                  the binary64 range: C is then left holding the right-hand side, and
                                  a synchronous single solve repeats the solve with SYLV_FP64 itself */
#define SYLV_ERR_STRUCTURE_A 101 /* A has two consecutive nonzero subdiagonal entries */
#define SYLV_ERR_STRUCTURE_B 102 /* B has two consecutive nonzero subdiagonal entries */
#define SYLV_ERR_NONFINITE 103   /* NaN or Inf in A, B or C */
#define SYLV_ERR_RANGE 104       /* an input tile's infinity norm exceeds Omega */
#define SYLV_ERR_TIMEOUT 105     /* a device-side wait exceeded opts->timeout_ms */
#define SYLV_ERR_CUDA 106        /* a CUDA runtime call failed */
#define SYLV_ERR_WORKSPACE 107   /* caller-provided workspace too small or misaligned */
#define SYLV_ERR_UNSUPPORTED 108 /* option combination not built (e.g. tile size) */

/* ---- precisions ------------------------------------------------------------ */
#define SYLV_FP64 0            /* robust tiled solve in binary64 (Algorithm 4) */
#define SYLV_FP64_NONROBUST 1  /* same tiling, no scaling at all (Algorithm 1 per tile) */
#define SYLV_FP32_REFINE 2     /* robust solve in binary32 + residual refinement in
                                  binary64-accurate arithmetic (not in the paper); the result has
                                  alpha = 1.  A solution beyond the binary64 range ends the
                                  refinement with SYLV_OVERFLOWED and C unchanged; a synchronous
                                  single solve (opts->sync) then solves again with SYLV_FP64 and
                                  returns that result (iters = 0, alpha <= 1), unless a caller
                                  workspace is too small for it */

typedef struct sylv_opts {
  int32_t transa;          /* 0: op(A) = A, 1: op(A) = A^T */
  int32_t transb;          /* 0: op(B) = B, 1: op(B) = B^T */
  int32_t precision;       /* SYLV_FP64, SYLV_FP64_NONROBUST or SYLV_FP32_REFINE */
  int32_t tile;            /* nominal tile size t (Sec. 2.2); 0 = automatic.  Tiles
                              hold t or t-1 rows so that no 2x2 block is split */
  double omega;            /* overflow threshold Omega; 0 = 2^1020 (2^124 for binary32); the binary32
                              correction solves of SYLV_FP32_REFINE use min(omega, 2^124) */
  double tol;              /* refinement: stop when max|dY| <= tol * max|Y|, or when the
                              corrections contract and the next one is predicted that small;
                              0 = 2^-43 */
  int32_t maxit;           /* refinement: at most this many correction solves; 0 = 6 */
  int32_t sync;            /* 1: wait, host result; 0: asynchronous, device result */
  int64_t timeout_ms;      /* bound on each device-side wait; 0 = 20000 */
  void* stream;            /* cudaStream_t; NULL = legacy default stream */
  void* workspace;         /* device memory for the solver's scratch, or NULL to let
                              the library allocate (and cache) it */
  size_t workspace_bytes;  /* size of `workspace` */
  int32_t isgn;            /* sign of the B term: +1 (or 0) solves op(A) Y + Y op(B) = alpha C,
                              -1 solves op(A) Y - Y op(B) = alpha C (LAPACK's ISGN; not in
                              the paper, which treats +1: the solver runs on -B) */
  int32_t max_sms;         /* cap on the SMs the persistent tile kernel occupies: its CTAs
                              on SMs with id >= max_sms leave at once (CTA 0 always runs);
                              0 = all.  For SM-scaling studies (the GPU analogue of
                              Sec. 4's core scaling); the solution is bitwise the same */
} sylv_opts;

typedef struct sylv_result {
  int64_t log2scale;  /* alpha = 2^log2scale (exact; never underflows) */
  double scale;       /* alpha as a double (0 when alpha < 2^-1074) */
  int32_t info;       /* SYLV_OK, SYLV_NEAR_SINGULAR, SYLV_SCALE_UNDERFLOW, ... */
  int32_t iters;      /* refinement corrections applied (FP32_REFINE), else 0 */
  double last_update; /* FP32_REFINE: estimated max|error| / max|Y| of the result: the last
                         correction's relative size, or, when the corrections' contraction
                         ended the loop, the predicted size of the next one */
  int32_t scale_events; /* number of scaling decisions taken (Sec. 4's "amount of scaling") */
  int32_t min_tile_exp; /* smallest local exponent before consistency scaling */
} sylv_result;

/* Fill *opts with the defaults described above (all zero except sync = 1). */
void sylv_default_opts(sylv_opts* opts);

/*
 * sylv_tri_solve -- robust FP64 solve of A*Y + Y*B = alpha*C (Algorithm 4).
 *   m, n       orders of A and B (m, n >= 0)
 *   A, lda     device, m x m upper quasi-triangular, read only
 *   B, ldb     device, n x n upper quasi-triangular, read only
 *   C, ldc     device, m x n; on exit Y
 *   tile       nominal tile size, 0 = automatic
 *   scale      HOST pointer; receives alpha (0 if it underflows)
 * Synchronous on the legacy default stream, library-managed workspace.
 * Returns SYLV_OK, SYLV_NEAR_SINGULAR, SYLV_SCALE_UNDERFLOW or an error code.
 */
int sylv_tri_solve(int64_t m, int64_t n, const double* A, int64_t lda, const double* B,
                   int64_t ldb, double* C, int64_t ldc, int64_t tile, double* scale);

/*
 * sylv_tri_solve_ex -- the same solve with options: op(A)/op(B) transposes,
 * precision mode (robust FP64 / non-robust FP64 / FP32 + refinement), stream,
 * workspace and asynchronous results.  `result` is a HOST pointer when
 * opts->sync != 0 and a DEVICE pointer otherwise (may be NULL: no result).
 * opts == NULL means sylv_default_opts.
 */
int sylv_tri_solve_ex(int64_t m, int64_t n, const double* A, int64_t lda, const double* B,
                      int64_t ldb, double* C, int64_t ldc, const sylv_opts* opts,
                      sylv_result* result);

/* Bytes of device workspace sylv_tri_solve_ex needs for these sizes and options
 * (opts may be NULL).  Workspace passed by the caller must be 256-byte aligned. */
size_t sylv_workspace_size(int64_t m, int64_t n, const sylv_opts* opts);

/*
 * Batched solves: `count` independent equations op(A_i) Y_i + Y_i op(B_i) =
 * alpha_i C_i of individual sizes, solved together by one persistent launch
 * whose task list interleaves the tiles of all equations level by level (a tile
 * of one equation only ever waits on tiles of the same equation, Sec. 2.2's task
 * dependences).  Not in the paper.
 *
 * opts->transa / opts->transb apply to every equation (the plan keeps
 * anti-transposed copies of A_i / B_i and reverses C_i in place around the solve).
 * With opts->precision = SYLV_FP32_REFINE every equation is refined as in
 * sylv_tri_solve_ex (binary32 robust correction solves, one batched tile-kernel
 * launch per correction; binary64-accurate residuals in double-float arithmetic on
 * the binary32 pipes); each equation stops on its own tolerance test, after which
 * its work is skipped, and results[i].iters / last_update report it.  The launch
 * sequence is the same whatever converges, so it stays capturable.  An equation
 * whose solution lies beyond the binary64 range reports SYLV_OVERFLOWED and keeps
 * its right-hand side in C_i (solve it again with SYLV_FP64).
 *
 * sylv_batch_create builds a plan: it validates the HOST arrays m[i], n[i],
 * lda[i], ldb[i], ldc[i] and the device pointers A[i], B[i], C[i] (HOST arrays of
 * device pointers), picks each equation's tile size (opts->tile, or the built-in
 * size table when 0), allocates the plan's device workspace and uploads the
 * descriptors (one host-to-device copy, then a stream synchronize).
 * sylv_batch_execute only enqueues kernels on `stream` (capturable in a CUDA
 * graph; replays re-solve in place, so C_i must be refilled by the caller between
 * replays).  sylv_batch_results waits for the stream and copies `count` results
 * to the HOST array `results`.  The plan's matrices must stay allocated while it
 * is used.  Returns SYLV_OK or an error code; per-equation status is in
 * results[i].info.
 */
typedef struct sylv_batch_plan sylv_batch_plan;
int sylv_batch_create(sylv_batch_plan** plan, int32_t count, const int64_t* m, const int64_t* n,
                      const double* const* A, const int64_t* lda, const double* const* B,
                      const int64_t* ldb, double* const* C, const int64_t* ldc,
                      const sylv_opts* opts);
/* As sylv_batch_create, with a tile size per equation: tiles[i] in {0, 2..64}
 * (0: opts->tile or the built-in choice), e.g. from an autotuner; NULL = none. */
int sylv_batch_create_tiles(sylv_batch_plan** plan, int32_t count, const int64_t* m, const int64_t* n,
                            const double* const* A, const int64_t* lda, const double* const* B,
                            const int64_t* ldb, double* const* C, const int64_t* ldc,
                            const int32_t* tiles, const sylv_opts* opts);
int sylv_batch_execute(sylv_batch_plan* plan, void* stream);
int sylv_batch_results(sylv_batch_plan* plan, sylv_result* results);
void sylv_batch_destroy(sylv_batch_plan* plan);

/* One-call form of the above: create, execute on opts->stream, wait, fill the
 * HOST array results[count], destroy. */
int sylv_tri_solve_batched(int32_t count, const int64_t* m, const int64_t* n,
                           const double* const* A, const int64_t* lda, const double* const* B,
                           const int64_t* ldb, double* const* C, const int64_t* ldc,
                           const sylv_opts* opts, sylv_result* results);

/*
 * sylv_tri_solve_backward -- adjoint of the FP64 solve for reverse-mode
 * differentiation (not in the paper).  The forward solve returned Y = alpha*X
 * with op(A) X + X op(B) = C, alpha a power of two held fixed (it is piecewise
 * constant in the inputs).  Given G = dL/dY (device, m x n, ldg) this computes
 *   Gamma   solving  op(A)^T Gamma + Gamma op(B)^T = G  (the same robust tiled
 *           solver with both transposes flipped, in opts->precision: FP64, or
 *           FP32 + refinement; Y, A, B unchanged),
 *   dL/dC = alpha * Gamma                     -> written over G,
 *   dL/dA = -Gamma Y^T  (op(A) = A)  or  -Y Gamma^T  (op(A) = A^T)   -> dA (m x m, ldda),
 *   dL/dB = -Y^T Gamma  (op(B) = B)  or  -Gamma^T Y  (op(B) = B^T)   -> dB (n x n, lddb),
 * since dL/dX = alpha*G and X = Y/alpha.  dA and dB are masked to the entries the
 * solver reads (upper triangle plus the nonzero subdiagonal entries that mark 2x2
 * blocks); all other entries are set to 0.  dA or dB may be NULL to skip them.
 * log2scale is the forward result's exponent (alpha = 2^log2scale).  If the adjoint
 * solve has to scale (its own factor alpha_G = 2^result->log2scale < 1), the call
 * removes alpha_G from all three outputs again on the device, by exact power-of-two
 * scaling (the exponent is read from the device result record, so the call does not
 * wait for the host); an output entry that leaves the binary64 range on the way
 * becomes +-Inf and the status is SYLV_OVERFLOWED.  result->log2scale still
 * reports alpha_G.  Y and G are device pointers.  With SYLV_FP32_REFINE the adjoint
 * solve returns alpha_G = 1: if Gamma lies beyond the binary64 range the status is
 * SYLV_OVERFLOWED and the three outputs are not gradients (call again with
 * SYLV_FP64, which scales).
 */
int sylv_tri_solve_backward(int64_t m, int64_t n, const double* A, int64_t lda, const double* B,
                            int64_t ldb, const double* Y, int64_t ldy, int64_t log2scale,
                            double* G, int64_t ldg, double* dA, int64_t ldda, double* dB,
                            int64_t lddb, const sylv_opts* opts, sylv_result* result);

/*
 * sylv_tri_solve_backward_batched -- sylv_tri_solve_backward for `count` equations
 * at once (HOST arrays of sizes, leading dimensions, device pointers and the
 * forward exponents log2scale[i]); the adjoint solves run as one batched launch
 * (both transposes flipped), the gradient products and the dC scaling as one
 * launch each.  dA / dB may be NULL (skip all) or hold NULL entries (skip one).
 * results[i] (HOST) receives each adjoint solve's record; as in the single form,
 * each equation's outputs come back with its adjoint factor alpha_G removed (status
 * SYLV_OVERFLOWED where an entry leaves the binary64 range).  Synchronizes
 * opts->stream; allocates a plan and a small descriptor buffer internally.
 */
int sylv_tri_solve_backward_batched(int32_t count, const int64_t* m, const int64_t* n,
                                    const double* const* A, const int64_t* lda,
                                    const double* const* B, const int64_t* ldb,
                                    const double* const* Y, const int64_t* ldy,
                                    const int64_t* log2scale, double* const* G, const int64_t* ldg,
                                    double* const* dA, const int64_t* ldda, double* const* dB,
                                    const int64_t* lddb, const sylv_opts* opts, sylv_result* results);

/*
 * sylv_tri_solve_noalloc -- the robust FP64 solve of sylv_tri_solve, for callers
 * that must not allocate device memory while they run: real-time loops that forbid
 * allocator calls after start-up (an allocation can block on the device or the
 * driver for an unbounded time), and hosts whose device memory belongs to another
 * allocator that the library cannot call into.  The paper has no counterpart; it is
 * a service of this library.
 *
 * It allocates nothing: its scratch is one fixed array of 16 MiB in device memory
 * that this library defines and every GPU that loads the library holds until the
 * process exits.  The caller passes the inputs and the output as for
 * sylv_tri_solve (device pointers; C is overwritten by Y); `tile` as for
 * sylv_tri_solve; `stream` is a cudaStream_t (NULL: legacy default stream).  The
 * call copies the result record to host memory and synchronizes `stream` before it
 * returns, filling the HOST record *result (may be NULL).
 * Problems whose bookkeeping does not fit the array are rejected on the host,
 * before any GPU work, with SYLV_ERR_WORKSPACE (about m, n <= 11000 fit at the
 * default tile); when the per-CTA stores fit only in part, the solve runs with
 * fewer CTAs.  The first call on a device looks up the array's device address
 * (a runtime call, once per device, with that device current).  All calls share
 * the one array and it keeps the last call's contents: each call clears what must
 * start at zero, but two calls that overlap on the GPU (different streams or
 * threads) race on it and give wrong results.  Status codes as for
 * sylv_tri_solve_ex.
 */
int sylv_tri_solve_noalloc(int64_t m, int64_t n, const double* A, int64_t lda, const double* B,
                           int64_t ldb, double* C, int64_t ldc, int64_t tile, void* stream,
                           sylv_result* result);

/*
 * sylv_tri_solve_triangular -- the robust triangular solve op(A) X = alpha C with
 * alpha in (0,1] a power of two chosen so that no intermediate exceeds Omega: the
 * solver with the B term removed (the robust triangular solver the paper builds on,
 * Sec. 2.1, and Algorithm 4 restricted to column updates).  Tiles of X depend only
 * on the tiles below them in the same column, so every column block proceeds in
 * parallel and the tile DAG has p levels instead of p + q - 1.
 *   m, n      order of A and number of right-hand sides (m, n >= 0)
 *   A, lda    device, m x m upper quasi-triangular (upper triangle + the first
 *             subdiagonal of its 2x2 blocks), read only; op(A) = A^T when
 *             opts->transa = 1
 *   C, ldc    device, m x n; on exit X
 *   opts      as for sylv_tri_solve_ex; precision SYLV_FP64 or SYLV_FP64_NONROBUST
 *             (SYLV_FP32_REFINE and transb are rejected with SYLV_ERR_UNSUPPORTED),
 *             isgn is ignored
 *   result    as for sylv_tri_solve_ex (host record in sync mode, device address
 *             otherwise)
 * Returns as sylv_tri_solve_ex; -1..-6 name the bad argument.
 */
int sylv_tri_solve_triangular(int64_t m, int64_t n, const double* A, int64_t lda, double* C, int64_t ldc,
                              const sylv_opts* opts, sylv_result* result);

/*
 * sylv_solve_schur -- the Bartels-Stewart wrapper around the robust solve (Sec. 1,
 * eqs. (3)-(5)): given real Schur forms A = U TA U^T and B = V TB V^T (U, V
 * orthogonal, TA, TB upper quasi-triangular, from an external eigensolver), solve
 *     A X + isgn X B = alpha C
 * as C~ = U^T C V, TA Y + isgn Y TB = alpha C~ (sylv_tri_solve_ex), X = U Y V^T.  The
 * four dense products run on the library's tensor-core GEMM in its binary64-accurate
 * form (bf16 operand slices by error-free splitting, exact integer accumulation of
 * the leading slice pairs): each product term is exact to within 2^-54 of (row
 * maximum) x (column maximum), as for sylv_residual.  A timeout of that GEMM's
 * pipeline waits gives SYLV_ERR_TIMEOUT (sync mode).
 *   U, ldu    device, m x m orthogonal, read only
 *   TA, ldta  device, m x m upper quasi-triangular, read only
 *   V, ldv    device, n x n orthogonal, read only
 *   TB, ldtb  device, n x n upper quasi-triangular, read only
 *   C, ldc    device, m x n; on exit X
 *   opts      as for sylv_tri_solve_ex (transa/transb must be 0; the workspace, if
 *             given, must hold sylv_schur_workspace_size(m, n, opts) bytes)
 *   result    as for sylv_tri_solve_ex
 * Returns as sylv_tri_solve_ex; -3/-4 U, -7/-8 V, -5/-6 TA, -9/-10 TB, -11/-12 C.
 */
int sylv_solve_schur(int64_t m, int64_t n, const double* U, int64_t ldu, const double* TA, int64_t ldta,
                     const double* V, int64_t ldv, const double* TB, int64_t ldtb, double* C, int64_t ldc,
                     const sylv_opts* opts, sylv_result* result);
/* Bytes of device workspace sylv_solve_schur needs for these sizes and options
 * (opts may be NULL; 0 for negative sizes or invalid options). */
size_t sylv_schur_workspace_size(int64_t m, int64_t n, const sylv_opts* opts);

/*
 * sylv_residual -- R = C - (A X + X B) to binary64 accuracy, the residual of
 * eq. (7) with alpha = 1 that the refinement of SYLV_FP32_REFINE evaluates for its
 * first correction (Sec. 2 defines the equation; the residual is the numerator of
 * eq. (9) without norms).
 *
 * A (m x m, lda) and B (n x n, ldb) are read in their upper quasi-triangular parts
 * only (upper triangle and first subdiagonal); X (m x n, ldx) and C (m x n, ldc) are
 * read in full; R (m x n, ldr) is written.  All are device pointers, column-major,
 * caller-owned; R may not overlap the inputs.  The products run on the bf16 tensor
 * cores by an error-free splitting of A and B by rows/columns and of X by
 * columns/rows into seven 8-bit slices each (Ozaki et al. 2012): each product term
 * is exact to within 2^-54 of (row maximum) x (column maximum), so R is within
 * about 2^-48 (|A||X| + |X||B|)_ij of the exact value when rows and columns are
 * balanced (a normwise guarantee otherwise).  The call uses the library's cached
 * device workspace (about 14 (m^2 + n^2 + 2mn) bytes), runs on
 * `stream` (null: the default stream) and synchronizes it.  Returns SYLV_OK, a
 * negative argument index, SYLV_ERR_UNSUPPORTED for m or n beyond the solver's
 * limit, SYLV_ERR_CUDA, or SYLV_ERR_TIMEOUT if a pipeline wait of the GEMM kernel
 * ran out (20 s).
 */
int sylv_residual(int64_t m, int64_t n, const double* A, int64_t lda, const double* B, int64_t ldb,
                  const double* X, int64_t ldx, const double* C, int64_t ldc, double* R, int64_t ldr,
                  void* stream);

/*
 * sylv_diag_wait_timeout -- diagnostic of the solver's bounded waits (not in the
 * paper).  Launches one CTA that waits, with the same bounded wait the tile-DAG
 * kernel uses for its ready flags, on a flag that nothing ever sets, and returns
 * the status the kernel recorded: SYLV_ERR_TIMEOUT once timeout_ms has passed
 * (the GPU context stays usable), or an error code if the launch failed.  It
 * allocates a few bytes of device memory and synchronizes `stream`.
 */
int sylv_diag_wait_timeout(int64_t timeout_ms, void* stream);

/*
 * sylv_diag_guards -- diagnostic of the solver's scaling guards.  Evaluates, on the
 * device, the very ProtectUpdate and ProtectDivision routines the tile kernels call
 * (Sec. 2.1), so a test can check their contracts directly:
 *   z_update[i]   = z <= 0 with 2^z (c[i] + t[i] x[i]) <= omega, for c, t, x in [0, omega];
 *   z_division[i] = the largest z <= 0 with 2^z |b[i]| / |d[i]| <= omega, for
 *                   |b[i]| <= omega and d[i] != 0.
 * All seven arrays hold `count` entries in device memory, caller-owned; omega is the
 * overflow threshold (>= 1, finite; the solver uses 2^1020 in binary64 and 2^124
 * for its binary32 correction solves).  Runs on `stream` (null: the default stream)
 * and synchronizes it.  Returns SYLV_OK, -1 (count), -2 (a null array), -9 (omega)
 * or SYLV_ERR_CUDA.  Allocates nothing.
 */
int sylv_diag_guards(int64_t count, const double* c, const double* t, const double* x, int32_t* z_update,
                     const double* b, const double* d, int32_t* z_division, double omega, void* stream);

/*
 * sylv_diag_fma_rate -- measures the peak rate of the FMA pipe that bounds the
 * solver's tile kernels (not in the paper): kind 0 = binary64 FMA (the FP64 solve),
 * 1 = binary32 FMA (the FP32 correction solves).  One launch of one full wave of
 * 256-thread CTAs (as many per SM as fit), each thread running 8 (binary64) or 16
 * (binary32) independent FMA chains for `iters` rounds, timed with CUDA events on
 * `stream` after a warm-up launch; *gflops receives 2 x chains x iters x threads /
 * time (two flops per FMA), *ms (may be NULL) the time.
 * Allocates 16 bytes and synchronizes `stream`.  Returns SYLV_OK, -1 (kind), -2
 * (iters outside [1, 2^32 - 1]), -3 (gflops NULL) or SYLV_ERR_CUDA.
 */
int sylv_diag_fma_rate(int32_t kind, int64_t iters, double* gflops, double* ms, void* stream);

/*
 * Kernel timing for benchmarks (not in the paper).  While enabled, every launch of
 * the tile-DAG kernel (the solver's dominant kernel) is bracketed by CUDA events
 * recorded on the stream it is launched on.  sylv_profile_read waits for those
 * events, returns the summed kernel time in milliseconds and the number of
 * launches since the last read, and releases the events.  Host-side state, not
 * thread-safe; sylv_profile(0) disables recording.
 */
int sylv_profile(int enable);
int sylv_profile_read(double* dag_ms, int64_t* dag_launches);

/* Static description of a status code. */
const char* sylv_error_string(int code);

/* Library version string. */
const char* sylv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SYLV_H */
