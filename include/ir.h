/*
 * ir.h -- C ABI of the GB300 mixed-precision iterative-refinement solver.
 *
 * The library solves dense A x = b on one NVIDIA GB300 GPU by Algorithm IR of
 * Kelley, "Using MultiPrecisionArrays.jl: Iterative Refinement in Julia"
 * (Sec. 1): a copy of the working-precision matrix A (type TW) is rounded to
 * the factorization precision TF and factored by LU with partial pivoting;
 * the loop { d = U^{-1} L^{-1} r ; x += d ; r = b - A x in precision TR }
 * runs until a termination rule on ||r|| holds (Sec. 5.1).
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major with a leading dimension lda >= n (LAPACK and
 *     Julia layout).  Vectors are contiguous.
 *   - Unless a name says "host", pointers are DEVICE pointers (cudaMalloc /
 *     torch allocations) on the device the context was created for.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  All device work is enqueued on it.
 *   - Pivots are 0-based: step k interchanged rows k and ipiv[k].
 *   - Every call returns an ir_status and never aborts the process.  On an
 *     error return nothing the call was to produce is valid.
 *   - The library allocates its own device workspace (the factorization copy,
 *     pivots, solve vectors) inside ir_factor; the caller owns A, b and x.
 */
#ifndef GB300_IR_H
#define GB300_IR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Precisions (the TW / TF / TR types of Sec. 1).  IR_TF32 is the tensor-core
 * format with 10 fraction bits; IR_BF16 / IR_F16 the 16-bit formats of Sec. 3. */
typedef enum { IR_F64 = 0, IR_F32 = 1, IR_TF32 = 2, IR_BF16 = 3, IR_F16 = 4 } ir_dtype;

typedef enum {
    IR_OK = 0,
    IR_EINVAL = 1,        /* bad argument (null pointer, n < 0, lda < n, unsupported dtype mix) */
    IR_ENOMEM = 2,        /* device allocation failed */
    IR_ECUDA = 3,         /* a CUDA runtime call failed */
    IR_ESINGULAR = 4,     /* exact zero pivot in the TF factorization (report.info) */
    IR_ENONFINITE = 5,    /* NaN/Inf in A or b, or overflow of the rounded copy */
    IR_ETIMEOUT = 6,      /* a bounded device-side wait gave up */
    IR_EUNSUPPORTED = 7   /* size or configuration outside what this build supports */
} ir_status;

/* Outcome of the refinement loop (numerical non-convergence is not an error). */
typedef enum {
    IR_CONVERGED = 0,     /* eq. (residterm) held, or the residual is exactly zero */
    IR_STAGNATED = 1,     /* eq. (stag), or eq. (wilkterm) when TR is wider than TW */
    IR_MAXIT = 2,         /* litmax residual computations without termination */
    IR_DIVERGED = 3,      /* the residual norm became non-finite */
    IR_FAILED = 4         /* the factorization had a zero pivot; no iteration ran */
} ir_solve_status;

/* Termination parameters: the TERM structure of Sec. 5.1.3.
 *   converged   if ||r|| == 0 (x is exact; r / ||r|| would be undefined)
 *               or, mode 0, ||r|| <= Cr * eps(TW) * ||b||  (eq. residterm)
 *                  (when abs_rel_tol > 0: ||r|| <= abs_rel_tol * ||b||)
 *               or, mode 1, ||r|| <= Ce * eps(TW) * (||b|| + ||A||_1 ||x||)
 *                  (eq. term, the normwise backward error; ||A||_1 is computed
 *                  in binary64 from A once per factorization, on first use)
 *   stagnated   if ||r_new|| >= Rmax ||r_old||           (eq. stag), TR == TW
 *               if ||d_new|| >= Rmax ||d_old||           (eq. wilkterm), TR wider than TW
 *   stop        after litmax residual computations.
 * Norms are infinity norms; eps(T) is 2^-52 (FP64) or 2^-23 (FP32). */
typedef struct {
    double Cr;            /* default 1.0 */
    double Ce;            /* default 1.0 (backward-error test, mode 1) */
    double Rmax;          /* default 0.5 */
    int litmax;           /* default 10, at most IR_MAX_HIST - 1 */
    int mode;             /* 0: small residual (default); 1: small backward error.
                             The batched driver supports mode 0 only (IR_EUNSUPPORTED). */
    double abs_rel_tol;   /* > 0 overrides Cr * eps(TW) */
} ir_term;

/* Factorization options (the keyword arguments TF and TR of mplu, Sec. 2.4).
 *   TW: IR_F64 or IR_F32 (type of A and b).  TF: IR_F32, IR_TF32, IR_BF16 or
 *   IR_F16.  TR: IR_F64.  fp16_scale = 1 multiplies A by s = 2^10 / max|a_ij|
 *   before the binary16 cast (ignored for other TF).  nb = 0 picks the block
 *   size. */
typedef struct {
    ir_dtype TW, TF, TR;
    int fp16_scale;       /* default 1 */
    int nb;               /* outer block size; 0 = default (64) */
    int autotune;         /* 1: tune the schedule on the caller's own input (see
                             ir_fact_schedule / ir_batch_schedule); default 0 */
    int group;            /* TF32 / bf16 / binary16: block steps whose update of the
                             far trailing columns is applied at once (1 .. 16;
                             0 = default 8, or the tuned value with autotune) */
    int onthefly;         /* 0 (default): low precision solves (LPS) -- binary32
                             triangular solves of fl32(P r / ||r||), scaled back
                             (eqs. vdlow / promotevd, Sec. 5.3); 1: mixed
                             precision solves (MPS, mplu(A; onthefly = true),
                             Sec. 5.3) -- r is kept in TW and the triangular
                             solves run in TW on the factors promoted exactly,
                             with no scaling by ||r||.  Used by ir_solve and
                             ir_solve_many (GMRES-IR / BiCGSTAB-IR keep their
                             preconditioner of Sec. 4.3). */
    int store_tf;         /* TF = IR_F16 / IR_BF16 only: 1 keeps the factors in TF,
                             as the paper's factorization copy is (Sec. 1, 2.5):
                             after the factorization every entry of L and U is
                             rounded to TF once, and the correction solves read
                             a 2-byte copy of them (half the bytes of binary32
                             factors) and promote each entry exactly.  0
                             (default): binary32 factors.  An entry that
                             overflows TF makes the factorization non-finite. */
} ir_opts;

#define IR_MAX_HIST 32

/* Iteration statistics (the `reporting = true` output of Sec. 2.2.1).
 * rhist[0] = ||b||; rhist[k] = ||r|| after the k-th correction; dhist[k] =
 * ||d_k||, one entry fewer than rhist. */
typedef struct {
    int iters;                    /* residual computations = entries of rhist - 1 */
    ir_solve_status status;
    double rhist[IR_MAX_HIST];
    double dhist[IR_MAX_HIST];
    int64_t info;                 /* first zero pivot (1-based) or 0 */
    double scale;                 /* s used for the factorization copy */
} ir_report;

typedef struct ir_ctx ir_ctx;
typedef struct ir_fact ir_fact;

/* Fill the paper's defaults (TW = F64, TF = F32, TR = F64; Cr = Ce = 1,
 * Rmax = 0.5, litmax = 10; Sec. 2.4 and 5.1.3). */
void ir_default_opts(ir_opts *opts);
void ir_default_term(ir_term *term);

/* Create a context on CUDA device `device` (selects it for the calling
 * thread).  *ctx receives a handle owned by the caller; free with ir_finalize. */
ir_status ir_init(int device, ir_ctx **ctx);
void ir_finalize(ir_ctx *ctx);

/* mplu (Sec. 2.4): round A to TF (A_F = I_W^F(s A), Sec. 1) into a library-
 * owned copy and factor it by LU with partial pivoting.
 *   0 <= n <= 77824, A: n x n in TW, column-major, lda >= max(1, n); a larger
 *   n gives IR_EUNSUPPORTED.  Up to n = 8192 every panel is factored by one
 *   thread-block cluster; a taller panel by one cooperative launch of up to one
 *   CTA per SM (512 rows each), whose CTAs exchange each column's pivot
 *   candidates through global memory; such a factorization is not replayed
 *   from a CUDA graph.
 * The handle BORROWS A for the residuals of ir_solve: A must stay alive and
 * unmodified until ir_fact_destroy or ir_refactor (the MPArray shares A's
 * storage, Sec. 2.5).  Asynchronous; a zero pivot or a non-finite copy is
 * reported by ir_solve or ir_fact_info. */
ir_status ir_factor(ir_ctx *ctx, int64_t n, const void *A, int64_t lda,
                    const ir_opts *opts, void *stream, ir_fact **out);

/* mplu!(MPF, B) (Sec. 2.5): factor another matrix of the same size and
 * precisions into the same storage.  The handle then borrows B. */
ir_status ir_refactor(ir_fact *fact, const void *B, int64_t ldb, void *stream);

/* Backslash on the factorization (Algorithm IR, Sec. 1): solve A x = b.
 *   b: n values in TW; x: n values in TW (the binary64 iterate rounded to TW).
 *   term may be NULL (defaults).  rep may be NULL.
 * Returns IR_ESINGULAR / IR_ENONFINITE when the factorization failed (rep
 * then carries info), IR_ENONFINITE for a non-finite b, IR_ETIMEOUT when a
 * device wait gave up.  The refinement loop runs on the device: the call
 * enqueues term->litmax corrections at once, each followed by a one-thread
 * kernel that applies the termination test of Sec. 5.1 to the device-side
 * histories; once it has decided, the remaining corrections' kernels return
 * without work.  The call synchronizes `stream` twice: once to read the
 * factorization's outcome before enqueueing, once at the end to read the
 * loop's result.  x is not written when the call fails. */
ir_status ir_solve(ir_fact *fact, const void *b, void *x, const ir_term *term,
                   void *stream, ir_report *rep);

/* Several right-hand sides on one factorization (Sec. 6.1: the factors are
 * reused, each solve costs O(N^2)): X(:, j) = A^{-1} B(:, j) for j < nrhs,
 * each column refined by its own IR loop and termination test (as ir_solve).
 *   B: n x nrhs in TW, column-major, ldb >= n; X likewise with ldx.
 *   reps: NULL or nrhs reports.  Returns the first error of any column. */
ir_status ir_solve_many(ir_fact *fact, int64_t nrhs, const void *B, int64_t ldb, void *X, int64_t ldx,
                        const ir_term *term, void *stream, ir_report *reps);

/* End-to-end solve from HOST memory: copies A and b to the device, factors,
 * refines and copies x back.  A_host: n x n column-major in TW (lda); b_host,
 * x_host: n values in TW.  Synchronous.  Host buffers may be pageable; pinned
 * buffers copy faster.  The device buffers and the factorization (with its
 * captured launch graph) are kept by the context for the next call of the
 * same shape and options, so repeated solves pay only the copies, the
 * factorization and the refinement; ir_finalize (or a call of another shape)
 * releases them.  Not for concurrent use of one context from several threads. */
ir_status ir_solve_host(ir_ctx *ctx, int64_t n, const void *A_host, int64_t lda,
                        const void *b_host, void *x_host, const ir_opts *opts,
                        const ir_term *term, void *stream, ir_report *rep);

/* One correction solve d = U^{-1} L^{-1} P v in binary32 (eq. vdlow without
 * the scaling): v, d are n binary32 device vectors (may alias). */
ir_status ir_lu_solve(ir_fact *fact, const float *v, float *d, void *stream);

/* Check of the bounded device waits (the paper has no counterpart): one
 * thread runs the wait the correction solves use for their inter-block
 * values, on a value of the factorization's solve workspace that no solve
 * ever writes, with the time limit limit_s (0 < limit_s <= 2 s, the limit
 * every product wait uses), and must give up.  Returns IR_ETIMEOUT when the
 * wait gave up as it should (the flag is then cleared again, so the
 * factorization and its context stay usable), IR_OK if it did not, IR_EINVAL
 * for a bad limit.  Synchronizes `stream`.  For tests and diagnostics. */
ir_status ir_check_wait_timeout(ir_fact *fact, double limit_s, void *stream);

/* Residual r = b - A x in binary64 (Algorithm IR, eq. xferrule: A and b in
 * TW are promoted exactly) and rnorm[0] = ||r||_inf.  A: n x n column-major
 * in TW (IR_F64 or IR_F32) with lda; b in TW; x, r, rnorm binary64; all
 * device pointers.  Uses library workspace from ctx. */
ir_status ir_residual(ir_ctx *ctx, int64_t n, ir_dtype TW, const void *A, int64_t lda,
                      const void *b, const double *x, double *r, double *rnorm,
                      void *stream);

/* Residual without device allocation (the paper has no counterpart): the
 * same r = b - A x and rnorm[0] = ||r||_inf as ir_residual, with the same
 * argument meaning and layout, for callers that must not call cudaMalloc --
 * code inside a framework whose caching allocator owns the device memory,
 * latency-critical loops that cannot afford cudaMalloc's implicit
 * synchronisation, deployments that allow allocation only at start-up.  Its
 * workspace is a fixed array of IR_RESIDUAL_NOALLOC_SCRATCH doubles (8 MiB)
 * in the library's device image, held by every GPU that loads the library
 * until exit.  No context is needed; the current device is used.
 *   n <= IR_RESIDUAL_NOALLOC_MAX_N, else IR_EUNSUPPORTED (nothing launched).
 *   The first successful call on a device looks up the array's address (once
 *   per device, with that device current): make it before any stream capture.
 *   A failed lookup is retried by the next call.  The address is kept until
 *   exit: resetting the device or its primary context afterwards is not
 *   supported.
 *   All calls share the array: calls that overlap on the GPU race and give
 *   wrong results; calls ordered on one stream are safe (each call writes
 *   every partial sum it reads and clears rnorm itself). */
#define IR_RESIDUAL_NOALLOC_SCRATCH (1 << 20)
#define IR_RESIDUAL_NOALLOC_MAX_N (1 << 20)
ir_status ir_residual_noalloc(int64_t n, ir_dtype TW, const void *A, int64_t lda,
                              const void *b, const double *x, double *r, double *rnorm,
                              void *stream);

/* ---- Batched solves ----------------------------------------------------------
 * The paper solves one system at a time; a batch runs the same steps as
 * ir_factor + ir_solve (the cast A_F = I_W^F(s A) of Sec. 1, LU with partial
 * pivoting in TF, Algorithm IR with the termination rules of Sec. 5.1, the
 * binary16 scaling s = 2^10 / max|a_ij|) for `count` independent systems of
 * uneven size inside ONE persistent kernel launch: one CTA per SM takes the
 * systems largest first from a device-side ticket.  The solves of a batch run
 * in binary32 by column sweeps (the reference BLAS trsv order); the residual
 * in binary64.  Sizes: 0 <= n_i <= IR_BATCH_MAX_N.
 *
 * Per-system outcome, written to device memory by the launch: */
#define IR_BATCH_MAX_N 512
typedef struct {
    int32_t status;      /* ir_solve_status */
    int32_t iters;       /* residual computations */
    int64_t info;        /* first zero pivot (1-based) or 0 */
    int32_t nonfinite;   /* 1: NaN/Inf in A or b, or overflow of the rounded copy */
    int32_t timeout;     /* 1: a bounded device-side wait gave up (status IR_FAILED) */
    double rnorm;        /* ||r||_inf after the last residual (||b|| when none ran) */
    double scale;        /* s of the rounded copy */
    int32_t tf;          /* ir_dtype of the factorization that produced x (see escalation) */
    int32_t pad;
    double bnorm;        /* ||b||_inf (rhist[0]) */
} ir_batch_result;

typedef struct ir_batch ir_batch;

/* Plan a batch: check the arguments, order the systems, upload their
 * descriptors and allocate the workspace (one slot of max_i n_i^2 binary32
 * values per resident CTA).  Synchronous; allocates device memory.
 *   count >= 0; n_host[i]: sizes; A_dev[i], b_dev[i], x_dev[i]: DEVICE
 *   pointers held in HOST arrays (A_i column-major n_i x n_i in TW, b_i and
 *   x_i n_i values in TW); lda_host may be NULL (lda_i = n_i), else
 *   lda_host[i] >= max(1, n_i).  opts: TW in {F64, F32}, TF in {F32, TF32,
 *   BF16, F16}, TR = F64, nb in {0, 64}.  term may be NULL (defaults).
 * The plan BORROWS every A_i, b_i and x_i: they must stay allocated until
 * ir_batch_destroy.  A size above IR_BATCH_MAX_N gives IR_EUNSUPPORTED. */
ir_status ir_batch_create(ir_ctx *ctx, int64_t count, const int64_t *n_host,
                          const void *const *A_dev, const int64_t *lda_host,
                          const void *const *b_dev, void *const *x_dev,
                          const ir_opts *opts, const ir_term *term, ir_batch **out);

/* Run a planned batch on `stream`: a 4-byte memset and one kernel launch,
 * with no allocation and no host synchronisation, so it can be captured in
 * a CUDA graph and replayed.  results_dev: `count` ir_batch_result in device
 * memory, in the order of the plan's arrays.  x_i is written unless
 * results_dev[i].status is IR_FAILED.  Runs of one plan must not overlap
 * (they share its workspace): order them on one stream. */
ir_status ir_batch_run(ir_batch *batch, ir_batch_result *results_dev, void *stream);
void ir_batch_destroy(ir_batch *batch);

/* Precision escalation (beyond the paper, whose Sec. 3 shows binary16 IR
 * failing on ill-conditioned systems): ir_batch_run, then every member that
 * neither converged nor stopped (stagnated, or litmax) with ||r|| <= rtol ||b||
 * is solved again from scratch with TF = tf2 (IR_F32 or IR_TF32; the plan's
 * TW, term and workspace), its result and x overwritten (results_dev[i].tf
 * tells which TF produced x).  rtol >= 0 (0: keep only converged members).
 * Selection and the second pass run on the device: no allocation, no host
 * synchronisation, capturable in a CUDA graph. */
ir_status ir_batch_run_escalate(ir_batch *batch, ir_dtype tf2, double rtol, ir_batch_result *results_dev,
                                void *stream);

/* One-shot batch: ir_batch_create + ir_batch_run + synchronisation of
 * `stream` + ir_batch_destroy. */
ir_status ir_factor_solve_batched(ir_ctx *ctx, int64_t count, const int64_t *n_host,
                                  const void *const *A_dev, const int64_t *lda_host,
                                  const void *const *b_dev, void *const *x_dev,
                                  const ir_opts *opts, const ir_term *term, void *stream,
                                  ir_batch_result *results_dev);

/* ---- GMRES-IR (Sec. 4.2-4.3) ---------------------------------------------
 * Each refinement step solves its correction equation A d = r by GMRES on the
 * left-preconditioned system P A d = P r, with P = U^{-1} L^{-1} (eq. pdef),
 * instead of applying P once.  Within GMRES everything is binary64: the
 * product A v (A promoted exactly), the Krylov basis (classical Gram-Schmidt,
 * done twice), the Hessenberg matrix and its Givens rotations.  P w is applied
 * as the refinement solve is: rho = ||w||_inf, binary32 solves of
 * fl32(w / rho), scaled back by rho (and by the binary16 scale s).
 * GMRES starts from d = 0 and stops after basissize iterations, when its
 * residual estimate |g_{k+1}| <= eta ||P r||_2, or on breakdown.
 * The outer loop and its termination are those of ir_solve, except that the
 * residual-stagnation test (eq. stag) uses Rmax_r in place of term->Rmax. */
#define IR_MAX_BASIS 64

typedef struct {
    int basissize;        /* default 10 (Sec. 4.3); 1 .. IR_MAX_BASIS */
    double eta;           /* default 1e-8 */
    double Rmax_r;        /* default 1.0: stop when the residual no longer decreases */
} ir_krylov_opts;

void ir_default_krylov_opts(ir_krylov_opts *kopts);

/* mpglu (Sec. 4.4): reserve the GMRES storage of a factorization -- the
 * Krylov basis, (basissize + 2) n binary64 values, and O(basissize^2)
 * scalars -- so that ir_solve_gmres allocates nothing.  ir_solve_gmres
 * reserves on first use (synchronously) when this was not called or was
 * called with a smaller basissize.  Freed by ir_fact_destroy. */
ir_status ir_gmres_reserve(ir_fact *fact, int basissize);

/* Backslash on the GMRES-IR factorization: solve A x = b.
 *   b, x: n values in TW (device).  term, kopts may be NULL (defaults).
 *   rep may be NULL; khist (host, may be NULL) receives IR_MAX_HIST ints,
 *   khist[k] = GMRES iterations of refinement step k (Sec. 4.5), for
 *   k < rep->iters.
 * Errors as ir_solve; IR_EINVAL for basissize outside 1 .. IR_MAX_BASIS or
 * eta < 0.  Synchronizes `stream` once per refinement step. */
ir_status ir_solve_gmres(ir_fact *fact, const void *b, void *x, const ir_term *term,
                         const ir_krylov_opts *kopts, void *stream, ir_report *rep, int *khist);

/* ---- BiCGSTAB-IR (Sec. 2.3, 4.2) ------------------------------------------
 * As ir_solve_gmres, with the correction equation P A d = P r solved by
 * BiCGSTAB (van der Vorst) in binary64 from d = 0: at most kopts->basissize
 * iterations (two products P A u each), stopping when the recurrence's
 * ||r||_2 (or ||s||_2 half-way) <= eta ||P r||_2 or on breakdown (a zero
 * <r^, r>, <r^, v> or <t, t>).  khist[k] = BiCGSTAB iterations of step k.
 * ir_bicgstab_reserve (mpblu's allocation, Sec. 4.4): 8 n binary64 values. */
ir_status ir_bicgstab_reserve(ir_fact *fact);
ir_status ir_solve_bicgstab(ir_fact *fact, const void *b, void *x, const ir_term *term,
                            const ir_krylov_opts *kopts, void *stream, ir_report *rep, int *khist);

/* The autotuned schedule (opts.autotune = 1; not in the paper).
 * Single system (n >= 1024): the SMs the lookahead's trailing update leaves
 * free for the next panel's cluster, picked among 8, 12, 16, 24, 32, and for
 * TF32 / bf16 / binary16 factors the block steps per group whose update of
 * the far trailing columns is applied at once (4, 8 or 16: K = 256, 512 or
 * 1024 on the tensor cores), picked by timing two factorizations of the
 * caller's A per candidate; remembered by the context per (n, TF).  nb is 64
 * (the tensor-core K block and the panel width).  group is 1 for binary32
 * factors (every block step updates the whole trailing matrix).  Batch (TF =
 * FP16/BF16): the smallest trailing block whose update goes to the tensor
 * cores (64, 128, 192, 256 or never), picked by timing two runs of the
 * planned batch per candidate inside ir_batch_create (x is overwritten; A, b
 * only read).  grid = persistent CTAs (one per SM). */
ir_status ir_fact_schedule(const ir_fact *fact, int *nb, int *panel_reserve_sms, int *group);
ir_status ir_batch_schedule(const ir_batch *batch, int *grid, int *tc_min_trail);

/* Pivots of the factorization (0-based, n entries) copied to host memory. */
ir_status ir_fact_pivots(const ir_fact *fact, int32_t *ipiv_host);

/* The factors L (unit lower, below the diagonal) and U (upper) of P A_F =
 * L U, binary32, copied to host memory column-major with leading dimension
 * ld >= n.  Synchronizes the device. */
ir_status ir_fact_factors(const ir_fact *fact, float *LU_host, int64_t ld);

/* Status of the factorization: 0-based-free info (first zero pivot, 1-based,
 * or 0) and whether the rounded copy held a non-finite value.  Synchronizes. */
ir_status ir_fact_info(const ir_fact *fact, int64_t *info, int *nonfinite);

void ir_fact_destroy(ir_fact *fact);
const char *ir_strerror(ir_status s);

/* Text of the most recent CUDA failure seen by this thread (diagnostics). */
const char *ir_last_error(void);

/* Instrumentation (no counterpart in the paper; used by the benchmark).
 * ir_kernel_launches: number of kernels this library has launched in the
 * process.  ir_profile_start: from now on, every launcher call is bracketed by
 * a pair of CUDA events on its stream.  ir_profile_stop: synchronizes the
 * device, writes per-kind total milliseconds and call counts for kinds
 * 0 .. max_kinds-1 (names from ir_profile_kind) and returns the number of
 * kinds (0 if profiling was off, -1 on a CUDA error). */
unsigned long long ir_kernel_launches(void);
void ir_profile_start(void);
int ir_profile_stop(double *ms, int *counts, int max_kinds);
const char *ir_profile_kind(int k);

#ifdef __cplusplus
}
#endif
#endif /* GB300_IR_H */
