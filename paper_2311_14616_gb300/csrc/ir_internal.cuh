// Internal declarations of the GB300 iterative-refinement library.
//
// Data layout in HBM (per factorization handle):
//   A      caller's working-precision matrix, column-major, borrowed (residual)
//   AF     factorization copy, binary32, ROW-major with padded row stride ldf
//          (row interchanges move contiguous rows; a panel row is contiguous)
//   Aop    rTF(L21) of the current block step, row-major (K contiguous), TF dtype
//   Bop    rTF(U12)^T of the current block step, row-major (K contiguous)
//   Linv/Uinv  inverses of the 128x128 diagonal blocks of L and U (row-major)
//   x      binary64 iterate (TR), r binary64 residual, y binary32 solve vector
//   dev    small block of device scalars (norms as ordered bit patterns, flags)
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include "../../include/ir.h"

namespace ir {

constexpr int kTrsvB = 128;       // row block of the triangular solves
constexpr int kPanelNB = 64;      // panel width = outer block size
constexpr int kPanelRows = 512;   // panel rows per CTA (two per thread)
constexpr int kPanelThreads = 256;
constexpr int kPanelMaxCluster = 16;
constexpr int kPanelMaxGrid = 152;  // CTAs of a panel taller than one cluster (one per SM, all resident)
constexpr int kPanelGridCounters = kPanelNB + 1;   // arrival counters of such a panel: one per column + one
constexpr int kPanelGridRec = 68;   // floats per exchanged pivot-candidate record
constexpr int kMaxN = kPanelRows * kPanelMaxGrid;  // 77824 rows: the tallest panel
constexpr int kMpsB = 64;         // row block of the mixed precision (binary64) solves
constexpr int kMaxGroup = 16;     // block steps per group of the tensor-core LU (64 x 16 = 1024 columns)

// Device-side scalars.  Non-negative doubles are ordered like their bit
// patterns, so maxima are kept with atomicMax on uint64 (deterministic).
struct DevScalars {
    unsigned long long rnorm_bits;   // ||r||_inf of the latest residual
    unsigned long long dnorm_bits;   // ||d||_inf of the latest correction
    unsigned long long xnorm_bits;   // ||x||_inf after the latest update (cleared with dnorm_bits)
    unsigned long long bnorm_bits;   // ||b||_inf
    unsigned long long amax_bits;    // max |a_ij| (binary16 scaling)
    unsigned long long anorm_bits;   // ||A||_1 (backward-error termination)
    double scale;                    // s of the factorization copy
    int info;                        // first zero pivot, 1-based (INT_MAX = none)
    int nonfinite;                   // 1: NaN/Inf met in A, b or the rounded copy
    int timeout;                     // 1: a bounded wait gave up
    int pad;
    unsigned long long one_bits;     // 1.0: the unit scale of mixed precision solves with TW = binary32
    unsigned int ticket[2];          // CTA ticket counters of the two solves
};

// State of one refinement loop run on the device (ir_solve): the termination
// test of Sec. 5.1 is evaluated by a one-thread kernel after every residual, so
// a whole solve is enqueued at once and the host reads this back at the end.
struct SolveLoop {
    int status;      // -1 while refining, else an ir_solve_status
    int k;           // corrections applied
    int done;        // 1: the remaining iterations' kernels return at once
    int err;         // 0, kLoopNonfinite (b or ||A||_1 not finite) or kLoopTimeout
    double rhist[IR_MAX_HIST];
    double dhist[IR_MAX_HIST];
};
constexpr int kLoopNonfinite = 1, kLoopTimeout = 2;

// The termination test's parameters (ir_term with the precision's unit roundoff).
struct TermArgs {
    double Cr, Ce, Rmax, abs_rel_tol, eps_w, rmax_r;
    int litmax, mode, tr_wider;
};

// Termination test of Sec. 5.1 after the k-th residual (rh[0..k], dh[0..k-1]):
// -1 to continue, else an ir_solve_status.  rmax_r: the factor of the
// residual-stagnation test.  With mode = 1 the small-residual test is the
// backward-error test (eq. term), anorm = ||A||_1, xnorm = ||x||_inf.  Every
// product and sum is rounded on its own (no fused multiply-add), so host and
// device decide alike.
__host__ __device__ inline double term_mul(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    volatile double p = a * b;
    return p;
#endif
}
__host__ __device__ inline double term_add(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dadd_rn(a, b);
#else
    volatile double q = a + b;
    return q;
#endif
}
__host__ __device__ inline int term_rule(const double *rh, const double *dh, int k, double bnorm,
                                         const TermArgs &t, double anorm, double xnorm) {
    const double rn = rh[k];
    if (!isfinite(rn)) return IR_DIVERGED;
    if (rn == 0.0) return IR_CONVERGED;    // exact solution: r / ||r|| (eq. vdlow) is undefined next
    if (t.tr_wider) {
        if (k >= 2 && dh[k - 1] >= term_mul(t.Rmax, dh[k - 2])) return IR_STAGNATED;   // eq. (wilkterm)
    } else {
        if (t.mode == 1) {
            const double be = term_mul(term_mul(t.Ce, t.eps_w), term_add(bnorm, term_mul(anorm, xnorm)));
            if (rn <= be) return IR_CONVERGED;                                        // eq. (term)
        } else {
            const double tol = t.abs_rel_tol > 0 ? t.abs_rel_tol : term_mul(t.Cr, t.eps_w);
            if (rn <= term_mul(tol, bnorm)) return IR_CONVERGED;                      // eq. (residterm)
        }
        if (k >= 1 && rn >= term_mul(t.rmax_r, rh[k - 1])) return IR_STAGNATED;       // eq. (stag)
    }
    if (k >= t.litmax) return IR_MAXIT;
    return -1;
}

// Scalars of a block of up to 4 right-hand sides refined together (ir_solve_many).
struct MultiScalars {
    unsigned long long rho[4];     // ||r_j||_inf (the scale of the next solve, then rhist)
    unsigned long long dnorm[4];   // ||d_j||_inf of the latest correction
    unsigned long long xnorm[4];   // ||x_j||_inf after it
    int active[4];                 // 1: column j is still refined
};

// GMRES state of one correction solve (device memory, written by the
// orthogonalization kernel's first CTA).  R is the Hessenberg matrix after the
// Givens rotations (upper triangular, column-major with leading dimension
// kMaxBasis), g the rotated right-hand side beta e_1.
constexpr int kMaxBasis = 64;
struct GmState {
    double beta;                        // ||P r||_2
    double g[kMaxBasis + 1];
    double cs[kMaxBasis], sn[kMaxBasis];
    double R[kMaxBasis * kMaxBasis];
    unsigned long long wnorm_bits;      // ||A v_j||_inf of the latest product
    int k;                              // GMRES iterations taken
    int done;                           // 1: the remaining iterations are skipped
};

// BiCGSTAB state of one correction solve (device memory).  The vectors live in
// the columns of the Krylov workspace: r, r^, p, v, s, t, d.
enum { kBiR = 0, kBiRh, kBiP, kBiV, kBiS, kBiT, kBiD, kBiCols };
struct BiState {
    double rho_old, rho, alpha, omega, z0;
    unsigned long long wnorm_bits;      // ||A p||_inf or ||A s||_inf of the latest product
    int k;                              // iterations taken
    int done;
};

}  // namespace ir

// Tuned factorization schedules, per (n, TF), kept by the context.
struct ir_tuned {
    int64_t n;
    int tf;
    int reserve_sms;
    int group;
};

struct ir_ctx {
    int device;
    int sms;
    ir_tuned tuned[16];      // ring of tuned schedules
    int ntuned;
    // ir_solve_host's device buffers and factorization, kept for the next
    // call of the same shape (released by ir_finalize or a different shape)
    struct ir_fact *host_f;
    void *host_dA, *host_db, *host_dx;
    int64_t host_n, host_lda;
    int host_tw, host_tf, host_scale, host_autotune;
    double *partials;        // residual split-K partial sums
    int64_t partials_cap;    // capacity in doubles
    double *rnorm_tmp;       // scratch scalar for ir_residual
};

struct ir_fact {
    ir_ctx *ctx;
    int64_t n;
    ir_dtype TW, TF, TR;
    int fp16_scale;
    int nb;
    int reserve_sms;         // SMs the trailing update leaves to the next panel's cluster (schedule)
    const void *A;
    int64_t lda;
    int64_t ldf;             // row stride of AF in floats (multiple of 32)
    float *AF;
    int32_t *ipiv;           // 0-based pivots
    int32_t *perm;           // (P A)[i] = A[perm[i]]
    int32_t *swap_list;      // 2 kMaxGroup x (1 + 2*2*NB) ints: count, then (dst, src) pairs, by step
    void *Aop, *Bop;         // tensor-core operands, 2 buffers each by step parity (NULL for TF = F32)
    int group;               // block steps per group of the tensor-core LU (far columns updated once per group)
    int onthefly;            // 1: mixed precision solves (Sec. 5.3) in ir_solve
    int store_tf;            // 1: factors kept in TF (2-byte copy AF16 read by the solves)
    void *AF16;
    // several right-hand sides refined together (ir_solve_many): 4 columns of x, r
    // and b (padded), the tagged solve words, the per-column scalars
    double *xm, *rm;
    void *bm;
    unsigned long long *mtags;
    ir::MultiScalars *mscal, *host_mscal;
    double *y64, *z64;       // MPS solve vectors (ceil(n / kMpsB) * kMpsB binary64 each; TW = binary64)
    int *mps_flags;          // MPS per-block publication flags (2 ceil(n / kMpsB))
    void *Agrp, *Bgrp;       // a group's operands: group x n rows x 64 (rTF of its L columns / U rows)
    cudaStream_t la_stream;  // low-priority stream of the lookahead schedule
    cudaEvent_t *la_events;  // fork/join events of the lookahead schedule
    int la_nevents;
    float *Linv, *Uinv;      // diagonal-block inverses, nblk x B x B (B = kTrsvB)
    int32_t *blk_subst;      // 2 x nblk: 1 = solve this diagonal block by substitution (ill-conditioned)
    unsigned long long *tags;  // 2 x nblk*64 tagged solve values (epoch << 32 | bits)
    unsigned epoch;            // tag of the latest solve
    double *x, *r;           // binary64 iterate and residual
    ir::DevScalars *dev;
    int anorm_valid;         // dev->anorm_bits holds ||A||_1 of the current A
    ir::DevScalars *host_dev;  // pinned mirror
    ir::SolveLoop *loop;       // device-side refinement loop of ir_solve
    float *panel_grec;         // pivot records of panels taller than one cluster (n > 8192)
    unsigned *panel_gcnt;      // and their arrival counters
    ir::SolveLoop *host_loop;  // pinned mirror
    // the factorization's launch sequence as a CUDA graph (captured for one A)
    cudaStream_t cap_stream;
    cudaGraphExec_t graph;
    const void *graph_A;
    int64_t graph_lda;
    unsigned long long graph_launches;  // kernels in the graph
    // GMRES-IR workspace (reserved on demand): Krylov basis V (gm_m + 1
    // columns of gm_ldv binary64), the product buffer W, the GMRES state
    int gm_m;
    int64_t gm_ldv;
    double *gm_V, *gm_W;
    ir::GmState *gm_st;
    int *gm_host_k;          // pinned mirror of gm_st->k
    // BiCGSTAB-IR workspace (reserved on demand): kBiCols columns of gm_ldv
    // binary64 and the state
    double *bi_V;
    ir::BiState *bi_st;
};

namespace ir {

// ---- launch accounting and optional per-launcher event timing --------------
void count_launch();                       // one call per kernel launch
void count_launches(unsigned long long k);  // k kernels launched at once (a graph replay)
unsigned long long launches();
// Record a failed CUDA call for ir_last_error() and map it to IR_ENOMEM / IR_ECUDA.
ir_status record_cuda_error(cudaError_t e, const char *what);

// ---- launchers (each returns the launch error) -----------------------------
cudaError_t launch_maxabs(int64_t n, ir_dtype tw, const void *A, int64_t lda, DevScalars *dev,
                          int sms, cudaStream_t s);
cudaError_t launch_cast(int64_t n, ir_dtype tw, const void *A, int64_t lda, ir_dtype tf,
                        int use_scale, float *AF, int64_t ldf, DevScalars *dev, cudaStream_t s);
cudaError_t launch_norm1(int64_t n, ir_dtype tw, const void *A, int64_t lda, unsigned long long *out_bits,
                         cudaStream_t s);
cudaError_t launch_init_rb(int64_t n, ir_dtype tw, const void *b, double *r, double *x,
                           DevScalars *dev, cudaStream_t s);
cudaError_t launch_store_x(int64_t n, ir_dtype tw, const double *x, void *out, cudaStream_t s,
                           const int *skip = nullptr);
// The device-side refinement loop (k_resid.cu): loop_start after x = 0, r = b
// (rhist[0] = ||b||, the flags of b and ||A||_1); loop_step after each residual
// (appends ||d||, ||r||, decides, clears ||d|| and ||x|| for the next step).
cudaError_t launch_loop_start(DevScalars *dev, SolveLoop *loop, const TermArgs &t, cudaStream_t s);
cudaError_t launch_loop_step(DevScalars *dev, SolveLoop *loop, const TermArgs &t, cudaStream_t s);

// Panel of the block step at column j.  Panels taller than one cluster holds
// (more than kPanelRows * kPanelMaxCluster rows) exchange their pivot records
// through grec (2 * kPanelMaxGrid * kPanelGridRec floats) and the counters gcnt
// (kPanelGridCounters, zeroed here) in one cooperative launch.
cudaError_t launch_panel(float *AF, int64_t ldf, int n, int j, int nbp, int32_t *ipiv,
                         int32_t *perm, int32_t *swap_list, DevScalars *dev, ir_dtype tf,
                         void *Aop, cudaStream_t s, float *grec = nullptr, unsigned *gcnt = nullptr);
cudaError_t launch_laswp(float *AF, int64_t ldf, int c0a, int c1a, int c0b, int c1b,
                         const int32_t *swap_list, cudaStream_t s);
// The interchange lists first .. first + count - 1 (of a ring of `ring` lists of
// list_ints ints) applied in order to the columns [c0, c1).
cudaError_t launch_laswp_lists(float *AF, int64_t ldf, int c0, int c1, const int32_t *lists, int list_ints, int ring,
                               int first, int count, cudaStream_t s);
cudaError_t launch_trsm(float *AF, int64_t ldf, int cb, int ce, int j, ir_dtype tf, void *Bop,
                        cudaStream_t s);
// The panel's row interchanges on the columns [cb, ce), then their U12 (one launch).
cudaError_t launch_laswp_trsm(float *AF, int64_t ldf, int cb, int ce, int j, ir_dtype tf, void *Bop,
                              const int32_t *swap_list, cudaStream_t s);
cudaError_t launch_gemm_simt(float *AF, int64_t ldf, int n, int j, int nb, int cb, int ce,
                             int max_ctas, cudaStream_t s);
cudaError_t launch_gemm_tc(float *AF, int64_t ldf, int n, int j, int nb, int cb, int ce,
                           ir_dtype tf, const void *Aop, const void *Bop, int sms, int max_ctas,
                           DevScalars *dev, cudaStream_t s);
// Group update of the tensor-core LU: rows [r0, r1) x columns [cb, ce) of A_F
// minus the products of slots [s0, s1) of the group operands (k_gemm_tc.cu).
cudaError_t launch_gemm_tc_group(float *AF, int64_t ldf, int c0, int G, int r0, int r1, int cb, int ce,
                                 int s0, int s1, ir_dtype tf, const void *Agrp, int64_t a_rows, const void *Bgrp,
                                 int64_t b_rows, int bbase, int sms, int max_ctas, DevScalars *dev,
                                 cudaStream_t s);
// U12 of the group of G block rows starting at c0 for the columns [cb, ce), with
// the group's own block steps between them on the tensor cores (k_gemm_tc.cu): L
// from the packed slots Agrp (a_rows rows each), rTF(U) of block t into slot t of
// Bgrp (b_rows rows each, row c - bbase for column c).
cudaError_t launch_u12_group_tc(float *AF, int64_t ldf, int c0, int G, int cb, int ce, ir_dtype tf,
                                const void *Agrp, int64_t a_rows, void *Bgrp, int64_t b_rows, int bbase,
                                DevScalars *dev, cudaStream_t s);
// rTF of the factor columns [c0, c0 + 64 G), rows [r0, r1), into G slots of `rows` rows.
cudaError_t launch_pack_slots(const float *AF, int64_t ldf, int c0, int G, int r0, int r1, int64_t rows, ir_dtype tf,
                              void *out, int sms, cudaStream_t s);
cudaError_t launch_iota(int n, int32_t *perm, cudaStream_t s);

cudaError_t launch_diag_inv(const float *AF, int64_t ldf, int n, float *Linv, float *Uinv,
                            int32_t *blk_subst, cudaStream_t s);
// Solve pair in one of three modes:
//   refinement (vin = pw = NULL): x += (||r|| s) fl64(U^{-1} L^{-1} fl32(P r / ||r||)), ||d||, ||x|| into dev;
//   raw (vin != NULL): dout = U^{-1} L^{-1} P vin in binary32;
//   preconditioner (pw != NULL): pw = (rho s) fl64(U^{-1} L^{-1} fl32(P r / rho)), rho from rho_bits.
// skip != NULL: every CTA returns at once while *skip != 0.
cudaError_t launch_trsv_pair(const float *AF, int64_t ldf, int n, const float *Linv,
                             const float *Uinv, const int32_t *blk_subst, const int32_t *perm, const double *r,
                             const float *vin, float *dout, double *x,
                             unsigned long long *tags, unsigned epoch, DevScalars *dev,
                             cudaStream_t s, const unsigned long long *rho_bits = nullptr,
                             double *pw = nullptr, const int *skip = nullptr, bool unit_rho = false,
                             const void *F16 = nullptr, ir_dtype tf16 = IR_F32);
// Several right-hand sides (4 columns; k_trsv.cu, k_resid.cu): the correction
// solve pair applying each factor tile to all columns, and the residual reading
// A once for all of them.  Column j: R + j ldr, X + j ldx, rho_bits[j], ...;
// tags: 2 x 4 x nblk*128 words.
constexpr int kMultiRhs = 4;
cudaError_t launch_trsv_multi(const float *AF, int64_t ldf, int n, const float *Linv, const float *Uinv,
                              const int32_t *blk_subst, const int32_t *perm, const double *R, int64_t ldr,
                              const unsigned long long *rho_bits, const int *active, double *X, int64_t ldx,
                              unsigned long long *dnorm_bits, unsigned long long *xnorm_bits,
                              unsigned long long *tags, unsigned epoch, DevScalars *dev, cudaStream_t s,
                              const void *F16, ir_dtype tf16);
cudaError_t launch_residual_multi(int64_t n, ir_dtype tw, const void *A, int64_t lda, const void *Bm, int64_t ldb,
                                  const double *X, int64_t ldx, double *R, int64_t ldr, double *partials,
                                  int64_t partials_cap, unsigned long long *rnorm_bits, int sms, cudaStream_t s);
// The factors kept in TF (binary16 / bfloat16): A_F rounded in place and copied
// to the 2-byte array F16 (row stride ldf); overflow raises dev->nonfinite.
cudaError_t launch_store_tf(float *AF, int64_t ldf, int n, ir_dtype tf, void *F16, DevScalars *dev, int sms,
                            cudaStream_t s);
// Mixed precision solve pair (k_trsv64.cu): x += s U^{-1} L^{-1} P r in binary64,
// blocks of kMpsB rows
// on the binary32 factors; ||d||, ||x|| into dev.
cudaError_t launch_mps_pair(const float *AF, int64_t ldf, int n, const int32_t *perm, const double *r, double *x,
                            double *y64, double *z64, int *flags, unsigned tag, DevScalars *dev, cudaStream_t s,
                            const int *skip = nullptr);
// One thread runs the solves' bounded tag wait on tags[0] for a tag that is
// never written, with the limit limit_ns; it sets *timeout when it gives up.
cudaError_t launch_wait_probe(const unsigned long long *tags, unsigned tag, unsigned long long limit_ns,
                              int *timeout, cudaStream_t s);
// r = b - A x (b == NULL: r = A x) and ||r||_inf into rnorm_bits; skip as above.
cudaError_t launch_residual(int64_t n, ir_dtype tw, const void *A, int64_t lda, const void *b,
                            const double *x, double *r, double *partials, int64_t partials_cap,
                            unsigned long long *rnorm_bits, int sms, cudaStream_t s,
                            const int *skip = nullptr);

// GMRES (k_krylov.cu).  j = -1: v_0 = V_0 / ||V_0||_2, beta, g = beta e_1.
// j >= 0: orthogonalize V_{j+1} = P A v_j against v_0..v_j (classical
// Gram-Schmidt twice), normalize, rotate column j of H, set done.
cudaError_t launch_gm_orth(int n, double *V, int64_t ldv, int j, int m, double eta, GmState *st,
                           cudaStream_t s);
// BiCGSTAB phases (k_krylov.cu): 0 start (r^ = r = z, ||z||_2), 1 rho and p,
// 2 alpha and s (after v = M p), 3 omega, d and r (after t = M s).
cudaError_t launch_bi_step(int phase, int n, double *Vb, int64_t ldv, int kmax, double eta, BiState *st,
                           cudaStream_t s);
// x += d; ||d||_inf, ||x||_inf.
cudaError_t launch_axpy_norms(int n, const double *d, double *x, unsigned long long *dnorm_bits,
                              unsigned long long *xnorm_bits, cudaStream_t s);
// d = V_k R^{-1} g; x += d; ||d||_inf into dnorm_bits, ||x||_inf into xnorm_bits.
cudaError_t launch_gm_update(int n, const double *V, int64_t ldv, const GmState *st, double *x,
                             unsigned long long *dnorm_bits, unsigned long long *xnorm_bits, cudaStream_t s);
int64_t residual_partials_needed(int64_t n, int sms);

// batched driver (many systems with n <= IR_BATCH_MAX_N, one persistent launch)
size_t batch_desc_bytes();
void batch_fill_desc(void *desc, int64_t i, const void *A, int64_t lda, const void *b, void *x, int n);
cudaError_t batch_grid(int sms, int64_t count, int *grid);
cudaError_t launch_batched(const void *sys, const int *order, int64_t count, unsigned *ticket, float *ws,
                           int64_t ws_stride, int grid, ir_dtype tw, ir_dtype tf, int fp16_scale,
                           const ir_term *t, int tc_min_trail, ir_batch_result *results, cudaStream_t s,
                           const unsigned *dcount = nullptr);
cudaError_t launch_select_unconverged(const ir_batch_result *results, const int *order, int64_t count,
                                      double rtol, int *order2, unsigned *count2, cudaStream_t s);

// ---- device helpers --------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// cuTensorMapEncodeTiled, reached through the runtime's driver entry point
// (the library links only the CUDA runtime).
typedef CUresult (*TensorMapEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                      const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                      CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                      CUtensorMapFloatOOBfill);
inline TensorMapEncodeFn tensor_map_encoder() {
    static TensorMapEncodeFn fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<TensorMapEncodeFn>(ptr);
    }
    return fn;
}

// Programmatic dependent launch: a kernel launched with set_pdl() may be
// scheduled while its predecessor on the stream is still running; it lets its
// own successor launch at once (pdl_trigger) and waits for the predecessor's
// completion and memory (pdl_wait) before it reads anything.  Both are no-ops
// for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
inline bool pdl_enabled() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("IR_NO_PDL");
        v = !(e && e[0] && e[0] != '0');
    }
    return v != 0;
}
// Fill a launch attribute for programmatic dependent launch; returns the number
// of attributes written (0 when disabled).
inline unsigned set_pdl(cudaLaunchAttribute *a) {
    if (!pdl_enabled()) return 0;
    a->id = cudaLaunchAttributeProgrammaticStreamSerialization;
    a->val.programmaticStreamSerializationAllowed = 1;
    return 1;
}

// ---- thread-block cluster helpers -------------------------------------------
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}
__device__ __forceinline__ unsigned map_cta(unsigned local_addr, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_addr), "r"(rank));
    return r;
}

// 16-byte store into another CTA's shared memory, counted (complete_tx) on that
// CTA's mbarrier; the receiver's acquire of the mbarrier phase makes it visible.
__device__ __forceinline__ void st_async_v4(unsigned rdst, float4 v, unsigned rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(rdst),
                 "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
                 "r"(__float_as_uint(v.w)), "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ void mbar_init_p(unsigned addr, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_arrive(unsigned addr, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(addr),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(unsigned addr, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}


// Bounded wait limit for inter-CTA flags (nanoseconds).
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *p, double v) {
    // |v| >= 0 (or NaN with the sign cleared): bit patterns order like values
    atomicMax(p, static_cast<unsigned long long>(__double_as_longlong(fabs(v))));
}

}  // namespace ir
