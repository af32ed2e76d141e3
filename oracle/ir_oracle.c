/*
 * CPU oracle for the iterative-refinement (IR) solver -- TEST INFRASTRUCTURE.
 *
 * This file is the plain, slow, obviously-correct restatement of the method of
 * Kelley, "Using MultiPrecisionArrays.jl: Iterative Refinement in Julia"
 * (Algorithm IR, Sec. 1; interprecision transfers, Sec. 5.3), used only by the
 * tests, by the build's smoke check and by the timed CPU baseline of bench.py.
 * The product (the CUDA library under paper_2311_14616_gb300/) never links,
 * calls or includes anything here, and this file shares nothing with it.
 *
 * Conventions
 *   - All matrices are column-major with a leading dimension (LAPACK layout).
 *   - Pivot vectors are 0-based: at step k, row k was interchanged with row ipiv[k].
 *   - Every fused multiply-add the method performs is written as fma()/fmaf();
 *     the file is compiled with -ffp-contract=off so that no other expression
 *     is contracted.  IEEE-754 fma and division are exactly specified, so the
 *     results are identical on every conforming host.
 *   - OpenMP only splits loops whose iterations are independent (columns of
 *     a rank-1 update, rows of a residual); every result is bitwise the same
 *     for any thread count.
 *   - dtype codes: 0 = binary64, 1 = binary32, 2 = TF32, 3 = bfloat16, 4 = binary16.
 *
 * Parity pins (see tests/test_oracle_pins.py): exact rational solves for N <= 6,
 * brute-force pivot order on tiny inputs, ||PA - LU|| / ||A|| <= 4 N u_F, the
 * rounding functions against numpy/torch conversions, the closed-form spectrum
 * of the Green's matrix, and the paper's printed residual histories.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define DT_F64 0
#define DT_F32 1
#define DT_TF32 2
#define DT_BF16 3
#define DT_F16 4

/* ------------------------------------------------------------------------ */
/* Rounding to the factorization precision TF (the copy operator I_W^F of     */
/* Sec. 1).                                                                  */
/* ------------------------------------------------------------------------ */

/* Round a double to the nearest number of a binary format with p fraction
 * bits, minimum normal exponent emin and maximum exponent emax (subnormals
 * included, overflow to +-inf).  ties_away = 0: ties to even; 1: ties away
 * from zero. */
static double round_format(double x, int p, int emin, int emax, int ties_away)
{
    if (x == 0.0 || isnan(x) || isinf(x)) return x;
    double a = fabs(x);
    int e;
    frexp(a, &e);                 /* a = m 2^e, m in [1/2, 1) */
    int E = e - 1;                /* floor(log2 a) */
    if (E < emin) E = emin;       /* subnormal range: fixed quantum */
    double q = ldexp(1.0, E - p); /* spacing of the format at a */
    double t = a / q;             /* exact: division by a power of two */
    double r = ties_away ? round(t) : nearbyint(t);
    double y = r * q;
    double maxfin = ldexp(2.0 - ldexp(1.0, -p), emax);
    if (y > maxfin) y = INFINITY;
    return copysign(y, x);
}

/* The value of x rounded to TF and held in binary32 (every TF value is a
 * binary32 number).  TF32 uses round-to-nearest, ties away from zero; bfloat16
 * and binary16 use round-to-nearest-even.  NaN is returned unchanged. */
float orc_round_tf(float x, int tf)
{
    switch (tf) {
    case DT_F32: return x;
    case DT_TF32: return (float)round_format((double)x, 10, -126, 127, 1);
    case DT_BF16: return (float)round_format((double)x, 7, -126, 127, 0);
    case DT_F16: return (float)round_format((double)x, 10, -14, 15, 0);
    default: return NAN;
    }
}

void orc_round_tf_array(int64_t n, const float *x, float *y, int tf)
{
    for (int64_t i = 0; i < n; ++i) y[i] = orc_round_tf(x[i], tf);
}

/* A_F = round_TF(fl32(s * a_ij)) for an n x n matrix A in TW (binary64 or
 * binary32), Sec. 1 (A_F = I_W^F(A)).  The product s * a_ij is formed in
 * binary64 (exact when s = 1).  Output AF is column-major with ld = ldf. */
void orc_cast(int64_t n, int tw, const void *A, int64_t lda, double s, int tf,
              float *AF, int64_t ldf)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) {
            double a = (tw == DT_F64) ? ((const double *)A)[i + j * lda]
                                      : (double)((const float *)A)[i + j * lda];
            AF[i + j * ldf] = orc_round_tf((float)(s * a), tf);
        }
}

/* max_ij |a_ij| in binary64 (the FP16 scaling of the factorization copy). */
double orc_maxabs(int64_t n, int tw, const void *A, int64_t lda)
{
    double m = 0.0;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) {
            double a = (tw == DT_F64) ? ((const double *)A)[i + j * lda]
                                      : (double)((const float *)A)[i + j * lda];
            if (fabs(a) > m || isnan(a)) m = isnan(a) ? a : fabs(a);
        }
    return m;
}

/* ------------------------------------------------------------------------ */
/* LU factorization with partial pivoting ("Factor A = LU in precision TF",  */
/* Algorithm IR; lu! in Sec. 2.1.1).                                          */
/* ------------------------------------------------------------------------ */

/* Unblocked right-looking LU with partial pivoting in binary64.
 * Step k: p = first row i >= k with maximal |a_ik|; interchange rows k and p
 * across all columns; scale the column the way LAPACK's getf2 does (which is
 * what Julia's lu! runs for binary32/binary64 matrices): l_ik = a_ik * fl(1/a_kk)
 * when |a_kk| is at least the smallest normal number, l_ik = a_ik / a_kk
 * otherwise; then a_ij = a_ij - l_ik a_kj for i, j > k.
 * A zero pivot is recorded (1-based, first one) in the return value and the
 * column is left unscaled (its entries below the diagonal are all zero). */
int64_t orc_getrf_f64(int64_t n, double *A, int64_t lda, int32_t *ipiv)
{
    int64_t info = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = k;
        double amax = fabs(A[k + k * lda]);
        for (int64_t i = k + 1; i < n; ++i)
            if (fabs(A[i + k * lda]) > amax) { amax = fabs(A[i + k * lda]); p = i; }
        ipiv[k] = (int32_t)p;
        if (p != k)
            for (int64_t j = 0; j < n; ++j) {
                double t = A[k + j * lda]; A[k + j * lda] = A[p + j * lda]; A[p + j * lda] = t;
            }
        double akk = A[k + k * lda];
        if (akk == 0.0) { if (!info) info = k + 1; continue; }
        if (fabs(akk) >= DBL_MIN) {
            const double r = 1.0 / akk;
            for (int64_t i = k + 1; i < n; ++i) A[i + k * lda] = A[i + k * lda] * r;
        } else {
            for (int64_t i = k + 1; i < n; ++i) A[i + k * lda] = A[i + k * lda] / akk;
        }
#pragma omp parallel for schedule(static)
        for (int64_t j = k + 1; j < n; ++j) {
            double u = A[k + j * lda];
            for (int64_t i = k + 1; i < n; ++i)
                A[i + j * lda] = fma(-A[i + k * lda], u, A[i + j * lda]);
        }
    }
    return info;
}

/* One pivot step of the binary32 factorization: choose the pivot row for
 * column k among rows k..n-1 (first maximal |a_ik|, or the forced row when
 * force >= 0), record max / runner-up / chosen magnitudes, interchange whole
 * rows, and scale column k as LAPACK's getf2 does (reciprocal of the pivot,
 * plain division below the smallest normal).  Returns the chosen row. */
static int64_t pivot_step_f32(int64_t n, float *A, int64_t lda, int64_t k,
                              int32_t force, float *gap, int64_t *info)
{
    int64_t p = k;
    float amax = fabsf(A[k + k * lda]);
    for (int64_t i = k + 1; i < n; ++i)
        if (fabsf(A[i + k * lda]) > amax) { amax = fabsf(A[i + k * lda]); p = i; }
    float second = -1.0f;
    for (int64_t i = k; i < n; ++i)
        if (i != p && fabsf(A[i + k * lda]) > second) second = fabsf(A[i + k * lda]);
    if (force >= 0) p = force;
    if (gap) { gap[3 * k] = amax; gap[3 * k + 1] = second; gap[3 * k + 2] = fabsf(A[p + k * lda]); }
    if (p != k)
        for (int64_t j = 0; j < n; ++j) {
            float t = A[k + j * lda]; A[k + j * lda] = A[p + j * lda]; A[p + j * lda] = t;
        }
    float akk = A[k + k * lda];
    if (akk == 0.0f) { if (!*info) *info = k + 1; return p; }
    if (fabsf(akk) >= FLT_MIN) {           /* LAPACK getf2: scale by the reciprocal */
        const float r = 1.0f / akk;
        for (int64_t i = k + 1; i < n; ++i) A[i + k * lda] = A[i + k * lda] * r;
    } else {
        for (int64_t i = k + 1; i < n; ++i) A[i + k * lda] = A[i + k * lda] / akk;
    }
    return p;
}

/* LU with partial pivoting of the factorization copy A_F (binary32 storage).
 *
 * tf = binary32: the unblocked right-looking algorithm of orc_getrf_f64 in
 * binary32, every update a_ij = fmaf(-l_ik, u_kj, a_ij) with k ascending.
 *
 * tf in {TF32, bfloat16, binary16}: the mixed-precision LU that runs the
 * trailing update on tensor cores with binary32 accumulation.  Columns are
 * taken in blocks of nb.  For the block starting at column j:
 *   1. the panel A[j:n, j:j+nb] is factored by the binary32 unblocked steps
 *      (interchanges applied to whole rows);
 *   2. U12 = L11^{-1} A12 by binary32 forward substitution, each entry an
 *      fmaf chain in ascending column order;
 *   3. A22_ic <- fl32( A22_ic - fl32( sum_m rTF(l_im) rTF(u_mc) ) ), where
 *      rTF rounds to TF and the sum of the (exact) products is accumulated
 *      left to right in binary64.
 *
 * force_piv (may be NULL): force_piv[k] >= 0 makes step k take that row.
 * gap (may be NULL, 3n floats): per step the largest candidate magnitude, the
 * runner-up and the magnitude of the row taken.  Returns info (1-based first
 * zero pivot, or 0). */
int64_t orc_getrf_tf(int64_t n, float *A, int64_t lda, int32_t *ipiv, int tf,
                     int64_t nb, const int32_t *force_piv, float *gap)
{
    int64_t info = 0;
    if (tf == DT_F32 || nb <= 0) nb = n > 0 ? n : 1;
    for (int64_t j = 0; j < n; j += nb) {
        int64_t jb = (n - j < nb) ? n - j : nb;
        int64_t je = j + jb;
        /* 1. panel */
        for (int64_t k = j; k < je; ++k) {
            int64_t p = pivot_step_f32(n, A, lda, k, force_piv ? force_piv[k] : -1, gap, &info);
            ipiv[k] = (int32_t)p;
#pragma omp parallel for schedule(static)
            for (int64_t c = k + 1; c < je; ++c) {
                float u = A[k + c * lda];
                for (int64_t i = k + 1; i < n; ++i)
                    A[i + c * lda] = fmaf(-A[i + k * lda], u, A[i + c * lda]);
            }
        }
        if (je >= n) break;
        /* 2. U12 = L11^{-1} A12 */
#pragma omp parallel for schedule(static)
        for (int64_t c = je; c < n; ++c)
            for (int64_t k = j; k < je; ++k)
                for (int64_t m = j; m < k; ++m)
                    A[k + c * lda] = fmaf(-A[k + m * lda], A[m + c * lda], A[k + c * lda]);
        /* 3. A22 -= rTF(L21) rTF(U12): the operands are rounded once per block */
        {
            const int64_t m = n - je;
            double *rl = (double *)malloc(sizeof(double) * (size_t)m * (size_t)jb);   /* rl[i][k] */
            double *ru = (double *)malloc(sizeof(double) * (size_t)m * (size_t)jb);   /* ru[c][k] */
            if (!rl || !ru) { free(rl); free(ru); return -1; }
            for (int64_t i = 0; i < m; ++i)
                for (int64_t k = 0; k < jb; ++k) {
                    rl[i * jb + k] = (double)orc_round_tf(A[(je + i) + (j + k) * lda], tf);
                    ru[i * jb + k] = (double)orc_round_tf(A[(j + k) + (je + i) * lda], tf);
                }
#pragma omp parallel for schedule(static)
            for (int64_t c = 0; c < m; ++c)
                for (int64_t i = 0; i < m; ++i) {
                    double acc = 0.0;
                    for (int64_t k = 0; k < jb; ++k) acc += rl[i * jb + k] * ru[c * jb + k];
                    A[(je + i) + (je + c) * lda] = A[(je + i) + (je + c) * lda] - (float)acc;
                }
            free(rl);
            free(ru);
        }
    }
    return info;
}

/* ------------------------------------------------------------------------ */
/* Triangular solves d = U^{-1} L^{-1} P v (Algorithm IR; eq. vdlow).         */
/* ------------------------------------------------------------------------ */

/* binary32: interchanges of ipiv applied in order, then the two triangular
 * solves in the order of the reference BLAS trsv for a column-major matrix
 * (the solve LAPACK getrs performs):
 *   forward, unit lower L: for j ascending, v_i -= l_ij v_j for all i > j;
 *   back, U: for j descending, v_j /= u_jj, then v_i -= u_ij v_j for all i < j.
 * Each entry therefore sees its updates in ascending j (forward) and in
 * descending j (back), each a single-rounding fma. */
void orc_getrs_f32(int64_t n, const float *LU, int64_t lda, const int32_t *ipiv, float *v)
{
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = ipiv[k];
        if (p != k) { float t = v[k]; v[k] = v[p]; v[p] = t; }
    }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j + 1; i < n; ++i) v[i] = fmaf(-LU[i + j * lda], v[j], v[i]);
    for (int64_t j = n - 1; j >= 0; --j) {
        v[j] = v[j] / LU[j + j * lda];
        for (int64_t i = 0; i < j; ++i) v[i] = fmaf(-LU[i + j * lda], v[j], v[i]);
    }
}

/* The same solve in binary64 (the plain double-precision LU solve). */
void orc_getrs_f64(int64_t n, const double *LU, int64_t lda, const int32_t *ipiv, double *v)
{
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = ipiv[k];
        if (p != k) { double t = v[k]; v[k] = v[p]; v[p] = t; }
    }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j + 1; i < n; ++i) v[i] = fma(-LU[i + j * lda], v[j], v[i]);
    for (int64_t j = n - 1; j >= 0; --j) {
        v[j] = v[j] / LU[j + j * lda];
        for (int64_t i = 0; i < j; ++i) v[i] = fma(-LU[i + j * lda], v[j], v[i]);
    }
}

/* ------------------------------------------------------------------------ */
/* Residual r = b - A x in the residual precision TR = binary64              */
/* (Algorithm IR; eq. xferrule: A in TW is promoted exactly).                */
/* ------------------------------------------------------------------------ */

/* r_i = b_i - s_i with s_i = sum_j a_ij x_j accumulated as the fma chain
 * s = fma(a_ij, x_j, s), j ascending (the order of a column-oriented matrix-
 * vector product; with it the oracle reproduces the residual histories the
 * paper prints digit for digit). */
void orc_residual(int64_t n, int tw, const void *A, int64_t lda, const double *b,
                  const double *x, double *r)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        if (tw == DT_F64) {
            const double *a = (const double *)A;
            for (int64_t j = 0; j < n; ++j) s = fma(a[i + j * lda], x[j], s);
        } else {
            const float *a = (const float *)A;
            for (int64_t j = 0; j < n; ++j) s = fma((double)a[i + j * lda], x[j], s);
        }
        r[i] = b[i] - s;
    }
}

/* The residual in the host's long double (x86: 64-bit significand; aarch64:
 * binary128), rounded to binary64 at the end.  Used to refine the binary64
 * reference solution x_ref to which every result's error is referred. */
void orc_residual_ext(int64_t n, int tw, const void *A, int64_t lda, const double *b,
                      const double *x, double *r)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        long double s = 0.0L;
        if (tw == DT_F64) {
            const double *a = (const double *)A;
            for (int64_t j = 0; j < n; ++j) s += (long double)a[i + j * lda] * (long double)x[j];
        } else {
            const float *a = (const float *)A;
            for (int64_t j = 0; j < n; ++j) s += (long double)a[i + j * lda] * (long double)x[j];
        }
        r[i] = (double)((long double)b[i] - s);
    }
}
