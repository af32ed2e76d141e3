// Residual r = b - A x in binary64 (Algorithm IR, residual in TR; eq. xferrule:
// A and b in TW are promoted exactly) and ||r||_inf; with b = NULL the same
// kernels form the product A x (the high-precision matrix-vector product of
// GMRES-IR, Sec. 4.3).
//
// Pass 1: CTA (row block, column split) forms the partial sums of 256 rows over
// a range of columns -- each thread two adjacent rows, loaded as one 16-byte
// (binary64) or 8-byte (binary32) vector per column, so a warp reads 512 B of
// a column-major A contiguously; x is staged in shared memory.
// Pass 2: r_i = b_i - sum of the partials in split order (deterministic), and
// the maximum |r_i| by an atomic maximum on ordered bit patterns.
#include "ir_internal.cuh"

namespace ir {
namespace {

constexpr int RT = 128;            // threads per CTA
constexpr int RB = 2 * RT;         // rows per CTA
constexpr int XCH = 512;           // x values staged per smem chunk

template <typename TW>
struct Vec2;
template <>
struct Vec2<double> { using T = double2; };
template <>
struct Vec2<float> { using T = float2; };

template <typename TW>
__global__ void __launch_bounds__(RT) k_resid_partial(int64_t n, const TW *A, int64_t lda,
                                                      const double *x, int64_t cols_per_split,
                                                      double *partials, int vec_ok, const int *skip) {
    if (skip && *skip) return;
    __shared__ double xs[XCH];
    const int64_t i = (int64_t)blockIdx.x * RB + 2 * threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.y * cols_per_split;
    int64_t c1 = c0 + cols_per_split;
    if (c1 > n) c1 = n;
    double s0 = 0.0, s1 = 0.0;
    const bool both = (i + 1 < n);
    for (int64_t cb = c0; cb < c1; cb += XCH) {
        const int64_t ce = (cb + XCH < c1) ? cb + XCH : c1;
        __syncthreads();
        for (int64_t c = cb + threadIdx.x; c < ce; c += RT) xs[c - cb] = x[c];
        __syncthreads();
        if (i >= n) continue;
        const TW *col = A + i + cb * lda;
        const int cnt = (int)(ce - cb);
        if (vec_ok && both) {
            using V = typename Vec2<TW>::T;
            int c = 0;
            for (; c + 4 <= cnt; c += 4) {
                const V a0 = __ldg(reinterpret_cast<const V *>(col + (int64_t)(c + 0) * lda));
                const V a1 = __ldg(reinterpret_cast<const V *>(col + (int64_t)(c + 1) * lda));
                const V a2 = __ldg(reinterpret_cast<const V *>(col + (int64_t)(c + 2) * lda));
                const V a3 = __ldg(reinterpret_cast<const V *>(col + (int64_t)(c + 3) * lda));
                s0 = fma((double)a0.x, xs[c + 0], s0); s1 = fma((double)a0.y, xs[c + 0], s1);
                s0 = fma((double)a1.x, xs[c + 1], s0); s1 = fma((double)a1.y, xs[c + 1], s1);
                s0 = fma((double)a2.x, xs[c + 2], s0); s1 = fma((double)a2.y, xs[c + 2], s1);
                s0 = fma((double)a3.x, xs[c + 3], s0); s1 = fma((double)a3.y, xs[c + 3], s1);
            }
            for (; c < cnt; ++c) {
                const V a = __ldg(reinterpret_cast<const V *>(col + (int64_t)c * lda));
                s0 = fma((double)a.x, xs[c], s0);
                s1 = fma((double)a.y, xs[c], s1);
            }
        } else {
            for (int c = 0; c < cnt; ++c) {
                s0 = fma((double)__ldg(col + (int64_t)c * lda), xs[c], s0);
                if (both) s1 = fma((double)__ldg(col + (int64_t)c * lda + 1), xs[c], s1);
            }
        }
    }
    if (i < n) partials[blockIdx.y * n + i] = s0;
    if (both) partials[blockIdx.y * n + i + 1] = s1;
}

template <typename TW>
__global__ void k_resid_final(int64_t n, const TW *b, const double *partials, int nsplit,
                              double *r, unsigned long long *rnorm_bits, const int *skip) {
    if (skip && *skip) return;
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = partials[i];
        for (int k = 1; k < nsplit; ++k) s += partials[(int64_t)k * n + i];
        const double ri = b ? (double)b[i] - s : s;
        r[i] = ri;
        m = fmax(m, fabs(ri));
        if (ri != ri) m = ri;   // keep a NaN visible to the norm
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double v = __shfl_xor_sync(0xffffffffu, m, o);
        m = (v != v || v > m) ? v : m;
    }
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(rnorm_bits, m);
}

// K columns at once: R(:, j) = B(:, j) - A X(:, j); A is read once for all
// columns, each thread keeping 2 rows x K sums (the same fma chain per column
// as k_resid_partial); partials[(split * K + j) * n + i].
template <typename TW, int K>
__global__ void __launch_bounds__(RT) k_mresid_partial(int64_t n, const TW *A, int64_t lda, const double *X,
                                                       int64_t ldx, int64_t cols_per_split, double *partials,
                                                       int vec_ok) {
    __shared__ double xs[K][XCH / 2];
    constexpr int XC = XCH / 2;
    const int64_t i = (int64_t)blockIdx.x * RB + 2 * threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.y * cols_per_split;
    int64_t c1 = c0 + cols_per_split;
    if (c1 > n) c1 = n;
    double s0[K], s1[K];
#pragma unroll
    for (int j = 0; j < K; ++j) s0[j] = s1[j] = 0.0;
    const bool both = (i + 1 < n);
    for (int64_t cb = c0; cb < c1; cb += XC) {
        const int64_t ce = (cb + XC < c1) ? cb + XC : c1;
        __syncthreads();
        for (int64_t e = threadIdx.x; e < K * (ce - cb); e += RT) {
            const int j = (int)(e / (ce - cb));
            const int64_t c = cb + e % (ce - cb);
            xs[j][c - cb] = X[j * ldx + c];
        }
        __syncthreads();
        if (i >= n) continue;
        const TW *col = A + i + cb * lda;
        const int cnt = (int)(ce - cb);
        if (vec_ok && both) {
            using V = typename Vec2<TW>::T;
            for (int c = 0; c < cnt; ++c) {
                const V a = __ldg(reinterpret_cast<const V *>(col + (int64_t)c * lda));
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    s0[j] = fma((double)a.x, xs[j][c], s0[j]);
                    s1[j] = fma((double)a.y, xs[j][c], s1[j]);
                }
            }
        } else {
            for (int c = 0; c < cnt; ++c) {
                const double a0 = (double)__ldg(col + (int64_t)c * lda);
                const double a1 = both ? (double)__ldg(col + (int64_t)c * lda + 1) : 0.0;
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    s0[j] = fma(a0, xs[j][c], s0[j]);
                    s1[j] = fma(a1, xs[j][c], s1[j]);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
        if (i < n) partials[((int64_t)blockIdx.y * K + j) * n + i] = s0[j];
        if (both) partials[((int64_t)blockIdx.y * K + j) * n + i + 1] = s1[j];
    }
}

template <typename TW, int K>
__global__ void k_mresid_final(int64_t n, const TW *Bm, int64_t ldb, const double *partials, int nsplit, double *R,
                               int64_t ldr, unsigned long long *rnorm_bits) {
    const int j = blockIdx.y;
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = partials[(int64_t)j * n + i];
        for (int k = 1; k < nsplit; ++k) s += partials[((int64_t)k * K + j) * n + i];
        const double ri = (double)Bm[j * ldb + i] - s;
        R[j * ldr + i] = ri;
        m = fmax(m, fabs(ri));
        if (ri != ri) m = ri;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double v = __shfl_xor_sync(0xffffffffu, m, o);
        m = (v != v || v > m) ? v : m;
    }
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(rnorm_bits + j, m);
}

int nsplit_for(int64_t n, int sms) {
    const int64_t rowblocks = (n + RB - 1) / RB;
    int64_t ns = (4 * (int64_t)sms + rowblocks - 1) / rowblocks;
    int64_t maxs = (n + 63) / 64;           // at least 64 columns per split
    if (ns > maxs) ns = maxs;
    if (ns < 1) ns = 1;
    return (int)ns;
}

}  // namespace

int64_t residual_partials_needed(int64_t n, int sms) { return (int64_t)nsplit_for(n, sms) * n; }

cudaError_t launch_residual(int64_t n, ir_dtype tw, const void *A, int64_t lda, const void *b,
                            const double *x, double *r, double *partials, int64_t partials_cap,
                            unsigned long long *rnorm_bits, int sms, cudaStream_t s, const int *skip) {
    if (n == 0) return cudaSuccess;
    const int ns = nsplit_for(n, sms);
    if ((int64_t)ns * n > partials_cap) return cudaErrorInvalidValue;
    const int64_t cps = (n + ns - 1) / ns;
    const int64_t rowblocks = (n + RB - 1) / RB;
    dim3 grid((unsigned)rowblocks, (unsigned)ns);
    const size_t esz = (tw == IR_F64) ? 8 : 4;
    const int vec_ok = ((lda % 2) == 0) && (((uintptr_t)A % (2 * esz)) == 0);
    cudaError_t e = cudaMemsetAsync(rnorm_bits, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int fg = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    if (tw == IR_F64) {
        count_launch();
        k_resid_partial<double><<<grid, RT, 0, s>>>(n, (const double *)A, lda, x, cps, partials, vec_ok, skip);
        count_launch();
        k_resid_final<double><<<fg, 256, 0, s>>>(n, (const double *)b, partials, ns, r, rnorm_bits, skip);
    } else {
        count_launch();
        k_resid_partial<float><<<grid, RT, 0, s>>>(n, (const float *)A, lda, x, cps, partials, vec_ok, skip);
        count_launch();
        k_resid_final<float><<<fg, 256, 0, s>>>(n, (const float *)b, partials, ns, r, rnorm_bits, skip);
    }
    return cudaGetLastError();
}

// R(:, j) = B(:, j) - A X(:, j) for j < 4 and ||R(:, j)||_inf into rnorm_bits[j];
// partials: nsplit * 4 * n doubles (residual_partials_needed(n, sms) * 4).
cudaError_t launch_residual_multi(int64_t n, ir_dtype tw, const void *A, int64_t lda, const void *Bm, int64_t ldb,
                                  const double *X, int64_t ldx, double *R, int64_t ldr, double *partials,
                                  int64_t partials_cap, unsigned long long *rnorm_bits, int sms, cudaStream_t s) {
    constexpr int K = 4;
    if (n == 0) return cudaSuccess;
    const int ns = nsplit_for(n, sms);
    if ((int64_t)ns * n * K > partials_cap) return cudaErrorInvalidValue;
    const int64_t cps = (n + ns - 1) / ns;
    const int64_t rowblocks = (n + RB - 1) / RB;
    dim3 grid((unsigned)rowblocks, (unsigned)ns);
    const size_t esz = (tw == IR_F64) ? 8 : 4;
    const int vec_ok = ((lda % 2) == 0) && (((uintptr_t)A % (2 * esz)) == 0);
    cudaError_t e = cudaMemsetAsync(rnorm_bits, 0, K * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int fg = (int)((n + 255) / 256 < 256 ? (n + 255) / 256 : 256);
    count_launch();
    count_launch();
    if (tw == IR_F64) {
        k_mresid_partial<double, K><<<grid, RT, 0, s>>>(n, (const double *)A, lda, X, ldx, cps, partials, vec_ok);
        k_mresid_final<double, K><<<dim3(fg, K), 256, 0, s>>>(n, (const double *)Bm, ldb, partials, ns, R, ldr,
                                                              rnorm_bits);
    } else {
        k_mresid_partial<float, K><<<grid, RT, 0, s>>>(n, (const float *)A, lda, X, ldx, cps, partials, vec_ok);
        k_mresid_final<float, K><<<dim3(fg, K), 256, 0, s>>>(n, (const float *)Bm, ldb, partials, ns, R, ldr,
                                                             rnorm_bits);
    }
    return cudaGetLastError();
}

// ---- the refinement loop on the device (Algorithm IR's "while ||r|| is too
// large"; the termination test of Sec. 5.1) --------------------------------
namespace {

__device__ __forceinline__ double bits_value(unsigned long long b) { return __longlong_as_double((long long)b); }

// After x = 0, r = b: rhist[0] = ||b||; a non-finite b (or ||A||_1) ends the
// solve before any correction; ||b|| = 0 ends it converged.
__global__ void k_loop_start(DevScalars *dev, SolveLoop *loop, TermArgs t) {
    const double bnorm = bits_value(dev->bnorm_bits);
    loop->k = 0;
    loop->rhist[0] = bnorm;
    loop->err = dev->nonfinite ? kLoopNonfinite : 0;
    loop->status = loop->err ? IR_FAILED : (bnorm == 0.0 ? IR_CONVERGED : -1);
    loop->done = loop->status >= 0 ? 1 : 0;
    dev->dnorm_bits = 0;
    dev->xnorm_bits = 0;
}

// After the k-th residual: ||d|| and ||r|| appended, the test decides.
__global__ void k_loop_step(DevScalars *dev, SolveLoop *loop, TermArgs t) {
    if (loop->done) return;
    if (dev->timeout) {                 // a bounded wait gave up: the iterate is not to be trusted
        loop->err = kLoopTimeout;
        loop->status = IR_FAILED;
        loop->done = 1;
        return;
    }
    const int k = loop->k + 1;
    loop->k = k;
    loop->dhist[k - 1] = bits_value(dev->dnorm_bits);
    loop->rhist[k] = bits_value(dev->rnorm_bits);
    const int st = term_rule(loop->rhist, loop->dhist, k, loop->rhist[0], t, bits_value(dev->anorm_bits),
                             bits_value(dev->xnorm_bits));
    loop->status = st;
    if (st >= 0) {
        loop->done = 1;
    } else {
        dev->dnorm_bits = 0;
        dev->xnorm_bits = 0;
    }
}

}  // namespace

cudaError_t launch_loop_start(DevScalars *dev, SolveLoop *loop, const TermArgs &t, cudaStream_t s) {
    count_launch();
    k_loop_start<<<1, 1, 0, s>>>(dev, loop, t);
    return cudaGetLastError();
}

cudaError_t launch_loop_step(DevScalars *dev, SolveLoop *loop, const TermArgs &t, cudaStream_t s) {
    count_launch();
    k_loop_step<<<1, 1, 0, s>>>(dev, loop, t);
    return cudaGetLastError();
}

}  // namespace ir
