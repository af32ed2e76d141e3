// Correction solve d = U^{-1} L^{-1} P v in binary32 (Algorithm IR; eqs.
// vdlow/promotevd of Sec. 5.3 for the scaling by ||r||).
//
// Blocked, synchronisation-free triangular solves: the rows are cut into
// blocks of B = 64; CTA b (taken in order through a ticket counter, so every
// block it waits on has already started) accumulates the products of its
// off-diagonal blocks with the solution blocks as they appear, then applies
// the inverse of its diagonal block (computed once after the factorization)
// and publishes its 64 values.  A published value is a 64-bit word
// (epoch << 32 | binary32 bits), so a reader learns "ready" and the value in
// one load; waits are bounded and a timeout is reported, never hung.
#include "ir_internal.cuh"

namespace ir {
namespace {

constexpr int B = kTrsvB;
constexpr int TT = 256;          // threads per solve CTA (8 warps x 8 rows)

// Inverse of the diagonal blocks: blockIdx.y = 0 -> L (unit lower), 1 -> U.
// Thread t computes column t of the inverse by substitution (binary32).
// Rows/columns beyond n are treated as identity.
__global__ void __launch_bounds__(B) k_diag_inv(const float *AF, int64_t ldf, int n, float *Linv,
                                                 float *Uinv) {
    __shared__ float Tb[B][B + 1];
    __shared__ float X[B][B + 1];
    const int b = blockIdx.x, upper = blockIdx.y, t = threadIdx.x;
    const int r0 = b * B;
    for (int i = 0; i < B; ++i) {
        const int gi = r0 + i, gc = r0 + t;
        float v;
        if (gi < n && gc < n) v = AF[(int64_t)gi * ldf + gc];
        else v = (i == t) ? 1.f : 0.f;
        Tb[i][t] = v;
    }
    __syncthreads();
    if (!upper) {
        for (int i = 0; i < B; ++i) {
            float x;
            if (i < t) x = 0.f;
            else if (i == t) x = 1.f;
            else {
                x = 0.f;
                for (int m = t; m < i; ++m) x = fmaf(-Tb[i][m], X[m][t], x);
            }
            X[i][t] = x;
        }
    } else {
        for (int i = B - 1; i >= 0; --i) {
            float x;
            if (i > t) x = 0.f;
            else {
                x = (i == t) ? 1.f : 0.f;
                for (int m = i + 1; m <= t; ++m) x = fmaf(-Tb[i][m], X[m][t], x);
                x = x / Tb[i][i];
            }
            X[i][t] = x;
        }
    }
    __syncthreads();
    float *dst = (upper ? Uinv : Linv) + (int64_t)b * B * B;
    for (int i = 0; i < B; ++i) dst[i * B + t] = X[i][t];
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Wait (bounded) until the word carries `tag`, return its binary32 value.
__device__ __forceinline__ float poll_tagged(const unsigned long long *p, unsigned tag,
                                             int *timeout) {
    unsigned long long v = ld_relaxed_u64(p);
    if ((unsigned)(v >> 32) == tag) return __uint_as_float((unsigned)v);
    const unsigned long long t0 = globaltimer();
    while (true) {
        v = ld_relaxed_u64(p);
        if ((unsigned)(v >> 32) == tag) return __uint_as_float((unsigned)v);
        if (*reinterpret_cast<volatile int *>(timeout) || globaltimer() - t0 > kWaitLimitNs) {
            atomicExch(timeout, 1);
            return 0.f;
        }
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// mode 0: v = fl32(r[perm[i]] / ||r||) (refinement step); mode 1: v = vin[perm[i]].
// Writes tagged y for the upper solve.
__global__ void __launch_bounds__(TT) k_trsv_lower(const float *AF, int64_t ldf, int n, int nblk,
                                                   const float *Linv, const int32_t *perm,
                                                   const double *r, const float *vin, int mode,
                                                   unsigned long long *ytag, unsigned tag,
                                                   DevScalars *dev) {
    __shared__ int s_bi;
    __shared__ float sv[B];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) s_bi = (int)atomicAdd(&dev->ticket[0], 1u);
    __syncthreads();
    const int bi = s_bi;
    const int r0 = bi * B;
    const int row0 = r0 + warp * 8;     // this warp's 8 rows
    float p[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) p[q] = 0.f;
    float la[8], lb[8];
    for (int bj = 0; bj < bi; ++bj) {
        const int c = bj * B + lane;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = row0 + q;
            la[q] = (i < n) ? __ldg(AF + (int64_t)i * ldf + c) : 0.f;
            lb[q] = (i < n) ? __ldg(AF + (int64_t)i * ldf + c + 32) : 0.f;
        }
        const float y0 = poll_tagged(ytag + c, tag, &dev->timeout);
        const float y1 = poll_tagged(ytag + c + 32, tag, &dev->timeout);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            p[q] = fmaf(la[q], y0, p[q]);
            p[q] = fmaf(lb[q], y1, p[q]);
        }
    }
    double rinv_scale = 0.0;
    if (mode == 0) rinv_scale = __longlong_as_double((long long)dev->rnorm_bits);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float sq = warp_sum(p[q]);
        if (lane == q) {
            const int i = row0 + q;
            float v = 0.f;
            if (i < n) {
                const int src = perm[i];
                v = (mode == 0) ? __double2float_rn(r[src] / rinv_scale) : vin[src];
            }
            sv[warp * 8 + q] = v - sq;
        }
    }
    __syncthreads();
    const float *Li = Linv + (int64_t)bi * B * B;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int il = warp * 8 + q;
        float acc = fmaf(Li[il * B + lane], sv[lane], Li[il * B + lane + 32] * sv[lane + 32]);
        acc = warp_sum(acc);
        if (lane == q) {
            const float y = (r0 + il < n) ? acc : 0.f;
            st_relaxed_u64(ytag + r0 + il, ((unsigned long long)tag << 32) | __float_as_uint(y));
        }
    }
}

// Back substitution with U, reading the tagged y of the lower solve.
// mode 0: d = (||r|| s) fl64(z); x += d; ||d|| into dev; mode 1: dout = z.
__global__ void __launch_bounds__(TT) k_trsv_upper(const float *AF, int64_t ldf, int n, int nblk,
                                                   const float *Uinv,
                                                   const unsigned long long *ytag,
                                                   unsigned long long *ztag, unsigned tag,
                                                   int mode, double *x, float *dout,
                                                   DevScalars *dev) {
    __shared__ int s_bi;
    __shared__ float sv[B];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) s_bi = nblk - 1 - (int)atomicAdd(&dev->ticket[1], 1u);
    __syncthreads();
    const int bi = s_bi;
    const int r0 = bi * B;
    const int row0 = r0 + warp * 8;
    float p[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) p[q] = 0.f;
    float la[8], lb[8];
    for (int bj = nblk - 1; bj > bi; --bj) {
        const int c = bj * B + lane;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = row0 + q;
            la[q] = (i < n && c < n) ? __ldg(AF + (int64_t)i * ldf + c) : 0.f;
            lb[q] = (i < n && c + 32 < n) ? __ldg(AF + (int64_t)i * ldf + c + 32) : 0.f;
        }
        const float z0 = poll_tagged(ztag + c, tag, &dev->timeout);
        const float z1 = poll_tagged(ztag + c + 32, tag, &dev->timeout);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            p[q] = fmaf(la[q], z0, p[q]);
            p[q] = fmaf(lb[q], z1, p[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float sq = warp_sum(p[q]);
        if (lane == q) {
            const int i = row0 + q;
            // the lower solve of this launch sequence wrote every y word already
            const float yv = (i < n) ? __uint_as_float((unsigned)ld_relaxed_u64(ytag + i)) : 0.f;
            sv[warp * 8 + q] = yv - sq;
        }
    }
    __syncthreads();
    const float *Ui = Uinv + (int64_t)bi * B * B;
    double scale = 0.0;
    if (mode == 0)
        scale = __longlong_as_double((long long)dev->rnorm_bits) * dev->scale;
    double dmax = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int il = warp * 8 + q;
        float acc = fmaf(Ui[il * B + lane], sv[lane], Ui[il * B + lane + 32] * sv[lane + 32]);
        acc = warp_sum(acc);
        if (lane == q) {
            const int i = r0 + il;
            const float z = (i < n) ? acc : 0.f;
            st_relaxed_u64(ztag + i, ((unsigned long long)tag << 32) | __float_as_uint(z));
            if (i < n) {
                if (mode == 0) {
                    const double d = scale * (double)z;
                    x[i] += d;
                    dmax = fmax(dmax, fabs(d));
                } else {
                    dout[i] = z;
                }
            }
        }
    }
    if (mode == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        if (lane == 0) atomic_max_nonneg(&dev->dnorm_bits, dmax);
    }
}

}  // namespace

cudaError_t launch_diag_inv(const float *AF, int64_t ldf, int n, float *Linv, float *Uinv,
                            cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int nblk = (n + B - 1) / B;
    count_launch();
    k_diag_inv<<<dim3(nblk, 2), B, 0, s>>>(AF, ldf, n, Linv, Uinv);
    return cudaGetLastError();
}

// ytag/ztag: 2 arrays of nblk*B tagged words (flags buffer).  Tickets are reset here.
cudaError_t launch_trsv_pair(const float *AF, int64_t ldf, int n, const float *Linv,
                             const float *Uinv, const int32_t *perm, const double *r,
                             const float *vin, float *dout, double *x,
                             unsigned long long *tags, unsigned epoch, DevScalars *dev,
                             cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int nblk = (n + B - 1) / B;
    cudaError_t e = cudaMemsetAsync(&dev->ticket[0], 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const int mode = vin ? 1 : 0;
    unsigned long long *ytag = tags, *ztag = tags + (int64_t)nblk * B;
    count_launch();
    k_trsv_lower<<<nblk, TT, 0, s>>>(AF, ldf, n, nblk, Linv, perm, r, vin, mode, ytag, epoch, dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    count_launch();
    k_trsv_upper<<<nblk, TT, 0, s>>>(AF, ldf, n, nblk, Uinv, ytag, ztag, epoch, mode, x, dout, dev);
    return cudaGetLastError();
}

}  // namespace ir
