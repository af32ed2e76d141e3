// Elementwise kernels: the copy to the factorization precision (A_F = I_W^F(s A),
// Sec. 1), the max |a_ij| pass of the binary16 scaling, and the setup/finish of
// the refinement vectors (x = 0, r = b, Algorithm IR).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ir_internal.cuh"

namespace ir {
namespace {

template <typename TW>
__device__ __forceinline__ double ld_w(const TW *p) { return static_cast<double>(__ldg(p)); }

// max |a_ij| over a column-major n x n matrix; NaN/Inf raise the non-finite flag.
// One warp per column at a time (the warps stride over the columns), lanes
// down the column with four loads in flight; the maximum does not depend on
// the order.
template <typename TW>
__global__ void __launch_bounds__(512) k_maxabs(int64_t n, const TW *A, int64_t lda, DevScalars *dev) {
    double m = 0.0;
    int bad = 0;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n; j += warps) {
        const TW *col = A + j * lda;
        int64_t i = lane;
        for (; i + 96 < n; i += 128) {
            const double a0 = ld_w(col + i), a1 = ld_w(col + i + 32), a2 = ld_w(col + i + 64),
                         a3 = ld_w(col + i + 96);
            if (!isfinite(a0) || !isfinite(a1) || !isfinite(a2) || !isfinite(a3)) bad = 1;
            m = fmax(fmax(m, fabs(a0)), fmax(fabs(a1), fmax(fabs(a2), fabs(a3))));
        }
        for (; i < n; i += 32) {
            const double a = ld_w(col + i);
            if (!isfinite(a)) bad = 1;
            m = fmax(m, fabs(a));
        }
    }
    // block reduction of the maximum
    __shared__ double sm[32];
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    bad = __syncthreads_or(bad);
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) {
            atomic_max_nonneg(&dev->amax_bits, m);
            if (bad) atomicExch(&dev->nonfinite, 1);
        }
    }
}

// The same over a contiguous matrix (lda = n, 16-byte aligned): one flat
// stream of 16-byte vectors, four in flight per thread.
template <typename TW, typename V>
__global__ void __launch_bounds__(512) k_maxabs_flat(int64_t total, const TW *A, DevScalars *dev) {
    constexpr int E = sizeof(V) / sizeof(TW);           // elements per vector
    double m = 0.0;
    int bad = 0;
    const V *A4 = reinterpret_cast<const V *>(A);
    const int64_t nv = total / E;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    auto take = [&](const V &v) {
        const TW *e = reinterpret_cast<const TW *>(&v);
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const double a = static_cast<double>(e[q]);
            if (!isfinite(a)) bad = 1;
            m = fmax(m, fabs(a));
        }
    };
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < nv; i += 4 * stride) {
        const V v0 = __ldg(A4 + i), v1 = __ldg(A4 + i + stride), v2 = __ldg(A4 + i + 2 * stride),
                v3 = __ldg(A4 + i + 3 * stride);
        take(v0);
        take(v1);
        take(v2);
        take(v3);
    }
    for (; i < nv; i += stride) take(__ldg(A4 + i));
    for (int64_t r = nv * E + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total; r += stride) {
        const double a = ld_w(A + r);
        if (!isfinite(a)) bad = 1;
        m = fmax(m, fabs(a));
    }
    __shared__ double sm[32];
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    bad = __syncthreads_or(bad);
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) {
            atomic_max_nonneg(&dev->amax_bits, m);
            if (bad) atomicExch(&dev->nonfinite, 1);
        }
    }
}

// Round a binary32 value to TF, kept in binary32 (hardware conversions:
// cvt.rna.tf32.f32 = nearest, ties away; bf16/fp16 = nearest, ties to even).
__device__ __forceinline__ float round_tf(float v, ir_dtype tf) {
    switch (tf) {
    case IR_TF32: {
        uint32_t u;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
        return __uint_as_float(u);
    }
    case IR_BF16: return __bfloat162float(__float2bfloat16_rn(v));
    case IR_F16: return __half2float(__float2half_rn(v));
    default: return v;
    }
}

// A (column-major, TW) -> AF (row-major binary32 holding TF values):
// AF[i][j] = rTF(fl32(s * a_ij)).  64 x 64 tiles through shared memory so that
// both the column-major read and the row-major write are coalesced; each
// thread has 16 loads in flight, and writes two adjacent values at a time.
constexpr int kCastTile = 64;
template <typename TW>
__global__ void __launch_bounds__(256) k_cast(int64_t n, const TW *A, int64_t lda, ir_dtype tf,
                                              int use_scale, float *AF, int64_t ldf,
                                              DevScalars *dev) {
    __shared__ float tile[kCastTile][kCastTile + 1];
    const int64_t i0 = (int64_t)blockIdx.x * kCastTile, j0 = (int64_t)blockIdx.y * kCastTile;
    double s = 1.0;
    if (use_scale) {
        double m = __longlong_as_double((long long)dev->amax_bits);
        s = (m > 0.0 && isfinite(m)) ? 1024.0 / m : 1.0;
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) dev->scale = s;
    int bad = 0;
    // read: threadIdx.x runs down a column (rows i0 + tx and i0 + 32 + tx), coalesced in column-major A
    double a[kCastTile / 8][2];
#pragma unroll
    for (int q = 0; q < kCastTile / 8; ++q) {
        const int64_t j = j0 + threadIdx.y + 8 * q;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t i = i0 + threadIdx.x + 32 * h;
            a[q][h] = (i < n && j < n) ? ld_w(A + i + j * lda) : 0.0;
        }
    }
#pragma unroll
    for (int q = 0; q < kCastTile / 8; ++q)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float v = round_tf(__double2float_rn(s * a[q][h]), tf);
            if (!isfinite(v)) bad = 1;
            tile[threadIdx.y + 8 * q][threadIdx.x + 32 * h] = v;    // tile[column][row]
        }
    __syncthreads();
    // write: threadIdx.x takes columns 2 tx, 2 tx + 1 of a row, coalesced in row-major AF
    const int64_t j = j0 + 2 * threadIdx.x;
#pragma unroll
    for (int q = 0; q < kCastTile / 8; ++q) {
        const int ii = threadIdx.y + 8 * q;
        const int64_t i = i0 + ii;
        if (i >= n) continue;
        float *dst = AF + i * ldf + j;
        if (j + 1 < n)
            *reinterpret_cast<float2 *>(dst) = make_float2(tile[2 * threadIdx.x][ii], tile[2 * threadIdx.x + 1][ii]);
        else if (j < n)
            dst[0] = tile[2 * threadIdx.x][ii];
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0 && threadIdx.y == 0) atomicExch(&dev->nonfinite, 1);
}

// x = 0, r = b promoted to binary64, ||b||_inf.
template <typename TW>
__global__ void k_init_rb(int64_t n, const TW *b, double *r, double *x, DevScalars *dev) {
    double m = 0.0;
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = static_cast<double>(b[i]);
        if (!isfinite(v)) bad = 1;
        r[i] = v;
        x[i] = 0.0;
        m = fmax(m, fabs(v));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    bad = __syncthreads_or(bad);
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) {
            atomic_max_nonneg(&dev->bnorm_bits, m);
            if (bad) atomicExch(&dev->nonfinite, 1);
        }
    }
}

template <typename TW>
__global__ void k_store_x(int64_t n, const double *x, TW *out, const int *skip) {
    if (skip && *skip) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = static_cast<TW>(x[i]);
}

int grid_for(int64_t work, int threads, int cap) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    return (int)(g < cap ? g : cap);
}

}  // namespace

// ||A||_1 = max_j sum_i |a_ij| in binary64 (Sec. 5.1.1, eq. term; the OPNORM of
// Sec. 5.2): one warp per column (coalesced over the column-major rows), lane
// partial sums in row order, then a butterfly; the maximum over columns by an
// atomic maximum on ordered bit patterns, so the result is deterministic.
template <typename TW>
__global__ void __launch_bounds__(256) k_norm1(int64_t n, const TW *A, int64_t lda, unsigned long long *out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    double m = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n; j += warps) {
        const TW *col = A + j * lda;
        double s = 0.0;
        for (int64_t i = lane; i < n; i += 32) s += fabs(ld_w(col + i));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        m = fmax(m, s);
        if (s != s) m = s;
    }
    if (lane == 0) atomic_max_nonneg(out, m);
}

cudaError_t launch_norm1(int64_t n, ir_dtype tw, const void *A, int64_t lda, unsigned long long *out_bits,
                         cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out_bits, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n == 0) return e;
    int64_t g = (n + 7) / 8;
    if (g > 1216) g = 1216;
    count_launch();
    if (tw == IR_F64)
        k_norm1<double><<<(unsigned)g, 256, 0, s>>>(n, (const double *)A, lda, out_bits);
    else
        k_norm1<float><<<(unsigned)g, 256, 0, s>>>(n, (const float *)A, lda, out_bits);
    return cudaGetLastError();
}

cudaError_t launch_maxabs(int64_t n, ir_dtype tw, const void *A, int64_t lda, DevScalars *dev,
                          int sms, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    count_launch();
    if (lda == n && (reinterpret_cast<uintptr_t>(A) & 15) == 0) {
        const int g = 4 * sms;          // 4 blocks of 512 threads per SM: 64 warps, four vectors each in flight
        if (tw == IR_F64)
            k_maxabs_flat<double, double2><<<g, 512, 0, s>>>(n * n, (const double *)A, dev);
        else
            k_maxabs_flat<float, float4><<<g, 512, 0, s>>>(n * n, (const float *)A, dev);
        return cudaGetLastError();
    }
    int g = grid_for(n * n, 512, sms * 8);
    if (tw == IR_F64)
        k_maxabs<double><<<g, 512, 0, s>>>(n, (const double *)A, lda, dev);
    else
        k_maxabs<float><<<g, 512, 0, s>>>(n, (const float *)A, lda, dev);
    return cudaGetLastError();
}

cudaError_t launch_cast(int64_t n, ir_dtype tw, const void *A, int64_t lda, ir_dtype tf,
                        int use_scale, float *AF, int64_t ldf, DevScalars *dev, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    dim3 grid((unsigned)((n + kCastTile - 1) / kCastTile), (unsigned)((n + kCastTile - 1) / kCastTile)), block(32, 8);
    count_launch();
    if (tw == IR_F64)
        k_cast<double><<<grid, block, 0, s>>>(n, (const double *)A, lda, tf, use_scale, AF, ldf, dev);
    else
        k_cast<float><<<grid, block, 0, s>>>(n, (const float *)A, lda, tf, use_scale, AF, ldf, dev);
    return cudaGetLastError();
}

cudaError_t launch_init_rb(int64_t n, ir_dtype tw, const void *b, double *r, double *x,
                           DevScalars *dev, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int g = grid_for(n, 256, 1024);
    count_launch();
    if (tw == IR_F64)
        k_init_rb<double><<<g, 256, 0, s>>>(n, (const double *)b, r, x, dev);
    else
        k_init_rb<float><<<g, 256, 0, s>>>(n, (const float *)b, r, x, dev);
    return cudaGetLastError();
}

cudaError_t launch_store_x(int64_t n, ir_dtype tw, const double *x, void *out, cudaStream_t s, const int *skip) {
    if (n == 0) return cudaSuccess;
    int g = grid_for(n, 256, 1024);
    count_launch();
    if (tw == IR_F64)
        k_store_x<double><<<g, 256, 0, s>>>(n, x, (double *)out, skip);
    else
        k_store_x<float><<<g, 256, 0, s>>>(n, x, (float *)out, skip);
    return cudaGetLastError();
}

}  // namespace ir
