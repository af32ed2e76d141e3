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

// Wait (bounded, with back-off) until the word carries `tag`; return its value.
__device__ __forceinline__ float poll_tagged(const unsigned long long *p, unsigned tag,
                                             int *timeout) {
    unsigned long long v = ld_relaxed_u64(p);
    if ((unsigned)(v >> 32) == tag) return __uint_as_float((unsigned)v);
    const unsigned long long t0 = globaltimer();
    unsigned ns = 32;
    while (true) {
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        v = ld_relaxed_u64(p);
        if ((unsigned)(v >> 32) == tag) return __uint_as_float((unsigned)v);
        if (*reinterpret_cast<volatile int *>(timeout) || globaltimer() - t0 > kWaitLimitNs) {
            atomicExch(timeout, 1);
            return 0.f;
        }
    }
}

// Sum of 8 per-lane values over the 32 lanes of a warp in 9 shuffles
// (recursive halving): lane l ends with the total of row q(l) =
// 4*bit4(l) + 2*bit3(l) + bit2(l).
__device__ __forceinline__ float reduce8(float (&v)[8], int lane) {
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
    float a[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float send = h16 ? v[q] : v[q + 4];
        const float keep = h16 ? v[q + 4] : v[q];
        a[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float b2[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const float send = h8 ? a[q] : a[q + 2];
        const float keep = h8 ? a[q + 2] : a[q];
        b2[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float c;
    {
        const float send = h4 ? b2[0] : b2[1];
        const float keep = h4 ? b2[1] : b2[0];
        c = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}
__device__ __forceinline__ int reduce8_row(int lane) {
    return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}

// Prefetch of one 64x64 off-diagonal tile slice: warp w rows 8w..8w+7,
// lane l columns l and l+32 of block column bj.
__device__ __forceinline__ void load_tile(const float *AF, int64_t ldf, int n, int row0, int bj,
                                          int lane, float (&la)[8], float (&lb)[8]) {
    const int c = bj * B + lane;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int i = row0 + q;
        la[q] = (i < n && c < n) ? __ldg(AF + (int64_t)i * ldf + c) : 0.f;
        lb[q] = (i < n && c + 32 < n) ? __ldg(AF + (int64_t)i * ldf + c + 32) : 0.f;
    }
}

// Accumulate the off-diagonal products of block bi: p[q] += sum_j A[row0+q][j] y_j
// over the predecessor blocks, in order; the next tile is in flight while the
// current one waits for its published values.
template <bool LOWER>
__device__ __forceinline__ void offdiag(const float *AF, int64_t ldf, int n, int nblk, int bi,
                                        const unsigned long long *tags, unsigned tag, float *ys,
                                        int *timeout, float (&p)[8]) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int row0 = bi * B + warp * 8;
    const int npred = LOWER ? bi : (nblk - 1 - bi);
    float la[8], lb[8], na[8], nb2[8];
    if (npred > 0) load_tile(AF, ldf, n, row0, LOWER ? 0 : nblk - 1, lane, la, lb);
    for (int it = 0; it < npred; ++it) {
        const int bj = LOWER ? it : (nblk - 1 - it);
        if (it + 1 < npred) load_tile(AF, ldf, n, row0, LOWER ? bj + 1 : bj - 1, lane, na, nb2);
        if (warp == 0) {
            ys[lane] = poll_tagged(tags + bj * B + lane, tag, timeout);
            ys[lane + 32] = poll_tagged(tags + bj * B + lane + 32, tag, timeout);
        }
        __syncthreads();
        const float y0 = ys[lane], y1 = ys[lane + 32];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            p[q] = fmaf(la[q], y0, p[q]);
            p[q] = fmaf(lb[q], y1, p[q]);
        }
        __syncthreads();                       // ys consumed before the next fetch
#pragma unroll
        for (int q = 0; q < 8; ++q) { la[q] = na[q]; lb[q] = nb2[q]; }
    }
}

// mode 0: v = fl32(r[perm[i]] / ||r||) (refinement step); mode 1: v = vin[perm[i]].
// Publishes tagged y for the upper solve.
__global__ void __launch_bounds__(TT) k_trsv_lower(const float *AF, int64_t ldf, int n, int nblk,
                                                   const float *Linv, const int32_t *perm,
                                                   const double *r, const float *vin, int mode,
                                                   unsigned long long *ytag, unsigned tag,
                                                   DevScalars *dev) {
    __shared__ int s_bi;
    __shared__ float sv[B], ys[B];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) s_bi = (int)atomicAdd(&dev->ticket[0], 1u);
    __syncthreads();
    const int bi = s_bi;
    const int r0 = bi * B;
    // diagonal-block inverse rows of this warp, and this block's right-hand side
    const float *Li = Linv + (int64_t)bi * B * B;
    float da[8], db[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        da[q] = __ldg(Li + (warp * 8 + q) * B + lane);
        db[q] = __ldg(Li + (warp * 8 + q) * B + lane + 32);
    }
    if (t < B) {
        const int i = r0 + t;
        float v = 0.f;
        if (i < n) {
            const int src = perm[i];
            if (mode == 0) {
                const double rn = __longlong_as_double((long long)dev->rnorm_bits);
                v = __double2float_rn(r[src] / rn);
            } else {
                v = vin[src];
            }
        }
        sv[t] = v;
    }
    float p[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) p[q] = 0.f;
    offdiag<true>(AF, ldf, n, nblk, bi, ytag, tag, ys, &dev->timeout, p);
    __syncthreads();
    {
        const float sq = reduce8(p, lane);
        if ((lane & 3) == 0) sv[warp * 8 + reduce8_row(lane)] -= sq;
    }
    __syncthreads();
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = fmaf(da[q], sv[lane], db[q] * sv[lane + 32]);
    const float y = reduce8(acc, lane);
    if ((lane & 3) == 0) {
        const int il = warp * 8 + reduce8_row(lane);
        const float yv = (r0 + il < n) ? y : 0.f;
        st_relaxed_u64(ytag + r0 + il, ((unsigned long long)tag << 32) | __float_as_uint(yv));
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
    __shared__ float sv[B], ys[B];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) s_bi = nblk - 1 - (int)atomicAdd(&dev->ticket[1], 1u);
    __syncthreads();
    const int bi = s_bi;
    const int r0 = bi * B;
    const float *Ui = Uinv + (int64_t)bi * B * B;
    float da[8], db[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        da[q] = __ldg(Ui + (warp * 8 + q) * B + lane);
        db[q] = __ldg(Ui + (warp * 8 + q) * B + lane + 32);
    }
    if (t < B) {
        // the lower solve of this launch sequence has written every y word already
        const int i = r0 + t;
        sv[t] = (i < n) ? __uint_as_float((unsigned)ld_relaxed_u64(ytag + i)) : 0.f;
    }
    float p[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) p[q] = 0.f;
    offdiag<false>(AF, ldf, n, nblk, bi, ztag, tag, ys, &dev->timeout, p);
    __syncthreads();
    {
        const float sq = reduce8(p, lane);
        if ((lane & 3) == 0) sv[warp * 8 + reduce8_row(lane)] -= sq;
    }
    __syncthreads();
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = fmaf(da[q], sv[lane], db[q] * sv[lane + 32]);
    const float z = reduce8(acc, lane);
    double dmax = 0.0;
    if ((lane & 3) == 0) {
        const int i = r0 + warp * 8 + reduce8_row(lane);
        const float zv = (i < n) ? z : 0.f;
        st_relaxed_u64(ztag + i, ((unsigned long long)tag << 32) | __float_as_uint(zv));
        if (i < n) {
            if (mode == 0) {
                const double scale = __longlong_as_double((long long)dev->rnorm_bits) * dev->scale;
                const double d = scale * (double)zv;
                x[i] += d;
                dmax = fabs(d);
            } else {
                dout[i] = zv;
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
