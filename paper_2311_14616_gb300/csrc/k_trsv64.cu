// Mixed precision solves (MPS, Sec. 5.3: interprecision transfers "on the
// fly"): the correction d = s U^{-1} L^{-1} P r evaluated in TW = binary64 on
// the binary32 factors, each factor entry promoted exactly when it is used.
// The residual r is not scaled by ||r|| (nothing is rounded below TW, so
// nothing can underflow); s is the binary16 scale of the factorization copy.
//
// The same blocked, synchronisation-free structure as the binary32 pair in
// k_trsv.cu: rows in blocks of B, CTA b takes its block through a ticket
// counter (every block it waits on has already started), accumulates the
// products of its off-diagonal tiles with the solution blocks as they are
// published, then solves its diagonal block by substitution (one warp, column
// sweeps in the reference-BLAS order of the oracle, the diagonal applied as a
// product with its reciprocal, formed beforehand by the whole CTA) and
// publishes its B binary64 values followed by a per-block flag carrying the
// solve's tag.  Waits are bounded (kWaitLimitNs) and report a timeout, never
// hang.  The binary64 pipe (2 fma per clock per SM) sets the cost: a B x B tile
// is B^2 / 2 clocks and the chain of N / B block steps waits for one tile and
// one substitution per step, so B = 64 (half the binary32 pair's block) halves
// the chain's length in time.
#include "ir_internal.cuh"

namespace ir {
namespace {

constexpr int B = kMpsB;         // rows per block
constexpr int TT = 512;          // 16 warps
constexpr int RW = B / 16;       // rows of the block per warp
constexpr int CPL = B / 32;      // columns of a tile per lane

struct Mps64Smem {
    double sv[B];                // right-hand side of the block, then its solution
    double ys[B];                // published values of the predecessor being applied
    double rdiag[B];             // 1 / u_ii of the block (upper solve)
    double Dt[B][B + 1];         // the diagonal block, promoted and transposed: Dt[j][i] = T[i][j]
};
constexpr size_t kMpsSmem = sizeof(Mps64Smem);
static_assert(B % 32 == 0 && TT == 16 * 32 && RW * 16 == B, "16 warps of RW rows; lanes over 32-column groups");

// Bounded wait (thread 0) until flag == tag; on timeout raise *timeout.
__device__ __forceinline__ void wait_flag(const int *flag, int tag, int *timeout) {
    if (ld_acquire(flag) == tag) return;
    const unsigned long long t0 = globaltimer();
    unsigned ns = 16;
    while (ld_acquire(flag) != tag) {
        __nanosleep(ns);
        if (ns < 64) ns <<= 1;
        if (*reinterpret_cast<volatile int *>(timeout) || globaltimer() - t0 > kWaitLimitNs) {
            atomicExch(timeout, 1);
            return;
        }
    }
}

// Rows RW w .. RW w + RW - 1 of block bi, lane l columns l + 32c of block column bj.
__device__ __forceinline__ void load_tile64(const float *AF, int64_t ldf, int n, int row0, int bj, int lane,
                                            float (&a)[RW][CPL]) {
#pragma unroll
    for (int q = 0; q < RW; ++q) {
        const int i = row0 + q;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int col = bj * B + lane + 32 * c;
            a[q][c] = (i < n && col < n) ? __ldg(AF + (int64_t)i * ldf + col) : 0.f;
        }
    }
}

// sv[i] -= sum over the predecessor blocks of T[i][j] v_j (binary64), in order.
template <bool LOWER>
__device__ __forceinline__ void offdiag64(const float *AF, int64_t ldf, int n, int nblk, int bi, const double *vals,
                                          const int *flags, int tag, Mps64Smem &sm, int *timeout) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int row0 = bi * B + warp * RW;
    const int npred = LOWER ? bi : (nblk - 1 - bi);
    double p[RW];
#pragma unroll
    for (int q = 0; q < RW; ++q) p[q] = 0.0;
    float la[RW][CPL], na[RW][CPL];
    if (npred > 0) load_tile64(AF, ldf, n, row0, LOWER ? 0 : nblk - 1, lane, la);
    for (int it = 0; it < npred; ++it) {
        const int bj = LOWER ? it : (nblk - 1 - it);
        if (it + 1 < npred) load_tile64(AF, ldf, n, row0, LOWER ? bj + 1 : bj - 1, lane, na);
        if (t == 0) wait_flag(flags + bj, tag, timeout);
        __syncthreads();
        if (t < B) sm.ys[t] = vals[(int64_t)bj * B + t];
        __syncthreads();
        double y[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) y[c] = sm.ys[lane + 32 * c];
#pragma unroll
        for (int q = 0; q < RW; ++q)
#pragma unroll
            for (int c = 0; c < CPL; ++c) p[q] = fma((double)la[q][c], y[c], p[q]);
        __syncthreads();                       // ys consumed before the next fetch
#pragma unroll
        for (int q = 0; q < RW; ++q)
#pragma unroll
            for (int c = 0; c < CPL; ++c) la[q][c] = na[q][c];
    }
    // row sums over the 32 lanes, then subtract from the right-hand side
#pragma unroll
    for (int q = 0; q < RW; ++q) {
        double v = p[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        p[q] = v;
    }
    if (lane < RW) {
        double mine = p[0];
#pragma unroll
        for (int q = 1; q < RW; ++q)
            if (lane == q) mine = p[q];
        sm.sv[warp * RW + lane] -= mine;
    }
}

// The diagonal block solved in place on sv in binary64 (one warp, lane l rows
// l + 32r).  Lower: unit diagonal, columns ascending; upper: columns
// descending, each entry multiplied by the reciprocal of its diagonal entry
// (rdiag) before its column is applied.
template <bool LOWER>
__device__ __forceinline__ void subst64(const Mps64Smem &sm, double *sv, int lane) {
    double v[CPL];
#pragma unroll
    for (int r = 0; r < CPL; ++r) v[r] = sv[lane + 32 * r];
    if (LOWER) {
#pragma unroll
        for (int jr = 0; jr < CPL; ++jr) {
#pragma unroll 4
            for (int jl = 0; jl < 32; ++jl) {
                const int j = 32 * jr + jl;
                const double vj = __shfl_sync(0xffffffffu, v[jr], jl);
#pragma unroll
                for (int r = 0; r < CPL; ++r)
                    if (r >= jr && lane + 32 * r > j) v[r] = fma(-sm.Dt[j][lane + 32 * r], vj, v[r]);
            }
        }
    } else {
#pragma unroll
        for (int jr = CPL - 1; jr >= 0; --jr) {
#pragma unroll 4
            for (int jl = 31; jl >= 0; --jl) {
                const int j = 32 * jr + jl;
                if (lane == jl) v[jr] = v[jr] * sm.rdiag[j];
                const double vj = __shfl_sync(0xffffffffu, v[jr], jl);
#pragma unroll
                for (int r = 0; r < CPL; ++r)
                    if (r <= jr && lane + 32 * r < j) v[r] = fma(-sm.Dt[j][lane + 32 * r], vj, v[r]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < CPL; ++r) sv[lane + 32 * r] = v[r];
}

// The diagonal block's triangle, promoted (once, by the whole CTA, so the
// substitution's chain does no conversions) and transposed; identity past row n.
template <bool LOWER>
__device__ __forceinline__ void stage_tri(const float *AF, int64_t ldf, int n, int r0, Mps64Smem &sm) {
    for (int e = threadIdx.x; e < B * B; e += TT) {
        const int i = e / B, j = e % B, gi = r0 + i, gj = r0 + j;
        float v = (i == j) ? 1.f : 0.f;
        if (gi < n && gj < n && (LOWER ? j < i : j >= i)) v = __ldg(AF + (int64_t)gi * ldf + gj);
        sm.Dt[j][i] = (double)v;
    }
}

// y = L^{-1} P r: v_i = r[perm[i]] (binary64, unscaled).
__global__ void __launch_bounds__(TT, 1) k_mps_lower(const float *AF, int64_t ldf, int n, int nblk,
                                                     const int32_t *perm, const double *r, double *y, int *yflag,
                                                     int tag, DevScalars *dev, const int *skip) {
    if (skip && *skip) return;      // uniform: written by an earlier launch
    extern __shared__ __align__(16) unsigned char mps_smem[];
    Mps64Smem &sm = *reinterpret_cast<Mps64Smem *>(mps_smem);
    __shared__ int s_bi;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) s_bi = (int)atomicAdd(&dev->ticket[0], 1u);
    __syncthreads();
    const int bi = s_bi, r0 = bi * B;
    stage_tri<true>(AF, ldf, n, r0, sm);
    if (t < B) sm.sv[t] = (r0 + t < n) ? r[perm[r0 + t]] : 0.0;
    __syncthreads();
    offdiag64<true>(AF, ldf, n, nblk, bi, y, yflag, tag, sm, &dev->timeout);
    __syncthreads();
    if (warp == 0) subst64<true>(sm, sm.sv, lane);
    __syncthreads();
    if (t < B) y[r0 + t] = (r0 + t < n) ? sm.sv[t] : 0.0;
    __syncthreads();
    if (t == 0) {
        __threadfence();
        st_release(yflag + bi, tag);
    }
}

// z = U^{-1} y, d = s z, x += d, ||d||_inf and ||x||_inf into dev.
__global__ void __launch_bounds__(TT, 1) k_mps_upper(const float *AF, int64_t ldf, int n, int nblk, const double *y,
                                                     double *z, int *zflag, int tag, double *x, DevScalars *dev,
                                                     const int *skip) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char mps_smem[];
    Mps64Smem &sm = *reinterpret_cast<Mps64Smem *>(mps_smem);
    __shared__ int s_bi;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) s_bi = nblk - 1 - (int)atomicAdd(&dev->ticket[1], 1u);
    __syncthreads();
    const int bi = s_bi, r0 = bi * B;
    stage_tri<false>(AF, ldf, n, r0, sm);
    if (t < B) sm.sv[t] = y[r0 + t];          // written by the lower solve's launch
    __syncthreads();
    if (t < B) sm.rdiag[t] = 1.0 / sm.Dt[t][t];   // identity past n: 1
    offdiag64<false>(AF, ldf, n, nblk, bi, z, zflag, tag, sm, &dev->timeout);
    __syncthreads();
    if (warp == 0) subst64<false>(sm, sm.sv, lane);
    __syncthreads();
    double dmax = 0.0, xmax = 0.0;
    if (t < B) {
        const int i = r0 + t;
        const double zv = (i < n) ? sm.sv[t] : 0.0;
        z[i] = zv;
        if (i < n) {
            const double d = dev->scale * zv;
            const double xn = x[i] + d;
            x[i] = xn;
            dmax = fabs(d);
            xmax = fabs(xn);
        }
    }
    __syncthreads();
    if (t == 0) {
        __threadfence();
        st_release(zflag + bi, tag);
    }
    if (t < B) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
            xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
        }
        if (lane == 0) {
            atomic_max_nonneg(&dev->dnorm_bits, dmax);
            atomic_max_nonneg(&dev->xnorm_bits, xmax);
        }
    }
}

}  // namespace

// The mixed precision solve pair (x += s U^{-1} L^{-1} P r in binary64).
// y64, z64: nblk * kMpsB binary64 each (nblk = ceil(n / kMpsB)); flags: 2 nblk
// ints; tag: a value no earlier solve on these flags has written (the epoch).
cudaError_t launch_mps_pair(const float *AF, int64_t ldf, int n, const int32_t *perm, const double *r, double *x,
                            double *y64, double *z64, int *flags, unsigned tag, DevScalars *dev, cudaStream_t s,
                            const int *skip) {
    if (n == 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mps_lower, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMpsSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_mps_upper, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMpsSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int nblk = (n + B - 1) / B;
    cudaError_t e = cudaMemsetAsync(&dev->ticket[0], 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const int itag = (int)(tag & 0x7FFFFFFFu);
    count_launch();
    k_mps_lower<<<nblk, TT, kMpsSmem, s>>>(AF, ldf, n, nblk, perm, r, y64, flags, itag, dev, skip);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    count_launch();
    k_mps_upper<<<nblk, TT, kMpsSmem, s>>>(AF, ldf, n, nblk, y64, z64, flags + nblk, itag, x, dev, skip);
    return cudaGetLastError();
}

}  // namespace ir
