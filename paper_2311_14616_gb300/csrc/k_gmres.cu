// GMRES for the correction equation of GMRES-IR (Sec. 4.2-4.3): the scalar
// and vector work between the preconditioned products P A v_j (formed by the
// residual kernels with b = NULL and the solve pair with P = U^{-1} L^{-1},
// eq. pdef).
//
// k_gm_orth: one thread-block cluster, one basis row per thread (512 rows per
// CTA, up to 16 CTAs = 8192 rows).  Classical Gram-Schmidt run twice against
// v_0..v_j, the 2-norm, the normalization of v_{j+1}, then the Givens step on
// column j of the Hessenberg matrix and the stopping test.  Every dot product
// is summed lane-butterfly -> warps in order -> CTAs in rank order through
// distributed shared memory, so all CTAs see bitwise the same values and the
// result does not depend on scheduling.
// k_gm_update: y = R^{-1} g (back substitution, k <= 64), d = V_k y, x += d.
#include <cooperative_groups.h>

#include "ir_internal.cuh"

namespace cg = cooperative_groups;

namespace ir {
namespace {

constexpr int OT = 512;               // threads per CTA = basis rows per CTA
constexpr int OW = OT / 32;
constexpr int kOrthMaxCluster = 16;
constexpr int kChunk = 8;             // basis columns loaded together

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// res[l] = sum_i V_il w_i for l < cnt, or (V == NULL, cnt = 1) res[0] = sum_i w_i^2,
// over the rows of the whole cluster.  mine: this CTA's slot of the exchange,
// a different one per call so that no CTA overwrites a slot another still reads.
__device__ void cluster_dots(const cg::cluster_group &cl, const double *V, int64_t ldv, int i, bool on,
                             double w, int cnt, double (*wsum)[kMaxBasis + 1], double *mine, double *res) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int l0 = 0; l0 < cnt; l0 += kChunk) {
        double v[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q)
            v[q] = (on && l0 + q < cnt) ? (V ? V[(int64_t)(l0 + q) * ldv + i] : w) : 0.0;
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            if (l0 + q >= cnt) break;
            const double p = warp_sum(v[q] * w);
            if (lane == 0) wsum[warp][l0 + q] = p;
        }
    }
    __syncthreads();
    if (t < cnt) {
        double s = 0.0;
        for (int q = 0; q < OW; ++q) s += wsum[q][t];
        mine[t] = s;
    }
    cl.sync();
    if (t < cnt) {
        double s = 0.0;
        for (unsigned r = 0; r < cl.num_blocks(); ++r) s += cl.map_shared_rank(mine, r)[t];
        res[t] = s;
    }
    __syncthreads();
}

// w -= V_{0..cnt-1} h (fma chain over ascending l).
__device__ __forceinline__ double subtract_projection(const double *V, int64_t ldv, int i, bool on, double w,
                                                      int cnt, const double *h) {
    if (!on) return w;
    for (int l0 = 0; l0 < cnt; l0 += kChunk) {
        double v[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q) v[q] = (l0 + q < cnt) ? V[(int64_t)(l0 + q) * ldv + i] : 0.0;
#pragma unroll
        for (int q = 0; q < kChunk; ++q)
            if (l0 + q < cnt) w = fma(-v[q], h[l0 + q], w);
    }
    return w;
}

// j = -1: column 0 holds P r; beta = ||P r||_2, v_0 = P r / beta, g_0 = beta.
// j >= 0: column j + 1 holds P A v_j; orthogonalize, normalize and rotate.
__global__ void __launch_bounds__(OT, 1) k_gm_orth(int n, double *V, int64_t ldv, int j, int m, double eta,
                                                    GmState *st) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ double wsum[OW][kMaxBasis + 1];
    __shared__ double part[3][kMaxBasis + 1];
    __shared__ double h[3][kMaxBasis + 1];
    if (j >= 0 && st->done) return;      // uniform: written by an earlier launch
    const int t = threadIdx.x;
    const unsigned rank = cl.block_rank();
    const int i = (int)rank * OT + t;
    const bool on = i < n;
    const int nv = j + 1;                 // vectors already in the basis
    double *col = V + (int64_t)(j + 1) * ldv;
    double w = on ? col[i] : 0.0;
    if (j >= 0) {
        cluster_dots(cl, V, ldv, i, on, w, nv, wsum, part[0], h[0]);
        w = subtract_projection(V, ldv, i, on, w, nv, h[0]);
        cluster_dots(cl, V, ldv, i, on, w, nv, wsum, part[1], h[1]);
        w = subtract_projection(V, ldv, i, on, w, nv, h[1]);
    }
    cluster_dots(cl, nullptr, ldv, i, on, w, 1, wsum, part[2], h[2]);
    const double hn = sqrt(h[2][0]);
    if (on && hn > 0.0) col[i] = w / hn;
    if (rank == 0 && t == 0) {
        if (j < 0) {
            st->beta = hn;
            st->g[0] = hn;
            st->k = 0;
            st->done = (hn > 0.0) ? 0 : 1;
        } else {
            double *Rc = st->R + (int64_t)j * kMaxBasis;      // column j
            for (int l = 0; l < nv; ++l) Rc[l] = __dadd_rn(h[0][l], h[1][l]);
            for (int l = 0; l < j; ++l) {                    // earlier rotations
                const double a = Rc[l], b = Rc[l + 1], c = st->cs[l], s = st->sn[l];
                Rc[l] = __dadd_rn(__dmul_rn(c, a), __dmul_rn(s, b));
                Rc[l + 1] = __dadd_rn(__dmul_rn(-s, a), __dmul_rn(c, b));
            }
            const double nu = hypot(Rc[j], hn);
            double c = 1.0, s = 0.0;
            if (nu != 0.0) {
                c = Rc[j] / nu;
                s = hn / nu;
            }
            Rc[j] = nu;
            st->cs[j] = c;
            st->sn[j] = s;
            const double gj = st->g[j];
            st->g[j + 1] = __dmul_rn(-s, gj);
            st->g[j] = __dmul_rn(c, gj);
            st->k = j + 1;
            st->done = (fabs(st->g[j + 1]) <= eta * st->beta || hn == 0.0 || j + 1 >= m) ? 1 : 0;
        }
    }
    cl.sync();      // no CTA leaves while another may still read its slots
}

__global__ void __launch_bounds__(256) k_gm_update(int n, const double *V, int64_t ldv, const GmState *st,
                                                    double *x, unsigned long long *dnorm_bits) {
    __shared__ double y[kMaxBasis];
    const int k = st->k;
    if (threadIdx.x == 0) {
        for (int i = k - 1; i >= 0; --i) {
            double acc = st->g[i];
            for (int l = i + 1; l < k; ++l) acc = __dsub_rn(acc, __dmul_rn(st->R[(int64_t)l * kMaxBasis + i], y[l]));
            const double rii = st->R[(int64_t)i * kMaxBasis + i];
            y[i] = (rii != 0.0) ? acc / rii : 0.0;
        }
    }
    __syncthreads();
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int l = 0; l < k; ++l) d = fma(V[(int64_t)l * ldv + i], y[l], d);
        x[i] += d;
        m = fmax(m, fabs(d));
        if (d != d) m = d;     // keep a NaN visible to the norm
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v = __shfl_xor_sync(0xffffffffu, m, o);
        m = (v != v || v > m) ? v : m;
    }
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(dnorm_bits, m);
}

}  // namespace

cudaError_t launch_gm_orth(int n, double *V, int64_t ldv, int j, int m, double eta, GmState *st,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int C = (n + OT - 1) / OT;
    if (C > kOrthMaxCluster || j >= kMaxBasis || m > kMaxBasis) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(k_gm_orth, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(OT, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute a[1];
    a[0].id = cudaLaunchAttributeClusterDimension;
    a[0].val.clusterDim.x = C;
    a[0].val.clusterDim.y = 1;
    a[0].val.clusterDim.z = 1;
    cfg.attrs = a;
    cfg.numAttrs = 1;
    count_launch();
    return cudaLaunchKernelEx(&cfg, k_gm_orth, n, V, ldv, j, m, eta, st);
}

cudaError_t launch_gm_update(int n, const double *V, int64_t ldv, const GmState *st, double *x,
                             unsigned long long *dnorm_bits, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int grid = (n + 255) / 256;
    if (grid > 64) grid = 64;
    count_launch();
    k_gm_update<<<grid, 256, 0, s>>>(n, V, ldv, st, x, dnorm_bits);
    return cudaGetLastError();
}

}  // namespace ir
