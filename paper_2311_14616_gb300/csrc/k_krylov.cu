// Krylov solvers for the correction equation of Krylov-IR (Sec. 4.2-4.3):
// the scalar and vector work of GMRES and of BiCGSTAB between the
// preconditioned products P A v (formed by the residual kernels with b = NULL
// and the solve pair with P = U^{-1} L^{-1}, eq. pdef).
//
// k_gm_orth: one thread-block cluster of up to 16 CTAs x 256 threads, one or
// two basis rows per thread (8192 rows at most).  Classical Gram-Schmidt run twice against
// v_0..v_j, the 2-norm, the normalization of v_{j+1}, then the Givens step on
// column j of the Hessenberg matrix and the stopping test.  Every dot product
// is summed lane-butterfly -> warps in order -> CTAs in rank order through
// distributed shared memory, so all CTAs see bitwise the same values and the
// result does not depend on scheduling.
// k_gm_update: y = R^{-1} g (back substitution, k <= 64), d = V_k y, x += d.
// k_bi_step: one phase of a BiCGSTAB iteration in one cluster, the same
// deterministic cluster sums; every scalar is formed by one thread and
// broadcast through shared memory.
#include <cooperative_groups.h>

#include "ir_internal.cuh"

namespace cg = cooperative_groups;

namespace ir {
namespace {

constexpr int OT = 256;               // threads per CTA
constexpr int OW = OT / 32;
constexpr int kOrthMaxCluster = 16;
constexpr int kChunk = 4;             // dot products reduced together

// Butterfly sum of one value over the warp (every lane ends with the total).
__device__ __forceinline__ double warp_sum1(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sums of four values by recursive halving: 6 binary64 additions per lane
// instead of 20 (binary64 throughput is the scarce resource on this part).
// Lane l ends with the total of value q(l) = 2 * bit4(l) + bit3(l).
__device__ __forceinline__ double warp_sum4(const double (&p)[4], int lane) {
    const bool h16 = lane & 16, h8 = lane & 8;
    double k0 = h16 ? p[2] : p[0], k1 = h16 ? p[3] : p[1];
    k0 += __shfl_xor_sync(0xffffffffu, h16 ? p[0] : p[2], 16);
    k1 += __shfl_xor_sync(0xffffffffu, h16 ? p[1] : p[3], 16);
    double k = h8 ? k1 : k0;
    k += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
    k += __shfl_xor_sync(0xffffffffu, k, 4);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    k += __shfl_xor_sync(0xffffffffu, k, 1);
    return k;
}

// Sum the per-warp partials of wsum[.][0..cnt) in warp order into this CTA's
// exchange slot, then the slots of all CTAs in rank order into res (every CTA
// gets bitwise the same totals).  mine is a different slot per call so that no
// CTA overwrites a slot another still reads.
__device__ __forceinline__ void cluster_total(const cg::cluster_group &cl, int cnt, double (*wsum)[kMaxBasis + 1],
                                              double *mine, double *res) {
    const int t = threadIdx.x;
    __syncthreads();
    if (t < cnt) {
        double v[OW];
#pragma unroll
        for (int q = 0; q < OW; ++q) v[q] = wsum[q][t];
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < OW; ++q) s += v[q];
        mine[t] = s;
    }
    cl.sync();
    if (t < cnt) {
        const unsigned C = cl.num_blocks();
        double v[kOrthMaxCluster];
#pragma unroll
        for (unsigned r = 0; r < kOrthMaxCluster; ++r) v[r] = (r < C) ? cl.map_shared_rank(mine, r)[t] : 0.0;
        double s = 0.0;
#pragma unroll
        for (unsigned r = 0; r < kOrthMaxCluster; ++r)
            if (r < C) s += v[r];
        res[t] = s;
    }
    __syncthreads();
}

// res[l] = sum over the cluster's rows of V_il w_i, l < cnt.  A thread's RPT
// rows are combined first (fma in row order), then warps, CTAs, the cluster.
template <int RPT>
__device__ void cluster_dots(const cg::cluster_group &cl, const double *V, int64_t ldv, const int (&i)[RPT],
                             const bool (&on)[RPT], const double (&w)[RPT], int cnt,
                             double (*wsum)[kMaxBasis + 1], double *mine, double *res) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int l0 = 0; l0 < cnt; l0 += kChunk) {
        double p[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            double acc = 0.0;
#pragma unroll
            for (int r = 0; r < RPT; ++r)
                if (on[r] && l0 + q < cnt) acc = fma(V[(int64_t)(l0 + q) * ldv + i[r]], w[r], acc);
            p[q] = acc;
        }
        const double sum = warp_sum4(p, lane);
        const int q = 2 * ((lane >> 4) & 1) + ((lane >> 3) & 1);
        if ((lane & 7) == 0 && l0 + q < cnt) wsum[warp][l0 + q] = sum;
    }
    cluster_total(cl, cnt, wsum, mine, res);
}

// res[0] = sum over the cluster's rows of w_i^2.
template <int RPT>
__device__ void cluster_norm2(const cg::cluster_group &cl, const bool (&on)[RPT], const double (&w)[RPT],
                              double (*wsum)[kMaxBasis + 1], double *mine, double *res) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc = 0.0;
#pragma unroll
    for (int r = 0; r < RPT; ++r)
        if (on[r]) acc = fma(w[r], w[r], acc);
    acc = warp_sum1(acc);
    if (lane == 0) wsum[warp][0] = acc;
    cluster_total(cl, 1, wsum, mine, res);
}

// w -= V_{0..cnt-1} h for each row (fma chain over ascending l).
template <int RPT>
__device__ __forceinline__ void subtract_projection(const double *V, int64_t ldv, const int (&i)[RPT],
                                                    const bool (&on)[RPT], double (&w)[RPT], int cnt,
                                                    const double *h) {
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        if (!on[r]) continue;
        for (int l0 = 0; l0 < cnt; l0 += kChunk) {
            double v[kChunk];
#pragma unroll
            for (int q = 0; q < kChunk; ++q) v[q] = (l0 + q < cnt) ? V[(int64_t)(l0 + q) * ldv + i[r]] : 0.0;
#pragma unroll
            for (int q = 0; q < kChunk; ++q)
                if (l0 + q < cnt) w[r] = fma(-v[q], h[l0 + q], w[r]);
        }
    }
}

// j = -1: column 0 holds P r; beta = ||P r||_2, v_0 = P r / beta, g_0 = beta.
// j >= 0: column j + 1 holds P A v_j; orthogonalize, normalize and rotate.
// CTA c of the cluster owns rows c RPT OT .. (c + 1) RPT OT - 1, thread t rows
// c RPT OT + t + r OT (coalesced).
template <int RPT>
__global__ void __launch_bounds__(OT, 1) k_gm_orth(int n, double *V, int64_t ldv, int j, int m, double eta,
                                                    GmState *st) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ double wsum[OW][kMaxBasis + 1];
    __shared__ double part[3][kMaxBasis + 1];
    __shared__ double h[3][kMaxBasis + 1];
    __shared__ double rot[2][kMaxBasis];   // the earlier rotations (c, s), read while the dots run
    __shared__ double gb[2];               // g_j, beta
    __shared__ double colj[kMaxBasis + 1]; // column j of H while it is rotated
    __shared__ double ninv[2];             // ||w||_2 and its reciprocal
    if (j >= 0 && st->done) return;      // uniform: written by an earlier launch
    const int t = threadIdx.x;
    const unsigned rank = cl.block_rank();
    if (rank == 0 && j >= 0) {
        if (t < j) {
            rot[0][t] = st->cs[t];
            rot[1][t] = st->sn[t];
        }
        if (t == 0) {
            gb[0] = st->g[j];
            gb[1] = st->beta;
        }
    }
    int i[RPT];
    bool on[RPT];
    double w[RPT];
    const int nv = j + 1;                 // vectors already in the basis
    double *col = V + (int64_t)(j + 1) * ldv;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        i[r] = (int)rank * RPT * OT + r * OT + t;
        on[r] = i[r] < n;
        w[r] = on[r] ? col[i[r]] : 0.0;
    }
    if (j >= 0) {
        cluster_dots<RPT>(cl, V, ldv, i, on, w, nv, wsum, part[0], h[0]);
        subtract_projection<RPT>(V, ldv, i, on, w, nv, h[0]);
        cluster_dots<RPT>(cl, V, ldv, i, on, w, nv, wsum, part[1], h[1]);
        subtract_projection<RPT>(V, ldv, i, on, w, nv, h[1]);
    }
    cluster_norm2<RPT>(cl, on, w, wsum, part[2], h[2]);
    // one thread takes the square root and the reciprocal (binary64 throughput is
    // scarce: every thread doing them costs microseconds); v_{j+1} = w * (1 / ||w||)
    if (t == 0) {
        const double nrm = sqrt(h[2][0]);
        ninv[0] = nrm;
        ninv[1] = (nrm > 0.0) ? 1.0 / nrm : 0.0;
    }
    __syncthreads();
    const double hn = ninv[0], inv = ninv[1];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
        if (on[r] && hn > 0.0) col[i[r]] = w[r] * inv;
    if (rank == 0 && t == 0) {
        if (j < 0) {
            st->beta = hn;
            st->g[0] = hn;
            st->k = 0;
            st->done = (hn > 0.0) ? 0 : 1;
        } else {
            double *Rc = colj;
            for (int l = 0; l < nv; ++l) Rc[l] = __dadd_rn(h[0][l], h[1][l]);
            for (int l = 0; l < j; ++l) {                    // earlier rotations
                const double a = Rc[l], b = Rc[l + 1], c = rot[0][l], s = rot[1][l];
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
            double *Rg = st->R + (int64_t)j * kMaxBasis;
            for (int l = 0; l < nv; ++l) Rg[l] = Rc[l];
            st->cs[j] = c;
            st->sn[j] = s;
            const double gj = gb[0], gn = __dmul_rn(-s, gj);
            st->g[j + 1] = gn;
            st->g[j] = __dmul_rn(c, gj);
            st->k = j + 1;
            st->done = (fabs(gn) <= eta * gb[1] || hn == 0.0 || j + 1 >= m) ? 1 : 0;
        }
    }
    cl.sync();      // no CTA leaves while another may still read its slots
}

__global__ void __launch_bounds__(256) k_gm_update(int n, const double *V, int64_t ldv, const GmState *st,
                                                    double *x, unsigned long long *dnorm_bits,
                                                    unsigned long long *xnorm_bits) {
    __shared__ double y[kMaxBasis];
    __shared__ double Rs[kMaxBasis * kMaxBasis];
    const int k = st->k;
    for (int e = threadIdx.x; e < k * kMaxBasis; e += blockDim.x) Rs[e] = st->R[e];   // columns 0..k-1
    if (threadIdx.x < k) y[threadIdx.x] = st->g[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = k - 1; i >= 0; --i) {
            double acc = y[i];
            for (int l = i + 1; l < k; ++l) acc = __dsub_rn(acc, __dmul_rn(Rs[l * kMaxBasis + i], y[l]));
            const double rii = Rs[i * kMaxBasis + i];
            y[i] = (rii != 0.0) ? acc / rii : 0.0;
        }
    }
    __syncthreads();
    double m = 0.0, xm = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int l = 0; l < k; ++l) d = fma(V[(int64_t)l * ldv + i], y[l], d);
        const double xn = x[i] + d;
        x[i] = xn;
        m = fmax(m, fabs(d));
        if (d != d) m = d;     // keep a NaN visible to the norm
        xm = fmax(xm, fabs(xn));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v = __shfl_xor_sync(0xffffffffu, m, o);
        m = (v != v || v > m) ? v : m;
        xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(dnorm_bits, m);
        atomic_max_nonneg(xnorm_bits, xm);
    }
}

// Warp sums of two values by recursive halving (5 additions per lane): lane l
// ends with the total of value bit4(l).
__device__ __forceinline__ double warp_sum2(double a, double b, int lane) {
    const bool h16 = lane & 16;
    double k = h16 ? b : a;
    k += __shfl_xor_sync(0xffffffffu, h16 ? a : b, 16);
    k += __shfl_xor_sync(0xffffffffu, k, 8);
    k += __shfl_xor_sync(0xffffffffu, k, 4);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    k += __shfl_xor_sync(0xffffffffu, k, 1);
    return k;
}

// res[0] = sum over the cluster's rows of a_i, res[1] = of b_i (per-thread
// partial sums a, b over the thread's rows).
__device__ __forceinline__ void cluster_sum2(const cg::cluster_group &cl, double a, double b,
                                             double (*wsum)[kMaxBasis + 1], double *mine, double *res) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double k = warp_sum2(a, b, lane);
    if ((lane & 15) == 0) wsum[warp][lane >> 4] = k;
    cluster_total(cl, 2, wsum, mine, res);
}

// One BiCGSTAB phase (van der Vorst) on P A d = z, z = P r in column kBiR.
//   0: z0 = ||z||_2; r^ = r; p = v = d = 0; rho_old = alpha = omega = 1.
//   1: rho = <r^, r>; beta = (rho / rho_old)(alpha / omega); p = r + beta (p - omega v).
//   2: (v = P A p) alpha = rho / <r^, v>; s = r - alpha v; k += 1;
//      ||s||_2 <= eta z0: d += alpha p, stop.
//   3: (t = P A s) omega = <t, s> / <t, t>; d += alpha p + omega s; r = s - omega t;
//      stop when ||r||_2 <= eta z0, omega = 0 or k = kmax.
// A zero rho, <r^, v> or <t, t> stops with the current d.
template <int RPT>
__global__ void __launch_bounds__(OT, 1) k_bi_step(int phase, int n, double *Vb, int64_t ldv, int kmax,
                                                    double eta, BiState *st) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ double wsum[OW][kMaxBasis + 1];
    __shared__ double part[3][kMaxBasis + 1];
    __shared__ double res[3][kMaxBasis + 1];
    __shared__ double sc[4];           // broadcast scalars
    __shared__ int stop;
    if (phase > 0 && st->done) return;     // uniform: written by an earlier launch
    const int t = threadIdx.x;
    const unsigned rank = cl.block_rank();
    double *r = Vb + kBiR * ldv, *rh = Vb + kBiRh * ldv, *p = Vb + kBiP * ldv, *v = Vb + kBiV * ldv;
    double *s = Vb + kBiS * ldv, *tv = Vb + kBiT * ldv, *d = Vb + kBiD * ldv;
    int i[RPT];
    bool on[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        i[q] = (int)rank * RPT * OT + q * OT + t;
        on[q] = i[q] < n;
    }
    const bool lead = (rank == 0 && t == 0);
    if (phase == 0) {
        double a = 0.0;
#pragma unroll
        for (int q = 0; q < RPT; ++q)
            if (on[q]) {
                const double z = r[i[q]];
                a = fma(z, z, a);
                rh[i[q]] = z;
                p[i[q]] = v[i[q]] = d[i[q]] = 0.0;
            }
        cluster_sum2(cl, a, 0.0, wsum, part[0], res[0]);
        if (lead) {
            const double z0 = sqrt(res[0][0]);
            st->z0 = z0;
            st->rho_old = st->alpha = st->omega = 1.0;
            st->k = 0;
            st->done = (z0 > 0.0 && kmax >= 1) ? 0 : 1;
        }
    } else if (phase == 1) {
        double a = 0.0;
#pragma unroll
        for (int q = 0; q < RPT; ++q)
            if (on[q]) a = fma(rh[i[q]], r[i[q]], a);
        cluster_sum2(cl, a, 0.0, wsum, part[0], res[0]);
        if (t == 0) {
            const double rho = res[0][0];
            sc[0] = (rho / st->rho_old) * (st->alpha / st->omega);   // beta
            sc[1] = st->omega;
            stop = (rho == 0.0);
            if (lead) {
                st->rho = rho;
                if (rho == 0.0) st->done = 1;
            }
        }
        __syncthreads();
        if (!stop) {
            const double beta = sc[0], om = sc[1];
#pragma unroll
            for (int q = 0; q < RPT; ++q)
                if (on[q]) p[i[q]] = r[i[q]] + beta * (p[i[q]] - om * v[i[q]]);
        }
    } else if (phase == 2) {
        double a = 0.0;
#pragma unroll
        for (int q = 0; q < RPT; ++q)
            if (on[q]) a = fma(rh[i[q]], v[i[q]], a);
        cluster_sum2(cl, a, 0.0, wsum, part[0], res[0]);
        if (t == 0) {
            const double sig = res[0][0];
            sc[0] = (sig != 0.0) ? st->rho / sig : 0.0;   // alpha
            stop = (sig == 0.0);
            if (lead && sig == 0.0) st->done = 1;
        }
        __syncthreads();
        if (!stop) {
            const double alpha = sc[0];
            double b2 = 0.0;
            double sv[RPT];
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                sv[q] = 0.0;
                if (on[q]) {
                    sv[q] = r[i[q]] - alpha * v[i[q]];
                    s[i[q]] = sv[q];
                    b2 = fma(sv[q], sv[q], b2);
                }
            }
            cluster_sum2(cl, b2, 0.0, wsum, part[1], res[1]);
            if (t == 0) stop = sqrt(res[1][0]) <= eta * st->z0;    // one thread: binary64 is scarce
            __syncthreads();
            const bool small = stop;
            if (small) {
#pragma unroll
                for (int q = 0; q < RPT; ++q)
                    if (on[q]) d[i[q]] = d[i[q]] + alpha * p[i[q]];
            }
            if (lead) {
                st->alpha = alpha;
                st->k += 1;
                if (small) st->done = 1;
            }
        }
    } else {
        double a = 0.0, b2 = 0.0;
#pragma unroll
        for (int q = 0; q < RPT; ++q)
            if (on[q]) {
                const double tq = tv[i[q]];
                a = fma(tq, s[i[q]], a);
                b2 = fma(tq, tq, b2);
            }
        cluster_sum2(cl, a, b2, wsum, part[0], res[0]);
        if (t == 0) {
            const double ts = res[0][0], tt = res[0][1];
            sc[0] = st->alpha;
            sc[1] = (tt != 0.0) ? ts / tt : 0.0;   // omega
            stop = (tt == 0.0);
        }
        __syncthreads();
        const double alpha = sc[0], om = sc[1];
        double c2 = 0.0;
#pragma unroll
        for (int q = 0; q < RPT; ++q)
            if (on[q]) {
                const double sq = s[i[q]];
                if (stop) {
                    d[i[q]] = d[i[q]] + alpha * p[i[q]];
                } else {
                    d[i[q]] = (d[i[q]] + alpha * p[i[q]]) + om * sq;
                    const double rq = sq - om * tv[i[q]];
                    r[i[q]] = rq;
                    c2 = fma(rq, rq, c2);
                }
            }
        cluster_sum2(cl, c2, 0.0, wsum, part[1], res[1]);
        if (lead) {
            const double rn = sqrt(res[1][0]);
            st->omega = om;
            st->rho_old = st->rho;
            if (stop || rn <= eta * st->z0 || om == 0.0 || st->k >= kmax) st->done = 1;
        }
    }
    cl.sync();      // no CTA leaves while another may still read its slots
}

__global__ void __launch_bounds__(256) k_axpy_norms(int n, const double *d, double *x,
                                                     unsigned long long *dnorm_bits,
                                                     unsigned long long *xnorm_bits) {
    double m = 0.0, xm = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double di = d[i], xn = x[i] + di;
        x[i] = xn;
        m = fmax(m, fabs(di));
        if (di != di) m = di;
        xm = fmax(xm, fabs(xn));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v = __shfl_xor_sync(0xffffffffu, m, o);
        m = (v != v || v > m) ? v : m;
        xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(dnorm_bits, m);
        atomic_max_nonneg(xnorm_bits, xm);
    }
}

}  // namespace

cudaError_t launch_gm_orth(int n, double *V, int64_t ldv, int j, int m, double eta, GmState *st,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    // one row per thread while 16 CTAs suffice, else two (n <= 8192)
    const int rpt = (n <= kOrthMaxCluster * OT) ? 1 : 2;
    const int C = (n + rpt * OT - 1) / (rpt * OT);
    if (C > kOrthMaxCluster || j >= kMaxBasis || m > kMaxBasis) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_gm_orth<1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gm_orth<2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
    if (rpt == 1) return cudaLaunchKernelEx(&cfg, k_gm_orth<1>, n, V, ldv, j, m, eta, st);
    return cudaLaunchKernelEx(&cfg, k_gm_orth<2>, n, V, ldv, j, m, eta, st);
}

cudaError_t launch_gm_update(int n, const double *V, int64_t ldv, const GmState *st, double *x,
                             unsigned long long *dnorm_bits, unsigned long long *xnorm_bits, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int grid = (n + 255) / 256;
    if (grid > 64) grid = 64;
    count_launch();
    k_gm_update<<<grid, 256, 0, s>>>(n, V, ldv, st, x, dnorm_bits, xnorm_bits);
    return cudaGetLastError();
}

}  // namespace ir

namespace ir {

cudaError_t launch_bi_step(int phase, int n, double *Vb, int64_t ldv, int kmax, double eta, BiState *st,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int rpt = (n <= kOrthMaxCluster * OT) ? 1 : 2;
    const int C = (n + rpt * OT - 1) / (rpt * OT);
    if (C > kOrthMaxCluster || phase < 0 || phase > 3) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_bi_step<1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bi_step<2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
    if (rpt == 1) return cudaLaunchKernelEx(&cfg, k_bi_step<1>, phase, n, Vb, ldv, kmax, eta, st);
    return cudaLaunchKernelEx(&cfg, k_bi_step<2>, phase, n, Vb, ldv, kmax, eta, st);
}

cudaError_t launch_axpy_norms(int n, const double *d, double *x, unsigned long long *dnorm_bits,
                              unsigned long long *xnorm_bits, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int grid = (n + 255) / 256;
    if (grid > 64) grid = 64;
    count_launch();
    k_axpy_norms<<<grid, 256, 0, s>>>(n, d, x, dnorm_bits, xnorm_bits);
    return cudaGetLastError();
}

}  // namespace ir
