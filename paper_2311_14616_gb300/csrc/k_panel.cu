// Panel factorization, row interchanges and the U12 triangular solve of the
// blocked LU with partial pivoting ("Factor A = LU in precision TF",
// Algorithm IR; lu! of Sec. 2.1.1).
//
// The binary32 operations are exactly those of the unblocked right-looking
// algorithm: pivot = first row of maximal |a_ik|, l_ik = a_ik * fl(1/a_kk)
// (LAPACK getf2; a division below the smallest normal), a_ij = fmaf(-l_ik,
// u_kj, a_ij) with k ascending for every element.  Blocking only regroups
// these chains, so the factors are bitwise those of the unblocked algorithm
// whenever the trailing update is binary32.
#include <cfloat>
#include <climits>
#include <cstddef>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ir_internal.cuh"

namespace ir {
namespace {

constexpr int NB = kPanelNB;
constexpr int T = kPanelT;
constexpr int NW = T / 32;

// Rows never move between threads during a panel: every thread keeps its
// row and tracks the row's current position, so an interchange is two integer
// compares and the panel's net permutation is known at the end.
//
// Candidate exchange: at step k every warp stages its best row as a 272-byte
// record (|a| bits, position, fl(1/a), the 64 row values, pad) and the CTA's
// best record is pushed with one bulk copy per destination into slot
// [k & 1][its rank] of every CTA of the cluster, counted on the receiver's
// mbarrier.  A receiver waits (bounded) for all records of the step.
constexpr int kRec = 68;                     // floats per record
struct PanelSmem {
    // records first, each 16-byte aligned (they are accessed as float4)
    alignas(16) float stage[2][NW][kRec];    // per-warp candidate records, by step parity
    alignas(16) float recv[2][kPanelMaxCluster][kRec];
    alignas(8) unsigned long long recv_bar[2];
    int piv_log[NB];             // p_k of every step (the panel's interchanges)
    int zero_piv;                // first zero pivot of this panel (1-based), or 0
    int abort_flag;
};
static_assert(offsetof(PanelSmem, stage) % 16 == 0 && offsetof(PanelSmem, recv) % 16 == 0 &&
                  (kRec * 4) % 16 == 0,
              "float4 records of the panel's shared memory must be 16-byte aligned");
// Dynamic shared memory after PanelSmem: Ls[NB][T] multipliers by step and
// thread, Us[NB][NB] pivot rows.
constexpr size_t kPanelDynSmem = sizeof(PanelSmem) + sizeof(float) * (size_t)NB * T + sizeof(float) * NB * NB + 16;

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

// Bulk copy of `bytes` (multiple of 16) from this CTA's shared memory into
// another CTA's shared memory, counted on that CTA's mbarrier.
__device__ __forceinline__ void bulk_to_cta(unsigned rdst, unsigned src, unsigned bytes, unsigned rbar) {
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(rdst),
                 "r"(src), "r"(bytes), "r"(rbar)
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

// Store one operand row (NB values, rounded to TF) into Aop/Bop.
__device__ __forceinline__ void store_op_row(void *op, int64_t row, const float *v, ir_dtype tf) {
    if (tf == IR_TF32) {
        float4 *dst = reinterpret_cast<float4 *>(static_cast<float *>(op) + row * NB);
#pragma unroll
        for (int c = 0; c < NB; c += 4)
            dst[c / 4] = make_float4(round_tf(v[c], tf), round_tf(v[c + 1], tf), round_tf(v[c + 2], tf),
                                     round_tf(v[c + 3], tf));
    } else if (tf == IR_BF16) {
        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(op) + row * NB);
#pragma unroll
        for (int c = 0; c < NB; c += 8) {
            __nv_bfloat162 p[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) p[q] = __floats2bfloat162_rn(v[c + 2 * q], v[c + 2 * q + 1]);
            dst[c / 8] = *reinterpret_cast<uint4 *>(p);
        }
    } else if (tf == IR_F16) {
        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<__half *>(op) + row * NB);
#pragma unroll
        for (int c = 0; c < NB; c += 8) {
            __half2 p[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) p[q] = __floats2half2_rn(v[c + 2 * q], v[c + 2 * q + 1]);
            dst[c / 8] = *reinterpret_cast<uint4 *>(p);
        }
    }
}

// One cluster factors the panel AF[j:n, j:j+nbp].  Thread t of CTA c keeps
// row j + c*T + t for the whole panel in a rotating register window: at step
// k, a[i] holds column j+k+i (zero past the panel), so the current column is
// always a[0] and the update a[i] <- fmaf(-l, u[i+1], a[i+1]) also shifts the
// window.  Per column k: warp candidate (largest |a|, ties to the lowest
// current position: redux.sync) staged as a record -> the CTA's best record
// pushed to every CTA (bulk copies, issued by one lane per destination) ->
// bounded wait on the local mbarrier -> every warp picks the pivot row from
// the received headers -> positions k and p swap labels -> scaling by the
// pivot's reciprocal and rank-1 update of the rows that are not pivot rows.
// The column loop touches no global memory.  At the end each thread writes
// its row to its final position: the multipliers of the steps before the row
// became a pivot row (its own column of Ls), then the U part staged at that
// step.  Rows that moved are listed as (destination, origin) pairs in
// swap_list (count in swap_list[0]) for the interchanges of the other
// columns, and perm is composed with the panel's permutation.
__global__ void __launch_bounds__(T, 1)
    k_panel(float *AF, int64_t ldf, int n, int j, int nbp, int32_t *ipiv, int32_t *perm,
            int32_t *swap_list, DevScalars *dev, ir_dtype tf, void *Aop, int has_trailing) {
    extern __shared__ __align__(16) unsigned char panel_smem[];
    PanelSmem &sm = *reinterpret_cast<PanelSmem *>(panel_smem);
    float *Ls = reinterpret_cast<float *>(panel_smem + sizeof(PanelSmem));   // [NB][T]
    float *Us = Ls + (size_t)NB * T;                                          // [NB][NB]
    const unsigned crank = cluster_rank();
    const unsigned csize = cluster_size();
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int home = (int)crank * T + t;             // this row's position at the start, relative to j
    const bool valid = j + home < n;
    const unsigned step_bytes = csize * (unsigned)(kRec * 4);

    int pos = home;          // current position, relative to j
    int kp = nbp;            // the step at which the row became the pivot row (nbp: never)
    if (crank == 0 && t == 0) swap_list[0] = 0;
    if (t == 0) {
        sm.zero_piv = 0;
        sm.abort_flag = 0;
        mbar_init_p(smem_u32(&sm.recv_bar[0]), 1);
        mbar_init_p(smem_u32(&sm.recv_bar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect_arrive(smem_u32(&sm.recv_bar[0]), step_bytes);
        if (nbp > 1) mbar_expect_arrive(smem_u32(&sm.recv_bar[1]), step_bytes);
    }
    float a[NB];
    if (valid) {
        const float4 *src = reinterpret_cast<const float4 *>(AF + (int64_t)(j + home) * ldf + j);
#pragma unroll
        for (int c = 0; c < NB; c += 4) {
            float4 v = (c < nbp) ? src[c / 4] : make_float4(0.f, 0.f, 0.f, 0.f);
            a[c] = v.x; a[c + 1] = v.y; a[c + 2] = v.z; a[c + 3] = v.w;
        }
#pragma unroll
        for (int c = 0; c < NB; ++c)
            if (c >= nbp) a[c] = 0.f;
    } else {
#pragma unroll
        for (int c = 0; c < NB; ++c) a[c] = 0.f;
    }
    cluster_sync_all();   // every CTA is running and its mbarriers are armed
    const unsigned long long deadline = globaltimer() + kWaitLimitNs;   // for all waits of this launch

    const unsigned recv_addr = smem_u32(&sm.recv[0][0][0]);
    const unsigned bar_addr = smem_u32(&sm.recv_bar[0]);

#pragma unroll 1
    for (int k = 0; k < nbp; ++k) {
        const int buf = k & 1;
        // 1. warp candidate: largest |a_ik| over the rows that are not pivot
        //    rows yet, ties to the lowest current position; staged as a record
        const bool cand = valid && kp == nbp;
        const unsigned key = cand ? __float_as_uint(fabsf(a[0])) : 0u;
        const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
        const int mpos = __reduce_min_sync(0xffffffffu, (cand && key == kmax) ? pos : INT_MAX);
        float *st = sm.stage[buf][warp];
        if (cand && pos == mpos) {
            float4 *s4 = reinterpret_cast<float4 *>(st);
            s4[0] = make_float4(__uint_as_float(kmax), __int_as_float(mpos), (a[0] != 0.f) ? 1.0f / a[0] : 0.f, a[0]);
#pragma unroll
            for (int q = 0; q < 15; ++q)
                s4[1 + q] = make_float4(a[4 * q + 1], a[4 * q + 2], a[4 * q + 3], a[4 * q + 4]);
            s4[16] = make_float4(a[61], a[62], a[63], 0.f);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> bulk copy
        }
        if (lane == 0 && mpos == INT_MAX) {
            st[0] = 0.f;
            st[1] = __int_as_float(INT_MAX);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
        // 2. the CTA's best record, pushed to every CTA of the cluster (one lane per destination)
        if (warp == 0) {
            const unsigned wk = lane < NW ? __float_as_uint(sm.stage[buf][lane][0]) : 0u;
            const int wp = lane < NW ? __float_as_int(sm.stage[buf][lane][1]) : INT_MAX;
            const unsigned bk = __reduce_max_sync(0xffffffffu, wk);
            const int bp = __reduce_min_sync(0xffffffffu, (wp != INT_MAX && wk == bk) ? wp : INT_MAX);
            const unsigned who = __ballot_sync(0xffffffffu, lane < NW && wp == bp);
            const int w = who ? __ffs(who) - 1 : 0;
            if (lane < (int)csize) {
                const unsigned rbar = map_cta(bar_addr + 8u * buf, (unsigned)lane);
                const unsigned slot = recv_addr + (unsigned)((buf * kPanelMaxCluster + (int)crank) * kRec * 4);
                bulk_to_cta(map_cta(slot, (unsigned)lane), smem_u32(sm.stage[buf][w]), kRec * 4, rbar);
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");   // the stage slot may be reused
            }
        }
        // 3. every warp waits (bounded) for the records of all CTAs of this step
        const unsigned par = (unsigned)(k >> 1) & 1u;
        if (lane == 0 && !sm.abort_flag) {
            while (!mbar_try_wait_cluster(bar_addr + 8u * buf, par)) {
                if (globaltimer() > deadline) {      // give up: report, carry on without waiting
                    sm.abort_flag = 1;
                    atomicExch(&dev->timeout, 1);
                    break;
                }
            }
        }
        __syncwarp();
        // re-arm this buffer for step k + 2 (before this CTA sends its next record)
        if (t == 0 && k + 2 < nbp && !sm.abort_flag) mbar_expect_arrive(bar_addr + 8u * buf, step_bytes);
        // 4. the pivot row, picked by every warp from the received headers
        const float *rb = sm.recv[buf][0];
        const unsigned ck = lane < (int)csize ? __float_as_uint(rb[lane * kRec]) : 0u;
        const int cp = lane < (int)csize ? __float_as_int(rb[lane * kRec + 1]) : INT_MAX;
        const unsigned ckmax = __reduce_max_sync(0xffffffffu, ck);
        const int ppos = __reduce_min_sync(0xffffffffu, (cp != INT_MAX && ck == ckmax) ? cp : INT_MAX);
        const unsigned cwho = __ballot_sync(0xffffffffu, lane < (int)csize && cp == ppos);
        const int wc = cwho ? __ffs(cwho) - 1 : 0;
        const float *u = rb + wc * kRec;                // u[3 + i] = pivot row, column j + k + i
        const float piv = u[3];
        const float r = u[2];
        if (t == 0) {
            sm.piv_log[k] = j + ppos;
            if (piv == 0.f && sm.zero_piv == 0) sm.zero_piv = j + k + 1;
        }
        // 5. interchange of positions k and ppos: labels only
        if (cand && pos == ppos) {
            pos = k;
            kp = k;
        } else if (pos == k) {
            pos = ppos;
        }
        if (warp == 1) {
            Us[k * NB + lane] = u[3 + lane];
            Us[k * NB + lane + 32] = u[35 + lane];
        }
        // 6. scale column k (getf2: by the reciprocal, divide below the smallest
        //    normal), update and shift the live part of the window
        if (valid && kp == nbp) {
            float l = a[0];
            if (piv != 0.f) l = (fabsf(piv) >= FLT_MIN) ? l * r : l / piv;
            Ls[k * T + t] = l;
            const float4 *us = reinterpret_cast<const float4 *>(u + 4);   // u[4 + c] = column k+1+c
            const int live = nbp - k;                                        // a[0..live-1] nonzero
#pragma unroll
            for (int q = 0; q < NB / 4; ++q) {
                if (4 * q < live) {
                    const float4 w = us[q];
                    a[4 * q + 0] = fmaf(-l, w.x, a[4 * q + 1]);
                    a[4 * q + 1] = fmaf(-l, w.y, a[4 * q + 2]);
                    a[4 * q + 2] = fmaf(-l, w.z, a[4 * q + 3]);
                    a[4 * q + 3] = (4 * q + 3 < NB - 1) ? fmaf(-l, w.w, a[4 * q + 4]) : 0.f;
                }
            }
        }
    }
    // net permutation of the panel: position j + pos now holds the row that started at j + home
    int porg = 0;
    const bool moved = valid && pos != home;
    if (moved) {
        int e = atomicAdd(&swap_list[0], 1);
        swap_list[1 + 2 * e] = j + pos;
        swap_list[2 + 2 * e] = j + home;
        porg = perm[j + home];
    }
    if (crank == 0) {
        for (int k = t; k < nbp; k += T) ipiv[j + k] = sm.piv_log[k];
        if (t == 0 && sm.zero_piv) atomicMin(&dev->info, sm.zero_piv);
    }
    cluster_sync_all();   // every perm read of the cluster is done
    if (moved) perm[j + pos] = porg;
    if (valid) {
        // the row at its final position: multipliers of steps < kp, then the U part staged at step kp
#pragma unroll
        for (int c = 0; c < NB; ++c) a[c] = (c < kp) ? Ls[c * T + t] : (c < nbp ? Us[kp * NB + (c - kp)] : 0.f);
        float4 *dst = reinterpret_cast<float4 *>(AF + (int64_t)(j + pos) * ldf + j);
#pragma unroll
        for (int c = 0; c < NB; c += 4)
            if (c < nbp) dst[c / 4] = make_float4(a[c], a[c + 1], a[c + 2], a[c + 3]);
        if (has_trailing && Aop != nullptr && pos >= NB) store_op_row(Aop, pos - NB, a, tf);
    }
    cluster_sync_all();   // no CTA leaves while its shared memory may be written
}

// Apply the panel's row permutation to the columns [c0a, c1a) and [c0b, c1b):
// A[dst][c] = A[src][c] for the (dst, src) pairs the panel listed.  All
// sources of a column are read before any destination is written.
constexpr int kLaswpT = 64;   // 2*NB*kLaswpT floats of staging stay under 48 KB
__global__ void __launch_bounds__(kLaswpT) k_laswp(float *AF, int64_t ldf, int c0a, int c1a, int c0b, int c1b,
                                                  const int32_t *swap_list) {
    __shared__ int sd[2 * NB], ss[2 * NB];
    __shared__ float vals[2 * NB][kLaswpT];
    const int cnt = swap_list[0];
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        sd[e] = swap_list[1 + 2 * e];
        ss[e] = swap_list[2 + 2 * e];
    }
    __syncthreads();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int na = c1a - c0a;
    if (c >= na + (c1b - c0b) || cnt == 0) return;
    c = (c < na) ? c0a + c : c0b + (c - na);
    for (int e = 0; e < cnt; ++e) vals[e][threadIdx.x] = AF[(int64_t)ss[e] * ldf + c];
    for (int e = 0; e < cnt; ++e) AF[(int64_t)sd[e] * ldf + c] = vals[e][threadIdx.x];
}

// U12 = L11^{-1} A12 for the block row j..j+NB and columns j+NB..n.  One
// thread per column, its NB values in registers, L11 in shared memory; each
// u_kc is the fmaf chain over m < k in ascending order.  For tensor-core
// updates the rounded values rTF(u_mc) are also written to Bop (row c).
__global__ void __launch_bounds__(128) k_trsm(float *AF, int64_t ldf, int cb, int ce, int j, ir_dtype tf,
                                              void *Bop) {
    __shared__ float L[NB][NB + 1];
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        int r = e / NB, m = e % NB;
        L[r][m] = AF[(int64_t)(j + r) * ldf + j + m];
    }
    __syncthreads();
    const int c = cb + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ce) return;
    float u[NB];
#pragma unroll
    for (int m = 0; m < NB; ++m) u[m] = AF[(int64_t)(j + m) * ldf + c];
#pragma unroll
    for (int k = 1; k < NB; ++k)
#pragma unroll
        for (int m = 0; m < k; ++m) u[k] = fmaf(-L[k][m], u[m], u[k]);
#pragma unroll
    for (int m = 1; m < NB; ++m) AF[(int64_t)(j + m) * ldf + c] = u[m];
    if (Bop != nullptr) store_op_row(Bop, c - (j + NB), u, tf);
}

__global__ void k_iota(int n, int32_t *perm) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) perm[i] = i;
}

}  // namespace

cudaError_t launch_panel(float *AF, int64_t ldf, int n, int j, int nbp, int32_t *ipiv,
                         int32_t *perm, int32_t *swap_list, DevScalars *dev, ir_dtype tf,
                         void *Aop, cudaStream_t s) {
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_panel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPanelDynSmem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    int M = n - j;
    int C = (M + T - 1) / T;
    if (C > kPanelMaxCluster) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(T, 1, 1);
    cfg.dynamicSmemBytes = kPanelDynSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int has_trailing = (j + NB < n) ? 1 : 0;
    count_launch();
    return cudaLaunchKernelEx(&cfg, k_panel, AF, ldf, n, j, nbp, ipiv, perm, swap_list, dev, tf, Aop,
                              has_trailing);
}

cudaError_t launch_laswp(float *AF, int64_t ldf, int c0a, int c1a, int c0b, int c1b, const int32_t *swap_list,
                         cudaStream_t s) {
    const int ncols = (c1a - c0a) + (c1b - c0b);
    if (ncols <= 0) return cudaSuccess;
    count_launch();
    k_laswp<<<(ncols + kLaswpT - 1) / kLaswpT, kLaswpT, 0, s>>>(AF, ldf, c0a, c1a, c0b, c1b, swap_list);
    return cudaGetLastError();
}

// U12 for the columns [cb, ce) of the block row j..j+NB.
cudaError_t launch_trsm(float *AF, int64_t ldf, int cb, int ce, int j, ir_dtype tf, void *Bop, cudaStream_t s) {
    const int ncols = ce - cb;
    if (ncols <= 0) return cudaSuccess;
    count_launch();
    k_trsm<<<(ncols + 127) / 128, 128, 0, s>>>(AF, ldf, cb, ce, j, tf, tf == IR_F32 ? nullptr : Bop);
    return cudaGetLastError();
}

cudaError_t launch_iota(int n, int32_t *perm, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    count_launch();
    k_iota<<<(n + 255) / 256, 256, 0, s>>>(n, perm);
    return cudaGetLastError();
}

}  // namespace ir
