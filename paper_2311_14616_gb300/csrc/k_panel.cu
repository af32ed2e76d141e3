// Panel factorization, row interchanges and the U12 triangular solve of the
// blocked LU with partial pivoting ("Factor A = LU in precision TF",
// Algorithm IR; lu! of Sec. 2.1.1).
//
// The binary32 operations are exactly those of the unblocked right-looking
// algorithm: pivot = first row of maximal |a_ik|, l_ik = a_ik / a_kk (IEEE
// division), a_ij = fmaf(-l_ik, u_kj, a_ij) with k ascending for every
// element.  Blocking only regroups these chains, so the factors are bitwise
// those of the unblocked algorithm whenever the trailing update is binary32.
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

// Every panel row carries the index of the row it started the panel in
// ("origin"), so the panel's net permutation is known at the end without
// replaying the interchanges.
//
// Candidate exchange: at step k every CTA pushes one 272-byte record
// (|a|, position, origin, the 64 row values, pad) into slot [k & 1][its rank]
// of every CTA of the cluster with st.async, which counts the bytes on the
// receiver's mbarrier; CTA 0 also pushes the record of row k (slot kDiagSlot).
// A receiver waits (bounded) on its own mbarrier for all records of the step.
constexpr int kRec = 68;                     // floats per record
constexpr int kDiagSlot = kPanelMaxCluster;  // slot of the row-k record
struct PanelSmem {
    // row arrays first, each 16-byte aligned (they are accessed as float4)
    alignas(16) float stage_row[NW][NB];     // per-warp candidate row
    alignas(16) float diag_row[NB];          // row k, written by its owner (CTA 0)
    alignas(16) float recv[2][kPanelMaxCluster + 1][kRec];
    alignas(16) float out[2][2][kRec];       // [parity][candidate, row k] records to send
    alignas(8) unsigned long long recv_bar[2];
    float stage_val[NW];
    int stage_pos[NW];
    int stage_org[NW];
    int diag_org;
    float win_r;                 // fl(1/pivot) for the step
    int win_pos, win_src, uorg, dorg;
    int piv_log[NB];             // p_k of every step (the panel's interchanges)
    int zero_piv;                // first zero pivot of this panel (1-based), or 0
    int abort_flag;
};
static_assert(offsetof(PanelSmem, stage_row) % 16 == 0 && offsetof(PanelSmem, diag_row) % 16 == 0 &&
                  offsetof(PanelSmem, recv) % 16 == 0 && offsetof(PanelSmem, out) % 16 == 0 &&
                  (kRec * 4) % 16 == 0,
              "float4 rows of the panel's shared memory must be 16-byte aligned");
// Dynamic shared memory after PanelSmem: Ls[NB][T] multipliers by step and
// position, Us[NB][NB] pivot rows (CTA 0).
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
__device__ __forceinline__ float ld_dsmem_f32(unsigned addr) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
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

// One cluster factors the panel AF[j:n, j:j+nbp].  CTA c of the cluster owns
// panel rows (positions) j + c*T + t, one per thread.  A thread keeps the
// not-yet-eliminated part of its row in a rotating register window: at step k,
// a[i] holds column j+k+i (zero past the panel), so the current column is
// always a[0] and the update a[i] <- fmaf(-l, u[i+1], a[i+1]) also shifts the
// window.  Per column k: warp argmax (redux.sync) -> CTA candidate -> records
// pushed to every CTA (st.async) -> bounded wait on the local mbarrier ->
// winner picked locally -> interchange of positions k and p -> scaling by the
// pivot's reciprocal (LAPACK getf2) and rank-1 update.
// The column loop touches no global memory: multipliers go to shared memory
// by step and position, pivot rows and the interchanges to shared memory; at
// the end every row gathers its multipliers by walking the interchanges
// backward (DSMEM reads).  The rows whose content moved are listed as
// (destination, origin) pairs in swap_list (count in swap_list[0]) for the
// gather of the other columns, and perm is composed with the panel's
// permutation.
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
    const int gi = j + (int)crank * T + t;           // this thread's row (position)
    const bool valid = gi < n;
    const unsigned step_bytes = (csize + 1u) * (unsigned)(kRec * 4);

    int org = gi;
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
        const float4 *src = reinterpret_cast<const float4 *>(AF + (int64_t)gi * ldf + j);
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
        const int pk = j + k;   // position being eliminated
        // 1. local candidate: first maximal |a_ik| over rows i >= pk (rows are
        //    owned in increasing order, so the lowest lane/warp/CTA wins ties)
        const bool cand = valid && gi >= pk;
        const unsigned key = cand ? __float_as_uint(fabsf(a[0])) : 0u;
        const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
        const unsigned tie = __ballot_sync(0xffffffffu, cand && key == kmax);
        if (tie && lane == __ffs(tie) - 1) {
#pragma unroll
            for (int c = 0; c < NB; c += 4)
                *reinterpret_cast<float4 *>(&sm.stage_row[warp][c]) = make_float4(a[c], a[c + 1], a[c + 2], a[c + 3]);
            sm.stage_org[warp] = org;
            sm.stage_val[warp] = __uint_as_float(kmax);
            sm.stage_pos[warp] = gi;
        }
        if (lane == 0 && !tie) { sm.stage_val[warp] = 0.f; sm.stage_pos[warp] = INT_MAX; }
        // row k is published by its owner (always CTA 0: positions j..j+NB-1)
        if (valid && gi == pk) {
#pragma unroll
            for (int c = 0; c < NB; c += 4)
                *reinterpret_cast<float4 *>(&sm.diag_row[c]) = make_float4(a[c], a[c + 1], a[c + 2], a[c + 3]);
            sm.diag_org = org;
        }
        __syncthreads();
        // 2. CTA candidate, pushed to every CTA of the cluster
        if (warp == 0) {
            const unsigned wk = lane < NW ? __float_as_uint(sm.stage_val[lane]) : 0u;
            const int wp = lane < NW ? sm.stage_pos[lane] : INT_MAX;
            const unsigned bk = __reduce_max_sync(0xffffffffu, wk);
            const unsigned who = __ballot_sync(0xffffffffu, wp != INT_MAX && wk == bk);
            const int w = who ? __ffs(who) - 1 : 0;
            const int bp = who ? __shfl_sync(0xffffffffu, wp, w) : INT_MAX;
            // compose the records in local shared memory, then one bulk copy per CTA
            float *rec = sm.out[buf][0];
            const float *row = sm.stage_row[w];
            for (int c = lane; c < NB; c += 32) rec[3 + c] = row[c];
            if (lane == 0) {
                rec[0] = __uint_as_float(bk);
                rec[1] = __int_as_float(bp);
                rec[2] = __int_as_float(sm.stage_org[w]);
                rec[kRec - 1] = 0.f;
            }
            if (crank == 0) {
                float *drec = sm.out[buf][1];
                for (int c = lane; c < NB; c += 32) drec[3 + c] = sm.diag_row[c];
                if (lane == 0) {
                    drec[0] = 0.f;
                    drec[1] = __int_as_float(pk);
                    drec[2] = __int_as_float(sm.diag_org);
                    drec[kRec - 1] = 0.f;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> bulk copy
            __syncwarp();
            if (lane < (int)csize) {
                const unsigned rbar = map_cta(bar_addr + 8u * buf, (unsigned)lane);
                const unsigned slot = recv_addr + (unsigned)((buf * (kPanelMaxCluster + 1) + (int)crank) * kRec * 4);
                bulk_to_cta(map_cta(slot, (unsigned)lane), smem_u32(rec), kRec * 4, rbar);
                if (crank == 0) {
                    const unsigned dslot = recv_addr + (unsigned)((buf * (kPanelMaxCluster + 1) + kDiagSlot) * kRec * 4);
                    bulk_to_cta(map_cta(dslot, (unsigned)lane), smem_u32(sm.out[buf][1]), kRec * 4, rbar);
                }
            }
            // 3. wait (bounded) for every record of this step
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
            // re-arm this buffer for step k + 2
            if (lane == 0 && k + 2 < nbp && !sm.abort_flag) mbar_expect_arrive(bar_addr + 8u * buf, step_bytes);
            __syncwarp();
            // 4. the winner, picked locally from the received headers
            const float *rb = sm.recv[buf][0];
            const unsigned ck = lane < (int)csize ? __float_as_uint(rb[lane * kRec]) : 0u;
            const int cp = lane < (int)csize ? __float_as_int(rb[lane * kRec + 1]) : INT_MAX;
            const unsigned ckmax = __reduce_max_sync(0xffffffffu, ck);
            const unsigned cwho = __ballot_sync(0xffffffffu, cp != INT_MAX && ck == ckmax);
            const int wc = cwho ? __ffs(cwho) - 1 : 0;
            if (lane == 0) {
                const float *wr = rb + wc * kRec;
                const float piv = wr[3];
                sm.win_pos = __float_as_int(wr[1]);
                sm.win_src = wc;
                sm.uorg = __float_as_int(wr[2]);
                sm.dorg = __float_as_int(sm.recv[buf][kDiagSlot][2]);
                sm.win_r = (piv != 0.f) ? 1.0f / piv : 0.f;
                sm.piv_log[k] = sm.win_pos;
            }
        }
        __syncthreads();
        const int p = sm.win_pos;
        const float *u = sm.recv[buf][sm.win_src];     // u[3 + i] = pivot row, column k + i
        const float piv = u[3];
        // 5. interchange of positions pk and p; the pivot row is final (kept in Us)
        if (valid && gi == pk) {
            org = sm.uorg;
        } else if (valid && gi == p) {
            const float *dr = sm.recv[buf][kDiagSlot] + 3;
#pragma unroll
            for (int c = 0; c < NB; ++c) a[c] = dr[c];
            org = sm.dorg;
        }
        if (crank == 0 && warp == 1) {
            Us[k * NB + lane] = u[3 + lane];
            Us[k * NB + lane + 32] = u[35 + lane];
        }
        if (piv == 0.f && t == 0 && sm.zero_piv == 0) sm.zero_piv = pk + 1;
        // 6. scale column k (getf2: by the reciprocal, divide below the smallest
        //    normal), update and shift the live part of the window
        if (valid && gi > pk) {
            float l = a[0];
            if (piv != 0.f) l = (fabsf(piv) >= FLT_MIN) ? l * sm.win_r : l / piv;
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
    // net permutation of the panel: position gi now holds the row from org
    int porg = 0;
    const bool moved = valid && org != gi;
    if (moved) {
        int e = atomicAdd(&swap_list[0], 1);
        swap_list[1 + 2 * e] = gi;
        swap_list[2 + 2 * e] = org;
        porg = perm[org];
    }
    if (crank == 0) {
        for (int k = t; k < nbp; k += T) ipiv[j + k] = sm.piv_log[k];
        if (t == 0 && sm.zero_piv) atomicMin(&dev->info, sm.zero_piv);
    }
    // all multipliers of the cluster are in shared memory; perm reads done
    cluster_sync_all();
    if (moved) perm[gi] = porg;
    if (valid) {
        // multipliers of this row's content: walk the interchanges backward
        // from the final position; at step k the content sat at position pos
        const int kend = (gi - j < nbp) ? gi - j : nbp;
        const unsigned ls_base = smem_u32(Ls);
        int pos = gi;
#pragma unroll
        for (int k = NB - 1; k >= 0; --k) {
            if (k < nbp) {
                if (k < kend) {
                    const int rel = pos - j;
                    a[k] = ld_dsmem_f32(map_cta(ls_base + 4u * (unsigned)(k * T + (rel % T)), (unsigned)(rel / T)));
                } else {
                    a[k] = 0.f;
                }
                const int pkk = j + k, pp = sm.piv_log[k];
                if (pos == pkk) pos = pp;
                else if (pos == pp) pos = pkk;
            } else {
                a[k] = 0.f;
            }
        }
        float *dst = AF + (int64_t)gi * ldf + j;
        if (kend == NB) {
#pragma unroll
            for (int c = 0; c < NB; c += 4)
                reinterpret_cast<float4 *>(dst)[c / 4] = make_float4(a[c], a[c + 1], a[c + 2], a[c + 3]);
        } else {
            // a pivot row of this panel: L part, then its U part from Us
#pragma unroll
            for (int c = 0; c < NB; ++c)
                if (c < kend) dst[c] = a[c];
            for (int c = kend; c < nbp; ++c) dst[c] = Us[kend * NB + (c - kend)];
        }
        if (has_trailing && Aop != nullptr && gi >= j + NB) store_op_row(Aop, gi - (j + NB), a, tf);
    }
    cluster_sync_all();   // no CTA leaves while its shared memory may be read
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
