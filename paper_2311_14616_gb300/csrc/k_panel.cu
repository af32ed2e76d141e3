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
#include "lu_tiles.cuh"

namespace ir {
namespace {

constexpr int NB = kPanelNB;
constexpr int T = kPanelThreads;    // threads per CTA
constexpr int RPC = kPanelRows;     // rows per CTA: thread t holds rows t and t + T
constexpr int NW = T / 32;

// Rows never move between threads during a panel: every thread keeps its two
// rows and tracks their current positions, so an interchange is a few integer
// compares and the panel's net permutation is known at the end.
//
// Candidate exchange: at step k every warp stages its best row as a record
// (|a| bits, position, fl(1/a), the row's 64 - k live values; at most 272
// bytes) and the CTA's best record is pushed, in chunks of 16 bytes (17 at
// step 0, one fewer every four steps), each stored by its own thread with
// st.async, into slot [k & 1][its rank] of every CTA of the cluster, counted
// on the receiver's mbarrier.  A receiver waits (bounded) for all records of
// the step.  Values past the live width are never sent: the receivers' update
// may read stale ones there, but only into window entries that are dead.
constexpr int kRec = 68;                     // floats per record
constexpr int kChunks = kRec / 4;            // 16-byte chunks per record
static_assert(kRec == kPanelGridRec, "the grid exchange buffers hold records of kRec floats");
struct PanelSmem {
    // records first, each 16-byte aligned (they are accessed as float4)
    alignas(16) float stage[2][NW][kRec];    // per-warp candidate records, by step parity
    alignas(16) float recv[2][kPanelMaxCluster][kRec];
    alignas(8) unsigned long long recv_bar[2];
    int piv_log[NB];             // p_k of every step (the panel's interchanges)
    int posv[RPC];               // epilogue: each row slot's final position (-1: none)
    int kpv[RPC];                // and the step at which it became the pivot row
    int zero_piv;                // first zero pivot of this panel (1-based), or 0
    int abort_flag;
};
static_assert(offsetof(PanelSmem, stage) % 16 == 0 && offsetof(PanelSmem, recv) % 16 == 0 &&
                  (kRec * 4) % 16 == 0,
              "float4 records of the panel's shared memory must be 16-byte aligned");
// Dynamic shared memory after PanelSmem: Ls[RPC][LS] multipliers by row slot and
// step (odd stride: the per-step column stores and the epilogue's row reads
// spread over the banks), Us[NB][NB] pivot rows.
constexpr int LS = NB + 1;
constexpr size_t kPanelDynSmem = sizeof(PanelSmem) + sizeof(float) * (size_t)RPC * LS + sizeof(float) * NB * NB + 16;

using lu::round_tf;

// Store values 4q .. 4q + 3 of one operand row (rounded to TF) into Aop/Bop.
__device__ __forceinline__ void store_op_chunk(void *op, int64_t row, int q, float4 v, ir_dtype tf) {
    if (tf == IR_TF32) {
        reinterpret_cast<float4 *>(static_cast<float *>(op) + row * NB)[q] =
            make_float4(round_tf(v.x, tf), round_tf(v.y, tf), round_tf(v.z, tf), round_tf(v.w, tf));
    } else if (tf == IR_BF16) {
        __nv_bfloat162 p[2] = {__floats2bfloat162_rn(v.x, v.y), __floats2bfloat162_rn(v.z, v.w)};
        reinterpret_cast<uint2 *>(static_cast<__nv_bfloat16 *>(op) + row * NB)[q] = *reinterpret_cast<uint2 *>(p);
    } else if (tf == IR_F16) {
        __half2 p[2] = {__floats2half2_rn(v.x, v.y), __floats2half2_rn(v.z, v.w)};
        reinterpret_cast<uint2 *>(static_cast<__half *>(op) + row * NB)[q] = *reinterpret_cast<uint2 *>(p);
    }
}

// 16-byte chunks of step k's record: the header (3 floats) and the 64 - k live values.
__device__ __forceinline__ int rec_chunks(int k) { return (70 - k) / 4; }

// Stage the first nch chunks of a row window as a candidate record: |a| bits,
// position, fl(1/a), the values (record[3 + i] = a[i]).
__device__ __forceinline__ void stage_record(float *st, const float (&a)[NB], unsigned key, int pos, int nch) {
    float4 *s4 = reinterpret_cast<float4 *>(st);
    s4[0] = make_float4(__uint_as_float(key), __int_as_float(pos), (a[0] != 0.f) ? __frcp_rn(a[0]) : 0.f, a[0]);
#pragma unroll
    for (int q = 0; q < 15; ++q)
        if (1 + q < nch) s4[1 + q] = make_float4(a[4 * q + 1], a[4 * q + 2], a[4 * q + 3], a[4 * q + 4]);
    if (16 < nch) s4[16] = make_float4(a[61], a[62], a[63], 0.f);
}

// One cluster factors the panel AF[j:n, j:j+nbp].  Thread t of CTA c keeps
// rows j + c*RPC + t and j + c*RPC + T + t for the whole panel in rotating
// register windows: at step k, a[i] holds column j+k+i for i < nbp - k (live),
// so the current column is always a[0] and the update a[i] <- fmaf(-l,
// u[i+1], a[i+1]) also shifts the window.  Per column k: thread, then warp
// candidate (largest |a|, ties to the lowest current position: redux.sync)
// staged as a record -> the CTA's best record pushed to every CTA (st.async,
// one thread per 16-byte chunk and destination) -> bounded wait on the local
// mbarrier -> every warp picks the pivot row from the received headers (a
// single-CTA cluster takes its best record directly) ->
// positions k and p swap labels -> scaling by the pivot's reciprocal and
// rank-1 update of the rows that are not pivot rows (both rows of a thread
// share the loads of the pivot row).  The column loop touches no global
// memory.  At the end each row is written to its final position: the
// multipliers of the steps before it became a pivot row, then the U part
// staged at that step.  Rows that moved are listed as (destination, origin)
// pairs in swap_list (count in swap_list[0]) for the interchanges of the
// other columns, and perm is composed with the panel's permutation.
// The exchange of the CTAs' best records, by the panel's height:
//   kModeCluster  2..16 CTAs of one thread-block cluster: st.async into every
//                 CTA's shared memory (M <= 8192 rows)
//   kModeSingle   one CTA: its best record is the pivot row (M <= 512)
//   kModeGrid     up to one CTA per SM, launched cooperatively (all resident):
//                 each CTA writes its record to global memory (grec, two slots
//                 per CTA by step parity) and arrives on the step's counter
//                 (gcnt[k], zeroed before the launch); each waits (bounded)
//                 until all have arrived, reads the headers through L2 and
//                 copies the winner's record into its shared memory (M > 8192)
constexpr int kModeCluster = 0, kModeSingle = 1, kModeGrid = 2;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of a kModeGrid launch on counter *cnt (zeroed before the
// launch, used once): bounded; on timeout the flags are raised and it returns.
__device__ __forceinline__ void grid_barrier(unsigned *cnt, unsigned target, unsigned long long deadline,
                                             volatile int *abort_flag, DevScalars *dev) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(cnt, 1u);
        if (!*abort_flag) {
            while (ld_acquire_gpu(cnt) < target) {
                if (globaltimer() > deadline) {
                    *abort_flag = 1;
                    atomicExch(&dev->timeout, 1);
                    break;
                }
            }
        }
    }
    __syncthreads();
}

template <int kMode>
__global__ void __launch_bounds__(T, 1)
    k_panel(float *AF, int64_t ldf, int n, int j, int nbp, int32_t *ipiv, int32_t *perm,
            int32_t *swap_list, DevScalars *dev, ir_dtype tf, void *Aop, int has_trailing, float *grec,
            unsigned *gcnt) {
    constexpr bool kSingle = (kMode == kModeSingle), kGrid = (kMode == kModeGrid);
    pdl_trigger();
    pdl_wait();
    extern __shared__ __align__(16) unsigned char panel_smem[];
    PanelSmem &sm = *reinterpret_cast<PanelSmem *>(panel_smem);
    float *Ls = reinterpret_cast<float *>(panel_smem + sizeof(PanelSmem));   // [RPC][LS]
    float *Us = Ls + (size_t)RPC * LS;                                        // [NB][NB]
    const unsigned crank = kGrid ? blockIdx.x : cluster_rank();
    const unsigned csize = kGrid ? gridDim.x : cluster_size();
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int home0 = (int)crank * RPC + t, home1 = home0 + T;   // start positions, relative to j
    const bool valid0 = j + home0 < n, valid1 = j + home1 < n;
    auto step_bytes = [&](int k) { return csize * 16u * (unsigned)rec_chunks(k); };
    const int nsend = (int)csize * kChunks;                       // record chunks to store per step

    int pos0 = home0, pos1 = home1;     // current positions, relative to j
    int kp0 = nbp, kp1 = nbp;           // the step at which each row became the pivot row (nbp: never)
    if (crank == 0 && t == 0) swap_list[0] = 0;
    if (t == 0) {
        sm.zero_piv = 0;
        sm.abort_flag = 0;
        mbar_init_p(smem_u32(&sm.recv_bar[0]), 1);
        mbar_init_p(smem_u32(&sm.recv_bar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (kMode == kModeCluster) {      // the other modes use no mbarrier
            mbar_expect_arrive(smem_u32(&sm.recv_bar[0]), step_bytes(0));
            if (nbp > 1) mbar_expect_arrive(smem_u32(&sm.recv_bar[1]), step_bytes(1));
        }
    }
    float a0[NB], a1[NB];
    {
        const float4 *s0 = reinterpret_cast<const float4 *>(AF + (int64_t)(j + home0) * ldf + j);
        const float4 *s1 = reinterpret_cast<const float4 *>(AF + (int64_t)(j + home1) * ldf + j);
#pragma unroll
        for (int c = 0; c < NB; c += 4) {
            const float4 v = (valid0 && c < nbp) ? s0[c / 4] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 w = (valid1 && c < nbp) ? s1[c / 4] : make_float4(0.f, 0.f, 0.f, 0.f);
            a0[c] = v.x; a0[c + 1] = v.y; a0[c + 2] = v.z; a0[c + 3] = v.w;
            a1[c] = w.x; a1[c + 1] = w.y; a1[c + 2] = w.z; a1[c + 3] = w.w;
        }
#pragma unroll
        for (int c = 0; c < NB; ++c)
            if (c >= nbp) a0[c] = a1[c] = 0.f;
    }
    if constexpr (kGrid)
        __syncthreads();
    else
        cluster_sync_all();   // every CTA is running and its mbarriers are armed
    const unsigned long long deadline = globaltimer() + kWaitLimitNs;   // for all waits of this launch

    const unsigned recv_addr = smem_u32(&sm.recv[0][0][0]);
    const unsigned bar_addr = smem_u32(&sm.recv_bar[0]);

    // 1. candidate of the thread (its two rows), then of the warp: largest
    //    |a_ik| over rows that are not pivot rows yet, ties to the lowest
    //    current position.  For step k + 1 it is formed inside step k's
    //    update, right after the new column k + 1, so that the reductions
    //    overlap the rest of the update.
    bool use1, tc;
    int tpos, mpos;
    unsigned kmax;
    auto candidate = [&]() {
        const bool c0 = valid0 && kp0 == nbp, c1 = valid1 && kp1 == nbp;
        const unsigned k0 = c0 ? __float_as_uint(fabsf(a0[0])) : 0u;
        const unsigned k1 = c1 ? __float_as_uint(fabsf(a1[0])) : 0u;
        use1 = c1 && (!c0 || k1 > k0 || (k1 == k0 && pos1 < pos0));
        tc = c0 || c1;
        const unsigned key = use1 ? k1 : k0;
        tpos = use1 ? pos1 : pos0;
        kmax = __reduce_max_sync(0xffffffffu, key);
        mpos = __reduce_min_sync(0xffffffffu, (tc && key == kmax) ? tpos : INT_MAX);
    };
    candidate();
#pragma unroll 1
    for (int k = 0; k < nbp; ++k) {
        const int buf = k & 1;
        // the warp's candidate, staged as a record
        const bool c0 = valid0 && kp0 == nbp, c1 = valid1 && kp1 == nbp;
        float *st = sm.stage[buf][warp];
        const int nch = rec_chunks(k);
        if (tc && tpos == mpos) {
            if (use1)
                stage_record(st, a1, kmax, mpos, nch);
            else
                stage_record(st, a0, kmax, mpos, nch);
        }
        if (lane == 0 && mpos == INT_MAX) {
            st[0] = 0.f;
            st[1] = __int_as_float(INT_MAX);
        }
        __syncthreads();
        // 2. the CTA's best record (the best of its warps' records)
        const unsigned wk = lane < NW ? __float_as_uint(sm.stage[buf][lane][0]) : 0u;
        const int wp = lane < NW ? __float_as_int(sm.stage[buf][lane][1]) : INT_MAX;
        const unsigned bk = __reduce_max_sync(0xffffffffu, wk);
        const int bp = __reduce_min_sync(0xffffffffu, (wp != INT_MAX && wk == bk) ? wp : INT_MAX);
        const unsigned who = __ballot_sync(0xffffffffu, lane < NW && wp == bp);
        const int w = who ? __ffs(who) - 1 : 0;
        const float *u;     // u[3 + i] = pivot row, column j + k + i
        int ppos;
        if constexpr (kSingle) {
            // a single CTA: its best record is the pivot row
            ppos = bp;
            u = sm.stage[buf][w];
        } else if constexpr (kGrid) {
            // the CTA's best record into its global slot, arrive, wait for all CTAs
            float4 *gslot = reinterpret_cast<float4 *>(grec + ((size_t)buf * csize + crank) * kRec);
            if (t < nch) gslot[t] = reinterpret_cast<const float4 *>(sm.stage[buf][w])[t];
            grid_barrier(gcnt + k, csize, deadline, &sm.abort_flag, dev);
            // the pivot: the best of all CTAs' headers (lane l reads CTAs l, l + 32, ...)
            unsigned ck = 0u;
            int cp = INT_MAX, cw = 0;
            for (int q = lane; q < (int)csize; q += 32) {
                const float *h = grec + ((size_t)buf * csize + q) * kRec;
                const unsigned hk = __float_as_uint(__ldcg(h));
                const int hp = __float_as_int(__ldcg(h + 1));
                if (hp != INT_MAX && (cp == INT_MAX || hk > ck || (hk == ck && hp < cp))) {
                    ck = hk;
                    cp = hp;
                    cw = q;
                }
            }
            const unsigned ckmax = __reduce_max_sync(0xffffffffu, cp != INT_MAX ? ck : 0u);
            ppos = __reduce_min_sync(0xffffffffu, (cp != INT_MAX && ck == ckmax) ? cp : INT_MAX);
            const unsigned cwho = __ballot_sync(0xffffffffu, cp != INT_MAX && cp == ppos);
            const int wc = __shfl_sync(0xffffffffu, cw, cwho ? __ffs(cwho) - 1 : 0);
            // the winner's record into shared memory (every warp picked the same one)
            float *rb = sm.recv[buf][0];
            if (warp == 0 && lane < nch)
                reinterpret_cast<float4 *>(rb)[lane] =
                    __ldcg(reinterpret_cast<const float4 *>(grec + ((size_t)buf * csize + wc) * kRec) + lane);
            __syncthreads();
            u = rb;
        } else {
            // pushed to every CTA of the cluster: chunk i % 17 of it (if live)
            // into CTA i / 17 for i = t, t + T, ... (st.async, counted on the
            // receiver's mbarrier)
            for (int snd = t; snd < nsend; snd += T) {
                const int dst = snd / kChunks, ch = snd % kChunks;
                if (ch >= nch) continue;
                const float4 v = reinterpret_cast<const float4 *>(sm.stage[buf][w])[ch];
                const unsigned slot = recv_addr + (unsigned)(((buf * kPanelMaxCluster + (int)crank) * kRec + 4 * ch) * 4);
                st_async_v4(map_cta(slot, (unsigned)dst), v, map_cta(bar_addr + 8u * buf, (unsigned)dst));
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
            if (t == 0 && k + 2 < nbp && !sm.abort_flag) mbar_expect_arrive(bar_addr + 8u * buf, step_bytes(k + 2));
            // 4. the pivot row, picked by every warp from the received headers
            const float *rb = sm.recv[buf][0];
            const unsigned ck = lane < (int)csize ? __float_as_uint(rb[lane * kRec]) : 0u;
            const int cp = lane < (int)csize ? __float_as_int(rb[lane * kRec + 1]) : INT_MAX;
            const unsigned ckmax = __reduce_max_sync(0xffffffffu, ck);
            ppos = __reduce_min_sync(0xffffffffu, (cp != INT_MAX && ck == ckmax) ? cp : INT_MAX);
            const unsigned cwho = __ballot_sync(0xffffffffu, lane < (int)csize && cp == ppos);
            const int wc = cwho ? __ffs(cwho) - 1 : 0;
            u = rb + wc * kRec;
        }
        const float piv = u[3];
        const float r = u[2];
        if (t == 0) {
            sm.piv_log[k] = j + ppos;
            if (piv == 0.f && sm.zero_piv == 0) sm.zero_piv = j + k + 1;
        }
        // 5. interchange of positions k and ppos: labels only
        if (c0 && pos0 == ppos) {
            pos0 = k;
            kp0 = k;
        } else if (pos0 == k) {
            pos0 = ppos;
        }
        if (c1 && pos1 == ppos) {
            pos1 = k;
            kp1 = k;
        } else if (pos1 == k) {
            pos1 = ppos;
        }
        if (warp == 1) {
            Us[k * NB + lane] = u[3 + lane];
            Us[k * NB + lane + 32] = u[35 + lane];
        }
        // 6. scale column k (getf2: by the reciprocal, divide below the smallest
        //    normal) and update the live part of both windows.  A window that is
        //    not updated any more (pivot row, or past the matrix) is shifted with
        //    l = 0; its contents are never used again.
        const bool u0 = valid0 && kp0 == nbp, u1 = valid1 && kp1 == nbp;
        float l0 = 0.f, l1 = 0.f;
        if (u0) {
            l0 = a0[0];
            if (piv != 0.f) l0 = (fabsf(piv) >= FLT_MIN) ? l0 * r : l0 / piv;
            Ls[t * LS + k] = l0;
        }
        if (u1) {
            l1 = a1[0];
            if (piv != 0.f) l1 = (fabsf(piv) >= FLT_MIN) ? l1 * r : l1 / piv;
            Ls[(T + t) * LS + k] = l1;
        }
        // After the update only window entries i < 63 - k are live, so the
        // update stops at the first 16-column chunk that holds none of them
        // (one uniform branch per chunk; inside a chunk the 4 loads of the
        // pivot row are issued ahead of the fmas).  Entries past the live width
        // are dead: they may hold stale values and are never read.
        const float4 *us = reinterpret_cast<const float4 *>(u + 4);   // u[4 + c] = column k+1+c
        {
            const float4 w = us[0];
            a0[0] = fmaf(-l0, w.x, a0[1]);
            a1[0] = fmaf(-l1, w.x, a1[1]);
        }
        if (k + 1 < nbp) candidate();
#pragma unroll
        for (int q = 0; q < NB / 4; ++q) {
            if (q % 4 == 0 && q > 0 && 4 * q >= NB - 1 - k) break;
            const float4 w = us[q];
            if (q > 0) a0[4 * q + 0] = fmaf(-l0, w.x, a0[4 * q + 1]);
            a0[4 * q + 1] = fmaf(-l0, w.y, a0[4 * q + 2]);
            a0[4 * q + 2] = fmaf(-l0, w.z, a0[4 * q + 3]);
            a0[4 * q + 3] = (4 * q + 3 < NB - 1) ? fmaf(-l0, w.w, a0[4 * q + 4]) : 0.f;
            if (q > 0) a1[4 * q + 0] = fmaf(-l1, w.x, a1[4 * q + 1]);
            a1[4 * q + 1] = fmaf(-l1, w.y, a1[4 * q + 2]);
            a1[4 * q + 2] = fmaf(-l1, w.z, a1[4 * q + 3]);
            a1[4 * q + 3] = (4 * q + 3 < NB - 1) ? fmaf(-l1, w.w, a1[4 * q + 4]) : 0.f;
        }
    }
    // net permutation of the panel: position j + pos now holds the row that started at j + home
    int porg0 = 0, porg1 = 0;
    const bool moved0 = valid0 && pos0 != home0, moved1 = valid1 && pos1 != home1;
    if (moved0) {
        const int e = atomicAdd(&swap_list[0], 1);
        swap_list[1 + 2 * e] = j + pos0;
        swap_list[2 + 2 * e] = j + home0;
        porg0 = perm[j + home0];
    }
    if (moved1) {
        const int e = atomicAdd(&swap_list[0], 1);
        swap_list[1 + 2 * e] = j + pos1;
        swap_list[2 + 2 * e] = j + home1;
        porg1 = perm[j + home1];
    }
    if constexpr (kGrid)    // every perm read of the grid is done; piv_log is complete
        grid_barrier(gcnt + NB, csize, deadline, &sm.abort_flag, dev);
    else
        cluster_sync_all();   // every perm read of the cluster is done; piv_log is complete
    if (crank == 0) {
        for (int k = t; k < nbp; k += T) ipiv[j + k] = sm.piv_log[k];
        if (t == 0 && sm.zero_piv) atomicMin(&dev->info, sm.zero_piv);
    }
    if (moved0) perm[j + pos0] = porg0;
    if (moved1) perm[j + pos1] = porg1;
    // Final rows, written a row (256 contiguous bytes) per half warp: the
    // multipliers of the steps before a row became the pivot row come from its
    // slot of Ls, the rest (its U part) from Us; each slot's destination and
    // pivot step go through shared memory.
    sm.posv[t] = valid0 ? pos0 : -1;
    sm.posv[t + T] = valid1 ? pos1 : -1;
    sm.kpv[t] = kp0;
    sm.kpv[t + T] = kp1;
    __syncthreads();
    {
        const int q = lane & 15;
        const bool ops = has_trailing && Aop != nullptr;
#pragma unroll 4
        for (int it = 0; it < RPC / (2 * NW); ++it) {
            const int sl = 2 * NW * it + 2 * warp + (lane >> 4);
            const int pos = sm.posv[sl];
            if (pos < 0) continue;
            const int kp = sm.kpv[sl];
            float v[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int c = 4 * q + i;
                v[i] = (c < kp) ? Ls[sl * LS + c] : (c < nbp ? Us[kp * NB + (c - kp)] : 0.f);
            }
            const float4 w = make_float4(v[0], v[1], v[2], v[3]);
            if (4 * q < nbp) reinterpret_cast<float4 *>(AF + (int64_t)(j + pos) * ldf + j)[q] = w;
            if (ops && pos >= NB) store_op_chunk(Aop, pos - NB, q, w, tf);
        }
    }
    if constexpr (!kGrid) cluster_sync_all();   // no CTA leaves while its shared memory may be written
}

// Apply the panel's row permutation to the columns [c0a, c1a) and [c0b, c1b):
// A[dst][c] = A[src][c] for the (dst, src) pairs the panel listed.  All
// sources of a column are read before any destination is written.
constexpr int kLaswpT = 64;   // 2*NB*kLaswpT floats of staging stay under 48 KB
__global__ void __launch_bounds__(kLaswpT) k_laswp(float *AF, int64_t ldf, int c0a, int c1a, int c0b, int c1b,
                                                  const int32_t *swap_list) {
    pdl_trigger();
    pdl_wait();
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

// The interchanges of several consecutive panels, in order, on the columns
// [c0, c1): lists `first` .. `first + count - 1` of a ring of `ring` swap lists
// (kListInts ints each).  One thread per column; each list's sources are read
// before its destinations are written, and list t + 1 sees list t's result.
__global__ void __launch_bounds__(kLaswpT) k_laswp_lists(float *AF, int64_t ldf, int c0, int c1,
                                                        const int32_t *lists, int list_ints, int ring, int first,
                                                        int count) {
    pdl_trigger();
    pdl_wait();
    __shared__ int sd[2 * NB], ss[2 * NB];
    __shared__ float vals[2 * NB][kLaswpT];
    const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    for (int t = 0; t < count; ++t) {
        const int32_t *sl = lists + (int64_t)((first + t) % ring) * list_ints;
        const int cnt = sl[0];
        __syncthreads();                         // the previous list's entries are no longer read
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            sd[e] = sl[1 + 2 * e];
            ss[e] = sl[2 + 2 * e];
        }
        __syncthreads();
        if (c < c1) {
            for (int e = 0; e < cnt; ++e) vals[e][threadIdx.x] = AF[(int64_t)ss[e] * ldf + c];
            for (int e = 0; e < cnt; ++e) AF[(int64_t)sd[e] * ldf + c] = vals[e][threadIdx.x];
        }
    }
}

// U12 = L11^{-1} A12 for the block row j..j+NB and the columns [cb, ce): one
// CTA of 256 threads per 64 columns (lu::trsm64).
constexpr int kNarrowCols = 64;

// The same after the panel's row interchanges on the CTA's own 64 columns
// (the next block column of the lookahead chain: one launch instead of two).
// Interchanges as k_laswp: all sources of a column are read before any of its
// destinations is written; the shared staging is reused for L11 afterwards.
__global__ void __launch_bounds__(256) k_laswp_trsm(float *AF, int64_t ldf, int cb, int ce, int j, ir_dtype tf,
                                                    void *Bop, const int32_t *swap_list) {
    pdl_trigger();
    pdl_wait();
    __shared__ int sd[2 * NB], ss[2 * NB];
    __shared__ __align__(16) float stage[2 * NB * kNarrowCols];   // interchange values, then L11
    const int c0 = cb + blockIdx.x * kNarrowCols;
    const int cnt = swap_list[0];
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        sd[e] = swap_list[1 + 2 * e];
        ss[e] = swap_list[2 + 2 * e];
    }
    __syncthreads();
    {
        // thread t: column t % 64, list entries t / 64, t / 64 + 4, ...
        const int cc = threadIdx.x % kNarrowCols, e0 = threadIdx.x / kNarrowCols;
        const int c = c0 + cc;
        if (c < ce)
            for (int e = e0; e < cnt; e += 256 / kNarrowCols) stage[e * kNarrowCols + cc] = AF[(int64_t)ss[e] * ldf + c];
        __syncthreads();
        if (c < ce)
            for (int e = e0; e < cnt; e += 256 / kNarrowCols) AF[(int64_t)sd[e] * ldf + c] = stage[e * kNarrowCols + cc];
        __syncthreads();     // the interchanged rows are in A_F before trsm64 reads them
    }
    lu::trsm64(AF, ldf, c0, ce, j, tf, Bop, reinterpret_cast<float (*)[lu::kLd]>(stage));
}
__global__ void __launch_bounds__(256) k_trsm_narrow(float *AF, int64_t ldf, int cb, int ce, int j, ir_dtype tf,
                                                     void *Bop) {
    pdl_trigger();
    pdl_wait();
    __shared__ __align__(16) float Lt[NB][lu::kLd];
    lu::trsm64(AF, ldf, cb + blockIdx.x * kNarrowCols, ce, j, tf, Bop, Lt);
}

__global__ void k_iota(int n, int32_t *perm) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) perm[i] = i;
}

}  // namespace

cudaError_t launch_panel(float *AF, int64_t ldf, int n, int j, int nbp, int32_t *ipiv,
                         int32_t *perm, int32_t *swap_list, DevScalars *dev, ir_dtype tf,
                         void *Aop, cudaStream_t s, float *grec, unsigned *gcnt) {
    static bool attr_done = false;
    if (!attr_done) {
        for (auto kern : {k_panel<kModeCluster>, k_panel<kModeSingle>, k_panel<kModeGrid>}) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPanelDynSmem);
            if (e != cudaSuccess) return e;
        }
        attr_done = true;
    }
    int M = n - j;
    int C = (M + RPC - 1) / RPC;
    const int has_trailing = (j + NB < n) ? 1 : 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(T, 1, 1);
    cfg.dynamicSmemBytes = kPanelDynSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    cfg.attrs = attr;
    if (C > kPanelMaxCluster) {
        // taller than one cluster holds: one cooperative launch, every CTA resident
        if (!grec || !gcnt || C > kPanelMaxGrid) return cudaErrorInvalidValue;
        cudaError_t e = cudaMemsetAsync(gcnt, 0, kPanelGridCounters * sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.numAttrs = 1;
        count_launch();
        return cudaLaunchKernelEx(&cfg, k_panel<kModeGrid>, AF, ldf, n, j, nbp, ipiv, perm, swap_list, dev, tf, Aop,
                                  has_trailing, grec, gcnt);
    }
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.numAttrs = 1 + set_pdl(&attr[1]);
    count_launch();
    return cudaLaunchKernelEx(&cfg, C == 1 ? k_panel<kModeSingle> : k_panel<kModeCluster>, AF, ldf, n, j, nbp, ipiv,
                              perm, swap_list, dev, tf, Aop, has_trailing, (float *)nullptr, (unsigned *)nullptr);
}

cudaError_t launch_laswp(float *AF, int64_t ldf, int c0a, int c1a, int c0b, int c1b, const int32_t *swap_list,
                         cudaStream_t s) {
    const int ncols = (c1a - c0a) + (c1b - c0b);
    if (ncols <= 0) return cudaSuccess;
    count_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((ncols + kLaswpT - 1) / kLaswpT, 1, 1);
    cfg.blockDim = dim3(kLaswpT, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    cfg.attrs = attr;
    cfg.numAttrs = set_pdl(&attr[0]);
    return cudaLaunchKernelEx(&cfg, k_laswp, AF, ldf, c0a, c1a, c0b, c1b, swap_list);
}

cudaError_t launch_laswp_lists(float *AF, int64_t ldf, int c0, int c1, const int32_t *lists, int list_ints, int ring,
                               int first, int count, cudaStream_t s) {
    if (c1 <= c0 || count <= 0) return cudaSuccess;
    count_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((c1 - c0 + kLaswpT - 1) / kLaswpT, 1, 1);
    cfg.blockDim = dim3(kLaswpT, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    cfg.attrs = attr;
    cfg.numAttrs = set_pdl(&attr[0]);
    return cudaLaunchKernelEx(&cfg, k_laswp_lists, AF, ldf, c0, c1, lists, list_ints, ring, first, count);
}

// U12 for the columns [cb, ce) of the block row j..j+NB.
cudaError_t launch_trsm(float *AF, int64_t ldf, int cb, int ce, int j, ir_dtype tf, void *Bop, cudaStream_t s) {
    const int ncols = ce - cb;
    if (ncols <= 0) return cudaSuccess;
    count_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((ncols + kNarrowCols - 1) / kNarrowCols, 1, 1);
    cfg.blockDim = dim3(4 * kNarrowCols, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    cfg.attrs = attr;
    cfg.numAttrs = set_pdl(&attr[0]);
    return cudaLaunchKernelEx(&cfg, k_trsm_narrow, AF, ldf, cb, ce, j, tf, tf == IR_F32 ? nullptr : Bop);
}

cudaError_t launch_laswp_trsm(float *AF, int64_t ldf, int cb, int ce, int j, ir_dtype tf, void *Bop,
                              const int32_t *swap_list, cudaStream_t s) {
    const int ncols = ce - cb;
    if (ncols <= 0) return cudaSuccess;
    count_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((ncols + kNarrowCols - 1) / kNarrowCols, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    cfg.attrs = attr;
    cfg.numAttrs = set_pdl(&attr[0]);
    return cudaLaunchKernelEx(&cfg, k_laswp_trsm, AF, ldf, cb, ce, j, tf, tf == IR_F32 ? nullptr : Bop, swap_list);
}

cudaError_t launch_iota(int n, int32_t *perm, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    count_launch();
    k_iota<<<(n + 255) / 256, 256, 0, s>>>(n, perm);
    return cudaGetLastError();
}

}  // namespace ir
