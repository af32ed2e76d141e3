// Tensor-core trailing update of the mixed-precision blocked LU:
//     C <- C - rTF(L21) rTF(U12)
// with the TF-rounded operands (TF32, bf16 or fp16) multiplied by
// tcgen05.mma with binary32 accumulation in tensor memory (TMEM), then
// subtracted from the binary32 matrix in the epilogue.
//
// The operands live in "slot" buffers: slot s holds the 64-column K block of
// one panel, K-major (rows x 64 values, the row's 64 K values contiguous), and
// a launch applies the slots [s0, s1) one after another.  One block step of
// the right-looking LU is one slot; a group of G block steps applied at once
// to the far trailing columns is G slots, which reads and writes the binary32
// C tile once for all of them instead of once per block step.  Each slot's 64
// products are summed in their own TMEM accumulator and subtracted from C in
// binary32 before the next slot's, so C <- fl32(C - D_s) block by block as in
// the right-looking algorithm; only the C tile's trips to memory are shared.
//
// Persistent, warp-specialised kernel, one CTA per SM:
//   warp 0      TMA producer: for every output tile the binary32 C tile (four
//               128x32 boxes) into one of CBUFS C buffers, then the operand
//               tiles of each slot, one 128-byte K atom (128 rows, 128-byte
//               swizzle) of A and of B per stage of a shared-memory ring
//   warp 1      allocates TMEM (a ring of 4 accumulators x 128 columns) and
//               issues the MMAs from one thread, one accumulator per slot;
//               tcgen05.commit frees each stage and signals the accumulator
//   warps 2-9   epilogue: each thread holds 64 values of its C row in
//               registers, and for every slot tcgen05.ld's the accumulator,
//               frees it and subtracts; then the tile goes back to shared
//               memory and one thread stores it with TMA (edges are clipped
//               by the tensor map, so ragged tiles need no guards)
// Every mbarrier wait is bounded (globaltimer); on timeout the CTA records
// the error, waits (bounded) for its own copies in flight, frees TMEM and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ir_internal.cuh"
#include "tc_util.cuh"

namespace ir {
namespace {

constexpr int BM = 128, BN = 128, K = kPanelNB;
constexpr int kAtomBytes = BM * 128;      // one 128-row x 128-byte swizzle tile = 16 KB
constexpr int kThreads = 320;             // 10 warps
constexpr int kEpiThreads = 256;
constexpr int kRing = 4;                  // slot accumulators in TMEM
constexpr unsigned kTmemCols = kRing * BN;

struct TcParams {
    int M, N;               // rows and columns of C
    int tiles_n, num_tiles;
    int a_row0, b_row0;     // operand-map row of C's first row (A) / first column (B)
    int s0, s1;             // slots [s0, s1) of both operand maps
    unsigned idesc;
    int *timeout;
};

// Bounded wait; returns false (and raises the flags) after the time limit or
// when another role already aborted.
__device__ __forceinline__ bool mbar_wait(unsigned addr, unsigned parity, volatile int *abort_flag,
                                          int *timeout) {
    if (mbar_try_wait(addr, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(addr, parity)) {
        if (*abort_flag) return false;
        if (globaltimer() - t0 > kWaitLimitNs) {
            *abort_flag = 1;
            if (timeout) atomicExch(timeout, 1);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned addr, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(addr),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap *map, int c0, int c1,
                                            unsigned mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            unsigned mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int c0, int c1, unsigned src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1), "r"(src)
                 : "memory");
}

constexpr int kCBoxBytes = BM * 32 * 4;       // one 128-row x 32-column binary32 box = 16 KB
constexpr int kCBufBytes = 4 * kCBoxBytes;    // a 128 x 128 C tile = 64 KB

// KATOMS: 128-byte K atoms per slot row (2 for TF32, 1 for 16-bit).  GROUP: the
// launch applies a group's slots to the far columns; the code is the same, the
// separate instantiation lets launch lists and profiles tell the two apart.
template <int KATOMS, int STAGES, int CBUFS, bool GROUP>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ CUtensorMap tmC, TcParams p) {
    constexpr bool kTF32 = (KATOMS == 2);
    constexpr int kAtomElems = kTF32 ? 32 : 64;          // elements per 128-byte K atom
    constexpr int kKSteps = 128 / 32;                    // MMAs per atom (32-byte K per MMA)
    constexpr unsigned kStageBytes = 2u * kAtomBytes;              // one K atom of A and of B
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const unsigned sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (sbase - smem_u32(smem_raw));
    const unsigned sA = sbase;                                   // STAGES x 16 KB
    const unsigned sB = sbase + STAGES * kAtomBytes;
    const unsigned sC = sbase + 2 * STAGES * kAtomBytes;         // CBUFS x 64 KB
    unsigned char *gC = gbase + 2 * STAGES * kAtomBytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(gC + CBUFS * kCBufBytes);
    const unsigned bar0 = smem_u32(bars);
    constexpr int kAcc0 = 2 * STAGES, kC0 = kAcc0 + 2 * kRing;
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
    auto accf_bar = [&](int b) { return bar0 + 8u * (kAcc0 + b); };
    auto acce_bar = [&](int b) { return bar0 + 8u * (kAcc0 + kRing + b); };
    auto cfull_bar = [&](int b) { return bar0 + 8u * (kC0 + b); };
    auto cempty_bar = [&](int b) { return bar0 + 8u * (kC0 + CBUFS + b); };
    auto cdone_bar = [&](int b) { return bar0 + 8u * (kC0 + 2 * CBUFS + b); };   // epilogue wrote C
    const unsigned drain_bar = bar0 + 8u * (kC0 + 3 * CBUFS);
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(bars + kC0 + 3 * CBUFS + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nslots = p.s1 - p.s0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < kRing; ++b) {
            mbar_init(accf_bar(b), 1);
            mbar_init(acce_bar(b), kEpiThreads);
        }
        for (int b = 0; b < CBUFS; ++b) {
            mbar_init(cfull_bar(b), 1);
            mbar_init(cempty_bar(b), 1);
            mbar_init(cdone_bar(b), kEpiThreads);
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            unsigned ph = 0;
            unsigned last_ph[STAGES], last_cph[CBUFS];  // parity of the latest fill of each buffer
            bool issued[STAGES], cissued[CBUFS];
            for (int q = 0; q < STAGES; ++q) issued[q] = false;
            for (int q = 0; q < CBUFS; ++q) cissued[q] = false;
            int it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < p.num_tiles; tile += gridDim.x, ++it) {
                const int tm = tile / p.tiles_n, tn = tile % p.tiles_n;
                // the C tile first: the epilogue needs it before the first slot's result
                const int cb = it % CBUFS;
                const unsigned cph = (unsigned)(it / CBUFS) & 1u;
                if (!mbar_wait(cempty_bar(cb), cph ^ 1u, abort_flag, p.timeout)) break;
                mbar_arrive_expect_tx(cfull_bar(cb), (unsigned)kCBufBytes);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    tma_load_2d(sC + cb * kCBufBytes + q * kCBoxBytes, &tmC, tn * BN + 32 * q, tm * BM, cfull_bar(cb));
                last_cph[cb] = cph;
                cissued[cb] = true;
                for (int sl = p.s0; ok && sl < p.s1; ++sl)
                    for (int q = 0; q < KATOMS; ++q) {        // one stage per 128-byte K atom
                        if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_flag, p.timeout)) { ok = false; break; }
                        mbar_arrive_expect_tx(full_bar(s), kStageBytes);
                        tma_load_3d(sA + s * kAtomBytes, &tmA, q * kAtomElems, p.a_row0 + tm * BM, sl, full_bar(s));
                        tma_load_3d(sB + s * kAtomBytes, &tmB, q * kAtomElems, p.b_row0 + tn * BN, sl, full_bar(s));
                        last_ph[s] = ph;
                        issued[s] = true;
                        if (++s == STAGES) { s = 0; ph ^= 1u; }
                    }
            }
            if (*abort_flag) {
                // drain: wait (bounded) until the copies this thread issued have landed
                volatile int no_abort = 0;
                for (int q = 0; q < STAGES; ++q)
                    if (issued[q]) mbar_wait(full_bar(q), last_ph[q], &no_abort, nullptr);
                for (int q = 0; q < CBUFS; ++q)
                    if (cissued[q]) mbar_wait(cfull_bar(q), last_cph[q], &no_abort, nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int s = 0;
            unsigned ph = 0;
            unsigned qa = 0;                    // slots issued so far: accumulator qa % kRing
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < p.num_tiles; tile += gridDim.x) {
                for (int sl = 0; sl < nslots; ++sl, ++qa) {
                    const int ab = (int)(qa % kRing);
                    const unsigned aph = (qa / kRing) & 1u;
                    if (!mbar_wait(acce_bar(ab), aph ^ 1u, abort_flag, p.timeout)) { ok = false; break; }
                    tc_fence_after();
                    const unsigned dt = tmem_base + (unsigned)(ab * BN);
                    for (int q = 0; q < KATOMS; ++q) {
                        if (!mbar_wait(full_bar(s), ph, abort_flag, p.timeout)) { ok = false; break; }
                        tc_fence_after();
#pragma unroll
                        for (int kk = 0; kk < kKSteps; ++kk) {
                            const uint64_t ad = make_desc(sA + s * kAtomBytes + kk * 32);
                            const uint64_t bd = make_desc(sB + s * kAtomBytes + kk * 32);
                            mma<kTF32>(dt, ad, bd, p.idesc, (q | kk) != 0);
                        }
                        mma_commit(empty_bar(s));
                        if (++s == STAGES) { s = 0; ph ^= 1u; }
                    }
                    if (!ok) break;
                    mma_commit(accf_bar(ab));
                }
            }
            if (*abort_flag) {
                // wait (bounded) until the tensor core has finished everything issued
                volatile int no_abort = 0;
                mma_commit(drain_bar);
                mbar_wait(drain_bar, 0u, &no_abort, nullptr);
            }
        }
    } else {
        // epilogue: warps 2..9; TMEM lane quarter = warp % 4 (tile rows 32q..32q+31),
        // column half = (warp - 2) / 4 (tile columns 64h..64h+63, two 32-column boxes)
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int r = quarter * 32 + lane;                 // row within the tile
        const bool leader = (warp == 2 && lane == 0);
        int it = 0;
        unsigned qa = 0;
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < p.num_tiles; tile += gridDim.x, ++it) {
            const int tm = tile / p.tiles_n, tn = tile % p.tiles_n;
            const int cb = it % CBUFS;
            const unsigned cph = (unsigned)(it / CBUFS) & 1u;
            if (!mbar_wait(cfull_bar(cb), cph, abort_flag, p.timeout)) break;
            // this thread's 64 values of row r, from the 128B-swizzled boxes:
            // 16-byte chunk c16 of row r sits at c16 ^ (r & 7)
            float c[64];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const unsigned char *box = gC + cb * kCBufBytes + (half * 2 + h) * kCBoxBytes + r * 128;
#pragma unroll
                for (int c16 = 0; c16 < 8; ++c16) {
                    const float4 v4 = *reinterpret_cast<const float4 *>(box + ((c16 ^ (r & 7)) << 4));
                    c[32 * h + 4 * c16 + 0] = v4.x;
                    c[32 * h + 4 * c16 + 1] = v4.y;
                    c[32 * h + 4 * c16 + 2] = v4.z;
                    c[32 * h + 4 * c16 + 3] = v4.w;
                }
            }
            for (int sl = 0; sl < nslots; ++sl, ++qa) {
                const int ab = (int)(qa % kRing);
                const unsigned aph = (qa / kRing) & 1u;
                if (!mbar_wait(accf_bar(ab), aph, abort_flag, p.timeout)) { ok = false; break; }
                tc_fence_after();
                float v0[32], v1[32];
                const unsigned tl = tmem_base + ((unsigned)(quarter * 32) << 16) + (unsigned)(ab * BN + half * 64);
                tmem_ld32(tl, v0);
                tmem_ld32(tl + 32, v1);
                tc_fence_before();
                mbar_arrive(acce_bar(ab));                 // the accumulator may be reused
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    c[q] -= v0[q];
                    c[32 + q] -= v1[q];
                }
            }
            if (!ok) break;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                unsigned char *box = gC + cb * kCBufBytes + (half * 2 + h) * kCBoxBytes + r * 128;
#pragma unroll
                for (int c16 = 0; c16 < 8; ++c16)
                    *reinterpret_cast<float4 *>(box + ((c16 ^ (r & 7)) << 4)) =
                        make_float4(c[32 * h + 4 * c16], c[32 * h + 4 * c16 + 1], c[32 * h + 4 * c16 + 2],
                                    c[32 * h + 4 * c16 + 3]);
            }
            // make the generic-proxy writes visible to the TMA store, then signal
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(cdone_bar(cb));
            if (leader) {
                if (!mbar_wait(cdone_bar(cb), cph, abort_flag, p.timeout)) break;
#pragma unroll
                for (int q = 0; q < 4; ++q) tma_store_2d(&tmC, tn * BN + 32 * q, tm * BM, sC + cb * kCBufBytes + q * kCBoxBytes);
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                mbar_arrive(cempty_bar(cb));               // the C buffer may be refilled
            }
        }
        if (leader) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                     : "memory");
    }
}

// Pack rTF of the binary32 factor columns [c0, c0 + 64 G) for the rows
// [r0, r1) into G slots of `rows` x 64 values each (slot s = columns
// c0 + 64 s .. c0 + 64 s + 63; row i of the matrix at slot row i - c0).
// One thread per 4 consecutive values of one row; A_F is row-major, so a row's
// 64 G values are contiguous and both the read and the write are coalesced.
template <typename T>
__global__ void __launch_bounds__(256) k_pack_slots(const float *AF, int64_t ldf, int c0, int G, int r0, int r1,
                                                    int64_t rows, ir_dtype tf, T *out) {
    const int q4 = 16 * G;                                  // float4 per row
    const int64_t total = (int64_t)(r1 - r0) * q4;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = r0 + (int)(e / q4), q = (int)(e % q4);
        const float4 v = *reinterpret_cast<const float4 *>(AF + (int64_t)i * ldf + c0 + 4 * q);
        const int s = q / 16, k = 4 * (q % 16);
        T *dst = out + ((int64_t)s * rows + (i - c0)) * K + k;
        if constexpr (sizeof(T) == 4) {
            uint32_t u[4];
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u[0]) : "f"(v.x));
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u[1]) : "f"(v.y));
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u[2]) : "f"(v.z));
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u[3]) : "f"(v.w));
            *reinterpret_cast<uint4 *>(dst) = make_uint4(u[0], u[1], u[2], u[3]);
        } else if (tf == IR_BF16) {
            __nv_bfloat162 p2[2] = {__floats2bfloat162_rn(v.x, v.y), __floats2bfloat162_rn(v.z, v.w)};
            *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<uint2 *>(p2);
        } else {
            __half2 p2[2] = {__floats2half2_rn(v.x, v.y), __floats2half2_rn(v.z, v.w)};
            *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<uint2 *>(p2);
        }
    }
}

// U12 of a group's rows on the tensor cores (the group's end, before the update
// of the rows below the group).  For the far columns and the group's 64-row
// blocks c = 0 .. G-1 in order:
//     C_c <- fl32(C_c - D_{c,a}),  D_{c,a} = rTF(L_{c,a}) rTF(U_a),  a = 0 .. c-1
// (each D a binary32 tensor-core sum of one block step's 64 products, as in the
// right-looking LU restricted to the group's rows), then U_c = L_cc^{-1} C_c by
// the binary32 fmaf chains of the unblocked LU (unit lower triangle, ascending
// k).  U_c goes back to A_F and, rounded to TF, into operand slot c, from which
// the later blocks of the group and the update of the rows below read it.
//
// The MMA computes the transpose D^T = rTF(U_a)^T rTF(L_{c,a})^T: M = 128 far
// columns (one per TMEM lane and per epilogue thread), N = the 64 rows of block
// c, K = 64; A = slot a of the U slots (a column's 64 K values contiguous), B =
// slot a of the L slots (a row's 64 K values contiguous): the K-major slot
// layouts of the group update.
//   warp 0     TMA producer: per pair (c, a) the U tile (128 x 64) and the L
//              tile (64 x 64) of slot a into one stage; before the first pair
//              that needs U_a it waits until the epilogue has published U_a
//   warp 1     TMEM (8 accumulators x 64 columns); MMAs, one accumulator per pair
//   warps 2-5 and 6-9  two epilogue groups taking the block rows in turn
//              (c even, c odd), one far column per thread: C_c into registers,
//              the pairs' accumulators subtracted in order, the triangular
//              solve, stores; while one group solves block c, the other
//              already subtracts block c + 1's products with U_0 .. U_{c-1}
// One CTA per 128 far columns.  Every wait is bounded; after a timeout the
// epilogue still runs its loops (no barrier is skipped) without waiting.
constexpr int kU12Acc = 8;                 // accumulators of 64 TMEM columns
constexpr int kU12Threads = 320;
constexpr int kLAtomBytes = 64 * 128;      // one 64-row x 128-byte swizzle tile = 8 KB
constexpr int kLtLd = K + 4;               // row stride of the staged diagonal block

struct U12Params {
    float *AF;
    int64_t ldf;
    int c0, G;              // the group's first column and its number of 64-row blocks
    int cb, ce;             // far columns [cb, ce)
    int bbase;              // slot row of column c in the U slots: c - bbase
    char *bop;              // U slots (bslot bytes apart), written by the epilogue
    int64_t bslot;
    ir_dtype tf;
    unsigned idesc;
    int *timeout;
};

template <int KATOMS, int STAGES>
__global__ void __launch_bounds__(kU12Threads, 1)
    k_u12_group_tc(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmL, U12Params p) {
    constexpr bool kTF32 = (KATOMS == 2);
    constexpr int kAtomElems = kTF32 ? 32 : 64;
    constexpr int kKSteps = 128 / 32;
    constexpr unsigned kStageBytes = KATOMS * (kAtomBytes + kLAtomBytes);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const unsigned sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (sbase - smem_u32(smem_raw));
    const unsigned sU = sbase;                                   // STAGES x KATOMS x 16 KB
    const unsigned sL = sbase + STAGES * KATOMS * kAtomBytes;    // STAGES x KATOMS x 8 KB
    float *Lt = reinterpret_cast<float *>(gbase + STAGES * KATOMS * (kAtomBytes + kLAtomBytes));  // [2][K][kLtLd]
    uint64_t *bars = reinterpret_cast<uint64_t *>(Lt + 2 * K * kLtLd);
    const unsigned bar0 = smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
    auto accf_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
    auto acce_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + kU12Acc + b); };
    const unsigned uready_bar = bar0 + 8u * (2 * STAGES + 2 * kU12Acc);
    const unsigned drain_bar = uready_bar + 8u;
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(bars + 2 * STAGES + 2 * kU12Acc + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < kU12Acc; ++b) {
            mbar_init(accf_bar(b), 1);
            mbar_init(acce_bar(b), 128);
        }
        mbar_init(uready_bar, 128);
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kU12Acc * 64)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int s = 0, known = 0;
            unsigned ph = 0;
            unsigned last_ph[STAGES];
            bool issued[STAGES];
            for (int q = 0; q < STAGES; ++q) issued[q] = false;
            const int urow = blockIdx.x * BM + (p.cb - p.bbase);
            bool ok = true;
            for (int c = 1; ok && c < p.G; ++c)
                for (int a = 0; a < c; ++a) {
                    if (a >= known) {      // U_a has to be published first
                        if (!mbar_wait(uready_bar, (unsigned)a & 1u, abort_flag, p.timeout)) { ok = false; break; }
                        known = a + 1;
                    }
                    if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_flag, p.timeout)) { ok = false; break; }
                    mbar_arrive_expect_tx(full_bar(s), kStageBytes);
#pragma unroll
                    for (int q = 0; q < KATOMS; ++q) {
                        tma_load_3d(sU + (s * KATOMS + q) * kAtomBytes, &tmU, q * kAtomElems, urow, a, full_bar(s));
                        tma_load_3d(sL + (s * KATOMS + q) * kLAtomBytes, &tmL, q * kAtomElems, K * c, a, full_bar(s));
                    }
                    last_ph[s] = ph;
                    issued[s] = true;
                    if (++s == STAGES) { s = 0; ph ^= 1u; }
                }
            if (*abort_flag) {
                volatile int no_abort = 0;
                for (int q = 0; q < STAGES; ++q)
                    if (issued[q]) mbar_wait(full_bar(q), last_ph[q], &no_abort, nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int s = 0;
            unsigned ph = 0, qa = 0;
            bool ok = true;
            for (int c = 1; ok && c < p.G; ++c)
                for (int a = 0; a < c; ++a, ++qa) {
                    const int ab = (int)(qa % kU12Acc);
                    if (!mbar_wait(acce_bar(ab), ((qa / kU12Acc) & 1u) ^ 1u, abort_flag, p.timeout)) { ok = false; break; }
                    tc_fence_after();
                    if (!mbar_wait(full_bar(s), ph, abort_flag, p.timeout)) { ok = false; break; }
                    tc_fence_after();
                    const unsigned dt = tmem_base + (unsigned)(ab * 64);
#pragma unroll
                    for (int q = 0; q < KATOMS; ++q)
#pragma unroll
                        for (int kk = 0; kk < kKSteps; ++kk) {
                            const uint64_t ad = make_desc(sU + (s * KATOMS + q) * kAtomBytes + kk * 32);
                            const uint64_t bd = make_desc(sL + (s * KATOMS + q) * kLAtomBytes + kk * 32);
                            mma<kTF32>(dt, ad, bd, p.idesc, (q | kk) != 0);
                        }
                    mma_commit(empty_bar(s));
                    if (++s == STAGES) { s = 0; ph ^= 1u; }
                    mma_commit(accf_bar(ab));
                }
            if (*abort_flag) {
                volatile int no_abort = 0;
                mma_commit(drain_bar);
                mbar_wait(drain_bar, 0u, &no_abort, nullptr);
            }
        }
    } else {
        // warps 2..9: group eg = (warp - 2) / 4 takes the block rows c = eg, eg + 2, ...;
        // TMEM lane quarter warp % 4; thread = far column x of the CTA
        const int eg = (warp - 2) >> 2;
        const int quarter = warp & 3;
        const int x = quarter * 32 + lane;
        const int ep = (threadIdx.x - 64) & 127;            // 0 .. 127 within the group
        const int col = p.cb + blockIdx.x * BM + x;
        const bool on = col < p.ce;
        const int esz = (p.tf == IR_TF32) ? 4 : 2;
        float *Ltg = Lt + eg * K * kLtLd;
        const unsigned gbar = 1u + (unsigned)eg;            // the group's named barrier
        for (int c = eg; c < p.G; c += 2) {
            unsigned qa = (unsigned)(c * (c - 1) / 2);      // pairs of the blocks before c
            const int rc = p.c0 + K * c;
            float u[K];
#pragma unroll
            for (int i = 0; i < K; ++i) u[i] = on ? p.AF[(int64_t)(rc + i) * p.ldf + col] : 0.f;
            asm volatile("bar.sync %0, 128;" ::"r"(gbar) : "memory");   // the group's previous solve is done with Lt
            // Lt[m][k] = l_km of the diagonal block (binary32)
#pragma unroll
            for (int i = 0; i < K * K / 4 / 128; ++i) {
                const int e = ep + 128 * i, k = e % K, m4 = e / K;
                const float4 v = *reinterpret_cast<const float4 *>(p.AF + (int64_t)(rc + k) * p.ldf + rc + 4 * m4);
                Ltg[(4 * m4 + 0) * kLtLd + k] = v.x;
                Ltg[(4 * m4 + 1) * kLtLd + k] = v.y;
                Ltg[(4 * m4 + 2) * kLtLd + k] = v.z;
                Ltg[(4 * m4 + 3) * kLtLd + k] = v.w;
            }
            for (int a = 0; a < c; ++a, ++qa) {
                const int ab = (int)(qa % kU12Acc);
                mbar_wait(accf_bar(ab), (qa / kU12Acc) & 1u, abort_flag, p.timeout);
                tc_fence_after();
                float v0[32], v1[32];
                const unsigned tl = tmem_base + ((unsigned)(quarter * 32) << 16) + (unsigned)(ab * 64);
                tmem_ld32(tl, v0);
                tmem_ld32(tl + 32, v1);
                tc_fence_before();
                mbar_arrive(acce_bar(ab));
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    u[q] -= v0[q];
                    u[32 + q] -= v1[q];
                }
            }
            asm volatile("bar.sync %0, 128;" ::"r"(gbar) : "memory");   // Lt is complete
#pragma unroll
            for (int m = 0; m < K - 1; ++m) {
                const float um = u[m];
                const float4 *l4 = reinterpret_cast<const float4 *>(Ltg + m * kLtLd);
#pragma unroll
                for (int k4 = (m + 1) / 4; k4 < K / 4; ++k4) {
                    const float4 l = l4[k4];
                    if (4 * k4 + 0 > m) u[4 * k4 + 0] = fmaf(-l.x, um, u[4 * k4 + 0]);
                    if (4 * k4 + 1 > m) u[4 * k4 + 1] = fmaf(-l.y, um, u[4 * k4 + 1]);
                    if (4 * k4 + 2 > m) u[4 * k4 + 2] = fmaf(-l.z, um, u[4 * k4 + 2]);
                    if (4 * k4 + 3 > m) u[4 * k4 + 3] = fmaf(-l.w, um, u[4 * k4 + 3]);
                }
            }
            if (on) {
#pragma unroll
                for (int i = 0; i < K; ++i) p.AF[(int64_t)(rc + i) * p.ldf + col] = u[i];
                char *dst = p.bop + (int64_t)c * p.bslot + (int64_t)(col - p.bbase) * K * esz;
                if (p.tf == IR_TF32) {
#pragma unroll
                    for (int i = 0; i < K; i += 4) {
                        uint32_t r4[4];
#pragma unroll
                        for (int h = 0; h < 4; ++h) asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r4[h]) : "f"(u[i + h]));
                        reinterpret_cast<uint4 *>(dst)[i / 4] = make_uint4(r4[0], r4[1], r4[2], r4[3]);
                    }
                } else if (p.tf == IR_BF16) {
#pragma unroll
                    for (int i = 0; i < K; i += 8) {
                        __nv_bfloat162 p2[4];
#pragma unroll
                        for (int h = 0; h < 4; ++h) p2[h] = __floats2bfloat162_rn(u[i + 2 * h], u[i + 2 * h + 1]);
                        reinterpret_cast<uint4 *>(dst)[i / 8] = *reinterpret_cast<uint4 *>(p2);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < K; i += 8) {
                        __half2 p2[4];
#pragma unroll
                        for (int h = 0; h < 4; ++h) p2[h] = __floats2half2_rn(u[i + 2 * h], u[i + 2 * h + 1]);
                        reinterpret_cast<uint4 *>(dst)[i / 8] = *reinterpret_cast<uint4 *>(p2);
                    }
                }
            }
            // the U slot rows are read back by TMA (async proxy) for the later blocks
            asm volatile("fence.proxy.async.global;" ::: "memory");
            mbar_arrive(uready_bar);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kU12Acc * 64)
                     : "memory");
    }
}

using EncodeTiledFn = TensorMapEncodeFn;
EncodeTiledFn get_encoder() { return tensor_map_encoder(); }

// Operand slots: `slots` x rows x K, K contiguous (K-major); box = one 128-byte
// K atom x box_rows rows x 1 slot.
bool make_slot_map(CUtensorMap *m, const void *base, int64_t rows, int slots, ir_dtype tf, int box_rows = BM) {
    EncodeTiledFn enc = get_encoder();
    if (!enc) return false;
    const int esz = (tf == IR_TF32) ? 4 : 2;
    const CUtensorMapDataType dt = (tf == IR_TF32) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : (tf == IR_BF16) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)slots};
    cuuint64_t strides[2] = {(cuuint64_t)K * esz, (cuuint64_t)rows * K * esz};
    cuuint32_t box[3] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, dt, 3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The binary32 trailing matrix C (rows x cols, row stride ld floats): boxes of
// 128 rows x 32 columns (128 bytes), 128-byte swizzle.
bool make_c_map(CUtensorMap *m, float *base, int rows, int cols, int64_t ld) {
    EncodeTiledFn enc = get_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {32, (cuuint32_t)BM};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Instruction descriptor for kind::tf32 / kind::f16: D = F32 (bits 4-5 = 1),
// A/B format (bits 7-9 / 10-12: F16 0, BF16 1, TF32 2), both K-major,
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
unsigned make_idesc(ir_dtype tf, int n_cols = BN) {
    const unsigned fmt = (tf == IR_TF32) ? 2u : (tf == IR_BF16) ? 1u : 0u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((unsigned)(n_cols >> 3) << 17) | ((unsigned)(BM >> 4) << 24);
}

template <int KATOMS, int STAGES, int CBUFS>
constexpr size_t smem_bytes() {
    return 1024 + 2 * STAGES * kAtomBytes + CBUFS * kCBufBytes + 8 * (2 * STAGES + 2 * kRing + 1 + 3 * CBUFS) + 16;
}
// 3 stages of one K atom (32 KB for A and B) and 2 C buffers (64 KB each)
static_assert(smem_bytes<1, 3, 2>() <= 232448, "16-bit configuration exceeds shared memory");
static_assert(smem_bytes<2, 3, 2>() <= 232448, "TF32 configuration exceeds shared memory");


template <int KATOMS, int STAGES>
constexpr size_t u12_smem_bytes() {
    return 1024 + (size_t)STAGES * KATOMS * (kAtomBytes + kLAtomBytes) + (size_t)2 * K * kLtLd * 4 +
           8 * (2 * STAGES + 2 * kU12Acc + 2) + 16;
}
static_assert(u12_smem_bytes<1, 4>() <= 232448 && u12_smem_bytes<2, 3>() <= 232448,
              "group U12 configuration exceeds shared memory");

// Launch one update of C (rows x cols, binary32, row stride ldf) by the slots
// [s0, s1) of the operand maps; a_row0 / b_row0: operand rows of C's first
// row / column.  max_ctas > 0: share the GPU with a concurrent panel (8-CTA
// clusters, two clusters fewer than fit at once).
cudaError_t launch_slots(float *C, int64_t ldf, int rows, int cols, const CUtensorMap &ta, const CUtensorMap &tb,
                         int a_row0, int b_row0, int s0, int s1, ir_dtype tf, int sms, int max_ctas,
                         DevScalars *dev, cudaStream_t s) {
    if (rows <= 0 || cols <= 0 || s1 <= s0) return cudaSuccess;
    TcParams p;
    p.M = rows;
    p.N = cols;
    const int tiles_m = (rows + BM - 1) / BM;
    p.tiles_n = (cols + BN - 1) / BN;
    p.num_tiles = tiles_m * p.tiles_n;
    p.a_row0 = a_row0;
    p.b_row0 = b_row0;
    p.s0 = s0;
    p.s1 = s1;
    p.idesc = make_idesc(tf);
    p.timeout = &dev->timeout;
    CUtensorMap tc;
    if (!make_c_map(&tc, C, rows, cols, ldf)) return cudaErrorInvalidValue;
    const bool share = max_ctas > 0;
    int grid = p.num_tiles < sms ? p.num_tiles : sms;
    auto launch = [&](auto kern, size_t smem) -> cudaError_t {
        count_launch();
        if (!share) {
            kern<<<grid, kThreads, smem, s>>>(ta, tb, tc, p);
            return cudaGetLastError();
        }
        cudaLaunchConfig_t cfg = {};
        cfg.blockDim = dim3(kThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 8;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(8 * 32, 1, 1);
        int maxc = 0;
        if (cudaOccupancyMaxActiveClusters(&maxc, kern, &cfg) != cudaSuccess) maxc = 0;
        (void)cudaGetLastError();
        int clusters = maxc - 2;
        if (clusters < 1) clusters = 1;
        const int need = (p.num_tiles + 7) / 8;
        if (clusters > need) clusters = need;
        cfg.gridDim = dim3(8 * clusters, 1, 1);
        return cudaLaunchKernelEx(&cfg, kern, ta, tb, tc, p);
    };
    auto go = [&](auto kern, size_t smem, bool &attr) -> cudaError_t {
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        return launch(kern, smem);
    };
    const bool group = s1 - s0 > 1;
    static bool a0 = false, a1 = false, a2 = false, a3 = false;
    if (tf == IR_TF32)
        return group ? go(k_gemm_tc<2, 3, 2, true>, smem_bytes<2, 3, 2>(), a0)
                     : go(k_gemm_tc<2, 3, 2, false>, smem_bytes<2, 3, 2>(), a1);
    return group ? go(k_gemm_tc<1, 3, 2, true>, smem_bytes<1, 3, 2>(), a2)
                 : go(k_gemm_tc<1, 3, 2, false>, smem_bytes<1, 3, 2>(), a3);
}

}  // namespace

// One block step: rows [j + nb, n) x columns [cb, ce) of the trailing matrix
// (cb a multiple of 64) by the step's operands (Aop: rows j + nb .. n - 1,
// Bop: columns j + nb .. n - 1, K = 64 each); at most max_ctas persistent
// CTAs (0: one per SM).
cudaError_t launch_gemm_tc(float *AF, int64_t ldf, int n, int j, int nb, int cb, int ce, ir_dtype tf,
                           const void *Aop, const void *Bop, int sms, int max_ctas, DevScalars *dev,
                           cudaStream_t s) {
    const int m = n - (j + nb);
    if (m <= 0 || ce <= cb) return cudaSuccess;
    if (nb != K) return cudaErrorInvalidValue;
    CUtensorMap ta, tb;
    if (!make_slot_map(&ta, Aop, m, 1, tf) || !make_slot_map(&tb, Bop, m, 1, tf)) return cudaErrorInvalidValue;
    return launch_slots(AF + (int64_t)(j + nb) * ldf + cb, ldf, m, ce - cb, ta, tb, 0, cb - (j + nb), 0, 1, tf,
                        sms, max_ctas, dev, s);
}

// Group update (see the file comment): C = rows [r0, r1) x columns [cb, ce) of
// A_F minus the products of the group's slots [s0, s1).  Agrp: G slots of
// a_rows rows (slot row i - c0 holds rTF of row i of the group's L columns);
// Bgrp: G slots of b_rows rows (slot row c - bbase holds rTF(U) of column c).
cudaError_t launch_gemm_tc_group(float *AF, int64_t ldf, int c0, int G, int r0, int r1, int cb, int ce,
                                 int s0, int s1, ir_dtype tf, const void *Agrp, int64_t a_rows, const void *Bgrp,
                                 int64_t b_rows, int bbase, int sms, int max_ctas, DevScalars *dev,
                                 cudaStream_t s) {
    if (r1 <= r0 || ce <= cb || s1 <= s0) return cudaSuccess;
    CUtensorMap ta, tb;
    if (!make_slot_map(&ta, Agrp, a_rows, G, tf) || !make_slot_map(&tb, Bgrp, b_rows, G, tf))
        return cudaErrorInvalidValue;
    return launch_slots(AF + (int64_t)r0 * ldf + cb, ldf, r1 - r0, ce - cb, ta, tb, r0 - c0, cb - bbase, s0, s1, tf,
                        sms, max_ctas, dev, s);
}

// U12 of the group's rows on the tensor cores (see k_u12_group_tc): far columns
// [cb, ce); Agrp: the group's L slots (slot row i - c0 for matrix row i, a_rows
// rows per slot); Bgrp: the U slots (slot row c - bbase for column c, b_rows rows
// per slot, written here).
cudaError_t launch_u12_group_tc(float *AF, int64_t ldf, int c0, int G, int cb, int ce, ir_dtype tf,
                                const void *Agrp, int64_t a_rows, void *Bgrp, int64_t b_rows, int bbase,
                                DevScalars *dev, cudaStream_t s) {
    if (ce <= cb || G <= 0) return cudaSuccess;
    if (cb < bbase || ce - bbase > b_rows || (int64_t)K * G > a_rows) return cudaErrorInvalidValue;
    CUtensorMap tu, tl;
    if (!make_slot_map(&tu, Bgrp, b_rows, G, tf) || !make_slot_map(&tl, Agrp, a_rows, G, tf, K))
        return cudaErrorInvalidValue;
    U12Params p;
    p.AF = AF;
    p.ldf = ldf;
    p.c0 = c0;
    p.G = G;
    p.cb = cb;
    p.ce = ce;
    p.bbase = bbase;
    p.bop = static_cast<char *>(Bgrp);
    p.bslot = b_rows * K * (int64_t)((tf == IR_TF32) ? 4 : 2);
    p.tf = tf;
    p.idesc = make_idesc(tf, K);
    p.timeout = &dev->timeout;
    const int grid = (ce - cb + BM - 1) / BM;
    static bool a16 = false, a32 = false;
    count_launch();
    if (tf == IR_TF32) {
        constexpr size_t sm = u12_smem_bytes<2, 3>();
        if (!a32) {
            cudaError_t e = cudaFuncSetAttribute(k_u12_group_tc<2, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            a32 = true;
        }
        k_u12_group_tc<2, 3><<<grid, kU12Threads, sm, s>>>(tu, tl, p);
    } else {
        constexpr size_t sm = u12_smem_bytes<1, 4>();
        if (!a16) {
            cudaError_t e = cudaFuncSetAttribute(k_u12_group_tc<1, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            a16 = true;
        }
        k_u12_group_tc<1, 4><<<grid, kU12Threads, sm, s>>>(tu, tl, p);
    }
    return cudaGetLastError();
}

// rTF of the factor columns [c0, c0 + 64 G), rows [r0, r1), into the G slots of
// `rows` rows each (row i at slot row i - c0).
cudaError_t launch_pack_slots(const float *AF, int64_t ldf, int c0, int G, int r0, int r1, int64_t rows, ir_dtype tf,
                              void *out, int sms, cudaStream_t s) {
    if (r1 <= r0 || G <= 0) return cudaSuccess;
    count_launch();
    const int64_t total = (int64_t)(r1 - r0) * 16 * G;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 8 * sms) blocks = 8 * sms;
    if (tf == IR_TF32)
        k_pack_slots<float><<<(int)blocks, 256, 0, s>>>(AF, ldf, c0, G, r0, r1, rows, tf, static_cast<float *>(out));
    else
        k_pack_slots<__half><<<(int)blocks, 256, 0, s>>>(AF, ldf, c0, G, r0, r1, rows, tf, static_cast<__half *>(out));
    return cudaGetLastError();
}

}  // namespace ir
