// Tensor-core trailing update of the mixed-precision blocked LU:
//     A22 <- A22 - rTF(L21) rTF(U12)
// with the TF-rounded operands (TF32, bf16 or fp16, written by the panel and
// U12 kernels) multiplied by tcgen05.mma with binary32 accumulation in tensor
// memory (TMEM), then subtracted from the binary32 matrix in the epilogue.
//
// Persistent, warp-specialised kernel, one CTA per SM:
//   warp 0      TMA producer: both operand tiles of a 128x128 output tile
//               (K = 64, 128-byte swizzle) into a shared-memory ring, and the
//               binary32 C tile itself (four 128x32 boxes) into one of two
//               C buffers
//   warp 1      allocates TMEM (2 accumulators x 128 columns) and issues the
//               MMAs from one thread; tcgen05.commit frees the stage and
//               signals the accumulator
//   warps 2-9   epilogue: tcgen05.ld the accumulator, C -= D in shared memory,
//               one thread stores the tile back with TMA (edges are clipped
//               by the tensor map, so ragged tiles need no guards)
// Every mbarrier wait is bounded (globaltimer); on timeout the CTA records
// the error, waits (bounded) for its own copies in flight, frees TMEM and
// returns.
#include <cuda.h>

#include "ir_internal.cuh"
#include "tc_util.cuh"

namespace ir {
namespace {

constexpr int BM = 128, BN = 128, K = kPanelNB;
constexpr int kAtomBytes = BM * 128;      // one 128-row x 128-byte swizzle tile = 16 KB
constexpr int kThreads = 320;             // 10 warps
constexpr int kEpiThreads = 256;
constexpr unsigned kTmemCols = 2 * BN;    // double-buffered accumulator

struct TcParams {
    float *C;
    int64_t ldc;
    int M, N;
    int tiles_n, num_tiles;
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
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int c0, int c1, unsigned src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1), "r"(src)
                 : "memory");
}

constexpr int kCBoxBytes = BM * 32 * 4;       // one 128-row x 32-column binary32 box = 16 KB
constexpr int kCBufBytes = 4 * kCBoxBytes;    // a 128 x 128 C tile = 64 KB
constexpr int kCBufs = 2;

template <int KATOMS, int STAGES>   // 128-byte K atoms per operand row: 2 for TF32, 1 for 16-bit
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ CUtensorMap tmC, TcParams p) {
    constexpr bool kTF32 = (KATOMS == 2);
    constexpr int kAtomElems = kTF32 ? 32 : 64;          // elements per 128-byte K atom
    constexpr int kKSteps = 128 / 32;                    // MMAs per atom (32-byte K per MMA)
    constexpr unsigned kStageBytes = 2u * KATOMS * kAtomBytes;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const unsigned sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (sbase - smem_u32(smem_raw));
    const unsigned sA = sbase;                                   // STAGES x KATOMS x 16 KB
    const unsigned sB = sbase + STAGES * KATOMS * kAtomBytes;
    const unsigned sC = sbase + 2 * STAGES * KATOMS * kAtomBytes; // kCBufs x 64 KB
    unsigned char *gC = gbase + 2 * STAGES * KATOMS * kAtomBytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(gC + kCBufs * kCBufBytes);
    const unsigned bar0 = smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
    auto accf_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
    auto acce_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 + b); };
    auto cfull_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 4 + b); };
    auto cempty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 6 + b); };
    auto cdone_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 8 + b); };   // epilogue wrote C
    const unsigned drain_bar = bar0 + 8u * (2 * STAGES + 10);
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(bars + 2 * STAGES + 11);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf_bar(b), 1);
            mbar_init(acce_bar(b), kEpiThreads);
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
            unsigned last_ph[STAGES], last_cph[kCBufs];  // parity of the latest fill of each buffer
            bool issued[STAGES], cissued[kCBufs];
            for (int q = 0; q < STAGES; ++q) issued[q] = false;
            for (int q = 0; q < kCBufs; ++q) cissued[q] = false;
            int it = 0;
            for (int tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x, ++it) {
                const int tm = tile / p.tiles_n, tn = tile % p.tiles_n;
                if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_flag, p.timeout)) break;
                mbar_arrive_expect_tx(full_bar(s), kStageBytes);
#pragma unroll
                for (int q = 0; q < KATOMS; ++q) {
                    tma_load_2d(sA + (s * KATOMS + q) * kAtomBytes, &tmA, q * kAtomElems, tm * BM, full_bar(s));
                    tma_load_2d(sB + (s * KATOMS + q) * kAtomBytes, &tmB, q * kAtomElems, tn * BN, full_bar(s));
                }
                last_ph[s] = ph;
                issued[s] = true;
                if (++s == STAGES) { s = 0; ph ^= 1u; }
                // the C tile
                const int cb = it & 1;
                const unsigned cph = (unsigned)(it >> 1) & 1u;
                if (!mbar_wait(cempty_bar(cb), cph ^ 1u, abort_flag, p.timeout)) break;
                mbar_arrive_expect_tx(cfull_bar(cb), (unsigned)kCBufBytes);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    tma_load_2d(sC + cb * kCBufBytes + q * kCBoxBytes, &tmC, tn * BN + 32 * q, tm * BM, cfull_bar(cb));
                last_cph[cb] = cph;
                cissued[cb] = true;
            }
            if (*abort_flag) {
                // drain: wait (bounded) until the copies this thread issued have landed
                volatile int no_abort = 0;
                for (int q = 0; q < STAGES; ++q)
                    if (issued[q]) mbar_wait(full_bar(q), last_ph[q], &no_abort, nullptr);
                for (int q = 0; q < kCBufs; ++q)
                    if (cissued[q]) mbar_wait(cfull_bar(q), last_cph[q], &no_abort, nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int s = 0;
            unsigned ph = 0;
            int it = 0;
            for (int tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x, ++it) {
                const int ab = it & 1;
                const unsigned aph = (unsigned)(it >> 1) & 1u;
                if (!mbar_wait(acce_bar(ab), aph ^ 1u, abort_flag, p.timeout)) break;
                tc_fence_after();
                if (!mbar_wait(full_bar(s), ph, abort_flag, p.timeout)) break;
                tc_fence_after();
                const unsigned dt = tmem_base + (unsigned)(ab * BN);
#pragma unroll
                for (int q = 0; q < KATOMS; ++q)
#pragma unroll
                    for (int kk = 0; kk < kKSteps; ++kk) {
                        const uint64_t ad = make_desc(sA + (s * KATOMS + q) * kAtomBytes + kk * 32);
                        const uint64_t bd = make_desc(sB + (s * KATOMS + q) * kAtomBytes + kk * 32);
                        mma<kTF32>(dt, ad, bd, p.idesc, (q | kk) != 0);
                    }
                mma_commit(empty_bar(s));
                mma_commit(accf_bar(ab));
                if (++s == STAGES) { s = 0; ph ^= 1u; }
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
        for (int tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x, ++it) {
            const int tm = tile / p.tiles_n, tn = tile % p.tiles_n;
            const int ab = it & 1, cb = it & 1;
            const unsigned aph = (unsigned)(it >> 1) & 1u;
            if (!mbar_wait(accf_bar(ab), aph, abort_flag, p.timeout)) break;
            tc_fence_after();
            float v0[32], v1[32];
            const unsigned tl = tmem_base + ((unsigned)(quarter * 32) << 16) + (unsigned)(ab * BN + half * 64);
            tmem_ld32(tl, v0);
            tmem_ld32(tl + 32, v1);
            tc_fence_before();
            mbar_arrive(acce_bar(ab));                     // the accumulator may be reused
            if (!mbar_wait(cfull_bar(cb), aph, abort_flag, p.timeout)) break;
            // C -= D in the 128B-swizzled boxes: 16-byte chunk c16 of row r sits at c16 ^ (r & 7)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float *v = h ? v1 : v0;
                unsigned char *box = gC + cb * kCBufBytes + (half * 2 + h) * kCBoxBytes + r * 128;
#pragma unroll
                for (int c16 = 0; c16 < 8; ++c16) {
                    float4 *q4 = reinterpret_cast<float4 *>(box + ((c16 ^ (r & 7)) << 4));
                    float4 c = *q4;
                    c.x -= v[4 * c16 + 0];
                    c.y -= v[4 * c16 + 1];
                    c.z -= v[4 * c16 + 2];
                    c.w -= v[4 * c16 + 3];
                    *q4 = c;
                }
            }
            // make the generic-proxy writes visible to the TMA store, then signal
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(cdone_bar(cb));
            if (leader) {
                if (!mbar_wait(cdone_bar(cb), aph, abort_flag, p.timeout)) break;
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

using EncodeTiledFn = TensorMapEncodeFn;
EncodeTiledFn get_encoder() { return tensor_map_encoder(); }

// rows x K operand, row-major, K contiguous; box = one 128-byte K atom x 128 rows.
bool make_map(CUtensorMap *m, const void *base, int rows, ir_dtype tf) {
    EncodeTiledFn enc = get_encoder();
    if (!enc) return false;
    const int esz = (tf == IR_TF32) ? 4 : 2;
    const CUtensorMapDataType dt = (tf == IR_TF32) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : (tf == IR_BF16) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)K * esz};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)BM};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
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
unsigned make_idesc(ir_dtype tf) {
    const unsigned fmt = (tf == IR_TF32) ? 2u : (tf == IR_BF16) ? 1u : 0u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((unsigned)(BN >> 3) << 17) | ((unsigned)(BM >> 4) << 24);
}

template <int KATOMS, int STAGES>
size_t smem_bytes() {
    return 1024 + 2 * STAGES * KATOMS * kAtomBytes + kCBufs * kCBufBytes + 8 * (2 * STAGES + 11) + 16;
}

}  // namespace

// Columns [cb, ce) of the trailing matrix (cb a multiple of 64); at most
// max_ctas persistent CTAs (0: one per SM).
cudaError_t launch_gemm_tc(float *AF, int64_t ldf, int n, int j, int nb, int cb, int ce, ir_dtype tf,
                           const void *Aop, const void *Bop, int sms, int max_ctas, DevScalars *dev,
                           cudaStream_t s) {
    const int m = n - (j + nb);
    if (m <= 0 || ce <= cb) return cudaSuccess;
    if (nb != K) return cudaErrorInvalidValue;
    const int ncols = ce - cb;
    const size_t esz = (tf == IR_TF32) ? 4 : 2;
    const void *Bsub = static_cast<const char *>(Bop) + (size_t)(cb - (j + nb)) * K * esz;
    CUtensorMap ta, tb;
    if (!make_map(&ta, Aop, m, tf) || !make_map(&tb, Bsub, ncols, tf)) return cudaErrorInvalidValue;
    TcParams p;
    p.C = AF + (int64_t)(j + nb) * ldf + cb;
    p.ldc = ldf;
    p.M = m;
    p.N = ncols;
    const int tiles_m = (m + BM - 1) / BM;
    p.tiles_n = (ncols + BN - 1) / BN;
    p.num_tiles = tiles_m * p.tiles_n;
    p.idesc = make_idesc(tf);
    p.timeout = &dev->timeout;
    CUtensorMap tc;
    if (!make_c_map(&tc, p.C, m, ncols, ldf)) return cudaErrorInvalidValue;
    const bool share = max_ctas > 0;
    int grid = p.num_tiles < sms ? p.num_tiles : sms;
    auto launch = [&](auto kern, size_t smem) -> cudaError_t {
        count_launch();
        if (!share) {
            kern<<<grid, kThreads, smem, s>>>(ta, tb, tc, p);
            return cudaGetLastError();
        }
        // share the GPU with a concurrent panel: clusters of 8 CTAs, two
        // clusters fewer than fit at once, so whole GPC slots stay free
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
    if (tf == IR_TF32) {
        static bool attr = false;
        const size_t sm = smem_bytes<2, 1>();
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        return launch(k_gemm_tc<2, 1>, sm);
    } else {
        static bool attr = false;
        const size_t sm = smem_bytes<1, 2>();
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        return launch(k_gemm_tc<1, 2>, sm);
    }
}

}  // namespace ir
