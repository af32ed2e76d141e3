// Device pieces of the blocked LU shared by several kernels: the U12 solve of
// 64 columns and the 64 x 64 trailing-update tile.  Both are the binary32
// fmaf chains of the unblocked right-looking algorithm (l_ik, u_kj, k
// ascending), so every kernel built from them gives the same bits.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ir_internal.cuh"

namespace ir {
namespace lu {

constexpr int NB = kPanelNB;
constexpr int kLd = NB + 4;       // row stride of the 64-wide shared tiles

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

// U12 = L11^{-1} A12 for the block row j..j+NB and the columns c0 .. c0 + 63
// (those below ce), in place; 256 threads, four per column, each holding 16
// rows; column-oriented: for m ascending the owner of row m broadcasts the
// final u_m (shuffle) and the rows below take fmaf(-l_km, u_m, u_k), so every
// entry is the fmaf chain over m < k in ascending order, as in the unblocked
// LU.  For tensor-core updates rTF(u_mc) is also written to Bop (row c).
// Lt: shared [NB][kLd].  Every thread of the CTA must call it.
__device__ __forceinline__ void trsm64(float *AF, int64_t ldf, int c0, int ce, int j, ir_dtype tf, void *Bop,
                                       float (*Lt)[kLd]) {
    {
        // all loads in flight before the (transposing) stores: row k, columns 4 m4 .. 4 m4 + 3;
        // k runs fastest over the lanes so that the transposed stores hit 32 banks
        float4 v[NB * NB / 4 / 256];
#pragma unroll
        for (int i = 0; i < NB * NB / 4 / 256; ++i) {
            const int e = threadIdx.x + i * 256, k = e % NB, m4 = e / NB;
            v[i] = *reinterpret_cast<const float4 *>(AF + (int64_t)(j + k) * ldf + j + 4 * m4);
        }
#pragma unroll
        for (int i = 0; i < NB * NB / 4 / 256; ++i) {
            const int e = threadIdx.x + i * 256, k = e % NB, m4 = e / NB;
            Lt[4 * m4 + 0][k] = v[i].x;
            Lt[4 * m4 + 1][k] = v[i].y;
            Lt[4 * m4 + 2][k] = v[i].z;
            Lt[4 * m4 + 3][k] = v[i].w;
        }
    }
    __syncthreads();
    const int t = threadIdx.x, lane = t & 31, q = t & 3;
    const int c = c0 + (t >> 2);
    const bool on = c < ce;
    float u[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) u[r] = on ? AF[(int64_t)(j + q * 16 + r) * ldf + c] : 0.f;
#pragma unroll
    for (int m = 0; m < NB - 1; ++m) {
        const float um = __shfl_sync(0xffffffffu, u[m % 16], (lane & ~3) | (m / 16));
        const float4 *l4 = reinterpret_cast<const float4 *>(&Lt[m][q * 16]);
#pragma unroll
        for (int r4 = 0; r4 < 4; ++r4) {
            const float4 l = l4[r4];
            const int k = q * 16 + 4 * r4;
            if (k + 0 > m) u[4 * r4 + 0] = fmaf(-l.x, um, u[4 * r4 + 0]);
            if (k + 1 > m) u[4 * r4 + 1] = fmaf(-l.y, um, u[4 * r4 + 1]);
            if (k + 2 > m) u[4 * r4 + 2] = fmaf(-l.z, um, u[4 * r4 + 2]);
            if (k + 3 > m) u[4 * r4 + 3] = fmaf(-l.w, um, u[4 * r4 + 3]);
        }
    }
    if (!on) return;
#pragma unroll
    for (int r = 0; r < 16; ++r)
        if (q * 16 + r > 0) AF[(int64_t)(j + q * 16 + r) * ldf + c] = u[r];
    if (Bop == nullptr) return;
    const int64_t row = c - (j + NB);
    if (tf == IR_TF32) {
        float4 *dst = reinterpret_cast<float4 *>(static_cast<float *>(Bop) + row * NB + q * 16);
#pragma unroll
        for (int r = 0; r < 16; r += 4)
            dst[r / 4] = make_float4(round_tf(u[r], tf), round_tf(u[r + 1], tf), round_tf(u[r + 2], tf),
                                     round_tf(u[r + 3], tf));
    } else if (tf == IR_BF16) {
        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(Bop) + row * NB + q * 16);
#pragma unroll
        for (int r = 0; r < 16; r += 8) {
            __nv_bfloat162 p2[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) p2[h] = __floats2bfloat162_rn(u[r + 2 * h], u[r + 2 * h + 1]);
            dst[r / 8] = *reinterpret_cast<uint4 *>(p2);
        }
    } else if (tf == IR_F16) {
        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<__half *>(Bop) + row * NB + q * 16);
#pragma unroll
        for (int r = 0; r < 16; r += 8) {
            __half2 p2[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) p2[h] = __floats2half2_rn(u[r + 2 * h], u[r + 2 * h + 1]);
            dst[r / 8] = *reinterpret_cast<uint4 *>(p2);
        }
    }
}

// A22 <- A22 - L21 U12 on the 64 x 64 tile of rows i0 .. i0 + 63 (below n) and
// columns cb .. cb + 63 (below ce), binary32: thread (ty, tx) of 256 owns rows
// 4 ty .. 4 ty + 3 and columns 4 tx .. 4 tx + 3, fmaf chains from C in
// ascending k.  As, Bs: shared [NB][kLd].  Every thread of the CTA must call it.
__device__ __forceinline__ void gemm_tile64(float *AF, int64_t ldf, int n, int j, int cb, int ce, int i0,
                                            float (*As)[kLd], float (*Bs)[kLd]) {
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    {
        // all eight 16-byte loads of a thread in flight before the stores; for L21 the
        // row runs fastest over the lanes so that the transposed stores hit 32 banks
        constexpr int R = NB * NB / 4 / 256;
        float4 va[R], vb[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int e = t + q * 256, ra = e % NB, ka = (e / NB) * 4, i = i0 + ra;
            const int rb = e >> 4, cq = (e & 15) * 4, c = cb + cq;
            va[q] = (i < n) ? *reinterpret_cast<const float4 *>(AF + (int64_t)i * ldf + j + ka)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
            vb[q] = (c < ce) ? *reinterpret_cast<const float4 *>(AF + (int64_t)(j + rb) * ldf + c)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int e = t + q * 256, ra = e % NB, ka = (e / NB) * 4, rb = e >> 4, cq = (e & 15) * 4;
            As[ka + 0][ra] = va[q].x; As[ka + 1][ra] = va[q].y; As[ka + 2][ra] = va[q].z; As[ka + 3][ra] = va[q].w;
            *reinterpret_cast<float4 *>(&Bs[rb][cq]) = vb[q];
        }
    }
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = i0 + ty * 4 + r, c = cb + tx * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < n && c < ce) v = *reinterpret_cast<const float4 *>(AF + (int64_t)i * ldf + c);
        acc[r][0] = v.x; acc[r][1] = v.y; acc[r][2] = v.z; acc[r][3] = v.w;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < NB; ++k) {
        const float4 a = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
        const float4 b = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
        const float ar[4] = {a.x, a.y, a.z, a.w}, br[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(-ar[r], br[q], acc[r][q]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = i0 + ty * 4 + r, c = cb + tx * 4;
        if (i < n && c < ce)
            *reinterpret_cast<float4 *>(AF + (int64_t)i * ldf + c) =
                make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    }
}

}  // namespace lu
}  // namespace ir
