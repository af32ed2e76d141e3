// Batched driver: many independent systems of uneven size n <= 512, each cast,
// factored and refined (Algorithm IR, Sec. 1; termination of Sec. 5.1) inside
// ONE persistent kernel launch.  Each CTA (512 threads, one per SM) takes the
// next system from a ticket counter; the systems come in longest-first order,
// so the long ones start first and the short ones fill the tail.
//
// Inside a CTA every step of the single-system path runs on a row-major
// binary32 copy W (row stride ldw = n rounded up to a multiple of 4, so rows
// start 16-byte aligned) in the CTA's workspace slot (global memory, L2-
// resident at these sizes); the IR vectors x, r, b (binary64) and the
// permutation live in shared memory.
//   cast          W = rTF(fl32(s A)), A streamed through shared memory by cp.async
//   panel         64 columns, one row per thread in a rotating register
//                 window for the whole panel (rows never move; interchanges
//                 only swap position labels), one CTA barrier per column
//                 (each warp stages its candidate row; every warp then
//                 picks the pivot row)
//   interchanges  gather of the moved rows for the columns outside the panel
//   U12           L11^{-1} A12 by fmaf chains (binary32, ascending k)
//   update        binary16 / bfloat16 factors: tcgen05.mma on the tensor
//                 cores (operands rounded to TF while staged in shared
//                 memory, binary32 accumulation in tensor memory, C -= D in
//                 the epilogue), 128x128 tiles, four per wave;
//                 binary32 / TF32 factors (and trailing blocks of <= 64
//                 rows): two groups of 256 threads, 64x64 tiles, 4x4 per
//                 thread; TF = binary32 runs the fmaf chain from C (so the
//                 factors are bitwise those of the unblocked LU), TF32 sums
//                 rTF(l) rTF(u) in binary32 and subtracts the sum
//   solves        the reference-BLAS trsv order (forward: columns ascending;
//                 back: columns descending, the division first), blocked by
//                 32 columns: one warp solves the diagonal block with
//                 shuffles, every row below (above) then applies the block's
//                 32 columns in that same order; one CTA barrier per block
//   residual      binary64, one row per thread, fma chain in ascending j
#include <cfloat>
#include <climits>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ir_internal.cuh"
#include "tc_util.cuh"

namespace ir {
namespace {

constexpr int BT = 512;           // threads per CTA
constexpr int BW = BT / 32;       // warps per CTA
constexpr int NB = 64;            // block size (as in the single-system LU)
constexpr int kRow = NB + 4;      // staged row: value i at index 3 + i
constexpr int kLd = NB + 4;       // row stride of the 64-wide shared tiles
constexpr int kMaxBatchN = IR_BATCH_MAX_N;
static_assert(kMaxBatchN <= BT, "one row per thread");

struct BSmem {
    alignas(16) float stage[2][BW][kRow];     // per-warp candidate rows, by step parity
    alignas(16) double xs[kMaxBatchN];        // iterate (binary64)
    alignas(16) double rs[kMaxBatchN];        // residual
    alignas(16) double bs[kMaxBatchN];        // right-hand side, promoted
    alignas(16) float vs[kMaxBatchN];         // solve values published by the sweeps
    int perm[kMaxBatchN];                     // (P A)[i] = A[perm[i]]
    float sval[2][BW];
    int spos[2][BW];                          // current position of each warp's candidate
    float srec[2][BW];                        // reciprocal of each candidate's pivot value
    int moved_cnt;
    int moved_dst[2 * NB], moved_src[2 * NB];
    unsigned long long red[BW];
    unsigned long long mma_bar;               // tensor-core completion (tcgen05.commit)
    unsigned tmem_base;
    int info, nonfinite, cur, abort;
};
static_assert(offsetof(BSmem, stage) % 16 == 0 && (kRow * 4) % 16 == 0, "staged rows must be 16-byte aligned");
constexpr size_t kBigFloats = (size_t)NB * BT;      // 128 KB of multi-use scratch, 1024-byte aligned
constexpr size_t kBatchSmem = 1024 + (kBigFloats + NB * NB) * sizeof(float) + sizeof(BSmem);
constexpr unsigned kTmemCols = 512;                 // four 128x128 binary32 accumulators
static_assert(kBatchSmem <= 227 * 1024, "shared memory per CTA");
static_assert(4 * NB * kLd <= (int)kBigFloats, "update tiles of both groups fit the scratch");
static_assert(2 * NB * 256 <= (int)kBigFloats, "interchange staging fits the scratch");
static_assert(2 * 512 * 128 <= (int)kBigFloats * 4, "both 16-bit operands (512 rows x 128 bytes) fit the scratch");

struct BatchSys {
    const void *A;
    const void *b;
    void *x;
    int64_t lda;
    int n;
    int pad;
};

struct BatchCfg {
    double Cr, Rmax, abs_rel_tol, eps_w;
    int litmax, tr_wider, fp16_scale, count;
    ir_dtype tw, tf;
    int tc_min_trail;      // smallest trailing block that takes the tensor-core update (tuned)
};

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

// |v| as an ordered bit pattern: for non-negative doubles the unsigned order of
// the bits is the order of the values, and a NaN (sign cleared) sorts above
// infinity, so integer maxima are the NaN-propagating maxima of |v| without
// any binary64 compare (binary64 runs at a small fraction of the binary32 rate).
__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7FFFFFFFFFFFFFFFull;
}

// max over the CTA of ordered bit patterns; every thread gets the result as a double
__device__ double block_max_bits(unsigned long long v, BSmem &sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    __syncthreads();
    if (lane == 0) sm.red[warp] = v;
    __syncthreads();
    unsigned long long m = sm.red[0];
#pragma unroll
    for (int w = 1; w < BW; ++w) m = sm.red[w] > m ? sm.red[w] : m;
    return __longlong_as_double(static_cast<long long>(m));
}

__device__ __forceinline__ void group_sync(int g) {
    asm volatile("bar.sync %0, 256;" ::"r"(1 + g) : "memory");
}

// ---------------------------------------------------------------------------
// panel: columns j0 .. j0+nbp-1 of W (rows j0..n-1).  Thread t keeps row
// j0 + t in a rotating register window for the whole panel; rows never move
// between threads.  Each thread tracks the row's current position (relative to
// j0), so an interchange is two integer compares, and the pivot search takes
// the largest |a_ik| with ties to the lowest current position (the first
// maximal entry, as in LAPACK's getf2).  A row that becomes the pivot row of
// step kp stops there; its U part is the staged copy of step kp.
// ---------------------------------------------------------------------------
__device__ void b_panel(float *W, int n, int ldw, int j0, int nbp, BSmem &sm, float *Ls, float *Us) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const bool valid = j0 + t < n;
    int pos = t;            // current position of this row, relative to j0
    int kp = nbp;           // the step at which it became the pivot row (nbp: never)
    float a[NB];
    {
        // 16-byte loads: j0 and ldw are multiples of 4, and a chunk that starts
        // before column n ends inside the padded row
        const float4 *src = reinterpret_cast<const float4 *>(W + (int64_t)(j0 + t) * ldw + j0);
#pragma unroll
        for (int q = 0; q < NB / 4; ++q) {
            const float4 v = (valid && 4 * q < nbp) ? src[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            a[4 * q + 0] = (4 * q + 0 < nbp) ? v.x : 0.f;
            a[4 * q + 1] = (4 * q + 1 < nbp) ? v.y : 0.f;
            a[4 * q + 2] = (4 * q + 2 < nbp) ? v.z : 0.f;
            a[4 * q + 3] = (4 * q + 3 < nbp) ? v.w : 0.f;
        }
    }
#pragma unroll 1
    for (int k = 0; k < nbp; ++k) {
        const int b = k & 1;
        const bool cand = valid && kp == nbp;
        const unsigned key = cand ? __float_as_uint(fabsf(a[0])) : 0u;
        const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
        const int mpos = __reduce_min_sync(0xffffffffu, (cand && key == kmax) ? pos : INT_MAX);
        if (cand && pos == mpos) {
            float *st = sm.stage[b][warp];
            st[3] = a[0];
#pragma unroll
            for (int q = 0; q < 15; ++q)
                *reinterpret_cast<float4 *>(st + 4 + 4 * q) =
                    make_float4(a[4 * q + 1], a[4 * q + 2], a[4 * q + 3], a[4 * q + 4]);
            st[64] = a[61];
            st[65] = a[62];
            st[66] = a[63];
            st[67] = 0.f;
            sm.sval[b][warp] = __uint_as_float(kmax);
            sm.spos[b][warp] = mpos;
            sm.srec[b][warp] = (a[0] != 0.f) ? 1.0f / a[0] : 0.f;
        }
        if (lane == 0 && mpos == INT_MAX) {
            sm.sval[b][warp] = 0.f;
            sm.spos[b][warp] = INT_MAX;
        }
        __syncthreads();
        // the pivot row: largest |value|, lowest position among equals
        const unsigned wk = lane < BW ? __float_as_uint(sm.sval[b][lane]) : 0u;
        const int wp = lane < BW ? sm.spos[b][lane] : INT_MAX;
        const unsigned bk = __reduce_max_sync(0xffffffffu, wk);
        const int ppos = __reduce_min_sync(0xffffffffu, (wp != INT_MAX && wk == bk) ? wp : INT_MAX);
        const unsigned who = __ballot_sync(0xffffffffu, lane < BW && wp == ppos);
        const int w = who ? __ffs(who) - 1 : 0;
        const float *u = sm.stage[b][w];          // u[3 + i] = pivot row, column j0 + k + i
        const float piv = u[3];
        const float r = sm.srec[b][w];
        if (t == 0 && piv == 0.f && sm.info == 0) sm.info = j0 + k + 1;
        // interchange positions k and ppos
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
        if (valid && kp == nbp) {
            // l = a * fl(1/pivot) (division when the pivot is subnormal): LAPACK getf2
            float l = a[0];
            if (piv != 0.f) l = (fabsf(piv) >= FLT_MIN) ? l * r : l / piv;
            Ls[k * BT + t] = l;
            const float4 *us = reinterpret_cast<const float4 *>(u + 4);
            const int live = nbp - k;
#pragma unroll
            for (int q = 0; q < NB / 4; ++q) {
                if (4 * q < live) {
                    const float4 ww = us[q];
                    a[4 * q + 0] = fmaf(-l, ww.x, a[4 * q + 1]);
                    a[4 * q + 1] = fmaf(-l, ww.y, a[4 * q + 2]);
                    a[4 * q + 2] = fmaf(-l, ww.z, a[4 * q + 3]);
                    a[4 * q + 3] = (q < NB / 4 - 1) ? fmaf(-l, ww.w, a[4 * q + 4]) : 0.f;
                }
            }
        }
    }
    // moved rows and the composed permutation
    if (t == 0) sm.moved_cnt = 0;
    __syncthreads();
    const bool moved = valid && pos != t;
    int porg = 0;
    if (moved) {
        const int e = atomicAdd(&sm.moved_cnt, 1);
        sm.moved_dst[e] = j0 + pos;
        sm.moved_src[e] = j0 + t;
        porg = sm.perm[j0 + t];
    }
    __syncthreads();
    if (moved) sm.perm[j0 + pos] = porg;
    // the row at its final position: multipliers of steps < kp, then the U part staged at step kp
    if (valid) {
        float4 *dst = reinterpret_cast<float4 *>(W + (int64_t)(j0 + pos) * ldw + j0);
#pragma unroll
        for (int q = 0; q < NB / 4; ++q) {
            if (4 * q < nbp) {
                float v[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = 4 * q + e;
                    v[e] = (c < kp) ? Ls[c * BT + t] : (c < nbp ? Us[kp * NB + (c - kp)] : 0.f);
                }
                dst[q] = make_float4(v[0], v[1], v[2], v[3]);
            }
        }
    }
    __syncthreads();
}

// The panel's row moves applied to the columns outside it (all sources read first).
__device__ void b_laswp(float *W, int n, int ldw, int j0, int nbp, BSmem &sm, float *stg) {
    const int t = threadIdx.x;
    const int cnt = sm.moved_cnt;
    if (cnt == 0) return;
    const int ncols = n - nbp;
    for (int c0 = 0; c0 < ncols; c0 += 256) {
        int c = c0 + (t & 255);
        const bool act = (t < 256) && c < ncols;
        if (c >= j0) c += nbp;
        if (act)
            for (int e = 0; e < cnt; ++e) stg[e * 256 + t] = W[(int64_t)sm.moved_src[e] * ldw + c];
        __syncthreads();
        if (act)
            for (int e = 0; e < cnt; ++e) W[(int64_t)sm.moved_dst[e] * ldw + c] = stg[e * 256 + t];
        __syncthreads();
    }
}

// U12 = L11^{-1} A12 for the block row j0..j0+63: one thread per column.
// Column-oriented (m outer) with each entry's fmaf chain in ascending m, the
// order in which the unblocked LU applies it.  Lt[m][k] = L11[k][m].
__device__ void b_trsm(float *W, int n, int ldw, int j0, float *Lt) {
    const int t = threadIdx.x;
    for (int e = t; e < NB * NB; e += BT) {
        const int k = e / NB, m = e % NB;
        Lt[m * kLd + k] = W[(int64_t)(j0 + k) * ldw + j0 + m];
    }
    __syncthreads();
    const int c = j0 + NB + t;
    if (c < n) {
        float u[NB];
        const float *src = W + (int64_t)j0 * ldw + c;
#pragma unroll
        for (int m = 0; m < NB; ++m) {
            u[m] = *src;
            src += ldw;
        }
        const float4 *L4 = reinterpret_cast<const float4 *>(Lt);
#pragma unroll
        for (int m = 0; m < NB - 1; ++m) {
#pragma unroll
            for (int k4 = (m + 1) & ~3; k4 < NB; k4 += 4) {
                const float4 l = L4[m * (kLd / 4) + k4 / 4];
                if (k4 + 0 > m) u[k4 + 0] = fmaf(-l.x, u[m], u[k4 + 0]);
                if (k4 + 1 > m) u[k4 + 1] = fmaf(-l.y, u[m], u[k4 + 1]);
                if (k4 + 2 > m) u[k4 + 2] = fmaf(-l.z, u[m], u[k4 + 2]);
                if (k4 + 3 > m) u[k4 + 3] = fmaf(-l.w, u[m], u[k4 + 3]);
            }
            asm volatile("" ::: "memory");    // keeps the L loads of later steps from piling up in registers
        }
        float *dst = W + (int64_t)(j0 + 1) * ldw + c;
#pragma unroll
        for (int m = 1; m < NB; ++m) {
            *dst = u[m];
            dst += ldw;
        }
    }
    __syncthreads();
}

// A22 -= L21 U12.  Two groups of 256 threads share the 64x64 tiles round-robin;
// thread (tr, tc) of a group owns rows 4tr..4tr+3 and columns 4tc..4tc+3.
__device__ void b_update(float *W, int n, int ldw, int j0, ir_dtype tf, float *smem) {
    const int t = threadIdx.x, g = t >> 8, u = t & 255;
    float *As = smem + g * 2 * NB * kLd;       // As[k][r] = rTF(L21[r][k])
    float *Bs = As + NB * kLd;                 // Bs[k][c] = rTF(U12[k][c])
    const int r0 = j0 + NB;
    const int tiles = (n - r0 + NB - 1) / NB;
    const int tr = u >> 4, tc = u & 15;
    const bool exact32 = (tf == IR_F32);
    int staged_ti = -1;
    for (int L = g; L < tiles * tiles; L += 2) {
        const int ti = L / tiles, tj = L % tiles;
        const int i0 = r0 + ti * NB, c0 = r0 + tj * NB;
        if (ti != staged_ti) {
            for (int e = u; e < NB * NB; e += 256) {
                const int rr = e >> 6, kk = e & 63, row = i0 + rr;
                As[kk * kLd + rr] = (row < n) ? round_tf(W[(int64_t)row * ldw + j0 + kk], tf) : 0.f;
            }
            staged_ti = ti;
        }
        for (int e = u; e < NB * NB; e += 256) {
            const int kk = e >> 6, cc = e & 63, col = c0 + cc;
            Bs[kk * kLd + cc] = (col < n) ? round_tf(W[(int64_t)(j0 + kk) * ldw + col], tf) : 0.f;
        }
        group_sync(g);
        const int ra = i0 + 4 * tr, ca = c0 + 4 * tc;
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                acc[i][q] = (exact32 && ra + i < n && ca + q < n) ? W[(int64_t)(ra + i) * ldw + ca + q] : 0.f;
        if (exact32) {
#pragma unroll 4
            for (int k = 0; k < NB; ++k) {
                const float4 av = *reinterpret_cast<const float4 *>(&As[k * kLd + 4 * tr]);
                const float4 bv = *reinterpret_cast<const float4 *>(&Bs[k * kLd + 4 * tc]);
                const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[i][q] = fmaf(-ar[i], br[q], acc[i][q]);
            }
        } else {
#pragma unroll 4
            for (int k = 0; k < NB; ++k) {
                const float4 av = *reinterpret_cast<const float4 *>(&As[k * kLd + 4 * tr]);
                const float4 bv = *reinterpret_cast<const float4 *>(&Bs[k * kLd + 4 * tc]);
                const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[i][q] = fmaf(ar[i], br[q], acc[i][q]);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = ra + i, col = ca + q;
                if (row < n && col < n) {
                    float *cp = W + (int64_t)row * ldw + col;
                    *cp = exact32 ? acc[i][q] : (*cp - acc[i][q]);
                }
            }
        group_sync(g);
    }
    __syncthreads();
}

// The forward solve with unit lower L in binary32: thread t holds v[t]
// (t < n) and returns its final value.  Column order as the reference BLAS
// trsv: every entry takes its updates v_i -= l_ij v_j in ascending j.
// Blocks of 32 columns: warp J first applies, for its own rows, the columns of
// block J - 1 (as every warp below does), then solves its diagonal block one
// column at a time with shuffles and publishes the 32 values; the row entries
// of the next block are loaded before the barrier so the wait hides them.
// Eight binary32 values rounded to TF (binary16 or bfloat16, nearest even) and
// packed as one 16-byte chunk, element 0 in the lowest half-word.
__device__ __forceinline__ uint4 pack8(const float *v, ir_dtype tf) {
    unsigned w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        if (tf == IR_BF16) {
            const __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * h], v[2 * h + 1]);
            w[h] = *reinterpret_cast<const unsigned *>(&p);
        } else {
            const __half2 p = __floats2half2_rn(v[2 * h], v[2 * h + 1]);
            w[h] = *reinterpret_cast<const unsigned *>(&p);
        }
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Bounded wait on an mbarrier phase (globaltimer limit); false when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned addr, unsigned parity) {
    if (mbar_try_wait(addr, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(addr, parity))
        if (globaltimer() - t0 > kWaitLimitNs) return false;
    return true;
}

// A22 -= rTF(L21) rTF(U12) on the tensor cores (TF = binary16 or bfloat16).
// Thread t stages row t of both operands: L21 row t and U12 column t, each
// 64 K values rounded to TF = 128 bytes, written K-major in the 128-byte
// swizzle (16-byte chunk q of row r at chunk q ^ (r & 7) of the row; eight
// rows make one 1024-byte atom), rows past the trailing block zero.  Output
// tiles of 128 x 128, four per wave in the 512 TMEM columns; one thread issues
// the 4 MMAs (K = 16 each) per tile and commits them to an mbarrier; then warp
// w reads TMEM lanes 32 (w % 4) .. + 31 of tile w / 4 and subtracts D from C.
// Returns false if a bounded wait gave up (the caller abandons the system).
__device__ bool b_update_tc(float *W, int n, int ldw, int j0, ir_dtype tf, unsigned char *big, BSmem &sm,
                            unsigned &mph) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int r0 = j0 + NB, m = n - r0;
    const int tiles = (m + 127) >> 7, pad = tiles << 7;
    unsigned char *gA = big, *gB = big + 64 * 1024;
    if (t < pad) {
        uint4 ca[8], cb[8];
        if (t < m) {
            const float4 *src = reinterpret_cast<const float4 *>(W + (int64_t)(r0 + t) * ldw + j0);
            float u[NB];
#pragma unroll
            for (int k = 0; k < NB; ++k) u[k] = W[(int64_t)(j0 + k) * ldw + r0 + t];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 x = src[2 * q], y = src[2 * q + 1];
                const float v[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
                ca[q] = pack8(v, tf);
                cb[q] = pack8(u + 8 * q, tf);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) ca[q] = cb[q] = make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            *reinterpret_cast<uint4 *>(gA + t * 128 + ((q ^ (t & 7)) << 4)) = ca[q];
            *reinterpret_cast<uint4 *>(gB + t * 128 + ((q ^ (t & 7)) << 4)) = cb[q];
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> MMA operand reads
    __syncthreads();
    const unsigned sA = smem_u32(gA), sB = smem_u32(gB), bar = smem_u32(&sm.mma_bar);
    const unsigned fmt = (tf == IR_BF16) ? 1u : 0u;
    const unsigned idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
    const int ntile = tiles * tiles;
    for (int w0 = 0; w0 < ntile; w0 += 4) {
        const int nw = (ntile - w0 < 4) ? ntile - w0 : 4;
        if (t == 0) {
            tc_fence_after();
            for (int a = 0; a < nw; ++a) {
                const int ti = (w0 + a) / tiles, tj = (w0 + a) % tiles;
#pragma unroll
                for (int kk = 0; kk < NB / 16; ++kk)
                    mma<false>(sm.tmem_base + (unsigned)(a * 128), make_desc(sA + ti * 16384 + kk * 32),
                               make_desc(sB + tj * 16384 + kk * 32), idesc, kk);
            }
            mma_commit(bar);
        }
        const bool ok = mbar_wait_bounded(bar, mph);
        mph ^= 1u;
        if (!__syncthreads_and(ok)) return false;
        tc_fence_after();
        const int a = warp >> 2, quarter = warp & 3;
        if (a < nw) {
            const int ti = (w0 + a) / tiles, tj = (w0 + a) % tiles;
            const int i = ti * 128 + quarter * 32 + lane;
#pragma unroll 1
            for (int h = 0; h < 4; ++h) {
                float v[32];
                tmem_ld32(sm.tmem_base + ((unsigned)(quarter * 32) << 16) + (unsigned)(a * 128 + h * 32), v);
                const int c0 = tj * 128 + h * 32;
                if (i < m) {
                    // 16-byte groups that start inside the block end inside the padded row
                    float4 *cp = reinterpret_cast<float4 *>(W + (int64_t)(r0 + i) * ldw + r0 + c0);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        if (c0 + 4 * q < m) {
                            float4 c = cp[q];
                            c.x -= v[4 * q];
                            c.y -= v[4 * q + 1];
                            c.z -= v[4 * q + 2];
                            c.w -= v[4 * q + 3];
                            cp[q] = c;
                        }
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    return true;
}

__device__ __forceinline__ void load_block(const float4 *row4, int c0, int n, bool on, float (&dst)[32]) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 v = (on && c0 + 4 * q < n) ? row4[(c0 >> 2) + q] : make_float4(0.f, 0.f, 0.f, 0.f);
        dst[4 * q] = v.x;
        dst[4 * q + 1] = v.y;
        dst[4 * q + 2] = v.z;
        dst[4 * q + 3] = v.w;
    }
}

__device__ float b_lower(const float *W, int n, int ldw, float vi, BSmem &sm) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const bool mine = t < n;
    const float4 *row4 = reinterpret_cast<const float4 *>(W + (int64_t)t * ldw);
    const int nblk = (n + 31) >> 5;
    float l[32], ln[32];
    load_block(row4, 0, n, mine, l);
    for (int J = 0; J < nblk; ++J) {
        const int c0 = J << 5, w = (n - c0 < 32) ? n - c0 : 32;
        load_block(row4, c0 + 32, n, mine && J + 1 < nblk && warp >= J + 1, ln);   // next block, in flight
        if (warp == J) {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                const float vj = __shfl_sync(0xffffffffu, vi, jj);
                if (mine && lane > jj && jj < w) vi = fmaf(-l[jj], vj, vi);
            }
            sm.vs[t] = vi;
        }
        __syncthreads();
        if (mine && warp > J) {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj)
                if (jj < w) vi = fmaf(-l[jj], sm.vs[c0 + jj], vi);
        }
#pragma unroll
        for (int q = 0; q < 32; ++q) l[q] = ln[q];
    }
    return vi;
}

// The back solve with U: the reference trsv column order, columns descending,
// each column's own entry divided by the diagonal before it is used; every
// entry takes its updates in descending j.  Blocks of 32 columns, last first.
__device__ float b_upper(const float *W, int n, int ldw, float vi, BSmem &sm) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const bool mine = t < n;
    const float4 *row4 = reinterpret_cast<const float4 *>(W + (int64_t)t * ldw);
    const int nblk = (n + 31) >> 5;
    float u[32], un[32];
    load_block(row4, (nblk - 1) << 5, n, mine && warp <= nblk - 1, u);
    for (int J = nblk - 1; J >= 0; --J) {
        const int c0 = J << 5, w = (n - c0 < 32) ? n - c0 : 32;
        load_block(row4, c0 - 32, n, mine && J >= 1 && warp <= J - 1, un);
        if (warp == J) {
#pragma unroll
            for (int jj = 31; jj >= 0; --jj) {
                if (jj < w) {
                    if (lane == jj) vi = vi / u[jj];
                    const float vj = __shfl_sync(0xffffffffu, vi, jj);
                    if (lane < jj) vi = fmaf(-u[jj], vj, vi);
                }
            }
            sm.vs[t] = vi;
        }
        __syncthreads();
        if (mine && warp < J) {
#pragma unroll
            for (int jj = 31; jj >= 0; --jj)
                if (jj < w) vi = fmaf(-u[jj], sm.vs[c0 + jj], vi);
        }
#pragma unroll
        for (int q = 0; q < 32; ++q) u[q] = un[q];
    }
    return vi;
}

template <typename TW>
__device__ void b_system(const BatchSys &S, float *W, const BatchCfg &cfg, ir_batch_result *res, BSmem &sm,
                         float *big, float *Us, bool use_tc, unsigned &mph) {
    const int t = threadIdx.x;
    const int n = S.n;
    const ir_dtype tf = cfg.tf;
    const int ldw = (n + 3) & ~3;
    const TW *A = static_cast<const TW *>(S.A);
    const TW *bv = static_cast<const TW *>(S.b);
    if (n == 0) {
        if (t == 0) {
            res->status = IR_CONVERGED;
            res->tf = cfg.tf;
            res->iters = 0;
            res->info = 0;
            res->nonfinite = 0;
            res->timeout = 0;
            res->rnorm = 0.0;
            res->scale = 1.0;
            res->bnorm = 0.0;
        }
        return;
    }
    if (t == 0) {
        sm.info = 0;
        sm.nonfinite = 0;
    }
    // s = 2^10 / max|a_ij| for binary16 (computed in binary64); thread t scans
    // row t with 16 loads in flight
    double s = 1.0;
    if (tf == IR_F16 && cfg.fp16_scale) {
        unsigned long long mloc = 0;
        if (t < n) {
            constexpr int R = 16;
            const TW *Ar = A + t;
            double cur[R], nxt[R];
#pragma unroll
            for (int q = 0; q < R; ++q) cur[q] = (q < n) ? (double)Ar[(int64_t)q * S.lda] : 0.0;
            for (int j0 = 0; j0 < n; j0 += R) {
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int j = j0 + R + q;
                    nxt[q] = (j < n) ? (double)Ar[(int64_t)j * S.lda] : 0.0;
                }
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const unsigned long long b = abs_bits(cur[q]);
                    mloc = b > mloc ? b : mloc;
                }
#pragma unroll
                for (int q = 0; q < R; ++q) cur[q] = nxt[q];
            }
        }
        const double mx = block_max_bits(mloc, sm);
        s = (mx > 0.0 && isfinite(mx)) ? 1024.0 / mx : 1.0;
    }
    // W = rTF(fl32(s a)): thread t converts row t.  A streams through shared
    // memory in blocks of 16 columns (8-byte cp.async, two blocks in flight);
    // each thread reads back only what it copied, so no barrier is needed.
    {
        constexpr int CB = 16;
        double *stg = reinterpret_cast<double *>(big);          // [2][CB][BT]
        const int nb = (n + CB - 1) / CB;
        const bool scaled = (s != 1.0);
        int bad = 0;
        auto issue = [&](int blk) {
            if (t < n && blk < nb) {
                const int j0 = blk * CB;
#pragma unroll
                for (int q = 0; q < CB; ++q) {
                    if (j0 + q < n) {
                        const unsigned dst = smem_u32(stg + ((blk & 1) * CB + q) * BT + t);
                        const TW *src = A + t + (int64_t)(j0 + q) * S.lda;
                        if (sizeof(TW) == 8)
                            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
                        else
                            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
                    }
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        issue(0);
        for (int blk = 0; blk < nb; ++blk) {
            issue(blk + 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
            if (t < n) {
                const int j0 = blk * CB;
                float f[CB];
#pragma unroll
                for (int q = 0; q < CB; ++q) {
                    double v = 0.0;
                    if (j0 + q < n) {
                        const double *e = stg + ((blk & 1) * CB + q) * BT + t;
                        v = (sizeof(TW) == 8) ? *e : (double)*reinterpret_cast<const float *>(e);
                    }
                    f[q] = round_tf(__double2float_rn(scaled ? s * v : v), tf);
                    bad |= (j0 + q < n) && !isfinite(f[q]);
                }
                float4 *dst = reinterpret_cast<float4 *>(W + (int64_t)t * ldw + j0);
#pragma unroll
                for (int q = 0; q < CB / 4; ++q)
                    if (j0 + 4 * q < n) dst[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        for (int k = t; k < n; k += BT) sm.perm[k] = k;
        if (__syncthreads_or(bad) && t == 0) sm.nonfinite = 1;
        __syncthreads();
    }
    // blocked LU with partial pivoting
    for (int j0 = 0; j0 < n; j0 += NB) {
        const int nbp = (n - j0 < NB) ? n - j0 : NB;
        b_panel(W, n, ldw, j0, nbp, sm, big, Us);
        b_laswp(W, n, ldw, j0, nbp, sm, big);
        if (j0 + nbp < n) {
            b_trsm(W, n, ldw, j0, big);
            if (use_tc && n - j0 - NB > cfg.tc_min_trail) {
                if (!b_update_tc(W, n, ldw, j0, tf, reinterpret_cast<unsigned char *>(big), sm, mph)) {
                    if (t == 0) {
                        sm.abort = 1;
                        res->status = IR_FAILED;
                        res->tf = cfg.tf;
                        res->iters = 0;
                        res->info = 0;
                        res->nonfinite = 0;
                        res->timeout = 1;
                        res->rnorm = 0.0;
                        res->scale = 1.0;
                        res->bnorm = 0.0;
                    }
                    __syncthreads();
                    return;
                }
            } else {
                b_update(W, n, ldw, j0, tf, big);
            }
        }
    }
    // x = 0, r = b, rhist[0] = ||b||
    unsigned long long bl = 0;
    int badb = 0;
    for (int i = t; i < n; i += BT) {
        const double v = (double)bv[i];
        const unsigned long long b = abs_bits(v);
        badb |= b >= 0x7FF0000000000000ull;
        sm.bs[i] = v;
        sm.rs[i] = v;
        sm.xs[i] = 0.0;
        bl = b > bl ? b : bl;
    }
    badb = __syncthreads_or(badb);
    const double bnorm = block_max_bits(bl, sm);
    const int info = sm.info;
    const int nonfinite = sm.nonfinite | badb;
    int status = -1, k = 0;
    if (nonfinite || info) status = IR_FAILED;
    else if (bnorm == 0.0) status = IR_CONVERGED;
    double rprev = bnorm, dprev = 0.0;
    while (status < 0) {
        // v = fl32(P r / rho), rho = ||r||_inf (eq. vdlow); d = rho s fl64(U^{-1} L^{-1} v) (eq. promotevd)
        const double rho = rprev;
        float vi = (t < n) ? __double2float_rn(sm.rs[sm.perm[t]] / rho) : 0.f;
        __syncthreads();
        vi = b_upper(W, n, ldw, b_lower(W, n, ldw, vi, sm), sm);
        unsigned long long dl = 0;
        if (t < n) {
            const double d = (rho * s) * (double)vi;
            sm.xs[t] += d;
            dl = abs_bits(d);
        }
        const double dn = block_max_bits(dl, sm);     // its barriers also publish xs
        // r = b - A x in binary64 (the fma chain of the oracle, ascending j)
        // (16 loads of the row in flight ahead of the chain: A streams from HBM)
        unsigned long long rl = 0;
        if (t < n) {
            constexpr int R = 16;
            const TW *Ar = A + t;
            const int64_t lda = S.lda;
            double cur[R], nxt[R];
#pragma unroll
            for (int q = 0; q < R; ++q) cur[q] = (q < n) ? (double)Ar[(int64_t)q * lda] : 0.0;
            double acc = 0.0;
            for (int j0 = 0; j0 < n; j0 += R) {
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int j = j0 + R + q;
                    nxt[q] = (j < n) ? (double)Ar[(int64_t)j * lda] : 0.0;
                }
#pragma unroll
                for (int q = 0; q < R; ++q)
                    if (j0 + q < n) acc = fma(cur[q], sm.xs[j0 + q], acc);
#pragma unroll
                for (int q = 0; q < R; ++q) cur[q] = nxt[q];
            }
            const double ri = sm.bs[t] - acc;
            sm.rs[t] = ri;
            rl = abs_bits(ri);
        }
        const double rn = block_max_bits(rl, sm);
        ++k;
        // termination (Sec. 5.1): the rule of the single-system path
        if (!isfinite(rn)) {
            status = IR_DIVERGED;
        } else if (rn == 0.0) {
            status = IR_CONVERGED;       // exact solution: r / ||r|| (eq. vdlow) is undefined next
        } else if (cfg.tr_wider) {
            if (k >= 2 && dn >= cfg.Rmax * dprev) status = IR_STAGNATED;     // eq. (wilkterm)
        } else {
            const double tol = cfg.abs_rel_tol > 0 ? cfg.abs_rel_tol : cfg.Cr * cfg.eps_w;
            if (rn <= tol * bnorm) status = IR_CONVERGED;                    // eq. (residterm)
            else if (rn >= cfg.Rmax * rprev) status = IR_STAGNATED;          // eq. (stag)
        }
        if (status < 0 && k >= cfg.litmax) status = IR_MAXIT;
        dprev = dn;
        rprev = rn;
    }
    if (status != IR_FAILED) {
        TW *xo = static_cast<TW *>(S.x);
        for (int i = t; i < n; i += BT) xo[i] = (TW)sm.xs[i];
    }
    if (t == 0) {
        res->status = status;
        res->tf = cfg.tf;
        res->iters = k;
        res->info = info;
        res->nonfinite = nonfinite;
        res->timeout = 0;
        res->rnorm = rprev;
        res->scale = s;
        res->bnorm = bnorm;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(BT, 1)
    k_batched(const BatchSys *sys, const int *order, const unsigned *dcount, unsigned *ticket, float *ws,
              int64_t ws_stride, BatchCfg cfg, ir_batch_result *results) {
    extern __shared__ __align__(16) unsigned char bsm[];
    const unsigned s0 = smem_u32(bsm);
    unsigned char *base = bsm + (((s0 + 1023u) & ~1023u) - s0);
    float *big = reinterpret_cast<float *>(base);                   // 1024-byte aligned
    float *Us = big + kBigFloats;
    BSmem &sm = *reinterpret_cast<BSmem *>(Us + NB * NB);
    float *W = ws + (int64_t)blockIdx.x * ws_stride;
    const bool use_tc = (cfg.tf == IR_F16 || cfg.tf == IR_BF16);
    const int count = dcount ? (int)*dcount : cfg.count;   // device count: the escalation pass
    if (threadIdx.x == 0) {
        sm.abort = 0;
        mbar_init(smem_u32(&sm.mma_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (use_tc && threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    unsigned mph = 0;
    for (;;) {
        if (threadIdx.x == 0) sm.cur = (int)atomicAdd(ticket, 1u);
        __syncthreads();
        const int idx = sm.cur;
        const int abort = sm.abort;
        __syncthreads();
        if (idx >= count || abort) break;
        const int id = order[idx];
        const BatchSys S = sys[id];
        if (cfg.tw == IR_F64)
            b_system<double>(S, W, cfg, results + id, sm, big, Us, use_tc, mph);
        else
            b_system<float>(S, W, cfg, results + id, sm, big, Us, use_tc, mph);
    }
    if (use_tc) {
        if (sm.abort) {
            // a wait gave up: let the tensor core finish what was issued (bounded) before freeing TMEM
            if (threadIdx.x == 0) mma_commit(smem_u32(&sm.mma_bar));
            mbar_wait_bounded(smem_u32(&sm.mma_bar), mph);
        }
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x < 32) {
            tc_fence_after();
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sm.tmem_base), "r"(kTmemCols)
                         : "memory");
        }
    }
}

// The members of order[0..count) to solve again, in the same (largest-first)
// order, into order2[0..*count2): one CTA, chunked block scan.  A member is
// kept when it converged, or stagnated / ran out of iterations with
// ||r|| <= rtol ||b||; every other one (failed, diverged, or stopped at a
// larger residual) is selected.
__global__ void __launch_bounds__(1024) k_select_unconverged(const ir_batch_result *results, const int *order,
                                                             int count, double rtol, int *order2,
                                                             unsigned *count2) {
    __shared__ int wsum[32];
    __shared__ int base;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < count; c0 += 1024) {
        const int idx = c0 + t;
        const int id = idx < count ? order[idx] : -1;
        int sel = 0;
        if (id >= 0) {
            const ir_batch_result &r = results[id];
            const bool small = (r.status == IR_STAGNATED || r.status == IR_MAXIT) && r.rnorm <= rtol * r.bnorm;
            sel = (r.status == IR_CONVERGED || small) ? 0 : 1;
        }
        const unsigned mask = __ballot_sync(0xffffffffu, sel);
        const int before = __popc(mask & ((1u << lane) - 1u));
        if (lane == 31) wsum[warp] = before + sel;
        __syncthreads();
        if (warp == 0) {
            const int v = wsum[lane];
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            wsum[lane] = incl - v;      // exclusive prefix of the warp totals
        }
        __syncthreads();
        if (sel) order2[base + wsum[warp] + before] = id;
        __syncthreads();
        if (t == 1023) base += wsum[31] + before + sel;
        __syncthreads();
    }
    if (t == 0) *count2 = (unsigned)base;
}

}  // namespace

cudaError_t launch_select_unconverged(const ir_batch_result *results, const int *order, int64_t count,
                                      double rtol, int *order2, unsigned *count2, cudaStream_t s) {
    count_launch();
    k_select_unconverged<<<1, 1024, 0, s>>>(results, order, (int)count, rtol, order2, count2);
    return cudaGetLastError();
}

size_t batch_desc_bytes() { return sizeof(BatchSys); }

void batch_fill_desc(void *desc, int64_t i, const void *A, int64_t lda, const void *b, void *x, int n) {
    BatchSys *d = static_cast<BatchSys *>(desc) + i;
    d->A = A;
    d->b = b;
    d->x = x;
    d->lda = lda;
    d->n = n;
    d->pad = 0;
}

cudaError_t batch_grid(int sms, int64_t count, int *grid) {
    cudaError_t e = cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched, BT, kBatchSmem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t g = (int64_t)sms * per_sm;
    *grid = (int)(count < g ? (count > 0 ? count : 1) : g);
    return cudaSuccess;
}

cudaError_t launch_batched(const void *sys, const int *order, int64_t count, unsigned *ticket, float *ws,
                           int64_t ws_stride, int grid, ir_dtype tw, ir_dtype tf, int fp16_scale, const ir_term *t,
                           int tc_min_trail, ir_batch_result *results, cudaStream_t s, const unsigned *dcount) {
    if (count <= 0) return cudaSuccess;
    BatchCfg c;
    c.Cr = t->Cr;
    c.Rmax = t->Rmax;
    c.abs_rel_tol = t->abs_rel_tol;
    c.eps_w = (tw == IR_F64) ? 2.220446049250313e-16 : 1.1920928955078125e-07;
    c.litmax = t->litmax;
    c.tr_wider = (tw == IR_F32) ? 1 : 0;
    c.fp16_scale = fp16_scale;
    c.count = (int)count;
    c.tw = tw;
    c.tf = tf;
    c.tc_min_trail = tc_min_trail;
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    count_launch();
    k_batched<<<grid, BT, kBatchSmem, s>>>(static_cast<const BatchSys *>(sys), order, dcount, ticket, ws, ws_stride,
                                           c, results);
    return cudaGetLastError();
}

}  // namespace ir
