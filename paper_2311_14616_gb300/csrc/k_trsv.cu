// Correction solve d = U^{-1} L^{-1} P v in binary32 (Algorithm IR; eqs.
// vdlow/promotevd of Sec. 5.3 for the scaling by ||r||).
//
// Blocked, synchronisation-free triangular solves: the rows are cut into
// blocks of B = 128; CTA b (taken in order through a ticket counter, so every
// block it waits on has already started) accumulates the products of its
// off-diagonal blocks with the solution blocks as they appear, then applies
// its diagonal block -- by the inverse computed once after the factorization,
// or by substitution (one warp, column sweep) when the block's condition
// number ||T|| ||T^{-1}|| exceeds kSubstKappa, where an explicit inverse would
// lose too much accuracy -- and publishes its 128 values.  The off-diagonal
// sums are compensated (see acc_pair).  A published value is a 64-bit word
// (epoch << 32 | binary32 bits), so a reader learns "ready" and the value in
// one load; waits are bounded and a timeout is reported, never hung.  The
// solve is a chain of N / B dependent block steps, so the block is large:
// 512 threads, warp w owns rows 8w .. 8w+7 of the block and lane l columns
// l, l+32, l+64, l+96 of every 128-column tile.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "ir_internal.cuh"

namespace ir {
namespace {

constexpr int B = kTrsvB;
constexpr int TT = 512;          // threads per solve CTA (16 warps x 8 rows)
constexpr int CPL = B / 32;      // columns of a tile per lane
static_assert(B == 128 && TT == 32 * (B / 8), "warp w owns rows 8w..8w+7 of the block");

// Inverse of the diagonal blocks: blockIdx.y = 0 -> L (unit lower), 1 -> U.
// The columns of X = T^{-1} are independent, so a cluster of kDiagCG CTAs
// shares a block, CTA q taking columns 32q .. 32q+31.  Right-looking, one step
// per row of the block: once row m of X is final, every row below (L) or above
// (U) takes its term -T[r][m] X[m][t].  Warp w owns the rows r = w mod 16 and
// lane l column 32q + l; one barrier per step, so the block's dependency chain
// is 128 short steps instead of one thread's 8k-long fmaf chain.  For L the
// terms of X[r][t] arrive in the order m = t, ..., r - 1 (the order of forward
// substitution); for U in the order m = t, ..., r + 1, and X[m][t] is divided
// by T[m][m] when row m becomes final.  Rows/columns beyond n are treated as
// identity.  The row sums of |X| for the condition number are summed over the
// cluster through distributed shared memory.
constexpr int kDiagCG = 4;                 // CTAs (column groups) per block
constexpr int kDiagC = B / kDiagCG;        // columns per CTA
constexpr int kDiagT = 512;
constexpr int kDiagRG = kDiagT / kDiagC;   // row groups (one per warp)
static_assert(kDiagC == 32 && kDiagRG == 16, "lane = column, warp = row group");
struct DiagSmem {
    float Tb[B][B + 1];
    float X[B][kDiagC + 1];
    float xr[B];                 // this CTA's part of the row sums of |X|
    float red[2][B / 32];
};
constexpr size_t kDiagSmem = sizeof(DiagSmem);
constexpr float kSubstKappa = 1e5f;   // blocks above this condition number are solved by substitution
__global__ void __launch_bounds__(kDiagT) k_diag_inv(const float *AF, int64_t ldf, int n, float *Linv,
                                                      float *Uinv, int32_t *blk_subst) {
    extern __shared__ __align__(16) unsigned char diag_smem[];
    DiagSmem &sm = *reinterpret_cast<DiagSmem *>(diag_smem);
    const int b = blockIdx.x, upper = blockIdx.y;
    const int q = (int)cluster_rank();
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int c0 = q * kDiagC, t = c0 + lane;    // this thread's column of the block
    const int r0 = b * B;
    for (int i = threadIdx.x >> 7; i < B; i += kDiagT / B) {
        const int c = threadIdx.x & (B - 1);
        const int gi = r0 + i, gc = r0 + c;
        float v;
        if (gi < n && gc < n) v = AF[(int64_t)gi * ldf + gc];
        else v = (i == c) ? 1.f : 0.f;
        sm.Tb[i][c] = v;
    }
    for (int i = g; i < B; i += kDiagRG) sm.X[i][lane] = (i == t) ? 1.f : 0.f;
    __syncthreads();
    if (!upper) {
#pragma unroll 1
        for (int m = c0; m < B - 1; ++m) {   // X[m][t] = 0 for t > m: steps m < c0 change nothing here
            if (t <= m) {
                const float xm = sm.X[m][lane];
#pragma unroll 2
                for (int r = m + 1 + ((g - (m + 1)) & (kDiagRG - 1)); r < B; r += kDiagRG)
                    sm.X[r][lane] = fmaf(-sm.Tb[r][m], xm, sm.X[r][lane]);
            }
            __syncthreads();
        }
    } else {
#pragma unroll 1
        for (int m = c0 + kDiagC - 1; m >= 0; --m) {   // rows m > c0 + 31 have no term in these columns
            float xm = 0.f;
            if (t >= m) xm = sm.X[m][lane] / sm.Tb[m][m];   // row m final (X[m][t] = 0 for t < m)
            __syncthreads();                                 // every warp has read the row
            if (t >= m) {
                if (g == (m & (kDiagRG - 1))) sm.X[m][lane] = xm;
#pragma unroll 2
                for (int r = g; r < m; r += kDiagRG) sm.X[r][lane] = fmaf(-sm.Tb[r][m], xm, sm.X[r][lane]);
            }
            __syncthreads();
        }
    }
    float *dst = (upper ? Uinv : Linv) + (int64_t)b * B * B;
    for (int i = g; i < B; i += kDiagRG) dst[i * B + t] = sm.X[i][lane];
    // kappa_inf of the triangle: max row sum of |T| times max row sum of |T^{-1}|
    if (threadIdx.x < B) {
        const int i = threadIdx.x;
        float xr = 0.f;
        for (int c = 0; c < kDiagC; ++c) xr += fabsf(sm.X[i][c]);
        sm.xr[i] = xr;
    }
    cluster_sync_all();   // every part of the row sums is in place
    if (q == 0 && threadIdx.x < B) {
        const int i = threadIdx.x;
        float tr = 0.f;
        for (int m = 0; m < B; ++m) {
            const float tv = upper ? (m >= i ? sm.Tb[i][m] : 0.f) : (m < i ? sm.Tb[i][m] : (m == i ? 1.f : 0.f));
            tr += fabsf(tv);
        }
        float xr = sm.xr[i];
        const unsigned a = smem_u32(&sm.xr[i]);
        for (int p = 1; p < kDiagCG; ++p) {
            float v;
            asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(map_cta(a, (unsigned)p)) : "memory");
            xr += v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tr = fmaxf(tr, __shfl_xor_sync(0xffffffffu, tr, o));
            xr = fmaxf(xr, __shfl_xor_sync(0xffffffffu, xr, o));
        }
        if ((i & 31) == 0) {
            sm.red[0][i >> 5] = tr;
            sm.red[1][i >> 5] = xr;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(B) : "memory");   // the 4 warps that hold the rows
        if (i == 0) {
            float tm = 0.f, xm = 0.f;
            for (int w = 0; w < B / 32; ++w) {
                tm = fmaxf(tm, sm.red[0][w]);
                xm = fmaxf(xm, sm.red[1][w]);
            }
            const float kappa = tm * xm;
            blk_subst[upper * gridDim.x + b] = !(kappa <= kSubstKappa);   // NaN: substitution too
        }
    }
    cluster_sync_all();   // no CTA leaves while its row sums may still be read
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Wait (bounded by limit_ns, with a short back-off) until the word carries `tag`;
// return its value.  On timeout: *timeout = 1 and 0 is returned.
__device__ __forceinline__ float poll_tagged(const unsigned long long *p, unsigned tag,
                                             int *timeout, unsigned long long limit_ns = kWaitLimitNs) {
    unsigned long long v = ld_relaxed_u64(p);
    if ((unsigned)(v >> 32) == tag) return __uint_as_float((unsigned)v);
    const unsigned long long t0 = globaltimer();
    unsigned ns = 16;
    while (true) {
        __nanosleep(ns);
        if (ns < 64) ns <<= 1;
        v = ld_relaxed_u64(p);
        if ((unsigned)(v >> 32) == tag) return __uint_as_float((unsigned)v);
        if (*reinterpret_cast<volatile int *>(timeout) || globaltimer() - t0 > limit_ns) {
            atomicExch(timeout, 1);
            return 0.f;
        }
    }
}

// The 128 published values of one block, read by one warp: the four words of
// a lane are loaded together, and only the ones not yet carrying `tag` are
// polled again (bounded, with a short back-off).
__device__ __forceinline__ void poll_block(const unsigned long long *p, unsigned tag, float *ys, int lane,
                                           int *timeout) {
    unsigned long long v[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) v[c] = ld_relaxed_u64(p + lane + 32 * c);
    bool ready = true;
#pragma unroll
    for (int c = 0; c < CPL; ++c) ready &= ((unsigned)(v[c] >> 32) == tag);
    if (!ready) {
#pragma unroll
        for (int c = 0; c < CPL; ++c)
            if ((unsigned)(v[c] >> 32) != tag)
                v[c] = ((unsigned long long)tag << 32) | __float_as_uint(poll_tagged(p + lane + 32 * c, tag, timeout));
    }
#pragma unroll
    for (int c = 0; c < CPL; ++c) ys[lane + 32 * c] = __uint_as_float((unsigned)v[c]);
}

// Sum of 8 per-lane values over the 32 lanes of a warp in 9 shuffles
// (recursive halving): lane l ends with the total of row q(l) =
// 4*bit4(l) + 2*bit3(l) + bit2(l).
__device__ __forceinline__ float reduce8(float (&v)[8], int lane) {
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
    float a[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float send = h16 ? v[q] : v[q + 4];
        const float keep = h16 ? v[q + 4] : v[q];
        a[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float b2[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const float send = h8 ? a[q] : a[q + 2];
        const float keep = h8 ? a[q + 2] : a[q];
        b2[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float c;
    {
        const float send = h4 ? b2[0] : b2[1];
        const float keep = h4 ? b2[1] : b2[0];
        c = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}
__device__ __forceinline__ int reduce8_row(int lane) {
    return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}

// Compensated (double-binary32) accumulation of the off-diagonal products.
// A triangular solve of an ill-conditioned factor cancels heavily, and a row
// sum rounded at every step relative to its partial magnitude would carry an
// error proportional to |sum| into the (much smaller) result.  Each lane adds
// the sum of its 4 products of a tile to a pair (hi, lo) with TwoSum (Knuth),
// the pairs of a row are reduced the same way, and the right-hand side is
// subtracted before the single final rounding.
// (The _rn intrinsics keep the compiler from contracting these steps into fmas.)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void acc_pair(float &hi, float &lo, float h2, float l2) {
    float s, e;
    two_sum(hi, h2, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, l2));
}

// reduce8 for (hi, lo) pairs: the same recursive halving, each addition compensated.
__device__ __forceinline__ void reduce8_pair(float (&h)[8], float (&l)[8], int lane, float &ho, float &lo_out) {
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
    float ah[4], al[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float sh = h16 ? h[q] : h[q + 4], sl = h16 ? l[q] : l[q + 4];
        ah[q] = h16 ? h[q + 4] : h[q];
        al[q] = h16 ? l[q + 4] : l[q];
        acc_pair(ah[q], al[q], __shfl_xor_sync(0xffffffffu, sh, 16), __shfl_xor_sync(0xffffffffu, sl, 16));
    }
    float bh[2], bl[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const float sh = h8 ? ah[q] : ah[q + 2], sl = h8 ? al[q] : al[q + 2];
        bh[q] = h8 ? ah[q + 2] : ah[q];
        bl[q] = h8 ? al[q + 2] : al[q];
        acc_pair(bh[q], bl[q], __shfl_xor_sync(0xffffffffu, sh, 8), __shfl_xor_sync(0xffffffffu, sl, 8));
    }
    float ch, cl;
    {
        const float sh = h4 ? bh[0] : bh[1], sl = h4 ? bl[0] : bl[1];
        ch = h4 ? bh[1] : bh[0];
        cl = h4 ? bl[1] : bl[0];
        acc_pair(ch, cl, __shfl_xor_sync(0xffffffffu, sh, 4), __shfl_xor_sync(0xffffffffu, sl, 4));
    }
    acc_pair(ch, cl, __shfl_xor_sync(0xffffffffu, ch, 2), __shfl_xor_sync(0xffffffffu, cl, 2));
    acc_pair(ch, cl, __shfl_xor_sync(0xffffffffu, ch, 1), __shfl_xor_sync(0xffffffffu, cl, 1));
    ho = ch;
    lo_out = cl;
}

// sv_i <- fl32(sv_i - (hi + lo)), the subtraction itself compensated.
__device__ __forceinline__ float sub_pair(float v, float hi, float lo) {
    float s, e;
    two_sum(v, -hi, s, e);
    return __fadd_rn(s, __fsub_rn(e, lo));
}

// Factor entries as binary32: the binary32 factors themselves, or the 2-byte
// copy kept in TF (binary16 / bfloat16), promoted exactly.
__device__ __forceinline__ float factor_value(const float *F, int64_t e) { return __ldg(F + e); }
__device__ __forceinline__ float factor_value(const __half *F, int64_t e) { return __half2float(__ldg(F + e)); }
__device__ __forceinline__ float factor_value(const __nv_bfloat16 *F, int64_t e) {
    return __bfloat162float(__ldg(F + e));
}

// One 128x128 off-diagonal tile slice: warp w rows 8w..8w+7, lane l columns
// l + 32c (c < 4) of block column bj.
template <typename T>
__device__ __forceinline__ void load_tile(const T *AF, int64_t ldf, int n, int row0, int bj,
                                          int lane, float (&a)[8][CPL]) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int i = row0 + q;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int col = bj * B + lane + 32 * c;
            a[q][c] = (i < n && col < n) ? factor_value(AF, (int64_t)i * ldf + col) : 0.f;
        }
    }
}

// Accumulate the off-diagonal products of block bi: (p[q], pl[q]) += sum_j
// A[row0+q][j] y_j over the predecessor blocks, in order (compensated); the
// next tile is in flight while the current one waits for its published values.
template <bool LOWER, typename T>
__device__ __forceinline__ void offdiag(const T *AF, int64_t ldf, int n, int nblk, int bi,
                                        const unsigned long long *tags, unsigned tag, float *ys,
                                        int *timeout, float (&p)[8], float (&pl)[8]) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int row0 = bi * B + warp * 8;
    const int npred = LOWER ? bi : (nblk - 1 - bi);
    float la[8][CPL], na[8][CPL];
    if (npred > 0) load_tile(AF, ldf, n, row0, LOWER ? 0 : nblk - 1, lane, la);
    for (int it = 0; it < npred; ++it) {
        const int bj = LOWER ? it : (nblk - 1 - it);
        if (it + 1 < npred) load_tile(AF, ldf, n, row0, LOWER ? bj + 1 : bj - 1, lane, na);
        if (warp == 0) poll_block(tags + bj * B, tag, ys, lane, timeout);
        __syncthreads();
        float y[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) y[c] = ys[lane + 32 * c];
        // the tile's 4 products of a lane in binary32, their sum added compensated
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float tp = __fmul_rn(la[q][0], y[0]);
#pragma unroll
            for (int c = 1; c < CPL; ++c) tp = fmaf(la[q][c], y[c], tp);
            acc_pair(p[q], pl[q], tp, 0.f);
        }
        __syncthreads();                       // ys consumed before the next fetch
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int c = 0; c < CPL; ++c) la[q][c] = na[q][c];
    }
}

// Rows 8w..8w+7 of the diagonal-block inverse times sv: lane l takes columns
// l + 32c; the 8 row sums end in lanes with (l & 3) == 0 (reduce8).
__device__ __forceinline__ float diag_apply(const float *Ds, const float *sv, int warp, int lane) {
    float acc[8];
    float s[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) s[c] = sv[lane + 32 * c];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        float a = 0.f;
#pragma unroll
        for (int c = 0; c < CPL; ++c) a = fmaf(Ds[(warp * 8 + q) * B + lane + 32 * c], s[c], a);
        acc[q] = a;
    }
    return reduce8(acc, lane);
}

// The diagonal block solved by substitution in place on sv (one warp, lane l
// rows l + 32r): Dt[j][i] = T[i][j] (row stride B + 1).  Lower: unit
// diagonal, columns ascending; upper: columns descending, each diagonal
// entry divided before its column is applied.
template <bool LOWER>
__device__ __forceinline__ void diag_subst(const float *Dt, float *sv, int lane) {
    float v[CPL];
#pragma unroll
    for (int r = 0; r < CPL; ++r) v[r] = sv[lane + 32 * r];
    // j = 32 jr + jl: jr is unrolled, so v[jr] stays a register
    if (LOWER) {
#pragma unroll
        for (int jr = 0; jr < CPL; ++jr) {
#pragma unroll 4
            for (int jl = 0; jl < 32; ++jl) {
                const int j = 32 * jr + jl;
                const float vj = __shfl_sync(0xffffffffu, v[jr], jl);
#pragma unroll
                for (int r = 0; r < CPL; ++r)
                    if (r >= jr && lane + 32 * r > j) v[r] = fmaf(-Dt[j * (B + 1) + lane + 32 * r], vj, v[r]);
            }
        }
    } else {
#pragma unroll
        for (int jr = CPL - 1; jr >= 0; --jr) {
#pragma unroll 4
            for (int jl = 31; jl >= 0; --jl) {
                const int j = 32 * jr + jl;
                if (lane == jl) v[jr] = v[jr] / Dt[j * (B + 1) + j];
                const float vj = __shfl_sync(0xffffffffu, v[jr], jl);
#pragma unroll
                for (int r = 0; r < CPL; ++r)
                    if (r <= jr && lane + 32 * r < j) v[r] = fmaf(-Dt[j * (B + 1) + lane + 32 * r], vj, v[r]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < CPL; ++r) sv[lane + 32 * r] = v[r];
}

// Shared-memory staging of the diagonal block: the inverse (row-major, B x B)
// or, for a block solved by substitution, the triangle transposed (stride
// B + 1; identity past row n).
template <bool LOWER>
__device__ __forceinline__ void stage_diag(const float *AF, int64_t ldf, int n, int r0, const float *inv,
                                           bool subst, float *Ds) {
    const int t = threadIdx.x;
    if (!subst) {
        const float4 *src = reinterpret_cast<const float4 *>(inv);
        for (int e = t; e < B * B / 4; e += TT) reinterpret_cast<float4 *>(Ds)[e] = __ldg(src + e);
    } else {
        for (int e = t; e < B * B; e += TT) {
            const int i = e / B, j = e % B, gi = r0 + i, gj = r0 + j;
            float v = (i == j) ? 1.f : 0.f;
            if (gi < n && gj < n && (LOWER ? j < i : j >= i)) v = __ldg(AF + (int64_t)gi * ldf + gj);
            Ds[j * (B + 1) + i] = v;
        }
    }
}

// mode 0 / 2: v = fl32(r[perm[i]] / rho), rho = *rho_bits (||r||; v = 0 when
// rho = 0); mode 1: v = vin[perm[i]].  Publishes tagged y for the upper solve.
template <typename T>
__global__ void __launch_bounds__(TT, 1) k_trsv_lower(const float *AF, const T *F, int64_t ldf, int n, int nblk,
                                                      const float *Linv, const int32_t *blk_subst,
                                                      const int32_t *perm, const double *r, const float *vin,
                                                      int mode, const unsigned long long *rho_bits,
                                                      const int *skip, unsigned long long *ytag, unsigned tag,
                                                      DevScalars *dev) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) float tsm[];
    float *Ds = tsm;                 // this block's diagonal inverse, or its transposed triangle
    float *sv = Ds + B * (B + 1);    // right-hand side of the block, then its solution
    float *ys = sv + B;              // published values of the predecessor being applied
    __shared__ int s_bi;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) s_bi = (int)atomicAdd(&dev->ticket[0], 1u);
    __syncthreads();
    const int bi = s_bi;
    const int r0 = bi * B;
    const bool subst = blk_subst[bi] != 0;
    stage_diag<true>(AF, ldf, n, r0, Linv + (int64_t)bi * B * B, subst, Ds);
    if (t < B) {
        const int i = r0 + t;
        float v = 0.f;
        if (i < n) {
            const int src = perm[i];
            if (mode != 1) {
                const double rn = __longlong_as_double((long long)*rho_bits);
                v = (rn == 0.0) ? 0.f : __double2float_rn(r[src] / rn);
            } else {
                v = vin[src];
            }
        }
        sv[t] = v;
    }
    float p[8], pl[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) p[q] = pl[q] = 0.f;
    offdiag<true>(F, ldf, n, nblk, bi, ytag, tag, ys, &dev->timeout, p, pl);
    __syncthreads();
    {
        float sh, sl;
        reduce8_pair(p, pl, lane, sh, sl);
        if ((lane & 3) == 0) {
            const int il = warp * 8 + reduce8_row(lane);
            sv[il] = sub_pair(sv[il], sh, sl);
        }
    }
    __syncthreads();
    if (subst) {
        if (warp == 0) diag_subst<true>(Ds, sv, lane);
    } else {
        const float y = diag_apply(Ds, sv, warp, lane);
        __syncthreads();
        if ((lane & 3) == 0) sv[warp * 8 + reduce8_row(lane)] = y;
    }
    __syncthreads();
    if (t < B) {
        const float yv = (r0 + t < n) ? sv[t] : 0.f;
        st_relaxed_u64(ytag + r0 + t, ((unsigned long long)tag << 32) | __float_as_uint(yv));
    }
}

// Back substitution with U, reading the tagged y of the lower solve.
// mode 0: d = (rho s) fl64(z); x += d; ||d||, ||x|| into dev; mode 1: dout = z;
// mode 2: x = (rho s) fl64(z).
template <typename T>
__global__ void __launch_bounds__(TT, 1) k_trsv_upper(const float *AF, const T *F, int64_t ldf, int n, int nblk,
                                                      const float *Uinv, const int32_t *blk_subst,
                                                      const unsigned long long *ytag,
                                                      unsigned long long *ztag, unsigned tag,
                                                      int mode, const unsigned long long *rho_bits,
                                                      const int *skip, double *x, float *dout,
                                                      DevScalars *dev) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) float tsm[];
    float *Ds = tsm;
    float *sv = Ds + B * (B + 1);
    float *ys = sv + B;
    __shared__ int s_bi;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) s_bi = nblk - 1 - (int)atomicAdd(&dev->ticket[1], 1u);
    __syncthreads();
    const int bi = s_bi;
    const int r0 = bi * B;
    const bool subst = blk_subst[nblk + bi] != 0;
    stage_diag<false>(AF, ldf, n, r0, Uinv + (int64_t)bi * B * B, subst, Ds);
    if (t < B) {
        // the lower solve of this launch sequence has written every y word already
        const int i = r0 + t;
        sv[t] = (i < n) ? __uint_as_float((unsigned)ld_relaxed_u64(ytag + i)) : 0.f;
    }
    float p[8], pl[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) p[q] = pl[q] = 0.f;
    offdiag<false>(F, ldf, n, nblk, bi, ztag, tag, ys, &dev->timeout, p, pl);
    __syncthreads();
    {
        float sh, sl;
        reduce8_pair(p, pl, lane, sh, sl);
        if ((lane & 3) == 0) {
            const int il = warp * 8 + reduce8_row(lane);
            sv[il] = sub_pair(sv[il], sh, sl);
        }
    }
    __syncthreads();
    if (subst) {
        if (warp == 0) diag_subst<false>(Ds, sv, lane);
    } else {
        const float z = diag_apply(Ds, sv, warp, lane);
        __syncthreads();
        if ((lane & 3) == 0) sv[warp * 8 + reduce8_row(lane)] = z;
    }
    __syncthreads();
    double dmax = 0.0, xmax = 0.0;
    if (t < B) {
        const int i = r0 + t;
        const float zv = (i < n) ? sv[t] : 0.f;
        st_relaxed_u64(ztag + i, ((unsigned long long)tag << 32) | __float_as_uint(zv));
        if (i < n) {
            if (mode != 1) {
                const double scale = __longlong_as_double((long long)*rho_bits) * dev->scale;
                const double d = scale * (double)zv;
                if (mode == 0) {
                    const double xn = x[i] + d;
                    x[i] = xn;
                    dmax = fabs(d);
                    xmax = fabs(xn);
                } else {
                    x[i] = d;
                }
            } else {
                dout[i] = zv;
            }
        }
    }
    if (mode == 0 && t < B) {
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

constexpr size_t kSolveSmem = sizeof(float) * (B * (B + 1) + 2 * B);

// ---- several right-hand sides at once ------------------------------------------
// The same blocked, synchronisation-free pair for K columns of right-hand
// sides: each factor tile is loaded once and applied to all K columns (per
// column the products, compensated sums, diagonal solves and the order of the
// blocks are those of k_trsv_lower / k_trsv_upper), so one block step of the
// chain serves K refinement loops.  Column j of the tagged words lives at
// tags + j * ntag.  active[j] = 0: column j takes v = 0 (d = 0, x unchanged).
constexpr int kRhs = 4;
constexpr size_t kMultiSmem = sizeof(float) * (B * (B + 1) + 2 * kRhs * B);

template <bool LOWER, typename T>
__device__ __forceinline__ void offdiag_multi(const T *F, int64_t ldf, int n, int nblk, int bi,
                                              const unsigned long long *tags, int64_t ntag, unsigned tag,
                                              float (*ys)[B], int *timeout, float (&p)[kRhs][8],
                                              float (&pl)[kRhs][8]) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int row0 = bi * B + warp * 8;
    const int npred = LOWER ? bi : (nblk - 1 - bi);
    float la[8][CPL], na[8][CPL];
    if (npred > 0) load_tile(F, ldf, n, row0, LOWER ? 0 : nblk - 1, lane, la);
    for (int it = 0; it < npred; ++it) {
        const int bj = LOWER ? it : (nblk - 1 - it);
        if (it + 1 < npred) load_tile(F, ldf, n, row0, LOWER ? bj + 1 : bj - 1, lane, na);
        if (warp < kRhs) poll_block(tags + warp * ntag + bj * B, tag, ys[warp], lane, timeout);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kRhs; ++j) {
            float y[CPL];
#pragma unroll
            for (int c = 0; c < CPL; ++c) y[c] = ys[j][lane + 32 * c];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float tp = __fmul_rn(la[q][0], y[0]);
#pragma unroll
                for (int c = 1; c < CPL; ++c) tp = fmaf(la[q][c], y[c], tp);
                acc_pair(p[j][q], pl[j][q], tp, 0.f);
            }
        }
        __syncthreads();                       // ys consumed before the next fetch
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int c = 0; c < CPL; ++c) la[q][c] = na[q][c];
    }
}

// sv[j] <- sv[j] - (off-diagonal sums of column j), then the diagonal block
// applied to every column (inverse, or substitution by warps 0 .. K-1).
template <bool LOWER>
__device__ __forceinline__ void finish_multi(const float *Ds, bool subst, float (*sv)[B], float (&p)[kRhs][8],
                                             float (&pl)[kRhs][8]) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int j = 0; j < kRhs; ++j) {
        float sh, sl;
        reduce8_pair(p[j], pl[j], lane, sh, sl);
        if ((lane & 3) == 0) {
            const int il = warp * 8 + reduce8_row(lane);
            sv[j][il] = sub_pair(sv[j][il], sh, sl);
        }
    }
    __syncthreads();
    if (subst) {
        if (warp < kRhs) diag_subst<LOWER>(Ds, sv[warp], lane);
    } else {
        float out[kRhs];
#pragma unroll
        for (int j = 0; j < kRhs; ++j) out[j] = diag_apply(Ds, sv[j], warp, lane);
        __syncthreads();
        if ((lane & 3) == 0)
#pragma unroll
            for (int j = 0; j < kRhs; ++j) sv[j][warp * 8 + reduce8_row(lane)] = out[j];
    }
    __syncthreads();
}

// v_ij = fl32(R[j][perm[i]] / rho_j) (0 when rho_j = 0 or column j inactive);
// publishes tagged y for the upper solve.
template <typename T>
__global__ void __launch_bounds__(TT, 1) k_mtrsv_lower(const float *AF, const T *F, int64_t ldf, int n, int nblk,
                                                       const float *Linv, const int32_t *blk_subst,
                                                       const int32_t *perm, const double *R, int64_t ldr,
                                                       const unsigned long long *rho_bits, const int *active,
                                                       unsigned long long *ytag, int64_t ntag, unsigned tag,
                                                       DevScalars *dev) {
    extern __shared__ __align__(16) float tsm[];
    float *Ds = tsm;
    float (*sv)[B] = reinterpret_cast<float (*)[B]>(Ds + B * (B + 1));
    float (*ys)[B] = sv + kRhs;
    __shared__ int s_bi;
    const int t = threadIdx.x;
    if (t == 0) s_bi = (int)atomicAdd(&dev->ticket[0], 1u);
    __syncthreads();
    const int bi = s_bi, r0 = bi * B;
    const bool subst = blk_subst[bi] != 0;
    stage_diag<true>(AF, ldf, n, r0, Linv + (int64_t)bi * B * B, subst, Ds);
    for (int e = t; e < kRhs * B; e += TT) {
        const int j = e / B, i = r0 + e % B;
        float v = 0.f;
        if (i < n && active[j]) {
            const double rn = __longlong_as_double((long long)rho_bits[j]);
            v = (rn == 0.0) ? 0.f : __double2float_rn(R[j * ldr + perm[i]] / rn);
        }
        sv[j][e % B] = v;
    }
    float p[kRhs][8], pl[kRhs][8];
#pragma unroll
    for (int j = 0; j < kRhs; ++j)
#pragma unroll
        for (int q = 0; q < 8; ++q) p[j][q] = pl[j][q] = 0.f;
    offdiag_multi<true>(F, ldf, n, nblk, bi, ytag, ntag, tag, ys, &dev->timeout, p, pl);
    __syncthreads();
    finish_multi<true>(Ds, subst, sv, p, pl);
    for (int e = t; e < kRhs * B; e += TT) {
        const int j = e / B, i = e % B;
        const float yv = (r0 + i < n) ? sv[j][i] : 0.f;
        st_relaxed_u64(ytag + j * ntag + r0 + i, ((unsigned long long)tag << 32) | __float_as_uint(yv));
    }
}

// z = U^{-1} y per column; d_ij = (rho_j s) fl64(z_ij), X[j][i] += d_ij for
// active columns; ||d_j||, ||x_j|| into dnorm_bits[j], xnorm_bits[j].
template <typename T>
__global__ void __launch_bounds__(TT, 1) k_mtrsv_upper(const float *AF, const T *F, int64_t ldf, int n, int nblk,
                                                       const float *Uinv, const int32_t *blk_subst,
                                                       const unsigned long long *ytag, unsigned long long *ztag,
                                                       int64_t ntag, unsigned tag,
                                                       const unsigned long long *rho_bits, const int *active,
                                                       double *X, int64_t ldx, unsigned long long *dnorm_bits,
                                                       unsigned long long *xnorm_bits, DevScalars *dev) {
    extern __shared__ __align__(16) float tsm[];
    float *Ds = tsm;
    float (*sv)[B] = reinterpret_cast<float (*)[B]>(Ds + B * (B + 1));
    float (*ys)[B] = sv + kRhs;
    __shared__ int s_bi;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) s_bi = nblk - 1 - (int)atomicAdd(&dev->ticket[1], 1u);
    __syncthreads();
    const int bi = s_bi, r0 = bi * B;
    const bool subst = blk_subst[nblk + bi] != 0;
    stage_diag<false>(AF, ldf, n, r0, Uinv + (int64_t)bi * B * B, subst, Ds);
    for (int e = t; e < kRhs * B; e += TT) {
        const int j = e / B, i = r0 + e % B;
        sv[j][e % B] = (i < n) ? __uint_as_float((unsigned)ld_relaxed_u64(ytag + j * ntag + i)) : 0.f;
    }
    float p[kRhs][8], pl[kRhs][8];
#pragma unroll
    for (int j = 0; j < kRhs; ++j)
#pragma unroll
        for (int q = 0; q < 8; ++q) p[j][q] = pl[j][q] = 0.f;
    offdiag_multi<false>(F, ldf, n, nblk, bi, ztag, ntag, tag, ys, &dev->timeout, p, pl);
    __syncthreads();
    finish_multi<false>(Ds, subst, sv, p, pl);
    // column j is handled by warps 4j .. 4j + 3 (128 rows, one per lane)
    const int j = warp >> 2, i = r0 + (warp & 3) * 32 + lane;
    const float zv = (i < n) ? sv[j][i - r0] : 0.f;
    st_relaxed_u64(ztag + j * ntag + i, ((unsigned long long)tag << 32) | __float_as_uint(zv));
    double dmax = 0.0, xmax = 0.0;
    if (i < n && active[j]) {
        const double scale = __longlong_as_double((long long)rho_bits[j]) * dev->scale;
        const double d = scale * (double)zv;
        const double xn = X[j * ldx + i] + d;
        X[j * ldx + i] = xn;
        dmax = fabs(d);
        xmax = fabs(xn);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
    }
    if (lane == 0 && active[j]) {
        atomic_max_nonneg(dnorm_bits + j, dmax);
        atomic_max_nonneg(xnorm_bits + j, xmax);
    }
}

// ---- the solve pair in one thread-block cluster ------------------------------
// For N <= 16 * 2 * B: CTA c of a cluster of C = min(16, nblk) CTAs owns the
// blocks c and c + C.  A finished block of y (lower solve) or z (upper solve)
// is pushed to every CTA of the cluster with st.async (32 chunks of 16 bytes
// per destination, one thread each), counted on that block's mbarrier in the
// receiving CTA, so a block step costs one on-chip transfer instead of a round
// trip through global memory, and y never leaves the cluster.  The 128 x 128
// factor tiles a CTA applies are streamed by TMA (one cp.async.bulk.tensor per
// tile) through a two-deep ring in shared memory, in the order the CTA
// applies them (lower: block step ascending, own blocks ascending; upper:
// descending), so two tiles are always in flight while the CTA waits.  For
// each of its blocks a CTA applies the tiles in the same order, with the same
// per-lane products, compensated sums and diagonal solves as k_trsv_lower /
// k_trsv_upper, so the results are the same bits.
constexpr int kClCtas = 16;
constexpr int kClOwn = 2;
constexpr int kClMaxBlk = kClCtas * kClOwn;
constexpr unsigned kTileBytes = B * B * 4;
struct ClSmem {
    alignas(16) float ybuf[kClMaxBlk][B];          // every block of y, as pushed
    alignas(16) float zbuf[kClMaxBlk][B];          // every block of z
    alignas(16) float rhs[kClOwn][B];              // this CTA's right-hand sides (lower)
    alignas(16) float sv[B];                       // the block being finished
    alignas(8) unsigned long long bar[2][kClMaxBlk];
    alignas(8) unsigned long long full[2];         // the tile ring: copy landed
    alignas(8) unsigned long long dsbar;           // the diagonal inverse copy landed
    int abort;
};
// ring (2 tiles, 128-byte aligned) | ClSmem | Ds
constexpr size_t kClSmem = 128 + 2 * (size_t)kTileBytes + sizeof(ClSmem) + sizeof(float) * B * (B + 1);

__device__ __forceinline__ void cl_tma_tile(unsigned dst, const CUtensorMap *map, int bj, int bi, unsigned mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bj * B), "r"(bi * B), "r"(mbar)
        : "memory");
}

// Wait for the phase `parity` of barrier `bar`: one thread spins, bounded by
// the launch's deadline, then the CTA meets at a barrier.  A wait that gives up
// flags the solve as abandoned and returns anyway, so every warp keeps the same
// control flow (after the deadline every wait returns at once; the results are
// then garbage and the timeout is reported).
__device__ __forceinline__ void cta_wait(ClSmem &sm, unsigned bar, unsigned parity, unsigned long long deadline,
                                         int *timeout) {
    if (threadIdx.x == 0) {
        while (!mbar_try_wait_cluster(bar, parity)) {
            if (globaltimer() > deadline) {
                if (!sm.abort) {
                    sm.abort = 1;
                    atomicExch(timeout, 1);
                }
                break;
            }
        }
    }
    __syncthreads();
}

// Copy a block's diagonal inverse (B x B binary32, contiguous) into Ds with one
// bulk asynchronous copy counted on sm.dsbar (issued by thread 0).
__device__ __forceinline__ void ds_copy(ClSmem &sm, float *Ds, const float *src) {
    if (threadIdx.x == 0) {
        const unsigned bar = smem_u32(&sm.dsbar);
        mbar_expect_arrive(bar, B * B * 4);
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(Ds)),
                     "l"(src), "r"(B * B * 4), "r"(bar)
                     : "memory");
    }
}

// Push sv (B values) into buf[bj] of every CTA of the cluster.
__device__ __forceinline__ void cl_push(ClSmem &sm, float (*buf)[B], int ph, int bj, unsigned C) {
    const int t = threadIdx.x;
    if (t < 32 * (int)C) {
        const int dst = t >> 5, ch = t & 31;
        const float4 v = reinterpret_cast<const float4 *>(sm.sv)[ch];
        st_async_v4(map_cta(smem_u32(&buf[bj][4 * ch]), (unsigned)dst), v,
                    map_cta(smem_u32(&sm.bar[ph][bj]), (unsigned)dst));
    }
}

// (p, pl) += tile . y, the tile in shared memory (row-major B x B): the
// per-lane products of offdiag, compensated.
__device__ __forceinline__ void cl_apply(const float *tile, const float *yb, int lane, int warp, float (&p)[8],
                                         float (&pl)[8]) {
    float y[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) y[c] = yb[lane + 32 * c];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float *row = tile + (warp * 8 + q) * B + lane;
        float tp = __fmul_rn(row[0], y[0]);
#pragma unroll
        for (int c = 1; c < CPL; ++c) tp = fmaf(row[32 * c], y[c], tp);
        acc_pair(p[q], pl[q], tp, 0.f);
    }
}

// sv <- rhs - sum (compensated), then the diagonal block (inverse or substitution).
template <bool LOWER>
__device__ __forceinline__ void cl_finish(ClSmem &sm, const float *Ds, bool subst, const float (&p)[8],
                                          const float (&pl)[8]) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    float pp[8], ppl[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        pp[q] = p[q];
        ppl[q] = pl[q];
    }
    __syncthreads();                     // sv holds the right-hand side
    {
        float sh, sl;
        reduce8_pair(pp, ppl, lane, sh, sl);
        if ((lane & 3) == 0) {
            const int il = warp * 8 + reduce8_row(lane);
            sm.sv[il] = sub_pair(sm.sv[il], sh, sl);
        }
    }
    __syncthreads();
    if (subst) {
        if (warp == 0) diag_subst<LOWER>(Ds, sm.sv, lane);
    } else {
        const float y = diag_apply(Ds, sm.sv, warp, lane);
        __syncthreads();
        if ((lane & 3) == 0) sm.sv[warp * 8 + reduce8_row(lane)] = y;
    }
    __syncthreads();
}

// Outputs of a finished z block (sv): mode 0 x += (rho s) z with the maxima of
// |d| and |x|; mode 1 dout = z; mode 2 x = (rho s) z.
__device__ __forceinline__ void cl_out(const float *sv, int r0, int n, int mode, double scale, double *x,
                                       float *dout, double &dmax, double &xmax) {
    const int t = threadIdx.x;
    const int i = r0 + t;
    if (t >= B || i >= n) return;
    const float zv = sv[t];
    if (mode == 1) {
        dout[i] = zv;
        return;
    }
    const double d = scale * (double)zv;
    if (mode == 0) {
        const double xn = x[i] + d;
        x[i] = xn;
        dmax = fmax(dmax, fabs(d));
        xmax = fmax(xmax, fabs(xn));
    } else {
        x[i] = d;
    }
}

#define OWN(o) ((int)c + (o) * (int)C)
// The tile sequence of a CTA: phase 0 (lower) tiles (OWN(o), bj) for bj
// ascending and o ascending with OWN(o) > bj; phase 1 (upper) tiles for bj
// descending and o descending with OWN(o) < bj; phase 2: none left.
struct TileSeq {
    int ph, o, bj;
};
__device__ __forceinline__ void seq_first_upper(TileSeq &q, int c, int C, int nown, int nblk) {
    q.ph = 1;
    q.bj = nblk - 1;
    q.o = (nown > 1 && OWN(1) < q.bj) ? 1 : ((OWN(0) < q.bj) ? 0 : -1);
    if (q.o < 0) q.ph = 2;
}
__device__ __forceinline__ void seq_first(TileSeq &q, int c, int C, int nown, int nblk) {
    q.ph = 0;
    q.bj = 0;
    q.o = (OWN(0) > 0) ? 0 : ((nown > 1 && OWN(1) > 0) ? 1 : -1);
    if (q.o < 0) seq_first_upper(q, c, C, nown, nblk);
}
__device__ __forceinline__ void seq_next(TileSeq &q, int c, int C, int nown, int nblk) {
    if (q.ph == 0) {
        if (q.o == 0 && nown > 1 && OWN(1) > q.bj) {
            q.o = 1;
            return;
        }
        q.bj += 1;
        q.o = (OWN(0) > q.bj) ? 0 : ((nown > 1 && OWN(1) > q.bj) ? 1 : -1);
        if (q.o < 0) seq_first_upper(q, c, C, nown, nblk);
    } else if (q.ph == 1) {
        if (q.o == 1 && OWN(0) < q.bj) {
            q.o = 0;
            return;
        }
        q.bj -= 1;
        q.o = (nown > 1 && OWN(1) < q.bj) ? 1 : ((OWN(0) < q.bj) ? 0 : -1);
        if (q.o < 0) q.ph = 2;
    }
}

__global__ void __launch_bounds__(TT, 1) k_trsv_cluster(const __grid_constant__ CUtensorMap tmAF, int64_t ldf, int n,
                                                        int nblk, const float *AF, const float *Linv,
                                                        const float *Uinv, const int32_t *blk_subst,
                                                        const int32_t *perm, const double *r, const float *vin,
                                                        int mode, const unsigned long long *rho_bits,
                                                        const int *skip, double *x, float *dout, DevScalars *dev) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char cl_smem[];
    const unsigned s0 = smem_u32(cl_smem);
    unsigned char *base = cl_smem + (((s0 + 127u) & ~127u) - s0);
    float *ring = reinterpret_cast<float *>(base);                                  // [2][B * B]
    ClSmem &sm = *reinterpret_cast<ClSmem *>(base + 2 * (size_t)kTileBytes);
    float *Ds = reinterpret_cast<float *>(base + 2 * (size_t)kTileBytes + sizeof(ClSmem));
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int C = (int)cluster_size(), c = (int)cluster_rank();
    const int nown = (OWN(1) < nblk) ? 2 : 1;
    if (t == 0) {
        sm.abort = 0;
        for (int b = 0; b < nblk; ++b) {
            mbar_init_p(smem_u32(&sm.bar[0][b]), 1);
            mbar_init_p(smem_u32(&sm.bar[1][b]), 1);
        }
        mbar_init_p(smem_u32(&sm.full[0]), 1);
        mbar_init_p(smem_u32(&sm.full[1]), 1);
        mbar_init_p(smem_u32(&sm.dsbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int b = 0; b < nblk; ++b) {
            mbar_expect_arrive(smem_u32(&sm.bar[0][b]), B * 4);
            mbar_expect_arrive(smem_u32(&sm.bar[1][b]), B * 4);
        }
    }
    // right-hand sides of this CTA's blocks: fl32(r[perm_i] / ||r||) (mode 0, 2) or vin[perm_i]
    if (t < B) {
        const double rn = (mode != 1) ? __longlong_as_double((long long)*rho_bits) : 1.0;
#pragma unroll
        for (int o = 0; o < kClOwn; ++o) {
            float v = 0.f;
            const int i = OWN(o) * B + t;
            if (o < nown && i < n) {
                const int src = perm[i];
                v = (mode != 1) ? ((rn == 0.0) ? 0.f : __double2float_rn(r[src] / rn)) : vin[src];
            }
            sm.rhs[o][t] = v;
        }
    }
    cluster_sync_all();     // every barrier of the cluster is armed before anything is pushed
    const unsigned long long deadline = globaltimer() + kWaitLimitNs;
    // the producer (thread 0) keeps two tiles of the sequence in flight
    TileSeq pq;
    int issued = 0, used = 0;
    seq_first(pq, c, C, nown, nblk);
    if (t == 0) {
        for (int k = 0; k < 2 && pq.ph < 2; ++k) {
            const unsigned fb = smem_u32(&sm.full[k]);
            mbar_expect_arrive(fb, kTileBytes);
            cl_tma_tile(smem_u32(ring + (size_t)k * B * B), &tmAF, pq.bj, OWN(pq.o), fb);
            seq_next(pq, c, C, nown, nblk);
            ++issued;
        }
    }
    // the next tile of the sequence, in shared memory
    auto tile_ready = [&]() -> const float * {
        const int k = used;
        cta_wait(sm, smem_u32(&sm.full[k & 1]), (unsigned)((k >> 1) & 1), deadline, &dev->timeout);
        return ring + (size_t)(k & 1) * B * B;
    };
    // the tile is consumed: its buffer takes the tile two ahead
    auto tile_done = [&]() {
        __syncthreads();
        const int k = used;
        if (t == 0 && pq.ph < 2) {
            const unsigned fb = smem_u32(&sm.full[k & 1]);
            mbar_expect_arrive(fb, kTileBytes);
            cl_tma_tile(smem_u32(ring + (size_t)(k & 1) * B * B), &tmAF, pq.bj, OWN(pq.o), fb);
            seq_next(pq, c, C, nown, nblk);
            ++issued;
        }
        ++used;
    };
    // the diagonal block of block bi in Ds: its inverse by a bulk copy (waited for
    // in ds_ready), or its transposed triangle for a block solved by substitution
    int ds_async = 0, ds_k = 0;
    auto ds_stage = [&](bool lower, int bi) {
        const bool subst = blk_subst[(lower ? 0 : nblk) + bi] != 0;
        if (subst) {
            if (lower)
                stage_diag<true>(AF, ldf, n, bi * B, nullptr, true, Ds);
            else
                stage_diag<false>(AF, ldf, n, bi * B, nullptr, true, Ds);
            ds_async = 0;
        } else {
            ds_copy(sm, Ds, (lower ? Linv : Uinv) + (int64_t)bi * B * B);
            ds_async = 1;
        }
    };
    auto ds_ready = [&]() {
        if (ds_async) {
            cta_wait(sm, smem_u32(&sm.dsbar), (unsigned)(ds_k & 1), deadline, &dev->timeout);
            ++ds_k;
            ds_async = 0;
        }
    };
    float p[kClOwn][8], pl[kClOwn][8];

    // ---------------- lower: y = L^{-1} v, blocks ascending ----------------
#pragma unroll
    for (int o = 0; o < kClOwn; ++o)
#pragma unroll
        for (int q = 0; q < 8; ++q) p[o][q] = pl[o][q] = 0.f;
    ds_stage(true, OWN(0));
    if (OWN(0) == 0) {                      // block 0 has no predecessors
        if (t < B) sm.sv[t] = sm.rhs[0][t];
        ds_ready();
        cl_finish<true>(sm, Ds, blk_subst[0] != 0, p[0], pl[0]);
        cl_push(sm, sm.ybuf, 0, 0, C);
        if (nown > 1) {
            __syncthreads();
            ds_stage(true, OWN(1));
        }
    }
    for (int bj = 0; bj + 1 < nblk; ++bj) {
        if (OWN(nown - 1) <= bj) break;               // nothing of this CTA below bj
        cta_wait(sm, smem_u32(&sm.bar[0][bj]), 0u, deadline, &dev->timeout);
        const float *yb = sm.ybuf[bj];
#pragma unroll
        for (int o = 0; o < kClOwn; ++o) {
            if (o >= nown || OWN(o) <= bj) continue;
            const float *tile = tile_ready();
            cl_apply(tile, yb, lane, warp, p[o], pl[o]);
            tile_done();
            if (OWN(o) == bj + 1) {                   // the chain: finish and push
                if (t < B) sm.sv[t] = sm.rhs[o][t];
                ds_ready();
                cl_finish<true>(sm, Ds, blk_subst[OWN(o)] != 0, p[o], pl[o]);
                cl_push(sm, sm.ybuf, 0, OWN(o), C);
                if (o + 1 < nown) {
                    __syncthreads();
                    ds_stage(true, OWN(o + 1));
                }
            }
        }
    }

    // ---------------- upper: z = U^{-1} y, blocks descending ----------------
    const double scale = (mode != 1) ? __longlong_as_double((long long)*rho_bits) * dev->scale : 1.0;
    double dmax = 0.0, xmax = 0.0;
    {
        const int hi = nown - 1;
#pragma unroll
        for (int o = 0; o < kClOwn; ++o)
#pragma unroll
            for (int q = 0; q < 8; ++q) p[o][q] = pl[o][q] = 0.f;
        __syncthreads();
        ds_stage(false, OWN(hi));
        // the y blocks of this CTA: the lower solve pushed them here too
        cta_wait(sm, smem_u32(&sm.bar[0][OWN(hi)]), 0u, deadline, &dev->timeout);
        if (OWN(hi) == nblk - 1) {
            if (t < B) sm.sv[t] = sm.ybuf[OWN(hi)][t];       // the last block has no successors
            ds_ready();
            if (hi == 1)      // (static indices keep the partial sums in registers)
                cl_finish<false>(sm, Ds, blk_subst[nblk + OWN(1)] != 0, p[1], pl[1]);
            else
                cl_finish<false>(sm, Ds, blk_subst[nblk + OWN(0)] != 0, p[0], pl[0]);
            cl_push(sm, sm.zbuf, 1, OWN(hi), C);
            cl_out(sm.sv, OWN(hi) * B, n, mode, scale, x, dout, dmax, xmax);
            if (hi > 0) {
                __syncthreads();
                ds_stage(false, OWN(0));
            }
        }
        for (int bj = nblk - 1; bj > 0; --bj) {
            if (OWN(0) >= bj) break;                 // nothing of this CTA above bj
            cta_wait(sm, smem_u32(&sm.bar[1][bj]), 0u, deadline, &dev->timeout);
            const float *zb = sm.zbuf[bj];
#pragma unroll
            for (int oo = 0; oo < kClOwn; ++oo) {
                const int o = kClOwn - 1 - oo;      // the higher block first
                if (o >= nown || OWN(o) >= bj) continue;
                const float *tile = tile_ready();
                cl_apply(tile, zb, lane, warp, p[o], pl[o]);
                tile_done();
                if (OWN(o) == bj - 1) {
                    cta_wait(sm, smem_u32(&sm.bar[0][OWN(o)]), 0u, deadline, &dev->timeout);
                    if (t < B) sm.sv[t] = sm.ybuf[OWN(o)][t];
                    ds_ready();
                    cl_finish<false>(sm, Ds, blk_subst[nblk + OWN(o)] != 0, p[o], pl[o]);
                    cl_push(sm, sm.zbuf, 1, OWN(o), C);
                    cl_out(sm.sv, OWN(o) * B, n, mode, scale, x, dout, dmax, xmax);
                    if (o > 0) {
                        __syncthreads();
                        ds_stage(false, OWN(o - 1));
                    }
                }
            }
        }
    }
    if (mode == 0 && t < B) {
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
    // Every push into this CTA and every tile copy it issued has landed
    // (bounded), then nobody leaves before the others.
    if (t == 0) {
        if (ds_async)                            // (only after an abandoned solve)
            while (!mbar_try_wait_cluster(smem_u32(&sm.dsbar), (unsigned)(ds_k & 1)))
                if (globaltimer() > deadline + kWaitLimitNs) break;
        for (int k = used; k < issued; ++k)      // (only after an abandoned solve)
            while (!mbar_try_wait_cluster(smem_u32(&sm.full[k & 1]), (unsigned)((k >> 1) & 1)))
                if (globaltimer() > deadline + kWaitLimitNs) break;
        if (!sm.abort) {
            for (int b = 0; b < nblk; ++b)
                for (int ph = 0; ph < 2; ++ph)
                    while (!mbar_try_wait_cluster(smem_u32(&sm.bar[ph][b]), 0u))
                        if (globaltimer() > deadline) {
                            atomicExch(&dev->timeout, 1);
                            break;
                        }
        }
    }
    __syncthreads();
    cluster_sync_all();
}
#undef OWN

// The correction solves' tag wait on a word that never receives `tag` (one
// thread): it must give up after limit_ns and raise *timeout.
__global__ void k_wait_probe(const unsigned long long *tags, unsigned tag, unsigned long long limit_ns,
                             int *timeout) {
    if (threadIdx.x == 0 && blockIdx.x == 0) (void)poll_tagged(tags, tag, timeout, limit_ns);
}

}  // namespace

cudaError_t launch_diag_inv(const float *AF, int64_t ldf, int n, float *Linv, float *Uinv,
                            int32_t *blk_subst, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_diag_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDiagSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int nblk = (n + B - 1) / B;
    count_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblk, 2, kDiagCG);
    cfg.blockDim = dim3(kDiagT, 1, 1);
    cfg.dynamicSmemBytes = kDiagSmem;
    cfg.stream = s;
    cudaLaunchAttribute cl[1];
    cl[0].id = cudaLaunchAttributeClusterDimension;
    cl[0].val.clusterDim.x = 1;
    cl[0].val.clusterDim.y = 1;
    cl[0].val.clusterDim.z = kDiagCG;
    cfg.attrs = cl;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_diag_inv, AF, ldf, n, Linv, Uinv, blk_subst);
}

static bool cluster_solve_enabled() {
    const char *e = getenv("IR_NO_CLUSTER_SOLVE");
    return !(e && e[0] && e[0] != '0');
}

// ytag/ztag: 2 arrays of nblk*B tagged words (flags buffer).  Tickets are reset here.
cudaError_t launch_wait_probe(const unsigned long long *tags, unsigned tag, unsigned long long limit_ns,
                              int *timeout, cudaStream_t s) {
    count_launch();
    k_wait_probe<<<1, 32, 0, s>>>(tags, tag, limit_ns, timeout);
    return cudaGetLastError();
}

cudaError_t launch_trsv_pair(const float *AF, int64_t ldf, int n, const float *Linv,
                             const float *Uinv, const int32_t *blk_subst, const int32_t *perm, const double *r,
                             const float *vin, float *dout, double *x,
                             unsigned long long *tags, unsigned epoch, DevScalars *dev,
                             cudaStream_t s, const unsigned long long *rho_bits, double *pw,
                             const int *skip, bool unit_rho, const void *F16, ir_dtype tf16) {
    if (n == 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaSuccess;
        const void *kerns[6] = {(const void *)k_trsv_lower<float>, (const void *)k_trsv_upper<float>,
                                (const void *)k_trsv_lower<__half>, (const void *)k_trsv_upper<__half>,
                                (const void *)k_trsv_lower<__nv_bfloat16>, (const void *)k_trsv_upper<__nv_bfloat16>};
        for (int q = 0; q < 6 && e == cudaSuccess; ++q)
            e = cudaFuncSetAttribute(kerns[q], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSolveSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int nblk = (n + B - 1) / B;
    cudaError_t e = cudaSuccess;
    const int mode = vin ? 1 : (pw ? 2 : 0);
    if (mode != 2) rho_bits = unit_rho ? &dev->one_bits : &dev->rnorm_bits;
    double *xo = (mode == 2) ? pw : x;
    if (!F16 && nblk <= kClMaxBlk && cluster_solve_enabled()) {
        static bool cattr = false;
        if (!cattr) {
            e = cudaFuncSetAttribute(k_trsv_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClSmem);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_trsv_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
            cattr = true;
        }
        // the factors as a 2-D tensor (n x n, row stride ldf), 128 x 128 boxes, zero fill past n
        CUtensorMap tm;
        TensorMapEncodeFn enc = tensor_map_encoder();
        if (!enc) return cudaErrorNotSupported;
        const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
        const cuuint64_t strides[1] = {(cuuint64_t)ldf * 4};
        const cuuint32_t box[2] = {(cuuint32_t)B, (cuuint32_t)B};
        const cuuint32_t estr[2] = {1, 1};
        if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(AF), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        const int C = nblk < kClCtas ? nblk : kClCtas;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C, 1, 1);
        cfg.blockDim = dim3(TT, 1, 1);
        cfg.dynamicSmemBytes = kClSmem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        count_launch();
        return cudaLaunchKernelEx(&cfg, k_trsv_cluster, tm, ldf, n, nblk, AF, Linv, Uinv, blk_subst, perm, r, vin,
                                  mode, rho_bits, skip, xo, dout, dev);
    }
    e = cudaMemsetAsync(&dev->ticket[0], 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    unsigned long long *ytag = tags, *ztag = tags + (int64_t)nblk * B;
    auto pair = [&](auto *F) -> cudaError_t {
        using T = std::remove_const_t<std::remove_pointer_t<decltype(F)>>;
        count_launch();
        k_trsv_lower<T><<<nblk, TT, kSolveSmem, s>>>(AF, F, ldf, n, nblk, Linv, blk_subst, perm, r, vin, mode,
                                                     rho_bits, skip, ytag, epoch, dev);
        cudaError_t e2 = cudaGetLastError();
        if (e2 != cudaSuccess) return e2;
        count_launch();
        k_trsv_upper<T><<<nblk, TT, kSolveSmem, s>>>(AF, F, ldf, n, nblk, Uinv, blk_subst, ytag, ztag, epoch, mode,
                                                     rho_bits, skip, xo, dout, dev);
        return cudaGetLastError();
    };
    if (!F16) return pair(AF);
    if (tf16 == IR_BF16) return pair(static_cast<const __nv_bfloat16 *>(F16));
    return pair(static_cast<const __half *>(F16));
}

// The solve pair for kRhs right-hand sides (see k_mtrsv_lower / k_mtrsv_upper).
cudaError_t launch_trsv_multi(const float *AF, int64_t ldf, int n, const float *Linv, const float *Uinv,
                              const int32_t *blk_subst, const int32_t *perm, const double *R, int64_t ldr,
                              const unsigned long long *rho_bits, const int *active, double *X, int64_t ldx,
                              unsigned long long *dnorm_bits, unsigned long long *xnorm_bits,
                              unsigned long long *tags, unsigned epoch, DevScalars *dev, cudaStream_t s,
                              const void *F16, ir_dtype tf16) {
    if (n == 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaSuccess;
        const void *kerns[6] = {(const void *)k_mtrsv_lower<float>, (const void *)k_mtrsv_upper<float>,
                                (const void *)k_mtrsv_lower<__half>, (const void *)k_mtrsv_upper<__half>,
                                (const void *)k_mtrsv_lower<__nv_bfloat16>,
                                (const void *)k_mtrsv_upper<__nv_bfloat16>};
        for (int q = 0; q < 6 && e == cudaSuccess; ++q)
            e = cudaFuncSetAttribute(kerns[q], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMultiSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int nblk = (n + B - 1) / B;
    const int64_t ntag = (int64_t)nblk * B;
    cudaError_t e = cudaMemsetAsync(&dev->ticket[0], 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    unsigned long long *ytag = tags, *ztag = tags + kRhs * ntag;
    auto pair = [&](auto *F) -> cudaError_t {
        using T = std::remove_const_t<std::remove_pointer_t<decltype(F)>>;
        count_launch();
        k_mtrsv_lower<T><<<nblk, TT, kMultiSmem, s>>>(AF, F, ldf, n, nblk, Linv, blk_subst, perm, R, ldr, rho_bits,
                                                      active, ytag, ntag, epoch, dev);
        cudaError_t e2 = cudaGetLastError();
        if (e2 != cudaSuccess) return e2;
        count_launch();
        k_mtrsv_upper<T><<<nblk, TT, kMultiSmem, s>>>(AF, F, ldf, n, nblk, Uinv, blk_subst, ytag, ztag, ntag, epoch,
                                                      rho_bits, active, X, ldx, dnorm_bits, xnorm_bits, dev);
        return cudaGetLastError();
    };
    if (!F16) return pair(AF);
    if (tf16 == IR_BF16) return pair(static_cast<const __nv_bfloat16 *>(F16));
    return pair(static_cast<const __half *>(F16));
}

// The factors kept in TF: every entry of A_F (L and U, rows and columns < n)
// rounded to TF in place (binary32 storage of the TF value) and written to the
// 2-byte copy F16 (same layout, row stride ldf); an entry that overflows TF
// raises the non-finite flag.
template <typename T>
__global__ void k_store_tf(float *AF, int64_t ldf, int n, T *F16, DevScalars *dev) {
    const int64_t total = (int64_t)n * n;
    int bad = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n, j = e % n;
        const float v = AF[i * ldf + j];
        T h;
        if constexpr (sizeof(T) == 2 && std::is_same<T, __half>::value) h = __float2half_rn(v);
        else h = __float2bfloat16_rn(v);
        float w;
        if constexpr (std::is_same<T, __half>::value) w = __half2float(h);
        else w = __bfloat162float(h);
        bad |= (isfinite(v) && !isfinite(w));
        AF[i * ldf + j] = w;
        F16[i * ldf + j] = h;
    }
    if (bad) atomicExch(&dev->nonfinite, 1);
}

cudaError_t launch_store_tf(float *AF, int64_t ldf, int n, ir_dtype tf, void *F16, DevScalars *dev, int sms,
                            cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    count_launch();
    const int64_t total = (int64_t)n * n;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 16 * sms) blocks = 16 * sms;
    if (tf == IR_BF16)
        k_store_tf<__nv_bfloat16><<<(int)blocks, 256, 0, s>>>(AF, ldf, n, static_cast<__nv_bfloat16 *>(F16), dev);
    else
        k_store_tf<__half><<<(int)blocks, 256, 0, s>>>(AF, ldf, n, static_cast<__half *>(F16), dev);
    return cudaGetLastError();
}

}  // namespace ir
