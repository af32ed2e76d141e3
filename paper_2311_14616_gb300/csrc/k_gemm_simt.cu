// binary32 trailing update of the blocked LU: A22 <- A22 - L21 U12 with every
// element updated by the fmaf chain acc = fmaf(-l_im, u_mc, acc), m ascending
// from the stored value -- the same operations as the unblocked right-looking
// algorithm, so the binary32 factors are bitwise those of the plain LU.
#include "ir_internal.cuh"
#include "lu_tiles.cuh"

namespace ir {
namespace {

constexpr int BM = 128, BN = 128, BK = 32, NB = kPanelNB;
constexpr int kShareCluster = 8;

// Columns [cb, ce) of the trailing matrix (cb, ce multiples of 64, or ce = n);
// tiles are taken in a grid-stride loop so the grid can leave SMs free.
__global__ void __launch_bounds__(256) k_gemm_simt(float *AF, int64_t ldf, int n, int j, int cb, int ce) {
    pdl_trigger();
    pdl_wait();
    __shared__ __align__(16) float As[BK][BM + 4];   // As[k][i] = L21[i][k]
    __shared__ __align__(16) float Bs[BK][BN + 4];   // Bs[k][c] = U12[k][c]
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int m = n - (j + NB);
    const int tiles_m = (m + BM - 1) / BM, tiles_n = (ce - cb + BN - 1) / BN;
    for (int tile = blockIdx.x; tile < tiles_m * tiles_n; tile += gridDim.x) {
    const int i0 = j + NB + (tile / tiles_n) * BM;
    const int c0 = cb + (tile % tiles_n) * BN;

    // C micro-tile: rows i0 + {ty*4 + r, 64 + ty*4 + r}, cols c0 + {tx*4 + q, 64 + tx*4 + q}
    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int i = i0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = c0 + h * 64 + tx * 4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < n && c < ce) v = *reinterpret_cast<const float4 *>(AF + (int64_t)i * ldf + c);
            acc[r][h * 4 + 0] = v.x; acc[r][h * 4 + 1] = v.y;
            acc[r][h * 4 + 2] = v.z; acc[r][h * 4 + 3] = v.w;
        }
    }
    for (int kb = 0; kb < NB; kb += BK) {
        // A tile: 128 rows x 32 k (each row 128 contiguous bytes), stored transposed
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = t + q * 256;
            const int row = idx >> 3, kq = (idx & 7) * 4;
            const int i = i0 + row;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < n) v = *reinterpret_cast<const float4 *>(AF + (int64_t)i * ldf + j + kb + kq);
            As[kq + 0][row] = v.x; As[kq + 1][row] = v.y; As[kq + 2][row] = v.z; As[kq + 3][row] = v.w;
        }
        // B tile: 32 k x 128 cols (rows of U12 are contiguous)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = t + q * 256;
            const int m = idx >> 5, cq = (idx & 31) * 4;
            const int c = c0 + cq;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c < ce) v = *reinterpret_cast<const float4 *>(AF + (int64_t)(j + kb + m) * ldf + c);
            *reinterpret_cast<float4 *>(&Bs[m][cq]) = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int m = 0; m < BK; ++m) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[m][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[m][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[m][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[m][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[r][q] = fmaf(-av[r], bv[q], acc[r][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int i = i0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
        if (i >= n) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = c0 + h * 64 + tx * 4;
            if (c < ce)
                *reinterpret_cast<float4 *>(AF + (int64_t)i * ldf + c) =
                    make_float4(acc[r][h * 4 + 0], acc[r][h * 4 + 1], acc[r][h * 4 + 2], acc[r][h * 4 + 3]);
        }
    }
    }
}

// The same update for a narrow column range (<= 64 columns: the next block
// column of the lookahead, on the critical path): 64 x 64 tiles
// (lu::gemm_tile64), so twice the CTAs of the wide kernel for the same rows.
constexpr int NT = 64;
__global__ void __launch_bounds__(256) k_gemm_simt_narrow(float *AF, int64_t ldf, int n, int j, int cb, int ce) {
    pdl_trigger();
    pdl_wait();
    __shared__ __align__(16) float As[NB][lu::kLd];
    __shared__ __align__(16) float Bs[NB][lu::kLd];
    lu::gemm_tile64(AF, ldf, n, j, cb, ce, j + NB + blockIdx.x * NT, As, Bs);
}

}  // namespace

// max_ctas > 0: share the GPU with a concurrent panel -- the update runs as
// clusters of 8 CTAs, two clusters fewer than fit at once, so that whole GPC
// slots stay free for the panel's cluster.
cudaError_t launch_gemm_simt(float *AF, int64_t ldf, int n, int j, int nb, int cb, int ce, int max_ctas,
                             cudaStream_t s) {
    const int m = n - (j + nb);
    if (m <= 0 || ce <= cb) return cudaSuccess;
    const int tiles = ((m + BM - 1) / BM) * ((ce - cb + BN - 1) / BN);
    count_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(256, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    cfg.attrs = attr;
    if (max_ctas <= 0 && ce - cb <= NT) {
        cfg.gridDim = dim3((m + NT - 1) / NT, 1, 1);
        cfg.numAttrs = set_pdl(&attr[0]);
        return cudaLaunchKernelEx(&cfg, k_gemm_simt_narrow, AF, ldf, n, j, cb, ce);
    }
    if (max_ctas <= 0) {
        cfg.gridDim = dim3(tiles, 1, 1);
        cfg.numAttrs = set_pdl(&attr[0]);
        return cudaLaunchKernelEx(&cfg, k_gemm_simt, AF, ldf, n, j, cb, ce);
    }
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kShareCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.numAttrs = 1;
    static int max_clusters = -1;
    if (max_clusters < 0) {
        cfg.gridDim = dim3(kShareCluster * 64, 1, 1);
        if (cudaOccupancyMaxActiveClusters(&max_clusters, k_gemm_simt, &cfg) != cudaSuccess) max_clusters = 0;
        (void)cudaGetLastError();
    }
    cfg.numAttrs = 1 + set_pdl(&attr[1]);
    int clusters = max_clusters - 2;
    if (clusters < 1) clusters = 1;
    const int need = (tiles + kShareCluster - 1) / kShareCluster;
    if (clusters > need) clusters = need;
    cfg.gridDim = dim3(clusters * kShareCluster, 1, 1);
    return cudaLaunchKernelEx(&cfg, k_gemm_simt, AF, ldf, n, j, cb, ce);
}

}  // namespace ir
