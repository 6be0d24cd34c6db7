// coarse.cu -- direct solve on the coarsest level (§3.1): dense FP64 Cholesky factor of the
// coarsest operator, then its explicit inverse, so that each V-cycle's coarse solve is one
// dense matrix-vector product spread over many warps.
//
// Factorisation: right-looking, 32-column panels.  Per panel one kernel factors the 32 x 32
// diagonal block (every block redundantly, in shared memory) and solves its rows of the
// panel; a second kernel updates the trailing lower triangle.  A pivot <= 0 stores its row
// (1-based) in *info and the remaining kernels return without work.
#include <math.h>

#include "amg_internal.cuh"

namespace amgk {

constexpr int kPanel = 32;

__global__ void dense_from_csr_kernel(int n, const int *rp, const int *ci, const double *v, double *a)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) a[(size_t)i * n + ci[e]] = v[e];
}

// factor the diagonal block [j0, j0+b) in shared memory; rows j0+b+blockIdx.x*128+t solve
// L_ib = A_ib L_bb^-T.  Block 0 writes the factored diagonal block back.
__global__ void __launch_bounds__(128) panel_kernel(int n, int j0, double *a, int *info)
{
    __shared__ double L[kPanel][kPanel + 1];
    if (*info) return;
    const int b = min(kPanel, n - j0);
    for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
        int r = t / b, c = t % b;
        L[r][c] = a[(size_t)(j0 + r) * n + j0 + c];
    }
    __syncthreads();
    for (int j = 0; j < b; ++j) {
        if (threadIdx.x == 0) {
            double d = L[j][j];
            if (!(d > 0.0)) {
                if (blockIdx.x == 0) atomicCAS(info, 0, j0 + j + 1);
                L[j][j] = 0.0;
            } else {
                L[j][j] = sqrt(d);
            }
        }
        __syncthreads();
        if (L[j][j] == 0.0) return;
        double ljj = L[j][j];
        for (int i = j + 1 + threadIdx.x; i < b; i += blockDim.x) L[i][j] = L[i][j] / ljj;
        __syncthreads();
        for (int t = threadIdx.x; t < (b - j - 1) * (b - j - 1); t += blockDim.x) {
            int i = j + 1 + t / (b - j - 1), k = j + 1 + t % (b - j - 1);
            if (k <= i) L[i][k] -= L[i][j] * L[k][j];
        }
        __syncthreads();
    }
    if (blockIdx.x == 0) {
        for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
            int r = t / b, c = t % b;
            if (c <= r) a[(size_t)(j0 + r) * n + j0 + c] = L[r][c];
        }
    }
    // rows below the block: forward substitution against L_bb
    int i = j0 + b + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double *row = a + (size_t)i * n + j0;
    double x[kPanel];
    for (int c = 0; c < b; ++c) {
        double s = row[c];
        for (int k = 0; k < c; ++k) s -= x[k] * L[c][k];
        x[c] = s / L[c][c];
    }
    for (int c = 0; c < b; ++c) row[c] = x[c];
}

// trailing update of the lower triangle: a_ik -= sum_t L_it L_kt over the panel columns
__global__ void __launch_bounds__(256) trailing_kernel(int n, int j0, double *a, const int *info)
{
    if (*info) return;
    const int b = min(kPanel, n - j0);
    const int s0 = j0 + b;
    const int m = n - s0;
    __shared__ double Li[32][kPanel + 1], Lk[32][kPanel + 1];
    const int ti = blockIdx.y * 32, tk = blockIdx.x * 32;
    if (tk > ti) return;      // strictly upper tiles
    for (int t = threadIdx.x; t < 32 * b; t += blockDim.x) {
        int r = t / b, c = t % b;
        Li[r][c] = (ti + r < m) ? a[(size_t)(s0 + ti + r) * n + j0 + c] : 0.0;
        Lk[r][c] = (tk + r < m) ? a[(size_t)(s0 + tk + r) * n + j0 + c] : 0.0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
        int r = t / 32, c = t % 32;
        int i = ti + r, k = tk + c;
        if (i >= m || k >= m || k > i) continue;
        double s = 0.0;
        for (int q = 0; q < b; ++q) s += Li[r][q] * Lk[c][q];
        a[(size_t)(s0 + i) * n + s0 + k] -= s;
    }
}

// column j of A^-1 = L^-T L^-1 e_j, one warp per column, written as row j (A^-1 is symmetric)
__global__ void inverse_kernel(int n, const double *L, double *inv, const int *info)
{
    if (*info) return;
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= n) return;
    double *y = inv + (size_t)j * n;
    for (int i = lane; i < n; i += 32) y[i] = 0.0;
    __syncwarp();
    // forward: L y = e_j (y_i = 0 for i < j)
    for (int i = j; i < n; ++i) {
        double s = 0.0;
        for (int k = j + lane; k < i; k += 32) s += L[(size_t)i * n + k] * y[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) y[i] = ((i == j ? 1.0 : 0.0) - s) / L[(size_t)i * n + i];
        __syncwarp();
    }
    // backward: L^T x = y
    for (int i = n - 1; i >= 0; --i) {
        double s = 0.0;
        for (int k = i + 1 + lane; k < n; k += 32) s += L[(size_t)k * n + i] * y[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) y[i] = (y[i] - s) / L[(size_t)i * n + i];
        __syncwarp();
    }
}

cudaError_t coarse_inverse(const DevCsr &A, double *work, double *inv, int *info_dev, cudaStream_t s)
{
    const int n = A.n;
    AMG_CUDA_TRY(cudaMemsetAsync(info_dev, 0, sizeof(int), s));
    if (n == 0) return cudaSuccess;
    AMG_CUDA_TRY(cudaMemsetAsync(work, 0, sizeof(double) * (size_t)n * n, s));
    dense_from_csr_kernel<<<grid_for(n, 128), 128, 0, s>>>(n, A.rp, A.ci, A.v, work); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    for (int j0 = 0; j0 < n; j0 += kPanel) {
        const int b = min(kPanel, n - j0);
        const int rows_below = n - j0 - b;
        const int pblocks = rows_below > 0 ? (rows_below + 127) / 128 : 1;
        panel_kernel<<<pblocks, 128, 0, s>>>(n, j0, work, info_dev); note_launch();
        if (rows_below > 0) {
            int tiles = (rows_below + 31) / 32;
            trailing_kernel<<<dim3(tiles, tiles), 256, 0, s>>>(n, j0, work, info_dev); note_launch();
        }
        AMG_CUDA_TRY(cudaGetLastError());
    }
    inverse_kernel<<<grid_for((int64_t)n * 32, 128), 128, 0, s>>>(n, work, inv, info_dev); note_launch();
    return cudaGetLastError();
}

}  // namespace amgk
