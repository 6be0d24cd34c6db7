// coarse.cu -- direct solve on the coarsest level (§3.1): dense FP64 Cholesky factor of the
// coarsest operator, then its explicit inverse, so that each V-cycle's coarse solve is one
// dense matrix-vector product spread over many warps.
//
// FP64 arithmetic runs at a small fraction of the FP32 rate on this GPU, so the work is cut
// so that no SM carries much more than its share and no step waits on a long chain of
// dependent global-memory round trips.
//
// Factorisation: right-looking, 32-column panels.  Per panel one kernel factors the 32 x 32
// diagonal block with a single warp in shared memory (every block redundantly, which is
// cheaper than another launch) and then solves 32 rows of the panel below it, one row per
// lane with the row held in registers; a second kernel updates the trailing lower triangle.
// A pivot <= 0 stores its row (1-based) in *info and every later kernel returns at once.
//
// Inverse: X = L^-T L^-1, column j by one warp: L y = e_j forward and L^T x = y backward, both
// in the axpy form (step i finishes y_i, then every lane updates the entries it owns with row
// i of L^T resp. L, read contiguously), so a step's critical path is one multiply and one
// shuffle.  Only x_i for i >= j is formed (the backward sweep stops at j); the strictly upper
// part is written from the symmetry of X.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "amg_internal.cuh"

namespace amgk {

constexpr int kPanel = 32;
constexpr int kInvWarps = 4;                 // columns per block of the inverse (at most)
constexpr int kInvSmem = 200 * 1024;         // dynamic shared memory cap of the inverse kernel

__global__ void dense_from_csr_kernel(int n, const int *rp, const int *ci, const double *v, double *a)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) a[(size_t)i * n + ci[e]] = v[e];
}

// One warp per block.  Factors the diagonal block [j0, j0 + b) in shared memory (lane r owns
// row r), then lane r solves row i = j0 + b + 32 blockIdx.x + r of the panel:
// L_ib = A_ib L_bb^-T.  Block 0 writes the factored block back.
__global__ void __launch_bounds__(32) panel_kernel(int n, int j0, double *a, int *info)
{
    __shared__ double Lb[kPanel][kPanel + 1];
    if (*info) return;
    const int b = min(kPanel, n - j0);
    const int r = threadIdx.x;
    if (r < b)
        for (int c = 0; c < b; ++c) Lb[r][c] = a[(size_t)(j0 + r) * n + j0 + c];
    __syncwarp();
    for (int j = 0; j < b; ++j) {
        const double d = Lb[j][j];
        if (!(d > 0.0)) {
            if (blockIdx.x == 0 && r == 0) atomicCAS(info, 0, j0 + j + 1);
            return;                                   // uniform over the warp
        }
        const double ljj = sqrt(d);
        __syncwarp();
        if (r == j) Lb[j][j] = ljj;
        if (r > j && r < b) Lb[r][j] = Lb[r][j] / ljj;
        __syncwarp();
        if (r > j && r < b) {
            const double lrj = Lb[r][j];
            for (int k = j + 1; k <= r; ++k) Lb[r][k] -= lrj * Lb[k][j];
        }
        __syncwarp();
    }
    if (blockIdx.x == 0 && r < b)
        for (int c = 0; c <= r; ++c) a[(size_t)(j0 + r) * n + j0 + c] = Lb[r][c];
    const int i = j0 + b + blockIdx.x * kPanel + r;
    if (i >= n) return;
    double *row = a + (size_t)i * n + j0;
    double x[kPanel];
#pragma unroll
    for (int c = 0; c < kPanel; ++c) {
        if (c < b) {
            double s = row[c];
#pragma unroll
            for (int k = 0; k < kPanel; ++k)
                if (k < c) s -= x[k] * Lb[c][k];
            x[c] = s / Lb[c][c];
        }
    }
#pragma unroll
    for (int c = 0; c < kPanel; ++c)
        if (c < b) row[c] = x[c];
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
        int rr = t / b, c = t % b;
        Li[rr][c] = (ti + rr < m) ? a[(size_t)(s0 + ti + rr) * n + j0 + c] : 0.0;
        Lk[rr][c] = (tk + rr < m) ? a[(size_t)(s0 + tk + rr) * n + j0 + c] : 0.0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
        int rr = t / 32, c = t % 32;
        int i = ti + rr, k = tk + c;
        if (i >= m || k >= m || k > i) continue;
        double s = 0.0;
        for (int q = 0; q < b; ++q) s += Li[rr][q] * Lk[c][q];
        a[(size_t)(s0 + i) * n + s0 + k] -= s;
    }
}

// lt = L^T (upper) and rdiag = 1 / L_ii, from the factored lower triangle of a
__global__ void transpose_lower_kernel(int n, const double *a, double *lt, double *rdiag, const int *info)
{
    if (*info) return;
    __shared__ double tile[32][33];
    const int bi = blockIdx.y * 32, bk = blockIdx.x * 32;     // source tile rows bi.., cols bk..
    if (bk > bi) return;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    for (int y = ty; y < 32; y += 8) {
        const int i = bi + y, k = bk + tx;
        tile[y][tx] = (i < n && k < n && k <= i) ? a[(size_t)i * n + k] : 0.0;
    }
    __syncthreads();
    for (int y = ty; y < 32; y += 8) {
        const int k = bk + y, i = bi + tx;                   // lt[k][i] = a[i][k]
        if (k < n && i < n && k <= i) lt[(size_t)k * n + i] = tile[tx][y];
    }
    if (bi == bk)
        for (int y = threadIdx.x; y < 32; y += blockDim.x)
            if (bi + y < n) rdiag[bi + y] = 1.0 / a[(size_t)(bi + y) * n + bi + y];
}

// One warp per column j.  Lane l owns y_k and x_k for k = j + l + 32 m (kept in the warp's
// slice of shared memory).  Forward: y_i *= 1/L_ii, then y_k -= L^T_ik y_i for k > i.
// Backward: x_i = y_i / L_ii, then y_k -= L_ik x_i for j <= k < i.  inv_ij = inv_ji = x_i.
__global__ void __launch_bounds__(32 * kInvWarps) inverse_kernel(int n, const double *L, const double *Lt,
                                                                  const double *rdiag, double *inv, const int *info)
{
    extern __shared__ double ys[];
    if (*info) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = blockIdx.x * (int)(blockDim.x >> 5) + w;
    if (j >= n) return;
    double *y = ys + (size_t)w * n;
    const int m = n - j;                               // entries j .. n-1, local index k - j
    for (int t = lane; t < m; t += 32) y[t] = (t == 0) ? 1.0 : 0.0;
    __syncwarp();
    // forward: L y = e_j
    for (int t = 0; t < m; ++t) {
        const int i = j + t;
        double yi = 0.0;
        if ((t & 31) == lane) {
            yi = y[t] * rdiag[i];
            y[t] = yi;
        }
        yi = __shfl_sync(0xffffffffu, yi, t & 31);
        const double *lrow = Lt + (size_t)i * n;       // row i of L^T: L_ki for k > i
        for (int u = t + 1 + ((lane - t - 1) & 31); u < m; u += 32) y[u] -= lrow[j + u] * yi;
    }
    // backward: L^T x = y, rows n-1 down to j
    for (int t = m - 1; t >= 0; --t) {
        const int i = j + t;
        double xi = 0.0;
        if ((t & 31) == lane) {
            xi = y[t] * rdiag[i];
            y[t] = xi;
        }
        xi = __shfl_sync(0xffffffffu, xi, t & 31);
        const double *lrow = L + (size_t)i * n;        // row i of L: L_ik for k < i
        for (int u = lane; u < t; u += 32) y[u] -= lrow[j + u] * xi;
    }
    __syncwarp();
    for (int t = lane; t < m; t += 32) {
        inv[(size_t)(j + t) * n + j] = y[t];
        inv[(size_t)j * n + j + t] = y[t];
    }
}

cudaError_t coarse_inverse(const DevCsr &A, double *work, double *inv, int *info_dev, cudaStream_t s)
{
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kInvSmem);
    });
    AMG_CUDA_TRY(attr);
    const int n = A.n;
    AMG_CUDA_TRY(cudaMemsetAsync(info_dev, 0, sizeof(int), s));
    if (n == 0) return cudaSuccess;
    // columns per block: as many as the shared-memory cap holds, at most kInvWarps
    const int warps = (int)std::min<size_t>(kInvWarps, (size_t)kInvSmem / ((size_t)n * sizeof(double)));
    if (warps < 1) return cudaErrorInvalidValue;
    double *lt = work + (size_t)n * n, *rdiag = lt + (size_t)n * n;
    AMG_CUDA_TRY(cudaMemsetAsync(work, 0, sizeof(double) * (size_t)n * n, s));
    dense_from_csr_kernel<<<grid_for(n, 128), 128, 0, s>>>(n, A.rp, A.ci, A.v, work); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    for (int j0 = 0; j0 < n; j0 += kPanel) {
        const int b = min(kPanel, n - j0);
        const int rows_below = n - j0 - b;
        const int pblocks = rows_below > 0 ? (rows_below + kPanel - 1) / kPanel : 1;
        panel_kernel<<<pblocks, kPanel, 0, s>>>(n, j0, work, info_dev); note_launch();
        if (rows_below > 0) {
            int tiles = (rows_below + 31) / 32;
            trailing_kernel<<<dim3(tiles, tiles), 256, 0, s>>>(n, j0, work, info_dev); note_launch();
        }
        AMG_CUDA_TRY(cudaGetLastError());
    }
    const int tb = (n + 31) / 32;
    transpose_lower_kernel<<<dim3(tb, tb), 256, 0, s>>>(n, work, lt, rdiag, info_dev); note_launch();
    const size_t smem = (size_t)warps * n * sizeof(double);
    inverse_kernel<<<(n + warps - 1) / warps, 32 * warps, smem, s>>>(n, work, lt, rdiag, inv, info_dev); note_launch();
    return cudaGetLastError();
}

}  // namespace amgk
