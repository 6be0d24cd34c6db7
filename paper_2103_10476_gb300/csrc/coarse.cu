// coarse.cu -- direct solve on the coarsest level (§3.1): the explicit inverse of the coarsest
// operator in FP64, so that each V-cycle's coarse solve is one dense matrix-vector product
// spread over many warps.
//
// FP64 arithmetic runs at a small fraction of the FP32 rate on this GPU: a warp's FP64
// instruction occupies a sub-partition's FP64 unit for tens of cycles, so a serial chain of
// FP64 operations (a Cholesky panel, a triangular solve) is slow however few flops it has,
// while independent FP64 work spread over every sub-partition runs at the full rate.  The
// inverse is therefore formed in two stages:
//   1. Cholesky factor and inverse in FP32 (the serial chains at the FP32 rate): X0.
//   2. Newton-Schulz refinement in FP64, X <- X (2I - A X), as dense products with one output
//      per thread.  The error E = max |I - A X| squares every step; the step taken with
//      E < 1e-10 is the last (two steps from an FP32 inverse of a well-conditioned operator).
// If the FP32 factorisation meets a pivot <= 0 (the operator is too ill-conditioned for FP32)
// or the refinement does not bring E below 1e-6, the inverse is formed directly in FP64 by
// the same factorisation and inverse kernels in double precision.
// A large coarsest level (more than kCgMinRows rows, at most one stored entry in eight) is
// what aggregation leaves when it stalls: no entry is strong any more, so the Jacobi-scaled
// operator S A S (S = diag(a_ii)^-1/2) is close to the identity (condition numbers 1.1-1.2 on
// the random-coefficient cubes).  Its inverse is then formed without a dense factorisation,
// by conjugate gradients on the n columns of S A S X = I at once in FP64 (every column with
// its own step lengths; one product of the sparse operator with all n columns per step), until
// every column's residual is below 1e-15; the result is accepted once the true residual
// max |I - S A S X| is below 1e-13, and scaled back, A^-1 = S X S.  The dense factorisation
// costs n^3 work however sparse the operator is (a 7,004-row level with 4.5 entries per row
// took seconds); this costs (nnz + 10 n) n per step.  When CG does not converge within
// kCgMaxSteps steps, or a column meets a non-positive curvature, the dense path below is taken.
// A nonsymmetric coarsest operator (GMRES outer iteration) has no Cholesky factor: its
// inverse starts from X0 = A^T / (||A||_1 ||A||_inf), for which ||I - A X0||_2 < 1 whenever A
// is nonsingular, and takes Newton-Schulz steps in FP32 until E < 1e-4, then in FP64.
//
// Factorisation (either precision): right-looking, 32-column panels.  Per panel one kernel
// factors the 32 x 32 diagonal block with a single warp in shared memory (every block
// redundantly, cheaper than another launch) and then solves 32 rows of the panel below it,
// one row per lane with the row in registers; a second kernel updates the trailing lower
// triangle.  A pivot <= 0 stores its row (1-based) in *info and every later kernel returns.
// Inverse: X = L^-T L^-1, column j by one warp in the axpy form (step i finishes y_i, then
// every lane updates the entries it owns from a contiguous row of L^T resp. L); the backward
// sweep stops at j and the strictly upper part is written from the symmetry of X.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "amg_internal.cuh"

namespace amgk {

constexpr int kPanel = 32;
constexpr int kInvWarps = 4;                 // columns per block of the inverse (at most)
constexpr int kInvSmem = 200 * 1024;         // dynamic shared memory cap of the inverse kernel
constexpr int kNewtonSteps = 4;              // refinement steps at most (E0 up to ~1e-2 converges)
constexpr int kGeneral32 = 64;               // nonsymmetric operators: FP32 steps from the scaled transpose
constexpr int kGeneral64 = 8;                //   and FP64 steps after them
constexpr int kGT = 16;                      // product tile: many blocks, so that every SM's FP64 units work
constexpr int kCgMinRows = 512;              // the CG path for sparse coarsest levels larger than this
constexpr int kCgMaxSteps = 240;             // CG steps at most before the dense path is taken
constexpr int kCgCheck = 4;                  // steps between convergence checks on the host
constexpr int kCgChunk = 32;                 // rows per partial column sum
constexpr int kCgLongRow = 128;              // longer rows are summed in segments by blocks of their own
constexpr int kCgSegment = 256;

__global__ void dense_from_csr_kernel(int n, const int *rp, const int *ci, const double *v, double *a)
{
    const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    for (int e = rp[i] + lane; e < rp[i + 1]; e += 32) a[(size_t)i * n + ci[e]] = v[e];
}

template <typename A, typename B>
__global__ void convert_dense_kernel(size_t count, const A *src, B *dst)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (B)src[i];
}

// One warp per block.  Factors the diagonal block [j0, j0 + b) in shared memory (lane r owns
// row r), then lane r solves row i = j0 + b + 32 blockIdx.x + r of the panel:
// L_ib = A_ib L_bb^-T.  Block 0 writes the factored block back.
template <typename T>
__global__ void __launch_bounds__(32) panel_kernel(int n, int j0, T *a, int *info)
{
    __shared__ T Lb[kPanel][kPanel + 1];
    if (*info) return;
    const int b = min(kPanel, n - j0);
    const int r = threadIdx.x;
    if (r < b)
        for (int c = 0; c < b; ++c) Lb[r][c] = a[(size_t)(j0 + r) * n + j0 + c];
    __syncwarp();
    for (int j = 0; j < b; ++j) {
        const T d = Lb[j][j];
        if (!(d > T(0))) {
            if (blockIdx.x == 0 && r == 0) atomicCAS(info, 0, j0 + j + 1);
            return;                                   // uniform over the warp
        }
        const T ljj = sqrt(d);
        __syncwarp();
        if (r == j) Lb[j][j] = ljj;
        if (r > j && r < b) Lb[r][j] = Lb[r][j] / ljj;
        __syncwarp();
        if (r > j && r < b) {
            const T lrj = Lb[r][j];
            for (int k = j + 1; k <= r; ++k) Lb[r][k] -= lrj * Lb[k][j];
        }
        __syncwarp();
    }
    if (blockIdx.x == 0 && r < b)
        for (int c = 0; c <= r; ++c) a[(size_t)(j0 + r) * n + j0 + c] = Lb[r][c];
    const int i = j0 + b + blockIdx.x * kPanel + r;
    if (i >= n) return;
    T *row = a + (size_t)i * n + j0;
    T x[kPanel];
#pragma unroll
    for (int c = 0; c < kPanel; ++c) {
        if (c < b) {
            T s = row[c];
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
template <typename T>
__global__ void __launch_bounds__(256) trailing_kernel(int n, int j0, T *a, const int *info)
{
    if (*info) return;
    const int b = min(kPanel, n - j0);
    const int s0 = j0 + b;
    const int m = n - s0;
    __shared__ T Li[32][kPanel + 1], Lk[32][kPanel + 1];
    const int ti = blockIdx.y * 32, tk = blockIdx.x * 32;
    if (tk > ti) return;      // strictly upper tiles
    for (int t = threadIdx.x; t < 32 * b; t += blockDim.x) {
        int rr = t / b, c = t % b;
        Li[rr][c] = (ti + rr < m) ? a[(size_t)(s0 + ti + rr) * n + j0 + c] : T(0);
        Lk[rr][c] = (tk + rr < m) ? a[(size_t)(s0 + tk + rr) * n + j0 + c] : T(0);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
        int rr = t / 32, c = t % 32;
        int i = ti + rr, k = tk + c;
        if (i >= m || k >= m || k > i) continue;
        T s = T(0);
        for (int q = 0; q < b; ++q) s += Li[rr][q] * Lk[c][q];
        a[(size_t)(s0 + i) * n + s0 + k] -= s;
    }
}

// lt = L^T (upper) and rdiag = 1 / L_ii, from the factored lower triangle of a
template <typename T>
__global__ void transpose_lower_kernel(int n, const T *a, T *lt, T *rdiag, const int *info)
{
    if (*info) return;
    __shared__ T tile[32][33];
    const int bi = blockIdx.y * 32, bk = blockIdx.x * 32;     // source tile rows bi.., cols bk..
    if (bk > bi) return;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    for (int y = ty; y < 32; y += 8) {
        const int i = bi + y, k = bk + tx;
        tile[y][tx] = (i < n && k < n && k <= i) ? a[(size_t)i * n + k] : T(0);
    }
    __syncthreads();
    for (int y = ty; y < 32; y += 8) {
        const int k = bk + y, i = bi + tx;                   // lt[k][i] = a[i][k]
        if (k < n && i < n && k <= i) lt[(size_t)k * n + i] = tile[tx][y];
    }
    if (bi == bk)
        for (int y = threadIdx.x; y < 32; y += blockDim.x)
            if (bi + y < n) rdiag[bi + y] = T(1) / a[(size_t)(bi + y) * n + bi + y];
}

// One warp per column j.  Lane l owns y_k and x_k for k = j + l + 32 m (kept in the warp's
// slice of shared memory).  Forward: y_i *= 1/L_ii, then y_k -= L^T_ik y_i for k > i.
// Backward: x_i = y_i / L_ii, then y_k -= L_ik x_i for j <= k < i.  inv_ij = inv_ji = x_i.
template <typename T>
__global__ void __launch_bounds__(32 * kInvWarps) inverse_kernel(int n, const T *L, const T *Lt, const T *rdiag,
                                                                  T *inv, const int *info)
{
    extern __shared__ __align__(16) unsigned char inv_smem[];
    if (*info) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = blockIdx.x * (int)(blockDim.x >> 5) + w;
    if (j >= n) return;
    T *y = (T *)inv_smem + (size_t)w * n;
    const int m = n - j;                               // entries j .. n-1, local index k - j
    for (int t = lane; t < m; t += 32) y[t] = (t == 0) ? T(1) : T(0);
    __syncwarp();
    for (int t = 0; t < m; ++t) {                      // forward: L y = e_j
        const int i = j + t;
        const T *lrow = Lt + (size_t)i * n;            // row i of L^T: L_ki for k > i
        const int u0 = t + 1 + ((lane - t - 1) & 31);
        // the row's first entry of this lane is requested before the chain's shuffle
        const T l0 = u0 < m ? lrow[j + u0] : T(0);
        T yi = T(0);
        if ((t & 31) == lane) {
            yi = y[t] * rdiag[i];
            y[t] = yi;
        }
        yi = __shfl_sync(0xffffffffu, yi, t & 31);
        if (u0 < m) y[u0] -= l0 * yi;
        for (int u = u0 + 32; u < m; u += 32) y[u] -= lrow[j + u] * yi;
    }
    for (int t = m - 1; t >= 0; --t) {                 // backward: L^T x = y, rows n-1 .. j
        const int i = j + t;
        const T *lrow = L + (size_t)i * n;             // row i of L: L_ik for k < i
        const T l0 = lane < t ? lrow[j + lane] : T(0);
        T xi = T(0);
        if ((t & 31) == lane) {
            xi = y[t] * rdiag[i];
            y[t] = xi;
        }
        xi = __shfl_sync(0xffffffffu, xi, t & 31);
        if (lane < t) y[lane] -= l0 * xi;
        for (int u = lane + 32; u < t; u += 32) y[u] -= lrow[j + u] * xi;
    }
    __syncwarp();
    for (int t = lane; t < m; t += 32) {
        inv[(size_t)(j + t) * n + j] = y[t];
        inv[(size_t)j * n + j + t] = y[t];
    }
}

// ------------------------------------------------------------------------------------ refinement
// Newton-Schulz state (device): [0] E of the previous step, [1] 1 once converged, [2] E of this
// step (as the bits of a non-negative double, for atomicMax).
struct NewtonState {
    double e_prev;
    int done, last;         // last: this step's update is the final one
    unsigned long long e_bits;
};

// C = P Q (n x n, FP64), one output per thread, 32 x 32 tiles staged in shared memory.
// MODE 0: C = P Q and state->e_bits = max |I - C| (the residual of X = Q against P = A);
// MODE 1: C = 2 X - X R with X = P, R = Q (the Newton update), or C = X once converged.
template <typename T, int MODE>
__global__ void __launch_bounds__(kGT * kGT) newton_gemm_kernel(int n, const T *P, const T *Q, T *C,
                                                                 NewtonState *state)
{
    __shared__ T Ps[kGT][kGT + 1], Qs[kGT][kGT + 1];
    const int done = state->done || (MODE == 0 && state->last);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int row = blockIdx.y * kGT + ty, col = blockIdx.x * kGT + tx;
    if (done) {
        if (MODE == 1 && row < n && col < n) C[(size_t)row * n + col] = P[(size_t)row * n + col];
        return;
    }
    T acc = T(0);
    for (int k0 = 0; k0 < n; k0 += kGT) {
        Ps[ty][tx] = (row < n && k0 + tx < n) ? P[(size_t)row * n + k0 + tx] : T(0);
        Qs[ty][tx] = (k0 + ty < n && col < n) ? Q[(size_t)(k0 + ty) * n + col] : T(0);
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kGT; ++k) acc += Ps[ty][k] * Qs[k][tx];
        __syncthreads();
    }
    if (row >= n || col >= n) return;
    if (MODE == 0) {
        C[(size_t)row * n + col] = acc;
        const double e = fabs((row == col ? 1.0 : 0.0) - (double)acc);
        // non-negative doubles order as their bit patterns
        atomicMax(&state->e_bits, (unsigned long long)__double_as_longlong(e));
    } else {
        C[(size_t)row * n + col] = T(2) * P[(size_t)row * n + col] - acc;
    }
}

// FP32 stage of the general inverse: done once E < 1e-4 (the FP64 steps take it from there)
__global__ void newton32_check_kernel(NewtonState *state)
{
    if (state->done) return;
    const double e = __longlong_as_double((long long)state->e_bits);
    if (e < 1e-4) state->done = 1;
    state->e_prev = e;
    state->e_bits = 0ULL;
}

// out[0] = max row sum of |a_ij|, out[1] = max column sum (as bit patterns of non-negative doubles)
__global__ void abs_sums_kernel(int n, const double *a, unsigned long long *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double r = 0.0, c = 0.0;
    for (int k = 0; k < n; ++k) {
        r += fabs(a[(size_t)t * n + k]);
        c += fabs(a[(size_t)k * n + t]);
    }
    atomicMax(&out[0], (unsigned long long)__double_as_longlong(r));
    atomicMax(&out[1], (unsigned long long)__double_as_longlong(c));
}

// X0 = A^T / (||A||_1 ||A||_inf) in FP32: ||I - A X0||_2 < 1 for every nonsingular A
__global__ void transpose_seed_kernel(int n, const double *a, const unsigned long long *sums, float *x)
{
    const double scale = 1.0 / (__longlong_as_double((long long)sums[0]) * __longlong_as_double((long long)sums[1]));
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * n; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / n, j = e % n;
        x[e] = (float)(a[j * n + i] * scale);
    }
}

// after a residual with error E: E < 1e-10 -> this update is the last (its error, about E^2,
// is at rounding level); E >= 1 or E no longer halving -> stop without it (a step after the
// last update only marks the end)
__global__ void newton_check_kernel(NewtonState *state)
{
    if (state->done) return;
    if (state->last) {
        state->done = 1;
        return;
    }
    const double e = __longlong_as_double((long long)state->e_bits);
    if (e < 1e-10) state->last = 1;
    else if (!(e < 1.0) || !(e < 0.5 * state->e_prev)) state->done = 1;
    state->e_prev = e;
    state->e_bits = 0ULL;
}

// ------------------------------------------------------------------------------------ large and sparse: CG
// s_i = a_ii^-1/2 and sv = s_i a_ij s_j (bad[0] counts rows whose diagonal is missing or not
// positive: the operator is then not SPD and the dense path reports it)
__global__ void jacobi_scale_kernel(int n, const int *rp, const int *ci, const double *v, double *sc, int *bad)
{
    // a warp per row (rows of thousands of entries occur on stalled levels)
    const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    double d = 0.0;
    for (int e = rp[i] + lane; e < rp[i + 1]; e += 32)
        if (ci[e] == i) d = v[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_xor_sync(0xffffffffu, d, o);
        d = d != 0.0 ? d : t;
    }
    if (lane != 0) return;
    if (!(d > 0.0)) {
        atomicAdd(bad, 1);
        sc[i] = 0.0;
        return;
    }
    sc[i] = 1.0 / sqrt(d);
}
__global__ void scale_values_kernel(int n, const int *rp, const int *ci, const double *v, const double *sc, double *sv)
{
    const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    for (int e = rp[i] + lane; e < rp[i + 1]; e += 32) sv[e] = sc[i] * v[e] * sc[ci[e]];
}

// Every CG kernel works on n x n row-major arrays with thread (column c = blockIdx.x * 256 +
// threadIdx.x, rows of chunk blockIdx.y); per-chunk partial column sums go to part[chunk][c]
// and are added in chunk order by cg_reduce_kernel (reproducible).
// MODE 0: Q = S A S P and part = P .* Q;  MODE 1 (check): part = max |I - S A S P| per column.
// Rows longer than long_len were summed by cg_long_partial/cg_long_reduce into Q beforehand.
template <int MODE>
__global__ void __launch_bounds__(256) cg_spmm_kernel(int n, const int *rp, const int *ci, const double *sv,
                                                       const double *P, double *Q, double *part, int long_len)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int i0 = blockIdx.y * kCgChunk, i1 = min(n, i0 + kCgChunk);
    double acc = 0.0;
    for (int i = i0; i < i1; ++i) {
        const size_t ic = (size_t)i * n + c;
        double q = 0.0;
        if (rp[i + 1] - rp[i] > long_len) {
            q = Q[ic];
        } else {
            for (int e = rp[i]; e < rp[i + 1]; ++e) q = fma(sv[e], P[(size_t)ci[e] * n + c], q);
        }
        if (MODE == 0) {
            if (rp[i + 1] - rp[i] <= long_len) Q[ic] = q;
            acc = fma(P[ic], q, acc);
        } else {
            acc = fmax(acc, fabs((i == c ? 1.0 : 0.0) - q));
        }
    }
    part[(size_t)blockIdx.y * n + c] = acc;
}

// Long rows of S A S: segment s (entries [seg_k0[s], seg_k1[s]) of one long row) times the
// n columns of P, into part_long[s][c]; then each long row's segments added in order into Q.
__global__ void __launch_bounds__(256) cg_long_partial_kernel(int n, const int *seg_k0, const int *seg_k1,
                                                               const int *ci, const double *sv, const double *P,
                                                               double *part_long)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int sg = blockIdx.y;
    double q = 0.0;
    for (int e = seg_k0[sg]; e < seg_k1[sg]; ++e) q = fma(sv[e], P[(size_t)ci[e] * n + c], q);
    part_long[(size_t)sg * n + c] = q;
}
__global__ void __launch_bounds__(256) cg_long_reduce_kernel(int n, const int *long_rows, const int *seg_first,
                                                              const double *part_long, double *Q)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int r = blockIdx.y;
    double q = 0.0;
    for (int sg = seg_first[r]; sg < seg_first[r + 1]; ++sg) q += part_long[(size_t)sg * n + c];
    Q[(size_t)long_rows[r] * n + c] = q;
}

// per column c: sum (MODE 0: alpha = rr / pq; MODE 1: beta = rr_new / rr, rr = rr_new) or
// max (MODE 2) of the chunk partials.  flags[0] += 1 for a non-positive curvature p.q;
// bits[0] = max_c rr (bit patterns of non-negative doubles order as the values).
template <int MODE>
__global__ void cg_reduce_kernel(int n, int chunks, const double *part, double *rr, double *coef, int *flags,
                                 unsigned long long *bits)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double t = 0.0;
    for (int k = 0; k < chunks; ++k) {
        const double x = part[(size_t)k * n + c];
        t = MODE == 2 ? fmax(t, x) : t + x;
    }
    if (MODE == 0) {
        const double r = rr[c];
        if (r > 0.0 && !(t > 0.0)) atomicAdd(flags, 1);
        coef[c] = (r > 0.0 && t > 0.0) ? r / t : 0.0;
    } else if (MODE == 1) {
        const double r = rr[c];
        coef[c] = r > 0.0 ? t / r : 0.0;
        rr[c] = t;
        atomicMax(bits, (unsigned long long)__double_as_longlong(t));
    } else {
        atomicMax(bits, (unsigned long long)__double_as_longlong(t));
    }
}

// X += alpha P, R -= alpha Q, part = R .* R
__global__ void __launch_bounds__(256) cg_update_kernel(int n, const double *alpha, const double *P, const double *Q,
                                                         double *X, double *R, double *part)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int i0 = blockIdx.y * kCgChunk, i1 = min(n, i0 + kCgChunk);
    const double a = alpha[c];
    double acc = 0.0;
    for (int i = i0; i < i1; ++i) {
        const size_t ic = (size_t)i * n + c;
        X[ic] = fma(a, P[ic], X[ic]);
        const double r = fma(-a, Q[ic], R[ic]);
        R[ic] = r;
        acc = fma(r, r, acc);
    }
    part[(size_t)blockIdx.y * n + c] = acc;
}

// P = R + beta P (FIRST: X = 0, R = P = I)
template <bool FIRST>
__global__ void __launch_bounds__(256) cg_direction_kernel(int n, const double *beta, double *X, double *R, double *P)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int i0 = blockIdx.y * kCgChunk, i1 = min(n, i0 + kCgChunk);
    const double bc = FIRST ? 0.0 : beta[c];
    for (int i = i0; i < i1; ++i) {
        const size_t ic = (size_t)i * n + c;
        if (FIRST) {
            const double e = (i == c) ? 1.0 : 0.0;
            X[ic] = 0.0;
            R[ic] = e;
            P[ic] = e;
        } else {
            P[ic] = fma(bc, P[ic], R[ic]);
        }
    }
}

// inv = S X S
__global__ void unscale_inverse_kernel(int n, const double *sc, const double *X, double *inv)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int i0 = blockIdx.y * kCgChunk, i1 = min(n, i0 + kCgChunk);
    for (int i = i0; i < i1; ++i) {
        const size_t ic = (size_t)i * n + c;
        inv[ic] = sc[i] * X[ic] * sc[c];
    }
}

// The CG path; *taken = false (inv untouched) when the operator does not qualify or CG does
// not reach the accuracy.  mats: four n^2 doubles (X, R, P, Q); aux: n + nnz + (chunks + 4) n
// doubles plus 16 bytes of flags.
cudaError_t cg_inverse(const DevCsr &A, double *mats, double *aux, size_t aux_doubles, double *inv, bool *taken,
                       cudaStream_t s)
{
    *taken = false;
    const int n = A.n;
    const size_t nn = (size_t)n * n;
    const int chunks = (n + kCgChunk - 1) / kCgChunk;
    if (n <= kCgMinRows || (size_t)A.nnz * 8 > nn) return cudaSuccess;
    const size_t need = (size_t)n + 16 + (size_t)A.nnz + 16 + (size_t)(chunks + 4) * n + 16;
    if (need > aux_doubles) return cudaSuccess;
    double *X = mats, *R = X + nn, *P = R + nn, *Q = P + nn;
    double *sc = aux, *sv = sc + n + 16, *part = sv + A.nnz + 16, *rr = part + (size_t)chunks * n;
    double *coef = rr + n;
    int *flags = (int *)(coef + n + 16);
    unsigned long long *bits = (unsigned long long *)(flags + 4);
    AMG_CUDA_TRY(cudaMemsetAsync(flags, 0, 4 * sizeof(int) + 2 * sizeof(unsigned long long), s));
    jacobi_scale_kernel<<<grid_for((int64_t)n * 32, 128), 128, 0, s>>>(n, A.rp, A.ci, A.v, sc, flags); note_launch();
    scale_values_kernel<<<grid_for((int64_t)n * 32, 128), 128, 0, s>>>(n, A.rp, A.ci, A.v, sc, sv); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    int hflag = 0;
    std::vector<int> hrp((size_t)n + 1);
    AMG_CUDA_TRY(cudaMemcpyAsync(&hflag, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(hrp.data(), A.rp, sizeof(int) * ((size_t)n + 1), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (hflag) return cudaSuccess;
    // rows longer than kCgLongRow: summed in segments of kCgSegment entries by blocks of their own
    std::vector<int> lrows, seg_first(1, 0), seg_k0, seg_k1;
    for (int i = 0; i < n; ++i) {
        const int len = hrp[(size_t)i + 1] - hrp[(size_t)i];
        if (len <= kCgLongRow) continue;
        lrows.push_back(i);
        for (int k = hrp[(size_t)i]; k < hrp[(size_t)i + 1]; k += kCgSegment) {
            seg_k0.push_back(k);
            seg_k1.push_back(std::min(k + kCgSegment, hrp[(size_t)i + 1]));
        }
        seg_first.push_back((int)seg_k0.size());
    }
    const int nlong = (int)lrows.size(), nseg = (int)seg_k0.size();
    const int long_len = nlong ? kCgLongRow : 0x7fffffff;
    double *part_long = nullptr;
    int *d_lists = nullptr;
    if (nlong) {
        AMG_CUDA_TRY(cudaMallocAsync(&part_long, sizeof(double) * (size_t)nseg * n, s));
        AMG_CUDA_TRY(cudaMallocAsync(&d_lists, sizeof(int) * (size_t)(2 * nlong + 1 + 2 * nseg), s));
        std::vector<int> packed;
        packed.insert(packed.end(), lrows.begin(), lrows.end());
        packed.insert(packed.end(), seg_first.begin(), seg_first.end());
        packed.insert(packed.end(), seg_k0.begin(), seg_k0.end());
        packed.insert(packed.end(), seg_k1.begin(), seg_k1.end());
        AMG_CUDA_TRY(cudaMemcpyAsync(d_lists, packed.data(), sizeof(int) * packed.size(), cudaMemcpyHostToDevice, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));       // the host vector goes out of scope
    }
    const int *d_lrows = d_lists, *d_segfirst = d_lists + nlong, *d_k0 = d_segfirst + nlong + 1, *d_k1 = d_k0 + nseg;
    struct Release {
        double *p; int *q; cudaStream_t s;
        ~Release() { if (p) cudaFreeAsync(p, s); if (q) cudaFreeAsync(q, s); }
    } release{part_long, d_lists, s};
    auto long_rows_product = [&](const double *Pm, double *Qm) {
        if (!nlong) return;
        cg_long_partial_kernel<<<dim3((n + 255) / 256, nseg), 256, 0, s>>>(n, d_k0, d_k1, A.ci, sv, Pm, part_long);
        note_launch();
        cg_long_reduce_kernel<<<dim3((n + 255) / 256, nlong), 256, 0, s>>>(n, d_lrows, d_segfirst, part_long, Qm);
        note_launch();
    };
    const dim3 blk(256), grd((n + 255) / 256, chunks);
    const int cgrid = (n + 255) / 256;
    cg_direction_kernel<true><<<grd, blk, 0, s>>>(n, nullptr, X, R, P); note_launch();
    std::vector<double> ones((size_t)n, 1.0);
    AMG_CUDA_TRY(cudaMemcpyAsync(rr, ones.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    bool converged = false;
    for (int k = 0; k < kCgMaxSteps && !converged; ++k) {
        if (k > 0) { cg_direction_kernel<false><<<grd, blk, 0, s>>>(n, coef, X, R, P); note_launch(); }
        long_rows_product(P, Q);
        cg_spmm_kernel<0><<<grd, blk, 0, s>>>(n, A.rp, A.ci, sv, P, Q, part, long_len); note_launch();
        cg_reduce_kernel<0><<<cgrid, 256, 0, s>>>(n, chunks, part, rr, coef, flags, bits); note_launch();
        cg_update_kernel<<<grd, blk, 0, s>>>(n, coef, P, Q, X, R, part); note_launch();
        AMG_CUDA_TRY(cudaMemsetAsync(bits, 0, sizeof(unsigned long long), s));
        cg_reduce_kernel<1><<<cgrid, 256, 0, s>>>(n, chunks, part, rr, coef, flags, bits); note_launch();
        AMG_CUDA_TRY(cudaGetLastError());
        if ((k + 1) % kCgCheck == 0 || k + 1 == kCgMaxSteps) {
            unsigned long long hb = 0;
            AMG_CUDA_TRY(cudaMemcpyAsync(&hflag, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
            AMG_CUDA_TRY(cudaMemcpyAsync(&hb, bits, sizeof hb, cudaMemcpyDeviceToHost, s));
            AMG_CUDA_TRY(cudaStreamSynchronize(s));
            if (hflag) return cudaSuccess;                       // not positive definite
            double rmax = 0.0;
            std::memcpy(&rmax, &hb, sizeof rmax);
            if (!(rmax == rmax)) return cudaSuccess;             // NaN
            converged = rmax <= 1e-30;                           // every column's ||r|| <= 1e-15
        }
    }
    if (!converged) return cudaSuccess;
    // the true residual
    AMG_CUDA_TRY(cudaMemsetAsync(bits + 1, 0, sizeof(unsigned long long), s));
    long_rows_product(X, Q);
    cg_spmm_kernel<1><<<grd, blk, 0, s>>>(n, A.rp, A.ci, sv, X, Q, part, long_len); note_launch();
    cg_reduce_kernel<2><<<cgrid, 256, 0, s>>>(n, chunks, part, nullptr, nullptr, nullptr, bits + 1); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    unsigned long long he = 0;
    AMG_CUDA_TRY(cudaMemcpyAsync(&he, bits + 1, sizeof he, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    double err = 0.0;
    std::memcpy(&err, &he, sizeof err);
    if (!(err < 1e-13)) return cudaSuccess;
    unscale_inverse_kernel<<<grd, blk, 0, s>>>(n, sc, X, inv); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    *taken = true;
    return cudaSuccess;
}

template <typename T>
cudaError_t factor_and_invert(int n, T *a, T *lt, T *rdiag, T *inv, int *info, cudaStream_t s)
{
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(inverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kInvSmem);
    });
    AMG_CUDA_TRY(attr);
    const int warps = (int)std::min<size_t>(kInvWarps, (size_t)kInvSmem / ((size_t)n * sizeof(T)));
    if (warps < 1) return cudaErrorInvalidValue;
    for (int j0 = 0; j0 < n; j0 += kPanel) {
        const int b = min(kPanel, n - j0);
        const int rows_below = n - j0 - b;
        const int pblocks = rows_below > 0 ? (rows_below + kPanel - 1) / kPanel : 1;
        panel_kernel<T><<<pblocks, kPanel, 0, s>>>(n, j0, a, info); note_launch();
        if (rows_below > 0) {
            int tiles = (rows_below + 31) / 32;
            trailing_kernel<T><<<dim3(tiles, tiles), 256, 0, s>>>(n, j0, a, info); note_launch();
        }
        AMG_CUDA_TRY(cudaGetLastError());
    }
    const int tb = (n + 31) / 32;
    transpose_lower_kernel<T><<<dim3(tb, tb), 256, 0, s>>>(n, a, lt, rdiag, info); note_launch();
    const size_t smem = (size_t)warps * n * sizeof(T);
    inverse_kernel<T><<<(n + warps - 1) / warps, 32 * warps, smem, s>>>(n, a, lt, rdiag, inv, info); note_launch();
    return cudaGetLastError();
}

size_t coarse_work_bytes(int n)
{
    const size_t nn = (size_t)n * n;
    return sizeof(double) * (4 * nn + n + 16) + sizeof(float) * (3 * nn + n + 16) + 2 * sizeof(NewtonState) + 256;
}

// FP64 Newton-Schulz steps from X (in cur), at most `steps`; the result is in *out.  Returns
// the error of the last iterate checked (the one returned is at least as good).
cudaError_t newton64(int n, const double *Ad, double *cur, double *nxt, double *R, NewtonState *st, int steps,
                     double **out, double *err, cudaStream_t s)
{
    NewtonState init{1e300, 0, 0, 0ULL};   // e_prev, done, last, e_bits
    AMG_CUDA_TRY(cudaMemcpyAsync(st, &init, sizeof init, cudaMemcpyHostToDevice, s));
    const dim3 blk(kGT, kGT), grd((n + kGT - 1) / kGT, (n + kGT - 1) / kGT);
    for (int k = 0; k < steps; ++k) {
        newton_gemm_kernel<double, 0><<<grd, blk, 0, s>>>(n, Ad, cur, R, st); note_launch();
        newton_check_kernel<<<1, 1, 0, s>>>(st); note_launch();
        newton_gemm_kernel<double, 1><<<grd, blk, 0, s>>>(n, cur, R, nxt, st); note_launch();
        std::swap(cur, nxt);
    }
    AMG_CUDA_TRY(cudaGetLastError());
    NewtonState fin{};
    AMG_CUDA_TRY(cudaMemcpyAsync(&fin, st, sizeof fin, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    *out = cur;
    *err = fin.e_prev;
    return cudaSuccess;
}

cudaError_t coarse_inverse(const DevCsr &A, void *work_v, double *inv, int *info_dev, cudaStream_t s, bool general)
{
    const int n = A.n;
    AMG_CUDA_TRY(cudaMemsetAsync(info_dev, 0, sizeof(int), s));
    if (n == 0) return cudaSuccess;
    const size_t nn = (size_t)n * n;
    double *Ad = (double *)work_v, *X = Ad + nn, *Y = X + nn, *R = Y + nn, *rd = R + nn;
    float *Af = (float *)(rd + n + 16), *Ltf = Af + nn, *rdf = Ltf + nn;
    NewtonState *st = (NewtonState *)(((uintptr_t)(rdf + n + 16) + 15) & ~(uintptr_t)15);
    const int cgrid = (int)std::min<size_t>((nn + 255) / 256, 4096);
    // a large, sparse SPD operator (aggregation stalled on it): the CG path first, in the memory
    // of the dense matrices
    if (!general && n > kCgMinRows && (size_t)A.nnz * 8 <= nn) {
        bool taken = false;
        AMG_CUDA_TRY(cg_inverse(A, Ad, (double *)Af, nn, inv, &taken, s));
        if (taken) return cudaSuccess;
    }
    AMG_CUDA_TRY(cudaMemsetAsync(Ad, 0, sizeof(double) * nn, s));
    dense_from_csr_kernel<<<grid_for((int64_t)n * 32, 128), 128, 0, s>>>(n, A.rp, A.ci, A.v, Ad); note_launch();
    convert_dense_kernel<double, float><<<cgrid, 256, 0, s>>>(nn, Ad, Af); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    if (general) {
        // a nonsymmetric operator: Newton-Schulz from the scaled transpose, first in FP32 until
        // E < 1e-4 (at most kGeneral32 steps), then in FP64
        float *Xf = (float *)Y, *Rf = (float *)Y + nn, *Xf2 = Ltf;
        unsigned long long *sums = (unsigned long long *)(st + 1);
        AMG_CUDA_TRY(cudaMemsetAsync(sums, 0, 2 * sizeof(unsigned long long), s));
        abs_sums_kernel<<<grid_for(n, 128), 128, 0, s>>>(n, Ad, sums); note_launch();
        transpose_seed_kernel<<<cgrid, 256, 0, s>>>(n, Ad, sums, Xf); note_launch();
        NewtonState init{1e300, 0, 0, 0ULL};
        AMG_CUDA_TRY(cudaMemcpyAsync(st, &init, sizeof init, cudaMemcpyHostToDevice, s));
        const dim3 blk(kGT, kGT), grd((n + kGT - 1) / kGT, (n + kGT - 1) / kGT);
        float *cur = Xf, *nxt = Xf2;
        for (int k = 0; k < kGeneral32; ++k) {
            newton_gemm_kernel<float, 0><<<grd, blk, 0, s>>>(n, Af, cur, Rf, st); note_launch();
            newton32_check_kernel<<<1, 1, 0, s>>>(st); note_launch();
            newton_gemm_kernel<float, 1><<<grd, blk, 0, s>>>(n, cur, Rf, nxt, st); note_launch();
            std::swap(cur, nxt);
            if ((k & 7) == 7 && k + 1 < kGeneral32) {
                // every 8 steps: stop once converged (the steps after it would only copy)
                NewtonState now{};
                AMG_CUDA_TRY(cudaMemcpyAsync(&now, st, sizeof now, cudaMemcpyDeviceToHost, s));
                AMG_CUDA_TRY(cudaStreamSynchronize(s));
                if (now.done) break;
            }
        }
        convert_dense_kernel<float, double><<<cgrid, 256, 0, s>>>(nn, cur, X); note_launch();
        AMG_CUDA_TRY(cudaGetLastError());
        double *res = nullptr, err = 0.0;
        AMG_CUDA_TRY(newton64(n, Ad, X, R, (double *)Y, st, kGeneral64, &res, &err, s));
        if (!(err < 1e-6))             // singular, or too ill-conditioned: info = -1 (all bits set)
            return cudaMemsetAsync(info_dev, 0xFF, sizeof(int), s);
        return cudaMemcpyAsync(inv, res, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s);
    }
    // stage 1: FP32 factor and inverse (X0 in Y's memory, as floats)
    float *Xf = (float *)Y;
    AMG_CUDA_TRY(factor_and_invert<float>(n, Af, Ltf, rdf, Xf, info_dev, s));
    int info = 0;
    AMG_CUDA_TRY(cudaMemcpyAsync(&info, info_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    bool refined = false;
    if (info == 0) {
        // stage 2: Newton-Schulz in FP64 from X0
        convert_dense_kernel<float, double><<<cgrid, 256, 0, s>>>(nn, Xf, X); note_launch();
        AMG_CUDA_TRY(cudaGetLastError());
        double *res = nullptr, err = 0.0;
        AMG_CUDA_TRY(newton64(n, Ad, X, Y, R, st, kNewtonSteps, &res, &err, s));
        refined = err < 1e-6;
        if (refined) AMG_CUDA_TRY(cudaMemcpyAsync(inv, res, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
    }
    if (refined) return cudaSuccess;
    // the direct FP64 path
    AMG_CUDA_TRY(cudaMemsetAsync(info_dev, 0, sizeof(int), s));
    return factor_and_invert<double>(n, Ad, X, rd, inv, info_dev, s);
}

}  // namespace amgk
