// multi.cu -- several right-hand sides of one system solved together (no counterpart in the
// paper; each column's arithmetic is that of amg_solve: PCG with one V-cycle of Algorithm 1
// per iteration, §3.1's smoother and coarse solve).
//
// The k columns live interleaved (entry i of column c at i K + c, K = 2, 4 or 8 >= k), so that
// every sparse product of the V-cycle and of the PCG reads each matrix entry once and gathers
// K contiguous values per column index: the matrix traffic of k solves is paid once.  Each
// column keeps its own PCG scalars and stopping test and stops at the iteration it would stop
// alone; a stopped column's x, r and p are no longer updated (its slots in the products are
// computed and ignored).  Padding columns (k < K) start with b = 0 and never run.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "hierarchy.cuh"
#include "tma.cuh"

namespace amgk {

struct MScal {          // per column (device)
    double rz, rz_next, rz_new, rz_cross, pq, alpha, beta, active;
};

namespace {

constexpr unsigned kAllM = 0xffffffffu;

double now_ms_host()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
constexpr int kMT = 256;                 // threads per block of the product kernels
constexpr int kMaxTileM = 6144;
enum { MM_Y = 0, MM_RESID = 1, MM_CHEB = 2, MM_PROLONG = 3, MM_DOT = 4 };

// per-column fixed-order block sum (every thread gets the block's K totals)
template <int K>
__device__ __forceinline__ void block_sums(double (&v)[K], double (&out)[K])
{
    __shared__ double sh[kMT / 32][K];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < K; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(kAllM, v[c], o);
        if (lane == 0) sh[w][c] = v[c];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < K; ++c) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q][c];
        out[c] = t;
    }
    __syncthreads();
}

// Y = A X (K columns) over the rows of one block, the block's value and column ranges staged in
// shared memory by two bulk copies (as the single-vector tile SpMV).  Modes: Y; RESID y = f - AX;
// CHEB r = f - AX, d = c1 d + c2 D^-1 r, y = x + d; PROLONG y += AX; DOT y = AX and per-column
// partial[c * gridDim + block] = sum over the block's rows of x_ic y_ic.
template <typename T, int LPR, int MODE, int K>
__global__ void __launch_bounds__(kMT) spmm_tile_kernel(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                         const T *__restrict__ v, const T *__restrict__ x, T *y,
                                                         const T *__restrict__ f, const T *__restrict__ invd, T *d,
                                                         T c1, T c2, int cap, double *partial, int *err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    constexpr int RPB = kMT / LPR;
    constexpr int VA = 16 / (int)sizeof(T);
    const int r0 = blockIdx.x * RPB;
    const int r1 = min(n, r0 + RPB);
    const int k0 = rp[r0], k1 = rp[r1];
    const int k0v = k0 & ~(VA - 1), k1v = (k1 + VA - 1) & ~(VA - 1);
    const int k0i = k0 & ~3, k1i = (k1 + 3) & ~3;
    const bool staged = cap > 0 && (k1v - k0v) <= cap + 2 * VA && (k1i - k0i) <= cap + 8 && k1 > k0;
    T *sv = (T *)smem;
    int *sc = (int *)(smem + tile_values_bytes<T>(cap));
    bool tile_ok = true;
    if (staged) {
        if (threadIdx.x == 0) mbar_init(&bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned bv = (unsigned)((k1v - k0v) * (int)sizeof(T)), bi = (unsigned)((k1i - k0i) * 4);
            mbar_expect_tx(&bar, bv + bi);
            bulk_g2s(sv, v + k0v, bv, &bar);
            bulk_g2s(sc, ci + k0i, bi, &bar);
        }
        tile_ok = __syncthreads_and(mbar_wait_bounded(&bar, 0, err));
    }
    const int row = r0 + threadIdx.x / LPR;
    const int lane = threadIdx.x % LPR;
    T acc[K];
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = T(0);
    if (row < r1 && tile_ok) {
        const int b = rp[row], e = rp[row + 1];
        for (int k = b + lane; k < e; k += LPR) {
            const T a = staged ? sv[k - k0v] : v[k];
            const T *xc = x + (size_t)(staged ? sc[k - k0i] : ci[k]) * K;
#pragma unroll
            for (int c = 0; c < K; ++c) acc[c] += a * xc[c];
        }
    }
#pragma unroll
    for (int c = 0; c < K; ++c)
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(kAllM, acc[c], o, LPR);
    double contrib[K];
#pragma unroll
    for (int c = 0; c < K; ++c) contrib[c] = 0.0;
    if (row < r1 && lane == 0 && tile_ok) {
        const size_t o = (size_t)row * K;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            if (MODE == MM_Y) {
                y[o + c] = acc[c];
            } else if (MODE == MM_RESID) {
                y[o + c] = f[o + c] - acc[c];
            } else if (MODE == MM_CHEB) {
                const T r = f[o + c] - acc[c];
                const T dn = c1 * d[o + c] + c2 * (invd[row] * r);
                d[o + c] = dn;
                y[o + c] = x[o + c] + dn;
            } else if (MODE == MM_PROLONG) {
                y[o + c] += acc[c];
            } else {
                y[o + c] = acc[c];
                contrib[c] = (double)x[o + c] * (double)acc[c];
            }
        }
    }
    if (MODE == MM_DOT) {
        double tot[K];
        block_sums<K>(contrib, tot);
        if (threadIdx.x == 0)
#pragma unroll
            for (int c = 0; c < K; ++c) partial[(size_t)c * gridDim.x + blockIdx.x] = tot[c];
    }
}

// The same products on the level's sliced-ELL copy (slices of 32 rows stored column-major, one
// lane per row: coalesced loads of values and columns), FP64, for Y, RESID, CHEB and DOT: a row's
// entries 0, 2, 4, ... and 1, 3, 5, ... are summed apart and added at the end, the arithmetic of
// spmm_tile_kernel with two lanes per row, and DOT rebuilds that kernel's per-128-row partials
// with its shuffle tree and order of warps: the same bits as the CSR form.
constexpr int kSliceRowsM = 32;
template <typename T, int MODE, int K>
__global__ void __launch_bounds__(kMT) spmm_sell_kernel(int n, const int *__restrict__ sp, const int *__restrict__ sw,
                                                         const int *__restrict__ sci, const T *__restrict__ sv,
                                                         const T *__restrict__ x, T *y, const T *__restrict__ f,
                                                         const T *__restrict__ invd, T *d, T c1, T c2,
                                                         double *partial, int nparts)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slice = blockIdx.x * (kMT / kSliceRowsM) + warp;
    const int row = slice * kSliceRowsM + lane;
    T acc[K];
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = T(0);
    if (slice * kSliceRowsM < n) {
        const int base = sp[slice] + lane, w = sw[slice];
        T s0[K], s1[K];
#pragma unroll
        for (int c = 0; c < K; ++c) { s0[c] = T(0); s1[c] = T(0); }
        int k = 0;
        for (; k + 1 < w; k += 2) {
            const T a0 = sv[base + kSliceRowsM * k], a1 = sv[base + kSliceRowsM * (k + 1)];
            const T *x0 = x + (size_t)sci[base + kSliceRowsM * k] * K;
            const T *x1 = x + (size_t)sci[base + kSliceRowsM * (k + 1)] * K;
#pragma unroll
            for (int c = 0; c < K; ++c) {
                s0[c] += a0 * x0[c];
                s1[c] += a1 * x1[c];
            }
        }
        if (k < w) {
            const T a0 = sv[base + kSliceRowsM * k];
            const T *x0 = x + (size_t)sci[base + kSliceRowsM * k] * K;
#pragma unroll
            for (int c = 0; c < K; ++c) s0[c] += a0 * x0[c];
        }
#pragma unroll
        for (int c = 0; c < K; ++c) acc[c] = s0[c] + s1[c];
    }
    double contrib[K];
#pragma unroll
    for (int c = 0; c < K; ++c) contrib[c] = 0.0;
    if (row < n) {
        const size_t o = (size_t)row * K;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            if (MODE == MM_Y) {
                y[o + c] = acc[c];
            } else if (MODE == MM_RESID) {
                y[o + c] = f[o + c] - acc[c];
            } else if (MODE == MM_CHEB) {
                const T r = f[o + c] - acc[c];
                const T dn = c1 * d[o + c] + c2 * (invd[row] * r);
                d[o + c] = dn;
                y[o + c] = x[o + c] + dn;
            } else {
                y[o + c] = acc[c];
                contrib[c] = (double)x[o + c] * (double)acc[c];
            }
        }
    }
    if (MODE == MM_DOT) {
        // CSR block b covers rows 128 b ... 128 b + 127, its warp w rows 16 w ... 16 w + 15 with
        // row j's term on lane 2 j; this block's rows are CSR blocks 2 blockIdx and 2 blockIdx + 1
        __shared__ double con[K][kMT];
        __shared__ double wsum[2][kMT / 32][K];
#pragma unroll
        for (int c = 0; c < K; ++c) con[c][threadIdx.x] = contrib[c];
        __syncthreads();
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
#pragma unroll
            for (int c = 0; c < K; ++c) {
                double v = (lane & 1) ? 0.0 : con[c][128 * hh + 16 * warp + (lane >> 1)];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kAllM, v, o);
                if (lane == 0) wsum[hh][warp][c] = v;
            }
        }
        __syncthreads();
        if (threadIdx.x < 2 * K) {
            const int hh = threadIdx.x / K, c = threadIdx.x % K;
            const int part = 2 * blockIdx.x + hh;
            if (part < nparts) {
                double t = 0.0;
                for (int q = 0; q < kMT / 32; ++q) t += wsum[hh][q][c];
                partial[(size_t)c * nparts + part] = t;
            }
        }
    }
}

template <typename T>
const T *sell_values_m(const SpmvPlan &pl);
template <>
const double *sell_values_m<double>(const SpmvPlan &pl) { return pl.sv64; }
template <>
const float *sell_values_m<float>(const SpmvPlan &pl) { return pl.sv32; }

template <typename T, int MODE, int K>
cudaError_t spmm(const SpmvPlan &pl, int n, const int *rp, const int *ci, const T *v, const T *x, T *y, const T *f,
                 const T *invd, T *d, T c1, T c2, double *partial, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    // FP64 only: with FP32 values the staged CSR tiles below were faster (1.51x against 1.11x
    // for eight right-hand sides of the 64^3 stretched cube against one at a time)
    if (sizeof(T) == 8 && MODE != MM_PROLONG && pl.ns > 0 && pl.lpr == 2 && pl.lr.count == 0 &&
        sell_values_m<T>(pl)) {
        const int blocks = (pl.ns + kMT / kSliceRowsM - 1) / (kMT / kSliceRowsM);
        const int nparts = (n + kMT / 2 - 1) / (kMT / 2);
        spmm_sell_kernel<T, MODE, K><<<blocks, kMT, 0, s>>>(n, pl.sp, pl.sw, pl.sci, sell_values_m<T>(pl), x, y, f,
                                                           invd, d, c1, c2, partial, nparts);
        note_launch();
        return cudaGetLastError();
    }
    const int smem = tile_bytes<T>(pl.cap);
    auto go = [&](auto kern, int lpr) -> cudaError_t {
        // the shared-memory limit is raised once per instantiation (no API call inside a capture)
        static std::once_flag once[5];
        static cudaError_t cfg[5];
        const int slot = lpr == 2 ? 0 : lpr == 4 ? 1 : lpr == 8 ? 2 : lpr == 16 ? 3 : 4;
        std::call_once(once[slot], [&] {
            cfg[slot] = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             tile_bytes<T>(kMaxTileM));
        });
        AMG_CUDA_TRY(cfg[slot]);
        const int blocks = (n + kMT / lpr - 1) / (kMT / lpr);
        kern<<<blocks, kMT, smem, s>>>(n, rp, ci, v, x, y, f, invd, d, c1, c2, pl.cap, partial, spmv_error_flag());
        note_launch();
        return cudaGetLastError();
    };
    switch (pl.lpr) {
    case 2: return go(spmm_tile_kernel<T, 2, MODE, K>, 2);
    case 4: return go(spmm_tile_kernel<T, 4, MODE, K>, 4);
    case 8: return go(spmm_tile_kernel<T, 8, MODE, K>, 8);
    case 16: return go(spmm_tile_kernel<T, 16, MODE, K>, 16);
    default: return go(spmm_tile_kernel<T, 32, MODE, K>, 32);
    }
}

// first Chebyshev step from x = 0 on K columns: d = D^-1 f / theta, x = d
template <typename T, int K>
__global__ void mcheb0_kernel(int n, const T *f, const T *invd, T inv_theta, T *d, T *x)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * K; e += (size_t)gridDim.x * blockDim.x) {
        const T di = (invd[e / K] * f[e]) * inv_theta;
        d[e] = di;
        x[e] = di;
    }
}

// coarsest level, K columns: x = Ainv f, one warp per row (FP64 sums)
template <typename T, int K>
__global__ void mcoarse_kernel(int n, const double *__restrict__ inv, const T *__restrict__ f, T *x)
{
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    double acc[K];
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = 0.0;
    for (int k = lane; k < n; k += 32) {
        const double a = inv[(size_t)row * n + k];
#pragma unroll
        for (int c = 0; c < K; ++c) acc[c] += a * (double)f[(size_t)k * K + c];
    }
#pragma unroll
    for (int c = 0; c < K; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(kAllM, acc[c], o);
        if (lane == 0) x[(size_t)row * K + c] = (T)acc[c];
    }
}

template <typename A, typename B>
__global__ void mconvert_kernel(size_t count, const A *src, B *dst)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
        dst[e] = (B)src[e];
}

// ------------------------------------------------------------------------------------ PCG, K columns
// partial[c * count + i] summed in index order by every block (the same total everywhere)
template <int K>
__device__ __forceinline__ void sums_all(const double *partial, int count, double (&out)[K])
{
    double a[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        a[c] = 0.0;
        for (int i = threadIdx.x; i < count; i += blockDim.x) a[c] += partial[(size_t)c * count + i];
    }
    block_sums<K>(a, out);
}

// per-column a . b over rows (interleaved), fixed-order: block partials, then every caller of
// sums_all adds them in block order
template <int K>
__global__ void __launch_bounds__(kMT) mdot_kernel(int n, const double *a, const double *b, double *partial)
{
    double acc[K];
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = 0.0;
    for (int i = blockIdx.x * kMT + threadIdx.x; i < n; i += gridDim.x * kMT)
#pragma unroll
        for (int c = 0; c < K; ++c) acc[c] += a[(size_t)i * K + c] * b[(size_t)i * K + c];
    double tot[K];
    block_sums<K>(acc, tot);
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < K; ++c) partial[(size_t)c * gridDim.x + blockIdx.x] = tot[c];
}

// one block: out[c] = sum of partial[c * count + i] (i ascending)
template <int K>
__global__ void __launch_bounds__(kMT) mstore_kernel(const double *partial, int count, double *out, int stride)
{
    double t[K];
    sums_all<K>(partial, count, t);
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < K; ++c) out[(size_t)c * stride] = t[c];
}

// alpha_c = rz_next_c / (p . q)_c; x += alpha p; r -= alpha q on active columns; r . r partials
template <int K>
__global__ void __launch_bounds__(kMT) mxr_kernel(int n, double *x, double *r, const double *p, const double *q,
                                                  MScal *sc, const double *pq_partial, int pq_count,
                                                  double *rr_partial)
{
    double pq[K];
    sums_all<K>(pq_partial, pq_count, pq);
    double alpha[K], act[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        act[c] = sc[c].active;
        alpha[c] = act[c] != 0.0 ? sc[c].rz_next / pq[c] : 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < K; ++c)
            if (act[c] != 0.0) { sc[c].pq = pq[c]; sc[c].alpha = alpha[c]; sc[c].rz = sc[c].rz_next; }
    double acc[K];
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = 0.0;
    for (int i = blockIdx.x * kMT + threadIdx.x; i < n; i += gridDim.x * kMT) {
        const size_t o = (size_t)i * K;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            if (act[c] != 0.0) {
                x[o + c] += alpha[c] * p[o + c];
                r[o + c] = r[o + c] - alpha[c] * q[o + c];
            }
            acc[c] += r[o + c] * r[o + c];
        }
    }
    double tot[K];
    block_sums<K>(acc, tot);
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < K; ++c) rr_partial[(size_t)c * gridDim.x + blockIdx.x] = tot[c];
}

// r . z and r . z_prev per column (partials), then (second kernel) beta and p = z + beta p
template <int K>
__global__ void __launch_bounds__(kMT) mrz_kernel(int n, const double *r, const double *z, const double *zp,
                                                  double *pa, double *pb)
{
    double a[K], b[K];
#pragma unroll
    for (int c = 0; c < K; ++c) { a[c] = 0.0; b[c] = 0.0; }
    for (int i = blockIdx.x * kMT + threadIdx.x; i < n; i += gridDim.x * kMT) {
        const size_t o = (size_t)i * K;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            a[c] += r[o + c] * z[o + c];
            if (zp) b[c] += r[o + c] * zp[o + c];
        }
    }
    double ta[K], tb[K];
    block_sums<K>(a, ta);
    block_sums<K>(b, tb);
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < K; ++c) {
            pa[(size_t)c * gridDim.x + blockIdx.x] = ta[c];
            pb[(size_t)c * gridDim.x + blockIdx.x] = tb[c];
        }
}

template <int K>
__global__ void __launch_bounds__(kMT) mp_kernel(int n, double *p, const double *z, MScal *sc, const double *pa,
                                                 const double *pb, int count, int flexible)
{
    double rzn[K], rzc[K];
    sums_all<K>(pa, count, rzn);
    sums_all<K>(pb, count, rzc);
    double beta[K], act[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        act[c] = sc[c].active;
        beta[c] = act[c] != 0.0 ? (flexible ? rzn[c] - rzc[c] : rzn[c]) / sc[c].rz : 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < K; ++c)
            if (act[c] != 0.0) { sc[c].beta = beta[c]; sc[c].rz_next = rzn[c]; sc[c].rz_new = rzn[c]; }
    for (int i = blockIdx.x * kMT + threadIdx.x; i < n; i += gridDim.x * kMT) {
        const size_t o = (size_t)i * K;
#pragma unroll
        for (int c = 0; c < K; ++c)
            if (act[c] != 0.0) p[o + c] = z[o + c] + beta[c] * p[o + c];
    }
}

// column j (length n, contiguous) <-> interleaved slot j; mask: copy only columns with mask[c]
template <int K>
__global__ void mpack_kernel(int n, const double *col, double *inter, int j)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        inter[(size_t)i * K + j] = col[i];
}
template <int K>
__global__ void munpack_kernel(int n, const double *inter, double *col, int j)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        col[i] = inter[(size_t)i * K + j];
}
template <int K>
__global__ void mactive_kernel(MScal *sc, const int *done)
{
    if (threadIdx.x < K) sc[threadIdx.x].active = done[threadIdx.x] ? 0.0 : 1.0;
}
template <int K>
__global__ void mcopy_cols_kernel(int n, const double *src, double *dst, const int *mask)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * K; e += (size_t)gridDim.x * blockDim.x)
        if (mask[e % K]) dst[e] = src[e];
}

}  // namespace

// work vectors of the multi-column solve, allocated with the hierarchy on first use
struct MultiWork {
    int K = 0;
    void *f[32] = {}, *x[32] = {}, *x2[32] = {}, *r[32] = {}, *d[32] = {};    // V-cycle, per level (T)
    double *b = nullptr, *xs = nullptr, *rs = nullptr, *zb[2] = {}, *p = nullptr, *q = nullptr, *t = nullptr;
    double *partial = nullptr, *pa = nullptr, *pb = nullptr, *rr = nullptr, *tt = nullptr, *bb = nullptr;
    MScal *sc = nullptr;
    int *mask = nullptr;
    double *host = nullptr;      // pinned: rr (K x kReduceBlocks), then per-column scalars
    int nparts = 0;              // partial slots per column of the products
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};   // one iteration (z parity in mixed precision)
    long long gkernels[2] = {0, 0};
    bool graph_failed = false;
};

namespace {

template <typename T>
cudaError_t multi_alloc(amg_hierarchy *h, MultiWork &w, int K)
{
    auto al = [&](void **p, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMallocAsync(p, bytes + 128, h->s);
        if (e == cudaSuccess) {
            h->allocs.push_back(*p);
            h->bytes += bytes + 128;
        }
        return e;
    };
    const size_t ts = sizeof(T);
    for (int L = 0; L < h->nlev; ++L) {
        const size_t n = (size_t)h->lev[L].A.n * K;
        for (void **v : {&w.f[L], &w.x[L], &w.x2[L], &w.r[L], &w.d[L]}) AMG_CUDA_TRY(al(v, n * ts));
    }
    const size_t n0 = (size_t)h->lev[0].A.n * K;
    for (double **v : {&w.b, &w.xs, &w.rs, &w.zb[0], &w.zb[1], &w.p, &w.q, &w.t})
        AMG_CUDA_TRY(al((void **)v, n0 * sizeof(double)));
    // the products' partials: one slot per block at the most lanes per row (8 rows per block)
    int maxb = kReduceBlocks;
    for (int L = 0; L < h->nlev; ++L) maxb = std::max(maxb, (h->lev[L].A.n + kMT / 32 - 1) / (kMT / 32) + 1);
    w.nparts = maxb;
    for (double **v : {&w.partial, &w.pa, &w.pb, &w.rr, &w.tt, &w.bb})
        AMG_CUDA_TRY(al((void **)v, sizeof(double) * (size_t)K * maxb));
    AMG_CUDA_TRY(al((void **)&w.sc, sizeof(MScal) * K));
    AMG_CUDA_TRY(al((void **)&w.mask, sizeof(int) * K));
    AMG_CUDA_TRY(cudaMallocHost(&w.host, sizeof(double) * ((size_t)K * kReduceBlocks + 4 * K)));
    w.K = K;
    return cudaSuccess;
}

struct ChebC {
    double theta, delta, sigma1;
};

template <typename T, int K>
cudaError_t mvcycle_level(const amg_hierarchy *h, MultiWork &w, int L, T **out, cudaStream_t s, T *final_out)
{
    const Level &lv = h->lev[L];
    const SolveCtx &c = h->ctx;
    const LevelView &vw = c.lev[L];
    T *x = (T *)w.x[L], *x2 = (T *)w.x2[L];
    const T *f = (const T *)w.f[L];
    const int n = lv.A.n;
    const bool coarse_cheb = L == h->nlev - 1 && c.coarse_degree > 0;
    if (L == h->nlev - 1 && !coarse_cheb) {
        if (n > 0)
            mcoarse_kernel<T, K><<<grid_for((int64_t)n * 32, 128), 128, 0, s>>>(n, h->coarse_inv, f, x); note_launch();
        *out = x;
        return cudaGetLastError();
    }
    const T *av = (const T *)vw.av, *invd = (const T *)vw.invdiag;
    T *d = (T *)w.d[L];
    const double lmax = c.cheb_boost * vw.lambda, lmin = lmax / c.cheb_ratio;
    // the smoother's interval, or the coarsest level's Chebyshev solve (its own interval and degree)
    const ChebC cc = coarse_cheb ? ChebC{c.coarse_theta, c.coarse_delta, c.coarse_theta / c.coarse_delta}
                                 : ChebC{0.5 * (lmax + lmin), 0.5 * (lmax - lmin), (lmax + lmin) / (lmax - lmin)};
    const int degree = coarse_cheb ? c.coarse_degree : c.cheb_degree;
    auto smooth = [&](bool zero, T *fin) -> cudaError_t {
        double rho = 1.0 / cc.sigma1;
        int k0 = 1;
        if (zero) {
            mcheb0_kernel<T, K><<<grid_for((int64_t)n * K, 256, 8192), 256, 0, s>>>(n, f, invd, (T)(1.0 / cc.theta), d,
                                                                                    x); note_launch();
            AMG_CUDA_TRY(cudaGetLastError());
        } else {
            T *dst = (fin && degree == 1) ? fin : x2;
            AMG_CUDA_TRY((spmm<T, MM_CHEB, K>(vw.plan_a, n, vw.arp, vw.aci, av, x, dst, f, invd, d, (T)0,
                                              (T)(1.0 / cc.theta), nullptr, s)));
            x2 = x;
            x = dst;
        }
        for (int k = k0; k < degree; ++k) {
            const double rho_new = 1.0 / (2.0 * cc.sigma1 - rho);
            const double c1 = rho_new * rho, c2 = 2.0 * rho_new / cc.delta;
            T *dst = (fin && k == degree - 1) ? fin : x2;
            AMG_CUDA_TRY((spmm<T, MM_CHEB, K>(vw.plan_a, n, vw.arp, vw.aci, av, x, dst, f, invd, d, (T)c1, (T)c2,
                                              nullptr, s)));
            x2 = x;
            x = dst;
            rho = rho_new;
        }
        return cudaSuccess;
    };
    AMG_CUDA_TRY(smooth(true, nullptr));
    if (coarse_cheb) {
        *out = x;
        return cudaSuccess;
    }
    const Level &cl = h->lev[L + 1];
    T *rv = (T *)w.r[L];
    AMG_CUDA_TRY((spmm<T, MM_RESID, K>(vw.plan_a, n, vw.arp, vw.aci, av, x, rv, f, nullptr, nullptr, (T)0, (T)0,
                                       nullptr, s)));
    AMG_CUDA_TRY((spmm<T, MM_Y, K>(vw.plan_r, cl.A.n, vw.rrp, vw.rci, (const T *)vw.rv, rv, (T *)w.f[L + 1], nullptr,
                                   nullptr, nullptr, (T)0, (T)0, nullptr, s)));
    T *xc = nullptr;
    AMG_CUDA_TRY((mvcycle_level<T, K>(h, w, L + 1, &xc, s, nullptr)));
    AMG_CUDA_TRY((spmm<T, MM_PROLONG, K>(vw.plan_p, n, vw.prp, vw.pci, (const T *)vw.pv, xc, x, nullptr, nullptr,
                                         nullptr, (T)0, (T)0, nullptr, s)));
    AMG_CUDA_TRY(smooth(false, final_out));
    *out = x;
    return cudaSuccess;
}

// z = V(r) on K columns (r, z interleaved FP64)
template <int K>
cudaError_t mvcycle(amg_hierarchy *h, MultiWork &w, const double *r, double *z, cudaStream_t s)
{
    const int n = h->lev[0].A.n;
    const size_t nk = (size_t)n * K;
    const int g = (int)std::min<size_t>((nk + 255) / 256, 8192);
    if (!h->ctx.mixed) {
        AMG_CUDA_TRY(cudaMemcpyAsync(w.f[0], r, sizeof(double) * nk, cudaMemcpyDeviceToDevice, s));
        double *out = nullptr;
        AMG_CUDA_TRY((mvcycle_level<double, K>(h, w, 0, &out, s, h->nlev > 1 ? z : nullptr)));
        if (out == z) return cudaSuccess;
        return cudaMemcpyAsync(z, out, sizeof(double) * nk, cudaMemcpyDeviceToDevice, s);
    }
    mconvert_kernel<double, float><<<g, 256, 0, s>>>(nk, r, (float *)w.f[0]); note_launch();
    float *out = nullptr;
    AMG_CUDA_TRY((mvcycle_level<float, K>(h, w, 0, &out, s, nullptr)));
    mconvert_kernel<float, double><<<g, 256, 0, s>>>(nk, out, z); note_launch();
    return cudaGetLastError();
}

// q = A p with the per-column p . q, then x, r and the r . r partials (copied to the host)
template <int K>
cudaError_t mhead(amg_hierarchy *h, MultiWork &w, cudaStream_t s)
{
    const Level &l0 = h->lev[0];
    const int n = l0.A.n;
    AMG_CUDA_TRY((spmm<double, MM_DOT, K>(h->plan0, n, l0.A.rp, l0.A.ci, l0.A.v, w.p, w.q, nullptr, nullptr, nullptr,
                                          0.0, 0.0, w.partial, s)));
    mxr_kernel<K><<<kReduceBlocks, kMT, 0, s>>>(n, w.xs, w.rs, w.p, w.q, w.sc, w.partial,
                                                spmv_block_count(n, h->plan0), w.rr); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    return cudaMemcpyAsync(w.host, w.rr, sizeof(double) * (size_t)K * kReduceBlocks, cudaMemcpyDeviceToHost, s);
}

// z = M r, the per-column r . z (and r . z_prev), p = z + beta p
template <int K>
cudaError_t mtail(amg_hierarchy *h, MultiWork &w, int parity, cudaStream_t s)
{
    const int n = h->lev[0].A.n;
    const bool flexible = h->ctx.mixed != 0;
    double *z = w.zb[parity], *zp = flexible ? w.zb[1 - parity] : nullptr;
    AMG_CUDA_TRY(mvcycle<K>(h, w, w.rs, z, s));
    mrz_kernel<K><<<kReduceBlocks, kMT, 0, s>>>(n, w.rs, z, zp, w.pa, w.pb); note_launch();
    mp_kernel<K><<<kReduceBlocks, kMT, 0, s>>>(n, w.p, z, w.sc, w.pa, w.pb, kReduceBlocks, zp ? 1 : 0); note_launch();
    return cudaGetLastError();
}

// one iteration (tail, then head) as a CUDA graph, captured on first use
template <int K>
cudaGraphExec_t mgraph(amg_hierarchy *h, MultiWork &w, int parity)
{
    if (w.graph_failed || !h->cap) return nullptr;
    if (w.gexec[parity]) return w.gexec[parity];
    cudaGraph_t g = nullptr;
    const long long before = launch_count();
    cudaError_t e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = mtail<K>(h, w, parity, h->cap);
        cudaError_t e2 = e1 == cudaSuccess ? mhead<K>(h, w, h->cap) : e1;
        e = cudaStreamEndCapture(h->cap, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&w.gexec[parity], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        w.graph_failed = true;      // iterations run eagerly from now on
        w.gexec[parity] = nullptr;
        return nullptr;
    }
    w.gkernels[parity] = launch_count() - before;
    note_launches(-w.gkernels[parity]);
    return w.gexec[parity];
}

void drop_multi_graphs(MultiWork &w)
{
    for (int k = 0; k < 2; ++k) {
        if (w.gexec[k]) cudaGraphExecDestroy(w.gexec[k]);
        w.gexec[k] = nullptr;
    }
}

#define MK(expr)                                                           \
    do {                                                                   \
        cudaError_t _e = (expr);                                           \
        if (_e != cudaSuccess) return fail_cuda(_e, #expr);                \
    } while (0)

// ||b_c - A x_c|| for every column into host tt[c] (t holds the residuals)
template <int K>
amg_status_t mresidual(amg_hierarchy *h, MultiWork &w, const double *xs, double *tt_host, cudaStream_t s)
{
    const Level &l0 = h->lev[0];
    const int n = l0.A.n;
    MK((spmm<double, MM_RESID, K>(h->plan0, n, l0.A.rp, l0.A.ci, l0.A.v, xs, w.t, w.b, nullptr, nullptr, 0.0, 0.0,
                                  nullptr, s)));
    mdot_kernel<K><<<kReduceBlocks, kMT, 0, s>>>(n, w.t, w.t, w.partial); note_launch();
    mstore_kernel<K><<<1, kMT, 0, s>>>(w.partial, kReduceBlocks, w.tt, 1); note_launch();
    MK(cudaGetLastError());
    MK(cudaMemcpyAsync(tt_host, w.tt, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
    MK(cudaStreamSynchronize(s));
    return AMG_OK;
}

template <int K>
amg_status_t solve_k(amg_hierarchy *h, int k, const double *B, double *X, double tol, amg_info_t *infos)
{
    cudaStream_t s = h->s;
    const double t0 = now_ms_host();
    if (!h->multi) h->multi = new MultiWork();
    MultiWork &w = *h->multi;
    if (w.K != K) {
        if (w.K != 0) {
            // another width was used before: start over with fresh vectors (the old ones stay
            // with the hierarchy until it is freed)
            drop_multi_graphs(w);
            if (w.host) cudaFreeHost(w.host);
            w = MultiWork();
        }
        cudaError_t e = h->ctx.mixed ? multi_alloc<float>(h, w, K) : multi_alloc<double>(h, w, K);
        if (e != cudaSuccess) return fail_cuda(e, "amg_solve_multi");
    }
    const Level &l0 = h->lev[0];
    const int n = l0.A.n;
    const size_t nk = (size_t)n * K;
    const int gp = grid_for(n, 256, 8192);
    std::vector<int> iters(K, 0), done(K, 0);
    std::vector<amg_status_t> res(K, AMG_ERR_NOT_CONVERGED);
    std::vector<double> nb(K, 0.0), tt(K, 0.0), relres(K, 0.0);
    std::vector<double> col((size_t)n);
    std::vector<MScal> scal(K);
    std::vector<int> mask(K, 0);
    int it = 0;
    // b (padding columns zero), x = 0, r = b
    MK(cudaMemsetAsync(w.b, 0, sizeof(double) * nk, s));
    for (int j = 0; j < k; ++j) {
        MK(copy_to_device(w.t, B + (size_t)j * n, sizeof(double) * (size_t)n, s));
        mpack_kernel<K><<<gp, 256, 0, s>>>(n, w.t, w.b, j); note_launch();
    }
    MK(cudaMemsetAsync(w.xs, 0, sizeof(double) * nk, s));
    MK(cudaMemcpyAsync(w.rs, w.b, sizeof(double) * nk, cudaMemcpyDeviceToDevice, s));
    mdot_kernel<K><<<kReduceBlocks, kMT, 0, s>>>(n, w.b, w.b, w.partial); note_launch();
    mstore_kernel<K><<<1, kMT, 0, s>>>(w.partial, kReduceBlocks, w.bb, 1); note_launch();
    MK(cudaGetLastError());
    MK(cudaMemcpyAsync(tt.data(), w.bb, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
    MK(cudaStreamSynchronize(s));
    int live = 0;
    for (int c = 0; c < K; ++c) {
        nb[c] = std::sqrt(tt[c]);
        if (c >= k || nb[c] == 0.0) {
            done[c] = 1;
            res[c] = AMG_OK;
        } else {
            ++live;
        }
        scal[c] = MScal{0, 0, 0, 0, 0, 0, 0, done[c] ? 0.0 : 1.0};
    }
    const bool flexible = h->ctx.mixed != 0;
    double *z0 = w.zb[0];
    if (live > 0) {
        MK(cudaMemcpyAsync(w.sc, scal.data(), sizeof(MScal) * K, cudaMemcpyHostToDevice, s));
        // z = M r, p = z, rz_next = r . z
        MK(mvcycle<K>(h, w, w.rs, z0, s));
        MK(cudaMemcpyAsync(w.p, z0, sizeof(double) * nk, cudaMemcpyDeviceToDevice, s));
        mdot_kernel<K><<<kReduceBlocks, kMT, 0, s>>>(n, w.rs, z0, w.partial); note_launch();
        mstore_kernel<K><<<1, kMT, 0, s>>>(w.partial, kReduceBlocks, &w.sc[0].rz_next, sizeof(MScal) / sizeof(double));
        note_launch();
        if (flexible) MK(cudaMemsetAsync(w.zb[1], 0, sizeof(double) * nk, s));
        MK(cudaGetLastError());
    }
    if (live > 0 && h->p.max_iter > 0) {
        MK(mhead<K>(h, w, s));
        ++it;
    }
    while (live > 0 && it > 0) {
        MK(cudaStreamSynchronize(s));
        std::fill(mask.begin(), mask.end(), 0);
        bool any = false;
        for (int c = 0; c < K; ++c) {
            if (done[c]) continue;
            double rr = 0.0;
            for (int q = 0; q < kReduceBlocks; ++q) rr += w.host[(size_t)c * kReduceBlocks + q];
            if (std::sqrt(rr) / nb[c] <= tol) { mask[c] = 1; any = true; }
        }
        if (any) {
            // the recurrence says converged: check b - A x of those columns
            amg_status_t st = mresidual<K>(h, w, w.xs, tt.data(), s);
            if (st != AMG_OK) return st;
            bool replace = false;
            for (int c = 0; c < K; ++c) {
                if (!mask[c]) continue;
                if (std::sqrt(tt[c]) / nb[c] <= tol) {
                    done[c] = 1;
                    res[c] = AMG_OK;
                    iters[c] = it;
                    --live;
                    mask[c] = 0;
                } else {
                    replace = true;
                }
            }
            if (replace) {
                MK(cudaMemcpyAsync(w.mask, mask.data(), sizeof(int) * K, cudaMemcpyHostToDevice, s));
                mcopy_cols_kernel<K><<<grid_for((int64_t)nk, 256, 8192), 256, 0, s>>>(n, w.t, w.rs, w.mask); note_launch();
                MK(cudaGetLastError());
            }
            // stopped columns: no further updates
            MK(cudaMemcpyAsync(w.mask, done.data(), sizeof(int) * K, cudaMemcpyHostToDevice, s));
            mactive_kernel<K><<<1, 32, 0, s>>>(w.sc, w.mask); note_launch();
            MK(cudaGetLastError());
        }
        if (live == 0 || it >= h->p.max_iter) break;
        const int parity = flexible ? (it & 1) : 0;
        cudaGraphExec_t gx = mgraph<K>(h, w, parity);
        if (gx) {
            MK(cudaGraphLaunch(gx, s));
            note_launches(w.gkernels[parity]);
        } else {
            MK(mtail<K>(h, w, parity, s));
            MK(mhead<K>(h, w, s));
        }
        ++it;
    }
    for (int c = 0; c < K; ++c)
        if (!done[c]) iters[c] = it;
    // true residuals and the solutions
    {
        amg_status_t st = mresidual<K>(h, w, w.xs, tt.data(), s);
        if (st != AMG_OK) return st;
        for (int j = 0; j < k; ++j) {
            relres[j] = nb[j] > 0.0 ? std::sqrt(tt[j]) / nb[j] : 0.0;
            munpack_kernel<K><<<gp, 256, 0, s>>>(n, w.xs, w.t, j); note_launch();
            MK(cudaGetLastError());
            MK(copy_to_host(X + (size_t)j * n, w.t, sizeof(double) * (size_t)n, s));
        }
    }
    amg_status_t overall = AMG_OK;
    for (int j = 0; j < k; ++j)
        if (res[j] != AMG_OK) overall = res[j];
    if (spmv_take_errors(s) != 0) {
        set_last_error("a bulk copy into shared memory did not complete in time");
        overall = AMG_ERR_INTERNAL;
    }
    if (infos) {
        double tot = 0.0;
        for (int L = 0; L < h->nlev; ++L) tot += (double)h->lev[L].A.nnz;
        for (int j = 0; j < k; ++j) {
            infos[j].iters = iters[j];
            infos[j].status = overall == AMG_ERR_INTERNAL ? AMG_ERR_INTERNAL : res[j];
            infos[j].relres_true = relres[j];
            infos[j].setup_ms = h->setup_ms;
            infos[j].solve_ms = now_ms_host() - t0;
            infos[j].levels = h->nlev;
            infos[j].op_complexity = h->fine_nnz > 0 ? tot / (double)h->fine_nnz : 0.0;
        }
    }
    return overall;
}

#undef MK

}  // namespace

void multi_release(amg_hierarchy *h)
{
    if (!h->multi) return;
    drop_multi_graphs(*h->multi);
    if (h->multi->host) cudaFreeHost(h->multi->host);
    delete h->multi;
    h->multi = nullptr;
}

}  // namespace amgk

using namespace amgk;

extern "C" amg_status_t amg_solve_multi(amg_handle_t h, int k, const double *B, double *X, double tol,
                                        amg_info_t *infos)
{
    if (!h || k < 0 || k > 8 || !(tol >= 0.0)) return AMG_ERR_INVALID_ARG;
    if (h->p.krylov != AMG_KRYLOV_CG) {
        set_last_error("several right-hand sides at once are solved by PCG only");
        return AMG_ERR_UNSUPPORTED;
    }
    if (k == 0) return AMG_OK;
    if (h->lev[0].A.n > 0 && (!B || !X)) return AMG_ERR_INVALID_ARG;
    if (k <= 2) return solve_k<2>(h, k, B, X, tol, infos);
    if (k <= 4) return solve_k<4>(h, k, B, X, tol, infos);
    return solve_k<8>(h, k, B, X, tol, infos);
}
