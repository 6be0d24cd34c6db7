// solve.cu -- solve-phase kernels: CSR SpMV with fused epilogues (residual, Chebyshev step,
// prolongation, dot product), the V-cycle of Algorithm 1 with degree-k Chebyshev smoothing,
// the coarsest-level dense solve and the PCG vector updates.
//
// SpMV layout: a group of LANES consecutive lanes per row (LANES in {4, 8, 16, 32}), lanes
// stride over the row's entries (coalesced column/value loads), partial sums combined with
// xor shuffles inside the group.  The working type T is double (FP64 path) or float (the
// mixed path's V-cycle); accumulation is in T.
#include "amg_internal.cuh"

namespace amgk {

constexpr unsigned kAll = 0xffffffffu;

enum SpmvMode {
    MODE_Y = 0,          // y = A x
    MODE_RESID = 1,      // y = f - A x
    MODE_CHEB = 2,       // r = f - A x; d = c1 d + c2 D^-1 r; y = x + d
    MODE_PROLONG = 3,    // y += A x
};

struct ChebArgs {
    const void *f = nullptr;
    const void *invdiag = nullptr;
    void *d = nullptr;
    double c1 = 0.0, c2 = 0.0;
};

template <typename T, int LANES, int MODE>
__global__ void __launch_bounds__(256) spmv_kernel(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                   const T *__restrict__ v, const T *__restrict__ x, T *y,
                                                   const T *__restrict__ f, const T *__restrict__ invdiag, T *d,
                                                   T c1, T c2)
{
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = gtid / LANES;
    const int sub = threadIdx.x & (LANES - 1);
    T sum = T(0);
    if (row < n) {
        const int b = rp[row], e = rp[row + 1];
        for (int k = b + sub; k < e; k += LANES) sum += v[k] * x[ci[k]];
    }
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(kAll, sum, o, LANES);
    if (row < n && sub == 0) {
        if (MODE == MODE_Y) {
            y[row] = sum;
        } else if (MODE == MODE_RESID) {
            y[row] = f[row] - sum;
        } else if (MODE == MODE_CHEB) {
            T r = f[row] - sum;
            T dn = c1 * d[row] + c2 * (invdiag[row] * r);
            d[row] = dn;
            y[row] = x[row] + dn;
        } else {
            y[row] += sum;
        }
    }
}

template <typename T, int MODE>
cudaError_t spmv_launch_mode(int lanes, int n, const int *rp, const int *ci, const T *v, const T *x, T *y, const T *f,
                             const T *invdiag, T *d, T c1, T c2, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = grid_for((int64_t)n * lanes, threads);
    switch (lanes) {
    case 4: spmv_kernel<T, 4, MODE><<<blocks, threads, 0, s>>>(n, rp, ci, v, x, y, f, invdiag, d, c1, c2); note_launch(); break;
    case 8: spmv_kernel<T, 8, MODE><<<blocks, threads, 0, s>>>(n, rp, ci, v, x, y, f, invdiag, d, c1, c2); note_launch(); break;
    case 16: spmv_kernel<T, 16, MODE><<<blocks, threads, 0, s>>>(n, rp, ci, v, x, y, f, invdiag, d, c1, c2); note_launch(); break;
    default: spmv_kernel<T, 32, MODE><<<blocks, threads, 0, s>>>(n, rp, ci, v, x, y, f, invdiag, d, c1, c2); note_launch(); break;
    }
    return cudaGetLastError();
}

int pick_lanes(double avg_row)
{
    if (avg_row <= 6.0) return 4;
    if (avg_row <= 12.0) return 8;
    if (avg_row <= 40.0) return 16;
    return 32;
}

// ------------------------------------------------------------------------------------ FP64 entry points
cudaError_t spmv_d(const DevCsr &A, int lanes, const double *x, double *y, cudaStream_t s)
{
    return spmv_launch_mode<double, MODE_Y>(lanes, A.n, A.rp, A.ci, A.v, x, y, nullptr, nullptr, nullptr, 0.0, 0.0, s);
}

cudaError_t residual_d(const DevCsr &A, int lanes, const double *b, const double *x, double *r, cudaStream_t s)
{
    return spmv_launch_mode<double, MODE_RESID>(lanes, A.n, A.rp, A.ci, A.v, x, r, b, nullptr, nullptr, 0.0, 0.0, s);
}

// q = A p with deterministic partial sums of p . q (fixed grid, fixed row-to-block mapping)
template <int LANES>
__global__ void __launch_bounds__(kReduceThreads) spmv_dot_kernel(int n, const int *__restrict__ rp,
                                                                  const int *__restrict__ ci,
                                                                  const double *__restrict__ v,
                                                                  const double *__restrict__ p, double *q,
                                                                  double *partial)
{
    const int sub = threadIdx.x & (LANES - 1);
    const int groups_total = kReduceBlocks * (kReduceThreads / LANES);
    double acc = 0.0;
    // the trip count is uniform within a warp: it runs while any of its row groups has a row
    for (int row = (blockIdx.x * kReduceThreads + threadIdx.x) / LANES; __any_sync(kAll, row < n);
         row += groups_total) {
        const bool valid = row < n;
        double sum = 0.0;
        if (valid) {
            const int b = rp[row], e = rp[row + 1];
            for (int k = b + sub; k < e; k += LANES) sum += v[k] * p[ci[k]];
        }
#pragma unroll
        for (int o = LANES / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(kAll, sum, o, LANES);
        if (valid && sub == 0) {
            q[row] = sum;
            acc += p[row] * sum;
        }
    }
    // block reduction in a fixed order
    __shared__ double sh[kReduceThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kAll, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kReduceThreads / 32; ++w) t += sh[w];
        partial[blockIdx.x] = t;
    }
}

cudaError_t spmv_dot(const DevCsr &A, int lanes, const double *p, double *q, double *partial, cudaStream_t s)
{
    switch (lanes) {
    case 4: spmv_dot_kernel<4><<<kReduceBlocks, kReduceThreads, 0, s>>>(A.n, A.rp, A.ci, A.v, p, q, partial); note_launch(); break;
    case 8: spmv_dot_kernel<8><<<kReduceBlocks, kReduceThreads, 0, s>>>(A.n, A.rp, A.ci, A.v, p, q, partial); note_launch(); break;
    case 16:
        spmv_dot_kernel<16><<<kReduceBlocks, kReduceThreads, 0, s>>>(A.n, A.rp, A.ci, A.v, p, q, partial); note_launch();
        break;
    default:
        spmv_dot_kernel<32><<<kReduceBlocks, kReduceThreads, 0, s>>>(A.n, A.rp, A.ci, A.v, p, q, partial); note_launch();
        break;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ PCG vector updates
__device__ __forceinline__ double block_sum_fixed(double v)
{
    __shared__ double sh[kReduceThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kAll, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kReduceThreads / 32; ++w) t += sh[w];
    return t;
}

// x += alpha p; r -= alpha q; partial sums of r . r
__global__ void __launch_bounds__(kReduceThreads) pcg_xr_kernel(int n, double *x, double *r, const double *p,
                                                                const double *q, const PcgScalars *sc,
                                                                double *partial)
{
    const double alpha = sc->alpha;
    double acc = 0.0;
    for (int i = blockIdx.x * kReduceThreads + threadIdx.x; i < n; i += kReduceBlocks * kReduceThreads) {
        x[i] += alpha * p[i];
        double ri = r[i] - alpha * q[i];
        r[i] = ri;
        acc += ri * ri;
    }
    double t = block_sum_fixed(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

cudaError_t pcg_update_xr(int n, double *x, double *r, const double *p, const double *q, const PcgScalars *sc,
                          double *partial, cudaStream_t s)
{
    pcg_xr_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, x, r, p, q, sc, partial); note_launch();
    return cudaGetLastError();
}

__global__ void pcg_p_kernel(int n, double *p, const double *z, const PcgScalars *sc)
{
    const double beta = sc->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = z[i] + beta * p[i];
}

cudaError_t pcg_update_p(int n, double *p, const double *z, const PcgScalars *sc, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    pcg_p_kernel<<<grid_for(n, 256, 8192), 256, 0, s>>>(n, p, z, sc); note_launch();
    return cudaGetLastError();
}

__device__ __forceinline__ double sum_partials(const double *partial)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < kReduceBlocks; i += kReduceThreads) acc += partial[i];
    return block_sum_fixed(acc);
}

// pq = sum(partial); alpha = rz / pq
__global__ void __launch_bounds__(kReduceThreads) pcg_alpha_kernel(const double *partial, PcgScalars *sc)
{
    double t = sum_partials(partial);
    if (threadIdx.x == 0) {
        sc->pq = t;
        sc->alpha = sc->rz / t;
    }
}
// rz_new = sum(partial); beta = rz_new / rz; rz = rz_new
__global__ void __launch_bounds__(kReduceThreads) pcg_beta_kernel(const double *partial, PcgScalars *sc)
{
    double t = sum_partials(partial);
    if (threadIdx.x == 0) {
        sc->beta = t / sc->rz;
        sc->rz = t;
    }
}
__global__ void __launch_bounds__(kReduceThreads) pcg_store_kernel(const double *partial, double *dst)
{
    double t = sum_partials(partial);
    if (threadIdx.x == 0) *dst = t;
}

cudaError_t pcg_alpha(const double *partial, PcgScalars *sc, cudaStream_t s)
{
    pcg_alpha_kernel<<<1, kReduceThreads, 0, s>>>(partial, sc); note_launch();
    return cudaGetLastError();
}
cudaError_t pcg_beta(const double *partial, PcgScalars *sc, cudaStream_t s)
{
    pcg_beta_kernel<<<1, kReduceThreads, 0, s>>>(partial, sc); note_launch();
    return cudaGetLastError();
}
cudaError_t pcg_store(const double *partial, double *dst, cudaStream_t s)
{
    pcg_store_kernel<<<1, kReduceThreads, 0, s>>>(partial, dst); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ V-cycle
// First Chebyshev step from x = 0: d = D^-1 f / theta, x = d
template <typename T>
__global__ void cheb_first_zero_kernel(int n, const T *f, const T *invdiag, T inv_theta, T *d, T *x)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T di = (invdiag[i] * f[i]) * inv_theta;
        d[i] = di;
        x[i] = di;
    }
}

// coarsest level: x = Ainv f (dense FP64), one warp per row
template <typename T>
__global__ void coarse_gemv_kernel(int n, const double *__restrict__ inv, const T *__restrict__ f, T *x)
{
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    double acc = 0.0;
    for (int k = lane; k < n; k += 32) acc += inv[(size_t)row * n + k] * (double)f[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kAll, acc, o);
    if (lane == 0) x[row] = (T)acc;
}

template <typename T>
__global__ void d2t_kernel(int n, const double *in, T *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = (T)in[i];
}
template <typename T>
__global__ void t2d_kernel(int n, const T *in, double *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = (double)in[i];
}

namespace {

struct ChebCoef {
    double theta, delta, sigma1;
};

// algorithmic bytes of one level-operator SpMV: values, columns and row pointers once,
// plus `vecs` vectors of length n in the working type
template <typename T>
double spmv_bytes(const LevelView &lv, int vecs)
{
    return (double)(sizeof(T) + 4) * (double)lv.nnz_a + 4.0 * (lv.n + 1) + (double)vecs * sizeof(T) * lv.n;
}

ChebCoef cheb_coef(double lambda, double ratio)
{
    double lmax = lambda, lmin = lambda / ratio;
    ChebCoef c;
    c.theta = 0.5 * (lmax + lmin);
    c.delta = 0.5 * (lmax - lmin);
    c.sigma1 = c.theta / c.delta;
    return c;
}

// Chebyshev smoothing of degree m on level L; x holds the iterate (x_is_zero: it is 0).
// Returns the buffer that holds the result (x or x2).
template <typename T>
cudaError_t chebyshev(const SolveCtx &c, int L, T *&x, T *&x2, bool x_is_zero, cudaStream_t s)
{
    const LevelView &lv = c.lev[L];
    const ChebCoef cc = cheb_coef(lv.lambda, c.cheb_ratio);
    double rho = 1.0 / cc.sigma1;
    const T *f = (const T *)lv.f;
    const T *inv = (const T *)lv.invdiag;
    T *d = (T *)lv.d;
    const T *av = (const T *)lv.av;
    if (x_is_zero) {
        cheb_first_zero_kernel<T><<<grid_for(lv.n, 256, 8192), 256, 0, s>>>(lv.n, f, inv, (T)(1.0 / cc.theta), d, x); note_launch();
        AMG_CUDA_TRY(cudaGetLastError());
    } else {
        ProfScope ps(L == 0 ? KC_VCYCLE_SPMV : KC_COUNT, s, spmv_bytes<T>(lv, 6));
        AMG_CUDA_TRY((spmv_launch_mode<T, MODE_CHEB>(lv.lanes_a, lv.n, lv.arp, lv.aci, av, x, x2, f, inv, d, (T)0,
                                                     (T)(1.0 / cc.theta), s)));
        T *t = x; x = x2; x2 = t;
    }
    for (int k = 1; k < c.cheb_degree; ++k) {
        double rho_new = 1.0 / (2.0 * cc.sigma1 - rho);
        double c1 = rho_new * rho, c2 = 2.0 * rho_new / cc.delta;
        ProfScope ps(L == 0 ? KC_VCYCLE_SPMV : KC_COUNT, s, spmv_bytes<T>(lv, 6));
        AMG_CUDA_TRY((spmv_launch_mode<T, MODE_CHEB>(lv.lanes_a, lv.n, lv.arp, lv.aci, av, x, x2, f, inv, d, (T)c1,
                                                     (T)c2, s)));
        T *t = x; x = x2; x2 = t;
        rho = rho_new;
    }
    return cudaSuccess;
}

// Algorithm 1 from level L with x = 0; on return *out points at the level's solution buffer.
template <typename T>
cudaError_t vcycle_level(const SolveCtx &c, int L, T **out, cudaStream_t s)
{
    const LevelView &lv = c.lev[L];
    T *x = (T *)lv.x, *x2 = (T *)lv.x2;
    if (L == c.nlev - 1) {
        if (lv.n > 0)
            coarse_gemv_kernel<T><<<grid_for((int64_t)lv.n * 32, 128), 128, 0, s>>>(lv.n, c.coarse_inv,
                                                                                  (const T *)lv.f, x); note_launch();
        *out = x;
        return cudaGetLastError();
    }
    const LevelView &cl = c.lev[L + 1];
    AMG_CUDA_TRY(chebyshev<T>(c, L, x, x2, true, s));
    // r = f - A x ; f_c = R r
    {
    ProfScope ps(L == 0 ? KC_VCYCLE_SPMV : KC_COUNT, s, spmv_bytes<T>(lv, 3));
    AMG_CUDA_TRY((spmv_launch_mode<T, MODE_RESID>(lv.lanes_a, lv.n, lv.arp, lv.aci, (const T *)lv.av, x, (T *)lv.r,
                                                  (const T *)lv.f, nullptr, nullptr, (T)0, (T)0, s)));
    }
    AMG_CUDA_TRY((spmv_launch_mode<T, MODE_Y>(lv.lanes_r, cl.n, lv.rrp, lv.rci, (const T *)lv.rv, (const T *)lv.r,
                                              (T *)cl.f, nullptr, nullptr, nullptr, (T)0, (T)0, s)));
    T *xc = nullptr;
    AMG_CUDA_TRY(vcycle_level<T>(c, L + 1, &xc, s));
    // x += P x_c
    AMG_CUDA_TRY((spmv_launch_mode<T, MODE_PROLONG>(lv.lanes_p, lv.n, lv.prp, lv.pci, (const T *)lv.pv, xc, x,
                                                    nullptr, nullptr, nullptr, (T)0, (T)0, s)));
    AMG_CUDA_TRY(chebyshev<T>(c, L, x, x2, false, s));
    *out = x;
    return cudaSuccess;
}

}  // namespace

cudaError_t vcycle(const SolveCtx &c, const double *r, double *z, cudaStream_t s)
{
    const LevelView &l0 = c.lev[0];
    if (l0.n == 0) return cudaSuccess;
    if (!c.mixed) {
        // the finest level reads r in place
        SolveCtx cc = c;
        cc.lev[0].f = (void *)r;
        double *out = nullptr;
        AMG_CUDA_TRY(vcycle_level<double>(cc, 0, &out, s));
        return cudaMemcpyAsync(z, out, sizeof(double) * (size_t)l0.n, cudaMemcpyDeviceToDevice, s);
    }
    d2t_kernel<float><<<grid_for(l0.n, 256, 8192), 256, 0, s>>>(l0.n, r, (float *)l0.f); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    float *out = nullptr;
    AMG_CUDA_TRY(vcycle_level<float>(c, 0, &out, s));
    t2d_kernel<float><<<grid_for(l0.n, 256, 8192), 256, 0, s>>>(l0.n, out, z); note_launch();
    return cudaGetLastError();
}

}  // namespace amgk
