// gmres.cu -- flexible GMRES(m) with the V-cycle as right preconditioner, the outer iteration
// for nonsymmetric operators (§3's wind pressure system is solved by GMRES preconditioned with
// smoothed aggregation; Saad, "A flexible inner-outer preconditioned GMRES algorithm", SIAM J.
// Sci. Comput. 14, 1993).
//
// Per cycle r = b - A x, v_0 = r / |r|; per step z_j = M v_j (one V-cycle), w = A z_j,
// classical Gram-Schmidt against v_0..v_j done twice (h = V^T w, then w -= V h), v_{j+1} =
// w / |w|.  The Hessenberg column is copied to the host, where Givens rotations keep it
// triangular and |g_{j+1}| is the minimiser's residual norm.  When that is <= tol |b|, at the
// end of a cycle or at the iteration limit: y from the triangular system, x += Z y, and the
// true residual decides (stop, or restart from x).  One synchronisation per step.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "hierarchy.cuh"

namespace amgk {

struct GmresWork {
    int m = 0, n = 0;
    double *V = nullptr, *Z = nullptr, *w = nullptr;   // V: (m+1) x n, Z: m x n
    double *partial = nullptr;        // kReduceBlocks x (m+1)
    double *hd = nullptr;             // device: 2 (m+1) projections, then |w|^2, then spare
    double *yd = nullptr;             // device copy of y
    double *host = nullptr;           // pinned: 2 (m+2) values
};

namespace {

constexpr int kGT = 256;

double now_ms_g()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

__device__ __forceinline__ double block_sum_g(double v)
{
    __shared__ double sh[kGT / 32];
    __shared__ double tot;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kGT / 32; ++k) t += sh[k];
        tot = t;
    }
    __syncthreads();
    const double r = tot;
    __syncthreads();
    return r;
}

// partial[i * gridDim + block] = sum over the block's rows of V_i . w, i < nv
__global__ void __launch_bounds__(kGT) gs_dots_kernel(int n, const double *V, int nv, const double *w,
                                                      double *partial)
{
    for (int i = 0; i < nv; ++i) {
        const double *vi = V + (size_t)i * n;
        double acc = 0.0;
        for (int e = blockIdx.x * kGT + threadIdx.x; e < n; e += gridDim.x * kGT) acc += vi[e] * w[e];
        const double t = block_sum_g(acc);
        if (threadIdx.x == 0) partial[(size_t)i * gridDim.x + blockIdx.x] = t;
    }
}

// out[i] = partial[i * count + 0..count) added in order; block i
__global__ void __launch_bounds__(kGT) gs_reduce_kernel(const double *partial, int count, double *out)
{
    const double *p = partial + (size_t)blockIdx.x * count;
    double acc = 0.0;
    for (int k = threadIdx.x; k < count; k += kGT) acc += p[k];
    const double t = block_sum_g(acc);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
}

// w -= sum_i h_i V_i (per entry, i ascending)
__global__ void gs_update_kernel(int n, const double *V, int nv, const double *h, double *w)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        double t = w[e];
        for (int i = 0; i < nv; ++i) t = t - h[i] * V[(size_t)i * n + e];
        w[e] = t;
    }
}

__global__ void scale_copy_kernel(int n, const double *w, double nrm, double *v)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) v[e] = w[e] / nrm;
}

// x += sum_k y_k Z_k (per entry, k ascending)
__global__ void xz_update_kernel(int n, const double *Z, int nk, const double *y, double *x)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        double t = x[e];
        for (int k = 0; k < nk; ++k) t = t + y[k] * Z[(size_t)k * n + e];
        x[e] = t;
    }
}

cudaError_t gmres_alloc(amg_hierarchy *h, GmresWork &g, int m)
{
    const int n = h->lev[0].A.n;
    auto al = [&](void **p, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMallocAsync(p, bytes + 128, h->s);
        if (e == cudaSuccess) {
            h->allocs.push_back(*p);
            h->bytes += bytes + 128;
        }
        return e;
    };
    const size_t nn = (size_t)(n > 0 ? n : 1);
    AMG_CUDA_TRY(al((void **)&g.V, sizeof(double) * nn * (size_t)(m + 1)));
    AMG_CUDA_TRY(al((void **)&g.Z, sizeof(double) * nn * (size_t)m));
    AMG_CUDA_TRY(al((void **)&g.w, sizeof(double) * nn));
    AMG_CUDA_TRY(al((void **)&g.partial, sizeof(double) * (size_t)kReduceBlocks * (size_t)(m + 1)));
    AMG_CUDA_TRY(al((void **)&g.hd, sizeof(double) * (size_t)(2 * (m + 1) + 4)));
    AMG_CUDA_TRY(al((void **)&g.yd, sizeof(double) * (size_t)(m + 1)));
    AMG_CUDA_TRY(cudaMallocHost(&g.host, sizeof(double) * (size_t)(2 * (m + 1) + 4)));
    g.m = m;
    g.n = n;
    return cudaSuccess;
}

#define GK(expr)                                                           \
    do {                                                                   \
        cudaError_t _e = (expr);                                           \
        if (_e != cudaSuccess) { st = fail_cuda(_e, #expr); goto done; }   \
    } while (0)

}  // namespace

void gmres_release(amg_hierarchy *h)
{
    if (!h->gmres) return;
    if (h->gmres->host) cudaFreeHost(h->gmres->host);
    delete h->gmres;
    h->gmres = nullptr;
}

amg_status_t fgmres_solve(amg_hierarchy *h, const double *b, double *x, double tol, amg_info_t *info)
{
    const int n = h->lev[0].A.n;
    const int m = h->p.restart;
    const double t0 = now_ms_g();
    cudaStream_t s = h->s;
    const DevCsr &A = h->lev[0].A;
    amg_status_t st = AMG_OK, result = AMG_OK;
    int it = 0;
    double nb = 0.0, relres = 0.0;
    std::vector<double> H((size_t)(m + 1) * m, 0.0), g((size_t)(m + 1), 0.0), cs((size_t)m, 0.0), sn((size_t)m, 0.0),
        y((size_t)m, 0.0);
    const int gp = grid_for(n, 256, 8192);
    if (!h->gmres) h->gmres = new GmresWork();
    GmresWork &W = *h->gmres;
    if (n > 0 && W.m != m) {
        if (W.host) cudaFreeHost(W.host);
        W = GmresWork();
        GK(gmres_alloc(h, W, m));
    }
    if (n == 0) goto finish;
    GK(copy_to_device(h->b, b, sizeof(double) * (size_t)n, s));
    GK(cudaMemsetAsync(h->x, 0, sizeof(double) * (size_t)n, s));
    {
        double bb = 0.0;
        GK(dot(h->b, h->b, n, h->partial, &h->sc->bb, s));
        GK(cudaMemcpyAsync(&bb, &h->sc->bb, sizeof(double), cudaMemcpyDeviceToHost, s));
        GK(cudaStreamSynchronize(s));
        nb = std::sqrt(bb);
    }
    if (nb == 0.0) goto finish;
    result = AMG_ERR_NOT_CONVERGED;
    while (it < h->p.max_iter) {
        // r = b - A x, v_0 = r / |r|
        GK(residual_d(A, h->plan0, h->b, h->x, W.w, s));
        GK(dot(W.w, W.w, n, h->partial, &h->sc->tmp, s));
        double rr = 0.0;
        GK(cudaMemcpyAsync(&rr, &h->sc->tmp, sizeof(double), cudaMemcpyDeviceToHost, s));
        GK(cudaStreamSynchronize(s));
        const double beta = std::sqrt(rr);
        if (beta / nb <= tol) { result = AMG_OK; break; }
        scale_copy_kernel<<<gp, 256, 0, s>>>(n, W.w, beta, W.V); note_launch();
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0;
        bool stop = false;
        for (; j < m && it < h->p.max_iter; ++j) {
            double *vj = W.V + (size_t)j * n, *zj = W.Z + (size_t)j * n;
            GK(vcycle(h->ctx, vj, zj, s));
            GK(spmv_d(A, h->plan0, zj, W.w, s));
            ++it;
            const int nv = j + 1;
            for (int pass = 0; pass < 2; ++pass) {
                double *hp = W.hd + (size_t)pass * (m + 1);
                gs_dots_kernel<<<kReduceBlocks, kGT, 0, s>>>(n, W.V, nv, W.w, W.partial); note_launch();
                gs_reduce_kernel<<<nv, kGT, 0, s>>>(W.partial, kReduceBlocks, hp); note_launch();
                gs_update_kernel<<<gp, 256, 0, s>>>(n, W.V, nv, hp, W.w); note_launch();
            }
            GK(cudaGetLastError());
            GK(dot(W.w, W.w, n, h->partial, W.hd + 2 * (m + 1), s));
            GK(cudaMemcpyAsync(W.host, W.hd, sizeof(double) * (size_t)(2 * (m + 1) + 1), cudaMemcpyDeviceToHost, s));
            GK(cudaStreamSynchronize(s));
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = (0.0 + W.host[i]) + W.host[(m + 1) + i];
            const double hn = std::sqrt(W.host[2 * (m + 1)]);
            H[(size_t)(j + 1) * m + j] = hn;
            if (hn > 0.0) {
                scale_copy_kernel<<<gp, 256, 0, s>>>(n, W.w, hn, W.V + (size_t)(j + 1) * n); note_launch();
            }
            for (int i = 0; i < j; ++i) {
                const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
            const double r = std::sqrt(a * a + c * c);
            cs[j] = a / r;
            sn[j] = c / r;
            H[(size_t)j * m + j] = r;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            if (std::fabs(g[j + 1]) / nb <= tol || hn == 0.0) {
                stop = true;
                ++j;
                break;
            }
        }
        // y = H(0:j, 0:j)^-1 g(0:j); x += Z y
        for (int i = j - 1; i >= 0; --i) {
            double sum = g[i];
            for (int k = i + 1; k < j; ++k) sum = sum - H[(size_t)i * m + k] * y[k];
            y[i] = sum / H[(size_t)i * m + i];
        }
        if (j > 0) {
            GK(cudaMemcpyAsync(W.yd, y.data(), sizeof(double) * (size_t)j, cudaMemcpyHostToDevice, s));
            xz_update_kernel<<<gp, 256, 0, s>>>(n, W.Z, j, W.yd, h->x); note_launch();
            GK(cudaGetLastError());
        }
        if (stop || it >= h->p.max_iter) {
            GK(residual_d(A, h->plan0, h->b, h->x, W.w, s));
            GK(dot(W.w, W.w, n, h->partial, &h->sc->tmp, s));
            double tt = 0.0;
            GK(cudaMemcpyAsync(&tt, &h->sc->tmp, sizeof(double), cudaMemcpyDeviceToHost, s));
            GK(cudaStreamSynchronize(s));
            if (std::sqrt(tt) / nb <= tol) { result = AMG_OK; break; }
        }
    }
finish:
    if (n > 0) {
        GK(residual_d(A, h->plan0, h->b, h->x, W.w, s));
        GK(dot(W.w, W.w, n, h->partial, &h->sc->tmp, s));
        double tt = 0.0;
        GK(cudaMemcpyAsync(&tt, &h->sc->tmp, sizeof(double), cudaMemcpyDeviceToHost, s));
        GK(copy_to_host(x, h->x, sizeof(double) * (size_t)n, s));
        GK(cudaStreamSynchronize(s));
        relres = nb > 0.0 ? std::sqrt(tt) / nb : 0.0;
    }
    st = result;
    if (spmv_take_errors(s) != 0) {
        set_last_error("a bulk copy into shared memory did not complete in time");
        st = AMG_ERR_INTERNAL;
    }
done:
    if (info) {
        info->iters = it;
        info->status = st;
        info->relres_true = relres;
        info->setup_ms = h->setup_ms;
        info->solve_ms = now_ms_g() - t0;
        info->levels = h->nlev;
        double tot = 0.0;
        for (int L = 0; L < h->nlev; ++L) tot += (double)h->lev[L].A.nnz;
        info->op_complexity = h->fine_nnz > 0 ? tot / (double)h->fine_nnz : 0.0;
    }
    return st;
}

#undef GK

}  // namespace amgk
