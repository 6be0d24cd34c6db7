// gmres.cu -- flexible GMRES(m) with the V-cycle as right preconditioner, the outer iteration
// for nonsymmetric operators (§3's wind pressure system is solved by GMRES preconditioned with
// smoothed aggregation; Saad, "A flexible inner-outer preconditioned GMRES algorithm", SIAM J.
// Sci. Comput. 14, 1993).
//
// Per cycle r = b - A x, v_0 = r / |r|; per step z_j = M v_j (one V-cycle), w = A z_j,
// classical Gram-Schmidt against v_0..v_j done twice (h = V^T w, then w -= V h), v_{j+1} =
// w / |w|.  The Hessenberg column goes to the host, where Givens rotations keep it triangular
// and |g_{j+1}| is the minimiser's residual norm.  When that is <= tol |b|, at the end of a
// cycle or at the iteration limit: y from the triangular system, x += Z y, and the true
// residual decides (stop, or restart from x).
//
// Execution: step j (v_j = w / |w| from the norm left on the device, the V-cycle, A z_j, both
// Gram-Schmidt passes, |w|^2, the copy of the column to pinned host memory) is one CUDA graph,
// captured on first use and replayed in later cycles and solves.  Step j+1 is launched before
// the host waits for step j, so the GPU does not idle while the host rotates the column; a
// step launched past the stop is discarded (it writes only v_{j+1}, z_{j+1}, w and its own
// column slot, none of which the update of x reads).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "hierarchy.cuh"

namespace amgk {

struct GmresWork {
    int m = 0, n = 0;
    int slot = 0;                     // doubles per step slot: 2 (m+1) projections, then |w|^2
    double *V = nullptr, *Z = nullptr, *w = nullptr;   // V: (m+1) x n, Z: m x n
    double *partial = nullptr;        // kDotBlocks x (m+1)
    double *hd = nullptr;             // device: m step slots, then r.r of the cycle's start
    double *yd = nullptr;             // device copy of y
    double *host = nullptr;           // pinned: m step slots, r.r, then y (m values)
    std::vector<cudaGraphExec_t> gx;  // step graphs (null until captured)
    std::vector<long long> gk;        // kernels in each step graph
    bool graph_failed = false;
    cudaEvent_t ev[2] = {nullptr, nullptr};
};

namespace {

constexpr int kGT = 256;
constexpr int kDotBlocks = kReduceBlocks;   // Gram-Schmidt dot products: 2 blocks of 256 per SM

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

// partial[i * gridDim + block] = sum over the block's rows of V_i . w, i < nv.  Up to kGC basis
// vectors per pass over w.  Each thread accumulates its grid-stride entries in ascending order,
// kGU strides' loads issued together; the warp then reduces all kGC sums at once by a transposing
// butterfly (after the exchanges at distances 16, 8 and 4, lane L holds a quarter-warp sum of
// vector L/4; distances 2 and 1 finish it): 9 FP64 additions a lane instead of 5 per vector, which
// matters where FP64 issues at a small fraction of the FP32 rate; the block adds its warps in order.
constexpr int kGC = 8;
constexpr int kGU = 4;
__global__ void __launch_bounds__(kGT) gs_dots_kernel(int n, const double *V, int nv, const double *w,
                                                      double *partial)
{
    __shared__ double sh[kGC][kGT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t stride = (size_t)gridDim.x * kGT;
    for (int i0 = 0; i0 < nv; i0 += kGC) {
        const int c = min(kGC, nv - i0);
        const double *Vb = V + (size_t)i0 * n;
        double acc[kGC];
#pragma unroll
        for (int q = 0; q < kGC; ++q) acc[q] = 0.0;
        for (size_t e0 = (size_t)blockIdx.x * kGT + threadIdx.x; e0 < (size_t)n; e0 += kGU * stride) {
            double we[kGU], vv[kGU][kGC];
#pragma unroll
            for (int u = 0; u < kGU; ++u) {
                const size_t e = e0 + u * stride;
                const bool in = e < (size_t)n;
                we[u] = in ? w[e] : 0.0;
#pragma unroll
                for (int q = 0; q < kGC; ++q) vv[u][q] = (in && q < c) ? Vb[(size_t)q * n + e] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kGU; ++u)
                if (e0 + u * stride < (size_t)n) {
#pragma unroll
                    for (int q = 0; q < kGC; ++q)
                        if (q < c) acc[q] += vv[u][q] * we[u];
                }
        }
        const unsigned full = 0xffffffffu;
        const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
        double r4[4], r2[2];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const double keep = b4 ? acc[j + 4] : acc[j], send = b4 ? acc[j] : acc[j + 4];
            r4[j] = keep + __shfl_xor_sync(full, send, 16);
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const double keep = b3 ? r4[j + 2] : r4[j], send = b3 ? r4[j] : r4[j + 2];
            r2[j] = keep + __shfl_xor_sync(full, send, 8);
        }
        double r1;
        {
            const double keep = b2 ? r2[1] : r2[0], send = b2 ? r2[0] : r2[1];
            r1 = keep + __shfl_xor_sync(full, send, 4);
        }
        r1 += __shfl_xor_sync(full, r1, 2);
        r1 += __shfl_xor_sync(full, r1, 1);
        if ((lane & 3) == 0) sh[lane >> 2][warp] = r1;
        __syncthreads();
        if (threadIdx.x < c) {
            double t = 0.0;
            for (int k = 0; k < kGT / 32; ++k) t += sh[threadIdx.x][k];
            partial[(size_t)(i0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
        }
        __syncthreads();
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

// w -= sum_i h_i V_i (per entry, i ascending); the coefficients staged in shared memory.  A
// step has at most restart basis vectors and amg_setup refuses restart above 512.
constexpr int kMaxBasis = 513;
__global__ void __launch_bounds__(256) gs_update_kernel(int n, const double *V, int nv, const double *h,
                                                        double *w)
{
    __shared__ double hs[kMaxBasis];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
    __syncthreads();
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        double t = w[e];
        int i = 0;
        for (; i + 4 <= nv; i += 4) {
            const double a0 = V[(size_t)i * n + e], a1 = V[(size_t)(i + 1) * n + e],
                         a2 = V[(size_t)(i + 2) * n + e], a3 = V[(size_t)(i + 3) * n + e];
            t = t - hs[i] * a0;
            t = t - hs[i + 1] * a1;
            t = t - hs[i + 2] * a2;
            t = t - hs[i + 3] * a3;
        }
        for (; i < nv; ++i) t = t - hs[i] * V[(size_t)i * n + e];
        w[e] = t;
    }
}

// v = w * (1 / sqrt(*nrm2)), the reciprocal formed once per block (v = 0 when the norm is 0: the
// step before broke down and the host stops)
__global__ void __launch_bounds__(256) scale_norm_kernel(int n, const double *w, const double *nrm2, double *v)
{
    __shared__ double inv;
    if (threadIdx.x == 0) {
        const double nrm = sqrt(*nrm2);
        inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    }
    __syncthreads();
    const double r = inv;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) v[e] = w[e] * r;
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

void release_host_side(GmresWork *W)
{
    for (cudaGraphExec_t g : W->gx)
        if (g) cudaGraphExecDestroy(g);
    for (int k = 0; k < 2; ++k)
        if (W->ev[k]) cudaEventDestroy(W->ev[k]);
    if (W->host) cudaFreeHost(W->host);
    delete W;
}

// device vectors (owned by the handle's allocation list), pinned host slots, two events
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
    g.slot = 2 * (m + 1) + 1;
    g.m = m;
    g.n = n;
    AMG_CUDA_TRY(al((void **)&g.V, sizeof(double) * nn * (size_t)(m + 1)));
    AMG_CUDA_TRY(al((void **)&g.Z, sizeof(double) * nn * (size_t)m));
    AMG_CUDA_TRY(al((void **)&g.w, sizeof(double) * nn));
    AMG_CUDA_TRY(al((void **)&g.partial, sizeof(double) * (size_t)kDotBlocks * (size_t)(m + 1)));
    AMG_CUDA_TRY(al((void **)&g.hd, sizeof(double) * ((size_t)m * g.slot + 1)));
    AMG_CUDA_TRY(al((void **)&g.yd, sizeof(double) * (size_t)(m + 1)));
    AMG_CUDA_TRY(cudaMallocHost(&g.host, sizeof(double) * ((size_t)m * g.slot + 1 + (size_t)m)));
    for (int k = 0; k < 2; ++k) AMG_CUDA_TRY(cudaEventCreateWithFlags(&g.ev[k], cudaEventDisableTiming));
    g.gx.assign((size_t)m, nullptr);
    g.gk.assign((size_t)m, 0);
    return cudaSuccess;
}

// step j of a cycle, enqueued on st (the body of step graph j)
cudaError_t step_body(amg_hierarchy *h, GmresWork &W, int j, cudaStream_t st)
{
    const int n = W.n, m = W.m;
    const int gp = grid_for(n, 256, 8192);
    double *vj = W.V + (size_t)j * n, *zj = W.Z + (size_t)j * n;
    double *slot = W.hd + (size_t)j * W.slot;
    const double *nrm2 = j == 0 ? W.hd + (size_t)m * W.slot : W.hd + (size_t)(j - 1) * W.slot + 2 * (m + 1);
    scale_norm_kernel<<<gp, 256, 0, st>>>(n, W.w, nrm2, vj); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    AMG_CUDA_TRY(vcycle(h->ctx, vj, zj, st));
    AMG_CUDA_TRY(spmv_d(h->lev[0].A, h->plan0, zj, W.w, st));
    const int nv = j + 1;
    for (int pass = 0; pass < 2; ++pass) {
        double *hp = slot + (size_t)pass * (m + 1);
        gs_dots_kernel<<<kDotBlocks, kGT, 0, st>>>(n, W.V, nv, W.w, W.partial); note_launch();
        gs_reduce_kernel<<<nv, kGT, 0, st>>>(W.partial, kDotBlocks, hp); note_launch();
        gs_update_kernel<<<gp, 256, 0, st>>>(n, W.V, nv, hp, W.w); note_launch();
    }
    AMG_CUDA_TRY(cudaGetLastError());
    AMG_CUDA_TRY(dot(W.w, W.w, n, h->partial, slot + 2 * (m + 1), st));
    return cudaMemcpyAsync(W.host + (size_t)j * W.slot, slot, sizeof(double) * (size_t)W.slot,
                           cudaMemcpyDeviceToHost, st);
}

// the graph of step j (captured on first use); null when steps run eagerly
cudaGraphExec_t step_graph(amg_hierarchy *h, GmresWork &W, int j)
{
    if (W.graph_failed || profiling_enabled()) return nullptr;
    if (W.gx[(size_t)j]) return W.gx[(size_t)j];
    cudaGraph_t g = nullptr;
    const long long launches_before = launch_count();
    cudaError_t e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = step_body(h, W, j, h->cap);
        e = cudaStreamEndCapture(h->cap, &g);
        if (e == cudaSuccess && e1 != cudaSuccess) e = e1;
    }
    cudaGraphExec_t gx = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gx, g, 0);
    if (g) cudaGraphDestroy(g);
    const long long kernels = launch_count() - launches_before;
    note_launches(-kernels);       // the capture itself launched nothing
    if (e != cudaSuccess) {
        cudaGetLastError();
        W.graph_failed = true;     // this handle's steps run eagerly from now on
        return nullptr;
    }
    W.gx[(size_t)j] = gx;
    W.gk[(size_t)j] = kernels;
    return gx;
}

cudaError_t launch_step(amg_hierarchy *h, GmresWork &W, int j, cudaStream_t s)
{
    cudaGraphExec_t gx = step_graph(h, W, j);
    if (gx) {
        AMG_CUDA_TRY(cudaGraphLaunch(gx, s));
        note_launches(W.gk[(size_t)j]);
    } else {
        AMG_CUDA_TRY(step_body(h, W, j, s));
    }
    return cudaEventRecord(W.ev[j & 1], s);
}

// w = b - A x and |w|^2 (left on the device where step 0 reads it, and in *out); synchronises s
cudaError_t true_residual2(amg_hierarchy *h, GmresWork &W, double *out, cudaStream_t s)
{
    double *dv = W.hd + (size_t)W.m * W.slot, *hv = W.host + (size_t)W.m * W.slot;
    AMG_CUDA_TRY(residual_d(h->lev[0].A, h->plan0, h->b, h->x, W.w, s));
    AMG_CUDA_TRY(dot(W.w, W.w, W.n, h->partial, dv, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(hv, dv, sizeof(double), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    *out = *hv;
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
    release_host_side(h->gmres);
    h->gmres = nullptr;
}

amg_status_t fgmres_solve(amg_hierarchy *h, const double *b, double *x, double tol, amg_info_t *info)
{
    const int n = h->lev[0].A.n;
    const int m = h->p.restart;
    const double t0 = now_ms_g();
    cudaStream_t s = h->s;
    amg_status_t st = AMG_OK, result = AMG_OK;
    int it = 0;
    double nb = 0.0, relres = 0.0;
    std::vector<double> H((size_t)(m + 1) * m, 0.0), g((size_t)(m + 1), 0.0), cs((size_t)m, 0.0), sn((size_t)m, 0.0);
    const int gp = grid_for(n, 256, 8192);
    GmresWork *W = h->gmres;
    if (n > 0 && !W) {
        W = new GmresWork();
        const cudaError_t e = gmres_alloc(h, *W, m);
        if (e != cudaSuccess) {
            release_host_side(W);      // device memory stays on the handle's list
            W = nullptr;
            st = fail_cuda(e, "gmres_alloc");
            goto done;
        }
        h->gmres = W;
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
        double *y = W->host + (size_t)m * W->slot + 1;
        double rr = 0.0;
        GK(true_residual2(h, *W, &rr, s));
        const double beta = std::sqrt(rr);
        if (beta / nb <= tol) { result = AMG_OK; break; }
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0;
        bool stop = false;
        GK(launch_step(h, *W, 0, s));
        for (; j < m && it < h->p.max_iter; ++j) {
            // step j+1 is launched exactly when the loop will reach it, unless this step stops
            if (j + 1 < m && it + 1 < h->p.max_iter) GK(launch_step(h, *W, j + 1, s));
            GK(cudaEventSynchronize(W->ev[j & 1]));
            ++it;
            const double *col = W->host + (size_t)j * W->slot;
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = (0.0 + col[i]) + col[(m + 1) + i];
            const double hn = std::sqrt(col[2 * (m + 1)]);
            H[(size_t)(j + 1) * m + j] = hn;
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
            GK(cudaMemcpyAsync(W->yd, y, sizeof(double) * (size_t)j, cudaMemcpyHostToDevice, s));
            xz_update_kernel<<<gp, 256, 0, s>>>(n, W->Z, j, W->yd, h->x); note_launch();
            GK(cudaGetLastError());
        }
        if (stop || it >= h->p.max_iter) {
            double tt = 0.0;
            GK(true_residual2(h, *W, &tt, s));
            if (std::sqrt(tt) / nb <= tol) { result = AMG_OK; break; }
        }
    }
finish:
    if (n > 0) {
        double tt = 0.0;
        GK(true_residual2(h, *W, &tt, s));
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
