// api.cu -- the C ABI: hierarchy setup (per level: strength, aggregation, tentative
// prolongator, optional pruning, filtering, smoothing diagonal and damping, smoothed
// prolongator, optional constraints, transpose, Galerkin product, Chebyshev eigenvalue; then
// the coarsest factorisation) and the preconditioned conjugate-gradient solve.
//
// Host code only orchestrates: every arithmetic step runs in the kernels of setup.cu,
// spgemm.cu, coarse.cu, solve.cu and util.cu.  The host reads back sizes (to allocate),
// eigenvalue estimates (to set omega and the Chebyshev interval) and the residual norm (to
// stop PCG).
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <utility>
#include <string>
#include <vector>

#include "amg_internal.cuh"
#include "hierarchy.cuh"

using namespace amgk;

namespace {

thread_local std::string g_last_error;

}  // namespace

namespace amgk {

void set_last_error(const std::string &msg) { g_last_error = msg; }

amg_status_t fail_cuda(cudaError_t e, const char *where)
{
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    cudaGetLastError();   // clear a sticky-free error so later calls start clean
    if (e == cudaErrorMemoryAllocation) return AMG_ERR_OOM;
    return AMG_ERR_CUDA;
}

}  // namespace amgk

namespace {

#define CK(expr)                                                          \
    do {                                                                  \
        cudaError_t _e = (expr);                                          \
        if (_e != cudaSuccess) { st = fail_cuda(_e, #expr); goto done; }  \
    } while (0)

// Device memory comes from the stream-ordered pool of the handle's stream (no device-wide
// synchronisation per allocation or free; freed blocks are kept by the pool for reuse).
// Every array carries 16 elements of padding: bulk copies widen ranges to 16-byte boundaries.
template <typename T>
cudaError_t dalloc(amg_hierarchy *h, T **p, size_t count)
{
    *p = nullptr;
    cudaError_t e = cudaMallocAsync((void **)p, (count + 16) * sizeof(T), h->s);
    if (e == cudaSuccess) {
        h->allocs.push_back((void *)*p);
        h->bytes += (count + 16) * sizeof(T);
    }
    return e;
}

void own(amg_hierarchy *h, const DevCsr &c)
{
    if (c.rp) h->allocs.push_back(c.rp);
    if (c.ci) h->allocs.push_back(c.ci);
    if (c.v) h->allocs.push_back(c.v);
    h->bytes += 12 * ((size_t)c.nnz + 16) + 4 * ((size_t)c.n + 17);
}

void release_all(amg_hierarchy *h)
{
    for (void *p : h->allocs) cudaFreeAsync(p, h->s);
    h->allocs.clear();
    cudaStreamSynchronize(h->s);
}

// keep freed memory in the device's default pool instead of returning it at every sync
void keep_pool_memory()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    static std::atomic<bool> done[64];   // setting the attribute twice is harmless
    if (dev < 0 || dev >= 64 || done[dev].load()) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[dev].store(true);
}

void free_async(void *p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
}

__global__ void validate_kernel(int n, const int *rp, const int *ci, int *bad)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int has = 0, prev = -1;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        int c = ci[e];
        if (c < 0 || c >= n || c <= prev) { atomicAdd(bad, 1); return; }
        prev = c;
        has |= (c == i);
    }
    if (!has) atomicAdd(bad, 1);
}

__global__ void ones_kernel(int n, double *b)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = 1.0;
}

__global__ void component_ones_kernel(int n, int bs, int k, double *B)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * k) return;
    const int j = (int)(t / n), i = (int)(t % n);
    B[t] = (i % bs == j) ? 1.0 : 0.0;
}

// stored bytes of a device CSR (int32 row pointers and columns, double values)
double csr_bytes(const DevCsr &c) { return 12.0 * (double)c.nnz + 4.0 * (c.n + 1); }

double now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

void amgk::trace_mark(amg_hierarchy *h, int level, int phase)
{
    if (!h->p.trace || level < 0 || level >= 32) return;
    cudaStreamSynchronize(h->s);
    const double t = now_ms();
    h->phase_ms[level][phase] += t - h->phase_t;
    h->phase_t = t;
}

namespace {

// one level of the hierarchy; *coarsest = 1 if the level cannot be coarsened further
// Whether a level operator gets a sliced-ELL copy for its products (params.spmv_layout): AUTO
// copies an operator with short rows when it is larger than L2 (the CSR kernel would stream it
// from HBM) or has rows enough for four 256-row sliced blocks per SM: one lane per row issues
// fewer FP64 instructions than two, but a level with fewer rows leaves the SMs without warps to
// cover the latency of its longer rows.
bool sell_wanted(const amg_hierarchy *h, const Level &lv, int l2, int nsm)
{
    const bool want = h->p.spmv_layout == AMG_LAYOUT_SELL ||
                      (h->p.spmv_layout == AMG_LAYOUT_AUTO &&
                       (12.0 * (double)lv.A.nnz > (double)l2 || (double)lv.A.n >= 1024.0 * nsm));
    return want && lv.plan_a.lpr == 2 && lv.A.n > 0 && lv.plan_a.sci == nullptr;
}

// The finest level's sliced-ELL copy (FP64 values) during setup, so that its power method reads
// it too; no copy when the offsets would overflow or the padding exceeds an eighth of the
// entries.  Synchronises s.
cudaError_t sell_build_fine(amg_hierarchy *h, Level &lv, cudaStream_t s)
{
    int dev = 0, l2 = 0, nsm = 0;
    AMG_CUDA_TRY(cudaGetDevice(&dev));
    AMG_CUDA_TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    AMG_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (!sell_wanted(h, lv, l2, nsm)) return cudaSuccess;
    const int nsl = sell_slices(lv.A.n);
    int *sw = nullptr, *sp = nullptr, *sci = nullptr;
    unsigned long long *t64 = nullptr, tot = 0;
    double *sv64 = nullptr;
    AMG_CUDA_TRY(dalloc(h, &sw, (size_t)nsl));
    AMG_CUDA_TRY(dalloc(h, &sp, (size_t)nsl + 1));
    AMG_CUDA_TRY(dalloc(h, &t64, 1));
    AMG_CUDA_TRY(sell_layout(lv.A.n, lv.A.rp, sw, sp, t64, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(&tot, t64, sizeof tot, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (tot > (unsigned long long)INT32_MAX - 64 || tot > (unsigned long long)lv.A.nnz + (unsigned long long)lv.A.nnz / 8)
        return cudaSuccess;
    AMG_CUDA_TRY(dalloc(h, &sci, (size_t)tot));
    AMG_CUDA_TRY(dalloc(h, &sv64, (size_t)tot));
    SpmvPlan &pa = lv.plan_a;
    pa.ns = nsl;
    pa.sw = sw;
    pa.sp = sp;
    AMG_CUDA_TRY(sell_fill_d(lv.A.n, lv.A.rp, lv.A.ci, lv.A.v, pa.ns, pa.sp, pa.sw, sci, sv64, s));
    pa.sci = sci;
    pa.sv64 = sv64;
    pa.sell_entries = (size_t)tot;
    return cudaSuccess;
}

amg_status_t build_level(amg_hierarchy *h, int L, int *coarsest)
{
    amg_status_t st = AMG_OK;
    cudaStream_t s = h->s;
    const amg_params_t &p = h->p;
    Level &lv = h->lev[L];
    DevCsr &A = lv.A;
    const int n = A.n;
    int *kept = nullptr, *grp = nullptr, *gci = nullptr, *mstart = nullptr, *members = nullptr, *fill = nullptr;
    int *flags = nullptr;
    unsigned long long *t0 = nullptr, *t1 = nullptr;
    int *rootof = nullptr, *join1 = nullptr;
    uint8_t *drop = nullptr;
    double *px = nullptr, *py = nullptr, *scal = nullptr, *lvals = nullptr, *ldiag = nullptr;
    uint8_t *own_mask = nullptr;
    int *nrp = nullptr, *nci = nullptr, *ptrp = nullptr, *ptci = nullptr;   // systems: node graph, Pt
    double *nF = nullptr, *fdiag = nullptr, *W = nullptr, *Qv = nullptr, *ptv = nullptr;
    uint8_t *nstrong = nullptr;
    int nnz_n = 0;
    DevCsr AP, Ac;
    int hflags[5] = {0, 0, 0, 0, 0};
    SpmvPlan plan_bar;
    int nagg = 0, rounds = 0, nnz_g = 0, nnz_bar = 0, nnz_p = 0, ovf = 0;
    *coarsest = 0;

    CK(dalloc(h, &lv.strong, (size_t)A.nnz));
    CK(dalloc(h, &lv.removed, (size_t)A.nnz));
    CK(cudaMallocAsync(&kept, sizeof(int) * (size_t)(n + 1), s));
    CK(cudaMallocAsync(&flags, sizeof(int) * 5, s));
    CK(cudaMemsetAsync(flags, 0, sizeof(int) * 5, s));
    if (h->block) {
        // a system of PDEs: block strength between nodes, MIS-2 of the node graph, QR
        // tentative prolongator, P = Pt - omega Dbar^-1 (Abar Pt)
        const int bs = lv.bs, k = lv.k, nn = n / bs;
        CK(cudaMallocAsync(&nrp, sizeof(int) * (size_t)(nn + 1), s));
        CK(node_counts(A, bs, nrp, s));
        CK(scan_exclusive(nrp, nrp, nn, s));
        CK(cudaMemcpyAsync(&nnz_n, nrp + nn, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        CK(cudaMallocAsync(&nci, sizeof(int) * (size_t)(nnz_n > 0 ? nnz_n : 1), s));
        CK(cudaMallocAsync(&nF, sizeof(double) * (size_t)(nnz_n > 0 ? nnz_n : 1), s));
        CK(cudaMallocAsync(&fdiag, sizeof(double) * (size_t)(nn > 0 ? nn : 1), s));
        CK(cudaMallocAsync(&nstrong, (size_t)(nnz_n > 0 ? nnz_n : 1), s));
        CK(node_fill(A, bs, nrp, nci, nF, fdiag, s));
        CK(node_strength(nn, nrp, nci, nF, fdiag, p.theta, nstrong, s));
        CK(block_masks(A, bs, nrp, nci, nstrong, lv.strong, lv.removed, kept, s));
        DevCsr G;
        G.n = nn;
        G.ncol = nn;
        G.nnz = nnz_n;
        G.rp = nrp;
        G.ci = nci;
        CK(cudaMallocAsync(&grp, sizeof(int) * (size_t)(nn + 1), s));
        CK(strong_graph_counts(G, nstrong, grp, s));
        CK(scan_exclusive(grp, grp, nn, s));
        CK(cudaMemcpyAsync(&nnz_g, grp + nn, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        CK(cudaMallocAsync(&gci, sizeof(int) * (size_t)(nnz_g > 0 ? nnz_g : 1), s));
        CK(strong_graph_fill(G, nstrong, grp, gci, s));
        trace_mark(h, L, AMG_PH_STRENGTH);
        CK(dalloc(h, &lv.agg, (size_t)nn));
        CK(dalloc(h, &lv.root, (size_t)nn));
        CK(cudaMallocAsync(&t0, sizeof(unsigned long long) * (size_t)(nn > 0 ? nn : 1), s));
        CK(cudaMallocAsync(&t1, sizeof(unsigned long long) * (size_t)(nn > 0 ? nn : 1), s));
        CK(cudaMallocAsync(&rootof, sizeof(int) * (size_t)(nn + 1), s));
        CK(cudaMallocAsync(&join1, sizeof(int) * (size_t)(nn + 1), s));
        {
            AggWork w{t0, t1, rootof, join1, flags + 2};
            cudaError_t e = aggregate_mis2(nn, grp, gci, p.seed, L, w, lv.agg, lv.root, &nagg, &rounds, s);
            if (e == cudaErrorInvalidValue) { g_last_error = "aggregation left a node unassigned"; st = AMG_ERR_INTERNAL; goto done; }
            CK(e);
        }
        lv.nagg = nagg;
        trace_mark(h, L, AMG_PH_AGGREGATE);
        if (nagg == 0 || (int64_t)nagg * k >= (int64_t)n) { *coarsest = 1; goto done; }
        const int nc = nagg * k;
        CK(cudaMallocAsync(&mstart, sizeof(int) * (size_t)(nagg + 1), s));
        CK(cudaMallocAsync(&members, sizeof(int) * (size_t)nn, s));
        CK(cudaMallocAsync(&fill, sizeof(int) * (size_t)(nagg + 1), s));
        CK(aggregate_members(nn, nagg, lv.agg, mstart, members, fill, s));
        CK(cudaMallocAsync(&W, sizeof(double) * (size_t)n * (size_t)k, s));
        CK(cudaMallocAsync(&Qv, sizeof(double) * (size_t)n * (size_t)k, s));
        CK(dalloc(h, &lv.Bc, (size_t)nc * (size_t)k));
        CK(block_tentative(n, bs, k, nagg, mstart, members, lv.B, W, Qv, lv.Bc, flags + 0, s));
        // filtered matrix: dropped entries lumped into the diagonal (Eq. 6)
        lv.Abar.n = n;
        lv.Abar.ncol = n;
        CK(dalloc(h, &lv.Abar.rp, (size_t)n + 1));
        CK(scan_exclusive(kept, lv.Abar.rp, n, s));
        CK(cudaMemcpyAsync(&nnz_bar, lv.Abar.rp + n, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hflags, flags, sizeof(int) * 5, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hflags[0]) {
            g_last_error = "an aggregate too small to carry the near-null space";
            st = AMG_ERR_UNSUPPORTED;
            goto done;
        }
        lv.Abar.nnz = nnz_bar;
        CK(dalloc(h, &lv.Abar.ci, (size_t)nnz_bar));
        CK(dalloc(h, &lv.Abar.v, (size_t)nnz_bar));
        CK(dalloc(h, &lv.Dsm, (size_t)n));
        CK(dalloc(h, &lv.lumpflag, (size_t)n));
        CK(filter(A, lv.removed, 0, p.tau, 0, p.sigma, lv.Abar, lv.Dsm, lv.lumpflag, flags + 1, s));
        CK(cudaMemcpyAsync(hflags, flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hflags[1]) { g_last_error = "zero diagonal in the filtered matrix"; st = AMG_ERR_ZERO_DIAG; goto done; }
        trace_mark(h, L, AMG_PH_FILTER);
        CK(cudaMallocAsync(&px, sizeof(double) * (size_t)n, s));
        CK(cudaMallocAsync(&py, sizeof(double) * (size_t)n, s));
        {
            int np = 2 * spmv_partials_needed(n);
            CK(cudaMallocAsync(&scal, sizeof(double) * (size_t)((np > kReduceBlocks ? np : kReduceBlocks) + 8), s));
        }
        {
            SpmvPlan *pls[2] = {&plan_bar, &lv.plan_a};
            const int *rps[2] = {lv.Abar.rp, A.rp};
            const int ns[2] = {n, n};
            const int64_t nz[2] = {lv.Abar.nnz, A.nnz};
            CK(spmv_plans(2, pls, rps, ns, nz, s));
        }
        if (p.lambda_override > 0.0) {
            lv.lambda_bar = p.lambda_override;
        } else {
            CK(power_lambda(lv.Abar, plan_bar, lv.Dsm, p.power_iters, power_stream_seed(p.seed, L, 1), px, py,
                            scal + 8, scal, scal + 1, s));
            CK(cudaMemcpyAsync(&lv.lambda_bar, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        }
        if (!(lv.lambda_bar > 0.0) || !std::isfinite(lv.lambda_bar)) {
            g_last_error = "eigenvalue estimate not positive";
            st = AMG_ERR_EIGEN;
            goto done;
        }
        lv.omega = 4.0 / (3.0 * lv.lambda_bar);
        CK(cudaMemcpyAsync(scal + 2, &lv.omega, sizeof(double), cudaMemcpyHostToDevice, s));
        trace_mark(h, L, AMG_PH_EIGEN);
        {
            DevCsr Pt;
            Pt.n = n;
            Pt.ncol = nc;
            Pt.nnz = (int64_t)n * k;
            CK(cudaMallocAsync(&ptrp, sizeof(int) * ((size_t)n + 17), s));
            CK(cudaMallocAsync(&ptci, sizeof(int) * ((size_t)n * k + 16), s));
            CK(cudaMallocAsync(&ptv, sizeof(double) * ((size_t)n * k + 16), s));
            Pt.rp = ptrp;
            Pt.ci = ptci;
            Pt.v = ptv;
            CK(block_pt(n, bs, k, lv.agg, Qv, Pt, s));
            cudaError_t e = spgemm(lv.Abar, Pt, lv.P, &ovf, s);
            if (e == cudaErrorInvalidValue && ovf) { g_last_error = "hash table overflow in Abar*Pt"; st = AMG_ERR_INTERNAL; goto done; }
            CK(e);
            own(h, lv.P);
            nnz_p = (int)lv.P.nnz;
        }
        CK(block_combine(n, bs, k, lv.agg, Qv, lv.Dsm, scal + 2, lv.P, s));
        CK(dalloc(h, &lv.cflag, (size_t)n));
        CK(cudaMemsetAsync(lv.cflag, 0, (size_t)n, s));
        lv.R.n = nc;
        lv.R.ncol = n;
        lv.R.nnz = nnz_p;
        CK(dalloc(h, &lv.R.rp, (size_t)nc + 1));
        CK(dalloc(h, &lv.R.ci, (size_t)nnz_p));
        CK(dalloc(h, &lv.R.v, (size_t)nnz_p));
        CK(transpose_counts(lv.P, lv.R.rp, s));
        CK(scan_exclusive(lv.R.rp, lv.R.rp, nc, s));
        CK(cudaFreeAsync(fill, s));
        fill = nullptr;
        CK(cudaMallocAsync(&fill, sizeof(int) * (size_t)(nc + 1), s));
        CK(transpose_fill(lv.P, lv.R, fill, s));
        trace_mark(h, L, AMG_PH_PROLONG);
        goto galerkin;
    }
    // Eq. (7), on A or (§3.1) on the distance Laplacian of the level's coordinates; the strong
    // graph's row lengths come with it unless the nonsymmetric case changes the strong set
    CK(cudaMallocAsync(&grp, sizeof(int) * (size_t)(n + 1), s));
    if (p.strength == AMG_STRENGTH_DISTANCE) {
        CK(cudaMallocAsync(&lvals, sizeof(double) * (size_t)(A.nnz > 0 ? A.nnz : 1), s));
        CK(cudaMallocAsync(&ldiag, sizeof(double) * (size_t)(n > 0 ? n : 1), s));
        CK(distance_laplacian(A, lv.coords, h->dim, lvals, ldiag, flags + 4, s));
        DevCsr Ld = A;
        Ld.v = lvals;
        CK(strength(Ld, ldiag, p.theta, lv.strong, lv.removed, kept, s, grp));
    } else {
        CK(strength(A, lv.diag, p.theta, lv.strong, lv.removed, kept, s, grp));
    }
    if (p.krylov == AMG_KRYLOV_GMRES) {
        // nonsymmetric operator: i-j strong when either direction passes Eq. (7)
        CK(cudaMallocAsync(&own_mask, (size_t)(A.nnz > 0 ? A.nnz : 1), s));
        CK(cudaMemcpyAsync(own_mask, lv.strong, (size_t)A.nnz, cudaMemcpyDeviceToDevice, s));
        CK(symmetrize_strength(A, own_mask, lv.strong, lv.removed, kept, s));
        CK(strong_graph_counts(A, lv.strong, grp, s));
    }
    // strong graph
    CK(scan_exclusive(grp, grp, n, s));
    CK(cudaMemcpyAsync(&nnz_g, grp + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaMallocAsync(&gci, sizeof(int) * (size_t)(nnz_g > 0 ? nnz_g : 1), s));
    CK(strong_graph_fill(A, lv.strong, grp, gci, s));
    trace_mark(h, L, AMG_PH_STRENGTH);
    // aggregation
    CK(dalloc(h, &lv.agg, (size_t)n));
    CK(dalloc(h, &lv.root, (size_t)n));
    CK(cudaMallocAsync(&t0, sizeof(unsigned long long) * (size_t)(n > 0 ? n : 1), s));
    CK(cudaMallocAsync(&t1, sizeof(unsigned long long) * (size_t)(n > 0 ? n : 1), s));
    CK(cudaMallocAsync(&rootof, sizeof(int) * (size_t)(n + 1), s));
    CK(cudaMallocAsync(&join1, sizeof(int) * (size_t)(n + 1), s));
    {
        AggWork w{t0, t1, rootof, join1, flags + 2};
        cudaError_t e = aggregate_mis2(n, grp, gci, p.seed, L, w, lv.agg, lv.root, &nagg, &rounds, s);
        if (e == cudaErrorInvalidValue) { g_last_error = "aggregation left a vertex unassigned"; st = AMG_ERR_INTERNAL; goto done; }
        CK(e);
    }
    lv.nagg = nagg;
    trace_mark(h, L, AMG_PH_AGGREGATE);
    if (nagg == n || nagg == 0) { *coarsest = 1; goto done; }
    // members and tentative-prolongator column norms
    CK(cudaMallocAsync(&mstart, sizeof(int) * (size_t)(nagg + 1), s));
    CK(cudaMallocAsync(&members, sizeof(int) * (size_t)n, s));
    CK(cudaMallocAsync(&fill, sizeof(int) * (size_t)(nagg + 1), s));
    CK(aggregate_members(n, nagg, lv.agg, mstart, members, fill, s));
    if (lv.coords) {
        Level &nx = h->lev[L + 1];
        CK(dalloc(h, &nx.coords, (size_t)nagg * (size_t)h->dim));
        CK(coarse_coords(nagg, mstart, members, lv.coords, h->dim, nx.coords, s));
    }
    CK(dalloc(h, &lv.nrm, (size_t)nagg));
    CK(aggregate_norms(nagg, mstart, members, lv.B, lv.nrm, flags + 0, s));
    // §2.5
    if (p.variants & AMG_VAR_SPRSFY) {
        CK(cudaMallocAsync(&drop, (size_t)(A.nnz > 0 ? A.nnz : 1), s));
        CK(sprsfy(A, lv.strong, lv.agg, lv.root, nagg, mstart, members, drop, lv.removed, kept, s));
    }
    // filtered matrix and smoothing diagonal
    lv.Abar.n = n;
    lv.Abar.ncol = n;
    CK(dalloc(h, &lv.Abar.rp, (size_t)n + 1));
    CK(scan_exclusive(kept, lv.Abar.rp, n, s));
    CK(cudaMemcpyAsync(&nnz_bar, lv.Abar.rp + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hflags, flags, sizeof(int) * 5, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hflags[4]) { g_last_error = "two coupled rows at the same coordinates"; st = AMG_ERR_INVALID_ARG; goto done; }
    if (hflags[0]) { g_last_error = "near-null space is zero on an aggregate"; st = AMG_ERR_INVALID_ARG; goto done; }
    lv.Abar.nnz = nnz_bar;
    CK(dalloc(h, &lv.Abar.ci, (size_t)nnz_bar));
    CK(dalloc(h, &lv.Abar.v, (size_t)nnz_bar));
    CK(dalloc(h, &lv.Dsm, (size_t)n));
    CK(dalloc(h, &lv.lumpflag, (size_t)n));
    CK(filter(A, lv.removed, (p.variants & AMG_VAR_OFFLMP) ? 1 : 0, p.tau, (p.variants & AMG_VAR_1NORM) ? 1 : 0,
              p.sigma, lv.Abar, lv.Dsm, lv.lumpflag, flags + 1, s));
    CK(cudaMemcpyAsync(hflags, flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!(p.variants & AMG_VAR_1NORM) && hflags[1]) {
        g_last_error = "zero diagonal in the filtered matrix";
        st = AMG_ERR_ZERO_DIAG;
        goto done;
    }
    trace_mark(h, L, AMG_PH_FILTER);
    // eigenvalue of Dsm^-1 Abar and omega = 4 / (3 lambda), Eq. (3)
    CK(cudaMallocAsync(&px, sizeof(double) * (size_t)n, s));
    CK(cudaMallocAsync(&py, sizeof(double) * (size_t)n, s));
    {
        // 8 scalars, then the partial sums of the power method's dot products
        // the power method's two partial sums per SpMV block
        int np = 2 * spmv_partials_needed(n);
        CK(cudaMallocAsync(&scal, sizeof(double) * (size_t)((np > kReduceBlocks ? np : kReduceBlocks) + 8), s));
    }
    // launch plans of the filtered matrix (λ̄ power method) and of A_l (λ* power method, and
    // every V-cycle), with one synchronisation
    {
        SpmvPlan *pls[2] = {&plan_bar, &lv.plan_a};
        const int *rps[2] = {lv.Abar.rp, A.rp};
        const int ns[2] = {n, n};
        const int64_t nz[2] = {lv.Abar.nnz, A.nnz};
        CK(spmv_plans(2, pls, rps, ns, nz, s));
    }
    if (p.lambda_override > 0.0) {
        lv.lambda_bar = p.lambda_override;
    } else if ((p.variants & AMG_VAR_1NORM) && p.onenorm_lambda == AMG_LAMBDA_ONE) {
        lv.lambda_bar = 1.0;
    } else {
        CK(power_lambda(lv.Abar, plan_bar, lv.Dsm, p.power_iters, power_stream_seed(p.seed, L, 1), px, py, scal + 8, scal,
                        scal + 1, s));
        CK(cudaMemcpyAsync(&lv.lambda_bar, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    if (!(lv.lambda_bar > 0.0) || !std::isfinite(lv.lambda_bar)) {
        char buf[128];
        snprintf(buf, sizeof buf, "eigenvalue estimate %.17g on level %d", lv.lambda_bar, L);
        g_last_error = buf;
        st = AMG_ERR_EIGEN;
        goto done;
    }
    lv.omega = 4.0 / (3.0 * lv.lambda_bar);
    CK(cudaMemcpyAsync(scal + 2, &lv.omega, sizeof(double), cudaMemcpyHostToDevice, s));
    trace_mark(h, L, AMG_PH_EIGEN);
    // smoothed prolongator (unit basis), Algorithm 3, column scaling
    lv.P.n = n;
    lv.P.ncol = nagg;
    CK(dalloc(h, &lv.P.rp, (size_t)n + 1));
    CK(smooth_counts(lv.Abar, lv.agg, lv.P.rp, s));
    CK(scan_exclusive(lv.P.rp, lv.P.rp, n, s));
    CK(cudaMemcpyAsync(&nnz_p, lv.P.rp + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    lv.P.nnz = nnz_p;
    CK(dalloc(h, &lv.P.ci, (size_t)nnz_p));
    CK(dalloc(h, &lv.P.v, (size_t)nnz_p));
    CK(smooth_fill(lv.Abar, lv.agg, lv.B, lv.Dsm, scal + 2, lv.P, s));
    CK(dalloc(h, &lv.cflag, (size_t)n));
    CK(cudaMemsetAsync(lv.cflag, 0, (size_t)n, s));
    if (p.variants & AMG_VAR_CNSTRNT) CK(constrain(lv.P, lv.agg, lv.B, lv.cflag, s));
    if (p.pt_scaling == AMG_PT_ORTHONORMAL) CK(scale_columns(lv.P, lv.nrm, s));
    // R = P^T
    lv.R.n = nagg;
    lv.R.ncol = n;
    lv.R.nnz = nnz_p;
    CK(dalloc(h, &lv.R.rp, (size_t)nagg + 1));
    CK(dalloc(h, &lv.R.ci, (size_t)nnz_p));
    CK(dalloc(h, &lv.R.v, (size_t)nnz_p));
    CK(transpose_counts(lv.P, lv.R.rp, s));
    CK(scan_exclusive(lv.R.rp, lv.R.rp, nagg, s));
    CK(transpose_fill(lv.P, lv.R, fill, s));
    trace_mark(h, L, AMG_PH_PROLONG);
galerkin:
    // Galerkin product with the original A, Eq. (2)
    {
        cudaError_t e;
        {
            ProfScope ps(KC_SPGEMM, s, 0.0);
            e = spgemm(A, lv.P, AP, &ovf, s);
            ps.bytes = csr_bytes(A) + csr_bytes(lv.P) + csr_bytes(AP);
        }
        if (e == cudaErrorInvalidValue && ovf) { g_last_error = "hash table overflow in A*P"; st = AMG_ERR_INTERNAL; goto done; }
        CK(e);
        trace_mark(h, L, AMG_PH_GALERKIN_AP);
        {
            ProfScope ps(KC_SPGEMM, s, 0.0);
            e = spgemm(lv.R, AP, Ac, &ovf, s);
            ps.bytes = csr_bytes(lv.R) + csr_bytes(AP) + csr_bytes(Ac);
        }
        if (e == cudaErrorInvalidValue && ovf) { g_last_error = "hash table overflow in R*(AP)"; st = AMG_ERR_INTERNAL; goto done; }
        CK(e);
        trace_mark(h, L, AMG_PH_GALERKIN_RAP);
    }
    // Chebyshev smoother: lambda_max(D^-1 A_L) and D^-1 (the finest level's power method on
    // its sliced-ELL copy, made here rather than with the other levels' copies)
    if (L == 0) CK(sell_build_fine(h, lv, s));
    CK(dalloc(h, &lv.invdiag, (size_t)n));
    if (p.precision == AMG_MIXED) CK(dalloc(h, &lv.invdiag_f, (size_t)n));
    CK(invert_diag(lv.diag, lv.invdiag, lv.invdiag_f, n, flags + 3, s));
    CK(power_lambda(A, lv.plan_a, lv.diag, p.power_iters, power_stream_seed(p.seed, L, 2), px, py, scal + 8, scal,
                    scal + 1, s));
    CK(cudaMemcpyAsync(&lv.lambda_cheb, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hflags, flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hflags[3]) { g_last_error = "zero diagonal in a level operator"; st = AMG_ERR_ZERO_DIAG; goto done; }
    if (!(lv.lambda_cheb > 0.0) || !std::isfinite(lv.lambda_cheb)) {
        g_last_error = "Chebyshev eigenvalue estimate not positive";
        st = AMG_ERR_EIGEN;
        goto done;
    }
    trace_mark(h, L, AMG_PH_SMOOTHER);
    // next level
    {
        Level &nx = h->lev[L + 1];
        nx.A = Ac;
        own(h, Ac);
        Ac = DevCsr();
        nx.bs = lv.k;
        nx.k = lv.k;
        if (h->block) {
            nx.B = lv.Bc;           // R_a of every aggregate: k vectors of length nagg k
            lv.Bc = nullptr;
        } else {
            CK(dalloc(h, &nx.B, (size_t)nagg));
            if (p.pt_scaling == AMG_PT_ORTHONORMAL)
                CK(cudaMemcpyAsync(nx.B, lv.nrm, sizeof(double) * (size_t)nagg, cudaMemcpyDeviceToDevice, s));
            else if (nagg > 0) {
                ones_kernel<<<grid_for(nagg, 256), 256, 0, s>>>(nagg, nx.B); note_launch();
            }
        }
        CK(cudaGetLastError());
    }
done:
    for (void *p : {(void *)kept, (void *)grp, (void *)gci, (void *)mstart, (void *)members, (void *)fill,
                    (void *)flags, (void *)t0, (void *)t1, (void *)rootof, (void *)join1, (void *)drop, (void *)px,
                    (void *)py, (void *)scal, (void *)AP.rp, (void *)AP.ci, (void *)AP.v, (void *)Ac.rp,
                    (void *)Ac.ci, (void *)Ac.v, (void *)lvals, (void *)ldiag, (void *)own_mask, (void *)nrp,
                    (void *)nci, (void *)nF, (void *)fdiag, (void *)nstrong, (void *)W, (void *)Qv, (void *)ptrp,
                    (void *)ptci, (void *)ptv})
        free_async(p, s);
    cudaStreamSynchronize(s);
    return st;
}

// Coarsest levels above this many rows (and sparse) may take the Chebyshev solve instead of the
// dense inverse
constexpr int kCoarsePolyMinRows = 512;

// The dense inverse of the coarsest operator into h->coarse_inv (coarse.cu: the Cholesky-based
// inverse, CG on the columns of a large sparse SPD operator, Newton-Schulz for a nonsymmetric
// one).  Synchronises h->s.
amg_status_t form_coarse_inverse(amg_hierarchy *h)
{
    amg_status_t st = AMG_OK;
    cudaStream_t s = h->s;
    const DevCsr &A = h->lev[h->nlev - 1].A;
    const int nc = A.n;
    double *inv = nullptr;
    void *cwork = nullptr;
    int *info_dev = nullptr;
    int info = 0;
    if (nc > 8192) {
        g_last_error = "coarsest level too large for the dense solve";
        return AMG_ERR_UNSUPPORTED;
    }
    CK(dalloc(h, &inv, (size_t)nc * nc));
    CK(cudaMallocAsync(&cwork, coarse_work_bytes(nc), s));
    CK(cudaMallocAsync(&info_dev, sizeof(int), s));
    CK(coarse_inverse(A, cwork, inv, info_dev, s, h->p.krylov == AMG_KRYLOV_GMRES));
    CK(cudaMemcpyAsync(&info, info_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (info < 0) { g_last_error = "coarsest operator singular or too ill-conditioned for its inverse"; st = AMG_ERR_COARSE_NOT_SPD; goto done; }
    if (info) { g_last_error = "coarsest operator not positive definite"; st = AMG_ERR_COARSE_NOT_SPD; goto done; }
    h->coarse_inv = inv;
done:
    free_async(cwork, s);
    free_async(info_dev, s);
    return st;
}

amg_status_t prepare_solve(amg_hierarchy *h)
{
    amg_status_t st = AMG_OK;
    cudaStream_t s = h->s;
    const bool mixed = h->p.precision == AMG_MIXED;
    const size_t ts = mixed ? sizeof(float) : sizeof(double);
    const int n0 = h->lev[0].A.n;
    SolveCtx &c = h->ctx;
    c = SolveCtx();
    c.nlev = h->nlev;
    c.cheb_degree = h->p.cheb_degree;
    c.cheb_ratio = h->p.cheb_ratio;
    c.cheb_boost = h->p.cheb_boost;
    c.mixed = mixed ? 1 : 0;
    for (int L = 0; L < h->nlev; ++L) {
        Level &lv = h->lev[L];
        const int n = lv.A.n;
        const bool last = (L == h->nlev - 1);
        CK(dalloc(h, (char **)&lv.vf, (size_t)n * ts));
        CK(dalloc(h, (char **)&lv.vx, (size_t)n * ts));
        LevelView &v = c.lev[L];
        v.n = n;
        v.f = lv.vf;
        v.x = lv.vx;
        if (!last) {
            CK(dalloc(h, (char **)&lv.vx2, (size_t)n * ts));
            CK(dalloc(h, (char **)&lv.vr, (size_t)n * ts));
            CK(dalloc(h, (char **)&lv.vd, (size_t)n * ts));
            v.x2 = lv.vx2;
            v.r = lv.vr;
            v.d = lv.vd;
            v.nc = lv.R.n;
            v.arp = lv.A.rp; v.aci = lv.A.ci;
            v.prp = lv.P.rp; v.pci = lv.P.ci;
            v.rrp = lv.R.rp; v.rci = lv.R.ci;
            v.lambda = lv.lambda_cheb;
            v.nnz_a = lv.A.nnz;
            // plan_a was made during setup; plan_p and plan_r below, all levels at once
            if (mixed) {
                CK(dalloc(h, &lv.Af, (size_t)lv.A.nnz));
                CK(dalloc(h, &lv.Pf, (size_t)lv.P.nnz));
                CK(dalloc(h, &lv.Rf, (size_t)lv.R.nnz));
                CK(convert_d2f(lv.A.v, lv.Af, lv.A.nnz, s));
                CK(convert_d2f(lv.P.v, lv.Pf, lv.P.nnz, s));
                CK(convert_d2f(lv.R.v, lv.Rf, lv.R.nnz, s));
                v.av = lv.Af; v.pv = lv.Pf; v.rv = lv.Rf; v.invdiag = lv.invdiag_f;
            } else {
                v.av = lv.A.v; v.pv = lv.P.v; v.rv = lv.R.v; v.invdiag = lv.invdiag;
            }
        } else if (h->coarse_degree > 0) {
            // the Chebyshev coarse solve: A, D^-1 and two more vectors of the coarsest level
            CK(dalloc(h, (char **)&lv.vx2, (size_t)n * ts));
            CK(dalloc(h, (char **)&lv.vd, (size_t)n * ts));
            v.x2 = lv.vx2;
            v.d = lv.vd;
            v.arp = lv.A.rp; v.aci = lv.A.ci;
            v.nnz_a = lv.A.nnz;
            if (mixed) {
                CK(dalloc(h, &lv.Af, (size_t)lv.A.nnz));
                CK(convert_d2f(lv.A.v, lv.Af, lv.A.nnz, s));
                v.av = lv.Af; v.invdiag = lv.invdiag_f;
            } else {
                v.av = lv.A.v; v.invdiag = lv.invdiag;
            }
        }
    }
    c.coarse_n = h->lev[h->nlev - 1].A.n;
    c.coarse_inv = h->coarse_inv;
    c.coarse_degree = h->coarse_degree;
    c.coarse_theta = h->coarse_theta;
    c.coarse_delta = h->coarse_delta;
    // PCG vectors
    CK(dalloc(h, &h->b, (size_t)n0));
    CK(dalloc(h, &h->x, (size_t)n0));
    CK(dalloc(h, &h->r, (size_t)n0));
    CK(dalloc(h, &h->z, (size_t)n0));
    CK(dalloc(h, &h->pv, (size_t)n0));
    CK(dalloc(h, &h->q, (size_t)n0));
    CK(dalloc(h, &h->t, (size_t)n0));
    h->zb[0] = h->z;
    if (mixed) {
        CK(dalloc(h, &h->z_prev, (size_t)n0));
        h->zb[1] = h->z_prev;
    }
    CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    {
        int np = spmv_partials_needed(n0);
        CK(dalloc(h, &h->partial, (size_t)(np > kReduceBlocks ? np : kReduceBlocks)));
        CK(dalloc(h, &h->partial2, (size_t)kReduceBlocks));
        CK(dalloc(h, &h->partial3, (size_t)kReduceBlocks));
        CK(cudaMallocHost(&h->rr_host, sizeof(double) * kReduceBlocks));
    }
    // launch plans of every P and R (and of A_0 when level 0 is the coarsest), one sync
    {
        std::vector<SpmvPlan *> pls;
        std::vector<const int *> rps;
        std::vector<int> ns;
        std::vector<int64_t> nz;
        for (int L = 0; L + 1 < h->nlev; ++L) {
            Level &lv = h->lev[L];
            pls.push_back(&lv.plan_p); rps.push_back(lv.P.rp); ns.push_back(lv.A.n); nz.push_back(lv.P.nnz);
            pls.push_back(&lv.plan_r); rps.push_back(lv.R.rp); ns.push_back(lv.R.n); nz.push_back(lv.R.nnz);
        }
        if (h->nlev == 1 && n0 > 0) {
            pls.push_back(&h->plan0); rps.push_back(h->lev[0].A.rp); ns.push_back(n0); nz.push_back(h->lev[0].A.nnz);
        }
        // sliced-ELL copies of the level operators with short rows (sell_wanted; their layout
        // first; the entry counts reach the host with the plans' synchronisation).  The finest
        // level's FP64 copy exists already (sell_build_fine).
        std::vector<int> sell_levels;
        unsigned long long *tot_host = (unsigned long long *)h->rr_host;
        int dev = 0, l2 = 0, nsm = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        for (int L = 0; L + 1 < h->nlev; ++L) {
            Level &lv = h->lev[L];
            if (!sell_wanted(h, lv, l2, nsm) || (int)sell_levels.size() >= kReduceBlocks) continue;
            const int nsl = sell_slices(lv.A.n);
            int *sw = nullptr, *sp = nullptr;
            unsigned long long *t64 = nullptr;
            CK(dalloc(h, &sw, (size_t)nsl));
            CK(dalloc(h, &sp, (size_t)nsl + 1));
            CK(dalloc(h, &t64, 1));
            CK(sell_layout(lv.A.n, lv.A.rp, sw, sp, t64, s));
            CK(cudaMemcpyAsync(tot_host + sell_levels.size(), t64, sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, s));
            lv.plan_a.sw = sw;
            lv.plan_a.sp = sp;
            sell_levels.push_back(L);
        }
        CK(spmv_plans((int)pls.size(), pls.data(), rps.data(), ns.data(), nz.data(), s));
        if (!sell_levels.empty()) CK(cudaStreamSynchronize(s));
        for (size_t k = 0; k < sell_levels.size(); ++k) {
            Level &lv = h->lev[sell_levels[k]];
            SpmvPlan &pa = lv.plan_a;
            // no copy when the offsets would overflow or the padding exceeds an eighth
            if (tot_host[k] > (unsigned long long)INT32_MAX - 64 ||
                tot_host[k] > (unsigned long long)lv.A.nnz + (unsigned long long)lv.A.nnz / 8)
                continue;
            pa.ns = sell_slices(lv.A.n);
            const size_t total = (size_t)tot_host[k];
            int *sci = nullptr;
            CK(dalloc(h, &sci, total));
            double *sv64 = nullptr;
            if (!mixed || sell_levels[k] == 0) CK(dalloc(h, &sv64, total));   // FP64 products: PCG, FP64 V-cycle
            CK(sell_fill_d(lv.A.n, lv.A.rp, lv.A.ci, lv.A.v, pa.ns, pa.sp, pa.sw, sci, sv64, s));
            pa.sci = sci;
            pa.sv64 = sv64;
            pa.sell_entries = total;
            if (mixed) {
                float *sv32 = nullptr;
                CK(dalloc(h, &sv32, total));
                CK(sell_fill_f(lv.A.n, lv.A.rp, lv.Af, pa.ns, pa.sp, pa.sw, sv32, s));
                pa.sv32 = sv32;
            }
        }
        // the FP32 values of a copy made during setup (the finest level's)
        for (int L = 0; mixed && L + 1 < h->nlev; ++L) {
            Level &lv = h->lev[L];
            SpmvPlan &pa = lv.plan_a;
            if (!pa.sci || pa.sv32) continue;
            float *sv32 = nullptr;
            CK(dalloc(h, &sv32, pa.sell_entries));
            CK(sell_fill_f(lv.A.n, lv.A.rp, lv.Af, pa.ns, pa.sp, pa.sw, sv32, s));
            pa.sv32 = sv32;
        }
        // rows far longer than their operator's mean leave the row tiles of every solve product
        {
            std::vector<SpmvPlan *> sp;
            std::vector<const int *> srp;
            std::vector<int> sn;
            std::vector<int64_t> snz;
            for (int L = 0; L + 1 < h->nlev; ++L) {
                Level &lv = h->lev[L];
                sp.push_back(&lv.plan_a); srp.push_back(lv.A.rp); sn.push_back(lv.A.n); snz.push_back(lv.A.nnz);
                sp.push_back(&lv.plan_p); srp.push_back(lv.P.rp); sn.push_back(lv.A.n); snz.push_back(lv.P.nnz);
                sp.push_back(&lv.plan_r); srp.push_back(lv.R.rp); sn.push_back(lv.R.n); snz.push_back(lv.R.nnz);
            }
            if (h->nlev == 1 && n0 > 0) {
                sp.push_back(&h->plan0); srp.push_back(h->lev[0].A.rp); sn.push_back(n0); snz.push_back(h->lev[0].A.nnz);
            }
            if (h->coarse_degree > 0) {
                Level &cl = h->lev[h->nlev - 1];
                sp.push_back(&cl.plan_a); srp.push_back(cl.A.rp); sn.push_back(cl.A.n); snz.push_back(cl.A.nnz);
            }
            CK(spmv_split_rows((int)sp.size(), sp.data(), srp.data(), sn.data(), snz.data(),
                               [h](int **list, size_t count) { return dalloc(h, list, count); }, s));
            // the prolongators' short rows: a thread per row (the products with P only)
            std::vector<SpmvPlan *> pp;
            std::vector<const int *> prp;
            std::vector<int> pn;
            std::vector<int64_t> pnz;
            for (int L = 0; L + 1 < h->nlev; ++L) {
                Level &lv = h->lev[L];
                pp.push_back(&lv.plan_p); prp.push_back(lv.P.rp); pn.push_back(lv.A.n); pnz.push_back(lv.P.nnz);
            }
            CK(spmv_short_rows((int)pp.size(), pp.data(), prp.data(), pn.data(), pnz.data(), s));
        }
        if (h->nlev > 1) h->plan0 = h->lev[0].plan_a;
        for (int L = 0; L + 1 < h->nlev; ++L) {
            Level &lv = h->lev[L];
            c.lev[L].plan_a = lv.plan_a;
            c.lev[L].plan_p = lv.plan_p;
            c.lev[L].plan_r = lv.plan_r;
        }
        if (h->coarse_degree > 0) c.lev[h->nlev - 1].plan_a = h->lev[h->nlev - 1].plan_a;
    }
    CK(dalloc(h, (char **)&h->sc, sizeof(PcgScalars)));
    CK(dalloc(h, &h->counters, 8));
    CK(cudaMemsetAsync(h->counters, 0, sizeof(unsigned) * 8, s));
done:
    return st;
}

// ----------------------------------------------------------------------- PCG iteration pieces
// tail: z = M^-1 r (V-cycle), then p = z + beta p;  head: q = A p with p.q, alpha, x and r
// update, r.r partial sums copied to the host.  Parity selects the z buffer in mixed mode.
cudaError_t pcg_tail(amg_hierarchy *h, int parity, cudaStream_t s)
{
    const int n = h->lev[0].A.n;
    double *z = h->zb[h->zb[1] ? parity : 0];
    double *zp = h->zb[1] ? h->zb[1 - parity] : nullptr;
    AMG_CUDA_TRY(vcycle(h->ctx, h->r, z, s));
    return pcg_update_p(n, h->pv, h->r, z, zp, h->sc, h->partial, h->partial3, h->counters, s);
}

cudaError_t pcg_head(amg_hierarchy *h, cudaStream_t s)
{
    const DevCsr &A = h->lev[0].A;
    const int n = A.n;
    {
        ProfScope ps(KC_PCG_SPMV, s, 12.0 * (double)A.nnz + 20.0 * n + 4.0);
        AMG_CUDA_TRY(spmv_dot(A, h->plan0, h->pv, h->q, h->partial, nullptr, nullptr, s));
    }
    AMG_CUDA_TRY(pcg_update_xr(n, h->x, h->r, h->pv, h->q, h->sc, h->partial, spmv_block_count(n, h->plan0),
                               h->partial2, s));
    return cudaMemcpyAsync(h->rr_host, h->partial2, sizeof(double) * kReduceBlocks, cudaMemcpyDeviceToHost, s);
}

// the graph of tail(parity) + head, captured on first use (and again when kernel timing is
// switched on or off, so that its timing events are in the graph exactly when wanted)
cudaGraphExec_t pcg_graph(amg_hierarchy *h, int parity)
{
    if (h->graph_failed) return nullptr;
    const int want = profiling_enabled() ? 1 : 0;
    if (h->gexec[parity] && h->gprof_on[parity] == want) return h->gexec[parity];
    if (h->gexec[parity]) {
        cudaGraphExecDestroy(h->gexec[parity]);
        h->gexec[parity] = nullptr;
        profile_release(h->gprof[parity]);
    }
    cudaGraph_t g = nullptr;
    const long long launches_before = launch_count();
    cudaError_t e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        if (want) profile_capture_begin(&h->gprof[parity]);
        cudaError_t e1 = pcg_tail(h, parity, h->cap);
        cudaError_t e2 = e1 == cudaSuccess ? pcg_head(h, h->cap) : e1;
        profile_capture_end();
        e = cudaStreamEndCapture(h->cap, &g);
        if (e == cudaSuccess && e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec[parity], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->graph_failed = true;     // this handle runs the iterations eagerly from now on
        h->gexec[parity] = nullptr;
        profile_release(h->gprof[parity]);
        return nullptr;
    }
    h->gprof_on[parity] = want;
    // the capture itself launched nothing; its kernels run at every replay
    h->gkernels[parity] = launch_count() - launches_before;
    note_launches(-h->gkernels[parity]);
    return h->gexec[parity];
}

}  // namespace

// ------------------------------------------------------------------------------------ integrity check
namespace {
__global__ void csr_check_kernel(int n, int ncol, int64_t nnz, const int *rp, const int *ci, int *bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int b = rp[i], e = rp[i + 1];
        if (b < 0 || e < b || e > nnz) {
            atomicAdd(bad, 1);
            continue;
        }
        for (int k = b; k < e; ++k)
            if (ci[k] < 0 || ci[k] >= ncol) {
                atomicAdd(bad, 1);
                break;
            }
    }
}

}  // namespace

amg_status_t amgk::ensure_coarse_inverse(amg_hierarchy *h)
{
    if (!h || h->coarse_inv || h->nlev < 1) return AMG_OK;
    const amg_status_t st = form_coarse_inverse(h);
    if (st == AMG_OK) h->ctx.coarse_inv = h->coarse_inv;
    return st;
}

int amgk::hierarchy_check(const amg_hierarchy *h, cudaStream_t s, std::string *detail)
{
    int *bad = nullptr;
    if (cudaMallocAsync(&bad, sizeof(int), s) != cudaSuccess) return -1;
    int total = 0;
    auto one = [&](const DevCsr &c, int L, const char *what) -> bool {
        if (c.n == 0) return true;
        int head[2] = {0, 0};
        int hb = 0;
        if (cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess) return false;
        csr_check_kernel<<<grid_for(c.n, 256, 4096), 256, 0, s>>>(c.n, c.ncol, c.nnz, c.rp, c.ci, bad); note_launch();
        if (cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return false;
        if (cudaMemcpyAsync(&head[0], c.rp, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return false;
        if (cudaMemcpyAsync(&head[1], c.rp + c.n, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return false;
        if (cudaStreamSynchronize(s) != cudaSuccess) return false;
        const int f = hb + (head[0] != 0) + (head[1] != (int)c.nnz);
        if (f && total == 0 && detail)
            *detail = std::string(what) + " of level " + std::to_string(L) + ": " + std::to_string(hb) +
                      " bad rows, rp[0]=" + std::to_string(head[0]) + " rp[n]=" + std::to_string(head[1]) +
                      " nnz=" + std::to_string(c.nnz);
        total += f;
        return true;
    };
    bool ok = true;
    for (int L = 0; L < h->nlev && ok; ++L) {
        ok = one(h->lev[L].A, L, "A");
        if (ok && L + 1 < h->nlev) ok = one(h->lev[L].P, L, "P") && one(h->lev[L].R, L, "R");
    }
    cudaFreeAsync(bad, s);
    cudaStreamSynchronize(s);
    return ok ? total : -1;
}

// ====================================================================================== ABI

extern "C" {

void amg_params_default(amg_params_t *p)
{
    if (!p) return;
    p->theta = 0.0;
    p->variants = 0;
    p->tau = 1.1;
    p->sigma = 1.0 / 3.0;
    p->cheb_degree = 2;
    p->cheb_ratio = 10.0;
    p->cheb_boost = 1.1;
    p->power_iters = 10;
    p->max_coarse = 500;
    p->max_levels = 10;
    p->precision = AMG_FP64;
    p->pt_scaling = AMG_PT_ORTHONORMAL;
    p->onenorm_lambda = AMG_LAMBDA_ONE;
    p->max_iter = 1000;
    p->seed = 0;
    p->lambda_override = 0.0;
    p->cuda_stream = nullptr;
    p->strength = AMG_STRENGTH_MATRIX;
    p->trace = 0;
    p->krylov = AMG_KRYLOV_CG;
    p->restart = 30;
    p->spmv_layout = AMG_LAYOUT_AUTO;
    p->block_size = 1;
    p->nullspace_dim = 1;
    p->coarse_solve = AMG_COARSE_AUTO;
}

amg_status_t amg_setup_trace(amg_handle_t h, int level, double *ms)
{
    if (!h || !ms || level < 0 || level >= h->nlev) return AMG_ERR_INVALID_ARG;
    for (int k = 0; k < AMG_PH_COUNT; ++k) ms[k] = h->phase_ms[level][k];
    return AMG_OK;
}

const char *amg_status_string(amg_status_t s)
{
    switch (s) {
    case AMG_OK: return "ok";
    case AMG_ERR_INVALID_ARG: return "invalid argument";
    case AMG_ERR_OOM: return "out of device memory";
    case AMG_ERR_CUDA: return "CUDA error";
    case AMG_ERR_ZERO_DIAG: return "zero diagonal";
    case AMG_ERR_EIGEN: return "eigenvalue estimate not positive";
    case AMG_ERR_COARSE_NOT_SPD: return "coarsest operator not positive definite";
    case AMG_ERR_NOT_CONVERGED: return "not converged";
    case AMG_ERR_BUDGET: return "memory budget exceeded";
    case AMG_ERR_UNSUPPORTED: return "unsupported size";
    case AMG_ERR_INTERNAL: return "internal limit";
    case AMG_PENDING: return "pending";
    }
    return "unknown status";
}

const char *amg_last_error(void) { return g_last_error.c_str(); }

int64_t amg_launch_count(void) { return (int64_t)launch_count(); }

amg_status_t amg_profile_enable(int on)
{
    if (on < 0 || on > 2) return AMG_ERR_INVALID_ARG;
    profile_enable(on);
    return AMG_OK;
}

amg_status_t amg_profile_read(int kclass, int64_t *launches, double *total_ms, double *total_bytes)
{
    if (kclass < 0 || kclass >= KC_COUNT || !launches || !total_ms || !total_bytes) return AMG_ERR_INVALID_ARG;
    long long l = 0;
    profile_read(kclass, &l, total_ms, total_bytes);
    *launches = l;
    return AMG_OK;
}

amg_status_t amg_free(amg_handle_t h)
{
    if (!h) return AMG_OK;
    for (int k = 0; k < 2; ++k) {
        if (h->gexec[k]) cudaGraphExecDestroy(h->gexec[k]);
        profile_release(h->gprof[k]);
    }
    if (h->cap) cudaStreamDestroy(h->cap);
    multi_release(h);
    gmres_release(h);
    release_all(h);
    if (h->rr_host) cudaFreeHost(h->rr_host);
    delete h;
    return AMG_OK;
}

amg_status_t amg_setup(const amg_csr_t *Ain, const double *nullspace, const amg_params_t *pin, amg_handle_t *out)
{
    return amg_setup_coords(Ain, nullspace, nullptr, 0, pin, out);
}

amg_status_t amg_setup_coords(const amg_csr_t *Ain, const double *nullspace, const double *coords, int dim,
                              const amg_params_t *pin, amg_handle_t *out)
{
    if (!out) return AMG_ERR_INVALID_ARG;
    *out = nullptr;
    if (!Ain || !pin) return AMG_ERR_INVALID_ARG;
    if (pin->strength != AMG_STRENGTH_MATRIX && pin->strength != AMG_STRENGTH_DISTANCE) {
        g_last_error = "unknown strength criterion";
        return AMG_ERR_INVALID_ARG;
    }
    if (coords && (dim < 1 || dim > 3)) {
        g_last_error = "coordinates need 1 to 3 values per row";
        return AMG_ERR_INVALID_ARG;
    }
    if (pin->strength == AMG_STRENGTH_DISTANCE && !coords && Ain->n > 0) {
        g_last_error = "the distance-Laplacian strength needs coordinates";
        return AMG_ERR_INVALID_ARG;
    }
    if (Ain->n < 0 || Ain->nnz < 0 || (Ain->n > 0 && (!Ain->row_ptr || !Ain->col || !Ain->val)))
        return AMG_ERR_INVALID_ARG;
    if (Ain->n > 0x7ffffffe || Ain->nnz > 0x7ffffffe) {
        g_last_error = "matrix too large for 32-bit indices";
        return AMG_ERR_UNSUPPORTED;
    }
    const amg_params_t &p = *pin;
    if (!(p.theta >= 0.0 && p.theta <= 1.0) || p.cheb_degree < 1 || !(p.cheb_ratio > 1.0) || !(p.cheb_boost > 0.0) ||
        p.power_iters < 1 ||
        p.max_coarse < 1 || p.max_levels < 1 || p.max_iter < 0 || !(p.tau > 0.0) || !(p.sigma < 1.0) ||
        (p.krylov != AMG_KRYLOV_CG && p.krylov != AMG_KRYLOV_GMRES) ||
        (p.krylov == AMG_KRYLOV_GMRES && (p.restart < 1 || p.restart > 512)) ||
        (p.spmv_layout != AMG_LAYOUT_AUTO && p.spmv_layout != AMG_LAYOUT_CSR && p.spmv_layout != AMG_LAYOUT_SELL) ||
        (p.coarse_solve != AMG_COARSE_AUTO && p.coarse_solve != AMG_COARSE_INVERSE)) {
        g_last_error = "parameter out of range";
        return AMG_ERR_INVALID_ARG;
    }
    const bool block = p.block_size > 1 || p.nullspace_dim > 1;
    if (p.block_size < 1 || p.block_size > block_max_bs() || p.nullspace_dim < 1 || p.nullspace_dim > block_max_k() ||
        Ain->n % p.block_size != 0 || (block && !nullspace && p.nullspace_dim != p.block_size)) {
        g_last_error = "block size or near-null-space dimension out of range (or no vectors given for k != bs)";
        return AMG_ERR_INVALID_ARG;
    }
    if (block && (p.variants != 0 || p.strength != AMG_STRENGTH_MATRIX)) {
        g_last_error = "systems of PDEs: the adaptations and the distance strength are defined for scalar problems";
        return AMG_ERR_UNSUPPORTED;
    }
    const double t_start = now_ms();
    keep_pool_memory();
    amg_hierarchy *h = new amg_hierarchy();
    h->p = p;
    h->block = block;
    h->phase_t = t_start;
    h->s = (cudaStream_t)p.cuda_stream;
    amg_status_t st = AMG_OK;
    cudaStream_t s = h->s;
    const int n = (int)Ain->n;
    const int nnz = (int)Ain->nnz;
    int *bad = nullptr;
    int hbad = 0;
    int64_t *rp64 = nullptr;
    const int maxL = p.max_levels < 32 ? p.max_levels : 32;
    int L = 0;
    {
        Level &l0 = h->lev[0];
        l0.A.n = n;
        l0.A.ncol = n;
        l0.A.nnz = nnz;
        CK(dalloc(h, &l0.A.rp, (size_t)n + 1));
        CK(dalloc(h, &l0.A.ci, (size_t)nnz));
        CK(dalloc(h, &l0.A.v, (size_t)nnz));
        CK(cudaMallocAsync(&bad, sizeof(int), s));
        CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
        CK(cudaMallocAsync(&rp64, sizeof(int64_t) * ((size_t)n + 1), s));
        CK(copy_to_device(rp64, Ain->row_ptr, sizeof(int64_t) * ((size_t)n + 1), s));
        CK(convert_rowptr_to32(rp64, l0.A.rp, n + 1, bad, s));
        if (nnz > 0) {
            CK(copy_to_device(l0.A.ci, Ain->col, sizeof(int) * (size_t)nnz, s));
            CK(copy_to_device(l0.A.v, Ain->val, sizeof(double) * (size_t)nnz, s));
        }
        CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        int64_t last = 0;
        if (n > 0) CK(cudaMemcpy(&last, rp64 + n, sizeof(int64_t), cudaMemcpyDeviceToHost));
        if (hbad || last != nnz) { g_last_error = "row pointer not monotone or not matching nnz"; st = AMG_ERR_INVALID_ARG; goto done; }
        if (n > 0) {
            validate_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, l0.A.rp, l0.A.ci, bad); note_launch();
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (hbad) { g_last_error = "columns unsorted, out of range, duplicated, or a missing diagonal"; st = AMG_ERR_INVALID_ARG; goto done; }
        }
        l0.bs = p.block_size;
        l0.k = p.nullspace_dim;
        CK(dalloc(h, &l0.B, (size_t)n * (size_t)l0.k));
        if (coords && n > 0) {
            h->dim = dim;
            CK(dalloc(h, &l0.coords, (size_t)n * (size_t)dim));
            CK(copy_to_device(l0.coords, coords, sizeof(double) * (size_t)n * (size_t)dim, s));
        }
        if (nullspace) CK(copy_to_device(l0.B, nullspace, sizeof(double) * (size_t)n * (size_t)l0.k, s));
        else if (n > 0 && !block) { ones_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, l0.B); note_launch(); }
        else if (n > 0) {
            // the constant of each component: vector j is 1 on the unknowns of component j
            component_ones_kernel<<<grid_for((int64_t)n * l0.k, 256), 256, 0, s>>>(n, l0.bs, l0.k, l0.B); note_launch();
        }
        CK(cudaGetLastError());
        h->fine_nnz = nnz;
        trace_mark(h, 0, AMG_PH_INPUT);
    }
    // levels
    for (L = 0;; ++L) {
        Level &lv = h->lev[L];
        CK(dalloc(h, &lv.diag, (size_t)lv.A.n));
        CK(diag_extract(lv.A, nullptr, lv.diag, s));
        trace_mark(h, L, AMG_PH_STRENGTH);
        if (lv.A.n <= p.max_coarse || L + 1 >= maxL) break;
        int coarsest = 0;
        st = build_level(h, L, &coarsest);
        if (st != AMG_OK) goto done;
        if (coarsest) break;
    }
    h->nlev = L + 1;
    // coarsest level: the Chebyshev solve where it applies, else the dense inverse
    {
        Level &cl = h->lev[L];
        const int nc = cl.A.n;
        if (p.coarse_solve == AMG_COARSE_AUTO && p.krylov != AMG_KRYLOV_GMRES && nc > kCoarsePolyMinRows &&
            cl.A.nnz * 8 <= (int64_t)nc * nc) {
            int hzero = 0;
            CK(dalloc(h, &cl.invdiag, (size_t)nc));
            if (p.precision == AMG_MIXED) CK(dalloc(h, &cl.invdiag_f, (size_t)nc));
            CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
            CK(invert_diag(cl.diag, cl.invdiag, cl.invdiag_f, nc, bad, s));
            CK(cudaMemcpyAsync(&hzero, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(spmv_plan(cl.A.rp, nc, cl.A.nnz, &cl.plan_a, s));     // synchronises s
            if (!hzero)
                CK(coarse_cheb_setup(cl.A, cl.plan_a, cl.invdiag, &h->coarse_degree, &h->coarse_theta,
                                     &h->coarse_delta, &h->coarse_check, s));
        }
        if (h->coarse_degree == 0) {
            st = form_coarse_inverse(h);
            if (st != AMG_OK) goto done;
        }
        trace_mark(h, L, AMG_PH_COARSE);
    }
    st = prepare_solve(h);
    trace_mark(h, 0, AMG_PH_PREPARE);
    if (st == AMG_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fail_cuda(e, "setup");
        else if (spmv_take_errors(s) != 0) {
            g_last_error = "a bulk copy into shared memory did not complete in time";
            st = AMG_ERR_INTERNAL;
        }
    }
done:
    free_async(bad, s);
    free_async(rp64, s);
    if (st != AMG_OK) {
        amg_free(h);
        return st;
    }
    h->setup_ms = now_ms() - t_start;
    *out = h;
    return AMG_OK;
}

amg_status_t amg_num_levels(amg_handle_t h, int *levels)
{
    if (!h || !levels) return AMG_ERR_INVALID_ARG;
    *levels = h->nlev;
    return AMG_OK;
}

amg_status_t amg_coarse_solver(amg_handle_t h, int *degree, double *theta, double *delta, double *check)
{
    if (!h) return AMG_ERR_INVALID_ARG;
    if (degree) *degree = h->coarse_degree;
    if (theta) *theta = h->coarse_theta;
    if (delta) *delta = h->coarse_delta;
    if (check) *check = h->coarse_check;
    return AMG_OK;
}

amg_status_t amg_level_info(amg_handle_t h, int level, int64_t *n, int64_t *nnz, int64_t *nagg)
{
    if (!h || level < 0 || level >= h->nlev) return AMG_ERR_INVALID_ARG;
    const Level &lv = h->lev[level];
    if (n) *n = lv.A.n;
    if (nnz) *nnz = lv.A.nnz;
    if (nagg) *nagg = (level == h->nlev - 1) ? 0 : lv.nagg;
    return AMG_OK;
}

amg_status_t amg_vcycle(amg_handle_t h, const double *r, double *z)
{
    if (!h || (!r && h->lev[0].A.n) || (!z && h->lev[0].A.n)) return AMG_ERR_INVALID_ARG;
    amg_status_t st = AMG_OK;
    cudaStream_t s = h->s;
    const int n = h->lev[0].A.n;
    if (n == 0) return AMG_OK;
    CK(copy_to_device(h->r, r, sizeof(double) * (size_t)n, s));
    CK(vcycle(h->ctx, h->r, h->z, s));
    CK(copy_to_host(z, h->z, sizeof(double) * (size_t)n, s));
    CK(cudaStreamSynchronize(s));
    if (spmv_take_errors(s) != 0) {
        g_last_error = "a bulk copy into shared memory did not complete in time";
        st = AMG_ERR_INTERNAL;
    }
done:
    return st;
}

amg_status_t amg_solve(amg_handle_t h, const double *b, double *x, double tol, amg_info_t *info)
{
    if (!h) return AMG_ERR_INVALID_ARG;
    const int n = h->lev[0].A.n;
    if (n > 0 && (!b || !x)) return AMG_ERR_INVALID_ARG;
    if (!(tol >= 0.0)) return AMG_ERR_INVALID_ARG;
    if (h->p.krylov == AMG_KRYLOV_GMRES) return fgmres_solve(h, b, x, tol, info);
    const double t0 = now_ms();
    amg_status_t st = AMG_OK;
    cudaStream_t s = h->s;
    const DevCsr &A = h->lev[0].A;
    const SpmvPlan &plan = h->plan0;
    int it = 0;
    double bb = 0.0, rr = 0.0, relres = 0.0, nb = 0.0;
    amg_status_t result = AMG_OK;
    if (n == 0) goto finish;
    CK(copy_to_device(h->b, b, sizeof(double) * (size_t)n, s));
    CK(cudaMemsetAsync(h->x, 0, sizeof(double) * (size_t)n, s));
    CK(cudaMemcpyAsync(h->r, h->b, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    CK(dot(h->b, h->b, n, h->partial, &h->sc->bb, s));
    CK(cudaMemcpyAsync(&bb, &h->sc->bb, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    nb = std::sqrt(bb);
    if (nb == 0.0) goto finish;
    CK(vcycle(h->ctx, h->r, h->zb[0], s));
    CK(cudaMemcpyAsync(h->pv, h->zb[0], sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    CK(dot(h->r, h->zb[0], n, h->partial, &h->sc->rz_next, s));
    result = AMG_ERR_NOT_CONVERGED;
    if (h->p.max_iter > 0) {
        CK(pcg_head(h, s));
        ++it;
    }
    while (it > 0) {
        CK(cudaStreamSynchronize(s));
        rr = 0.0;
        for (int k = 0; k < kReduceBlocks; ++k) rr += h->rr_host[k];
        if (std::sqrt(rr) / nb <= tol) {
            CK(residual_d(A, plan, h->b, h->x, h->t, s));
            CK(dot(h->t, h->t, n, h->partial, &h->sc->tmp, s));
            double tt = 0.0;
            CK(cudaMemcpyAsync(&tt, &h->sc->tmp, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (std::sqrt(tt) / nb <= tol) { result = AMG_OK; break; }
            CK(cudaMemcpyAsync(h->r, h->t, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        }
        if (it >= h->p.max_iter) break;
        const int parity = h->zb[1] ? (it & 1) : 0;
        cudaGraphExec_t gx = pcg_graph(h, parity);
        if (gx) {
            CK(cudaGraphLaunch(gx, s));
            note_launches(h->gkernels[parity]);
            ++it;
            CK(cudaStreamSynchronize(s));
            profile_account(h->gprof[parity]);
            continue;
        }
        CK(pcg_tail(h, parity, s));
        CK(pcg_head(h, s));
        ++it;
    }
finish:
    if (n > 0) {
        CK(residual_d(A, plan, h->b, h->x, h->t, s));
        CK(dot(h->t, h->t, n, h->partial, &h->sc->tmp, s));
        double tt = 0.0;
        CK(cudaMemcpyAsync(&tt, &h->sc->tmp, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(copy_to_host(x, h->x, sizeof(double) * (size_t)n, s));
        CK(cudaStreamSynchronize(s));
        relres = nb > 0.0 ? std::sqrt(tt) / nb : 0.0;
    }
    st = result;
    if (spmv_take_errors(s) != 0) {
        g_last_error = "a bulk copy into shared memory did not complete in time";
        st = AMG_ERR_INTERNAL;
    }
done:
    if (info) {
        info->iters = it;
        info->status = st;
        info->relres_true = relres;
        info->setup_ms = h->setup_ms;
        info->solve_ms = now_ms() - t0;
        info->levels = h->nlev;
        double tot = 0.0;
        for (int L = 0; L < h->nlev; ++L) tot += (double)h->lev[L].A.nnz;
        info->op_complexity = h->fine_nnz > 0 ? tot / (double)h->fine_nnz : 0.0;
    }
    return st;
}

}  // extern "C"

namespace {

struct ExportSrc {
    const void *ptr = nullptr;
    int64_t count = 0;
    int kind = 0;     // 0 raw bytes of elem size, 1 int32 row pointer widened to int64
    size_t elem = 1;
};

ExportSrc export_src(const amg_hierarchy *h, int level, int what)
{
    ExportSrc e;
    const Level &lv = h->lev[level];
    const bool last = level == h->nlev - 1;
    auto rowptr = [&](const DevCsr &c, int rows) {
        ExportSrc r;
        if (!c.rp) return r;
        r.ptr = c.rp; r.count = rows + 1; r.kind = 1; r.elem = 8;
        return r;
    };
    auto arr = [&](const void *p, int64_t cnt, size_t el) {
        ExportSrc r;
        if (!p) return r;
        r.ptr = p; r.count = cnt; r.elem = el;
        return r;
    };
    switch (what) {
    case AMG_EX_A_ROWPTR: return rowptr(lv.A, lv.A.n);
    case AMG_EX_A_COL: return arr(lv.A.ci, lv.A.nnz, 4);
    case AMG_EX_A_VAL: return arr(lv.A.v, lv.A.nnz, 8);
    case AMG_EX_NULLSPACE: return arr(lv.B, (int64_t)lv.A.n * lv.k, 8);
    case AMG_EX_COORDS: return arr(lv.coords, (int64_t)lv.A.n * h->dim, 8);
    default: break;
    }
    if (last) return e;
    switch (what) {
    case AMG_EX_STRONG: return arr(lv.strong, lv.A.nnz, 1);
    case AMG_EX_REMOVED: return arr(lv.removed, lv.A.nnz, 1);
    case AMG_EX_LUMPFLAG: return arr(lv.lumpflag, lv.A.n, 1);
    case AMG_EX_ABAR_ROWPTR: return rowptr(lv.Abar, lv.Abar.n);
    case AMG_EX_ABAR_COL: return arr(lv.Abar.ci, lv.Abar.nnz, 4);
    case AMG_EX_ABAR_VAL: return arr(lv.Abar.v, lv.Abar.nnz, 8);
    case AMG_EX_AGG: return arr(lv.agg, lv.A.n / lv.bs, 4);
    case AMG_EX_ROOT: return arr(lv.root, lv.A.n / lv.bs, 1);
    case AMG_EX_P_ROWPTR: return rowptr(lv.P, lv.P.n);
    case AMG_EX_P_COL: return arr(lv.P.ci, lv.P.nnz, 4);
    case AMG_EX_P_VAL: return arr(lv.P.v, lv.P.nnz, 8);
    case AMG_EX_R_ROWPTR: return rowptr(lv.R, lv.R.n);
    case AMG_EX_R_COL: return arr(lv.R.ci, lv.R.nnz, 4);
    case AMG_EX_R_VAL: return arr(lv.R.v, lv.R.nnz, 8);
    case AMG_EX_DSMOOTH: return arr(lv.Dsm, lv.A.n, 8);
    case AMG_EX_CFLAG: return arr(lv.cflag, lv.A.n, 1);
    case AMG_EX_SCALARS: e.count = 4; e.elem = 8; e.kind = 2; return e;
    default: return e;
    }
}

}  // namespace

extern "C" {

amg_status_t amg_export_count(amg_handle_t h, int level, int what, int64_t *count)
{
    if (!h || !count || level < 0 || level >= h->nlev) return AMG_ERR_INVALID_ARG;
    if (what < 0 || what > AMG_EX_COORDS) return AMG_ERR_INVALID_ARG;
    *count = export_src(h, level, what).count;
    return AMG_OK;
}

amg_status_t amg_export(amg_handle_t h, int level, int what, void *dst)
{
    if (!h || !dst || level < 0 || level >= h->nlev) return AMG_ERR_INVALID_ARG;
    if (what < 0 || what > AMG_EX_COORDS) return AMG_ERR_INVALID_ARG;
    ExportSrc e = export_src(h, level, what);
    if (e.count == 0) return AMG_OK;
    const Level &lv = h->lev[level];
    if (e.kind == 2) {
        double sc[4] = {lv.lambda_bar, lv.omega, lv.lambda_cheb, (double)lv.nagg};
        std::memcpy(dst, sc, sizeof sc);
        return AMG_OK;
    }
    cudaError_t err;
    if (e.kind == 1) {
        std::vector<int> tmp((size_t)e.count);
        err = copy_to_host(tmp.data(), e.ptr, sizeof(int) * (size_t)e.count, nullptr);
        if (err != cudaSuccess) return fail_cuda(err, "amg_export");
        int64_t *o = (int64_t *)dst;
        for (int64_t i = 0; i < e.count; ++i) o[i] = tmp[(size_t)i];
        return AMG_OK;
    }
    err = copy_to_host(dst, e.ptr, e.elem * (size_t)e.count, nullptr);
    if (err != cudaSuccess) return fail_cuda(err, "amg_export");
    return AMG_OK;
}

amg_status_t amg_csr_release(amg_dcsr_t *C)
{
    if (!C) return AMG_OK;
    cudaFree(C->row_ptr);
    cudaFree(C->col);
    cudaFree(C->val);
    C->row_ptr = nullptr; C->col = nullptr; C->val = nullptr;
    C->nrow = C->ncol = C->nnz = 0;
    return AMG_OK;
}

amg_status_t amg_dcsr_download(const amg_dcsr_t *C, int64_t *row_ptr, int32_t *col, double *val)
{
    if (!C || !row_ptr || (C->nnz > 0 && (!col || !val))) return AMG_ERR_INVALID_ARG;
    cudaError_t e = copy_to_host(row_ptr, C->row_ptr, sizeof(int64_t) * (size_t)(C->nrow + 1), nullptr);
    if (e == cudaSuccess && C->nnz > 0) e = copy_to_host(col, C->col, sizeof(int32_t) * (size_t)C->nnz, nullptr);
    if (e == cudaSuccess && C->nnz > 0) e = copy_to_host(val, C->val, sizeof(double) * (size_t)C->nnz, nullptr);
    return e == cudaSuccess ? AMG_OK : fail_cuda(e, "amg_dcsr_download");
}

amg_status_t amg_spgemm_noalloc(const amg_csr_t *A, int64_t ncolA, const amg_csr_t *B, int64_t ncolB, void *stream,
                                int64_t *C_row_ptr, int32_t *C_col, double *C_val, int64_t capacity, int64_t *nnz_out)
{
    if (!A || !B || !C_row_ptr || !nnz_out || capacity < 0 || (capacity > 0 && (!C_col || !C_val)))
        return AMG_ERR_INVALID_ARG;
    *nnz_out = 0;
    if (!A->on_device || !B->on_device) {
        g_last_error = "amg_spgemm_noalloc: A and B must be device arrays";
        return AMG_ERR_INVALID_ARG;
    }
    if (A->n < 0 || B->n < 0 || ncolA != B->n || ncolB < 0 || ncolB > 0x7ffffffe || A->nnz < 0 || B->nnz < 0 ||
        A->nnz > 0x7ffffffe || B->nnz > 0x7ffffffe || A->n > 0x7ffffffe || B->n > 0x7ffffffe || !A->row_ptr ||
        !B->row_ptr || (A->nnz > 0 && (!A->col || !A->val)) || (B->nnz > 0 && (!B->col || !B->val)))
        return AMG_ERR_INVALID_ARG;
    int code = 0;
    std::string msg;
    cudaError_t e = spgemm_noalloc((int)A->n, (int)ncolA, A->row_ptr, A->col, A->val, A->nnz, (int)B->n, (int)ncolB,
                                   B->row_ptr, B->col, B->val, B->nnz, C_row_ptr, C_col, C_val, capacity, nnz_out,
                                   &code, &msg, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail_cuda(e, "amg_spgemm_noalloc");
    if (code) g_last_error = msg;
    switch (code) {
    case 0: return AMG_OK;
    case 1: return AMG_ERR_UNSUPPORTED;
    case 2: return AMG_ERR_BUDGET;
    case 3: return AMG_ERR_INVALID_ARG;
    default: return AMG_ERR_INTERNAL;
    }
}

amg_status_t amg_spgemm(const amg_csr_t *A, int64_t ncolA, const amg_csr_t *B, int64_t ncolB, void *stream,
                        amg_dcsr_t *C)
{
    if (!A || !B || !C) return AMG_ERR_INVALID_ARG;
    *C = amg_dcsr_t{0, 0, 0, nullptr, nullptr, nullptr};
    if (A->n < 0 || B->n < 0 || ncolA != B->n || ncolB < 0 || A->n > 0x7ffffffe || B->n > 0x7ffffffe ||
        A->nnz > 0x7ffffffe || B->nnz > 0x7ffffffe || ncolB > 0x7ffffffe)
        return AMG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    amg_status_t st = AMG_OK;
    DevCsr dA, dB, dC;
    int64_t *rp64 = nullptr;
    int *bad = nullptr;
    int ovf = 0, hbad = 0;
    const amg_csr_t *src[2] = {A, B};
    DevCsr *dst[2] = {&dA, &dB};
    CK(cudaMalloc(&bad, sizeof(int)));
    CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
    for (int t = 0; t < 2; ++t) {
        const amg_csr_t *m = src[t];
        DevCsr *d = dst[t];
        d->n = (int)m->n;
        d->ncol = t == 0 ? (int)ncolA : (int)ncolB;
        d->nnz = m->nnz;
        CK(cudaMalloc(&d->rp, sizeof(int) * (size_t)(m->n + 1)));
        CK(cudaMalloc(&d->ci, sizeof(int) * (size_t)(m->nnz > 0 ? m->nnz : 1)));
        CK(cudaMalloc(&d->v, sizeof(double) * (size_t)(m->nnz > 0 ? m->nnz : 1)));
        CK(cudaMalloc(&rp64, sizeof(int64_t) * (size_t)(m->n + 1)));
        CK(copy_to_device(rp64, m->row_ptr, sizeof(int64_t) * (size_t)(m->n + 1), s));
        CK(convert_rowptr_to32(rp64, d->rp, (int)m->n + 1, bad, s));
        if (m->nnz > 0) {
            CK(copy_to_device(d->ci, m->col, sizeof(int) * (size_t)m->nnz, s));
            CK(copy_to_device(d->v, m->val, sizeof(double) * (size_t)m->nnz, s));
        }
        CK(cudaStreamSynchronize(s));
        cudaFree(rp64);
        rp64 = nullptr;
    }
    CK(cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost));
    if (hbad) { st = AMG_ERR_INVALID_ARG; goto done; }
    {
        cudaError_t e = spgemm(dA, dB, dC, &ovf, s);
        if (e == cudaErrorInvalidValue && ovf) { g_last_error = "hash table overflow"; st = AMG_ERR_INTERNAL; goto done; }
        CK(e);
    }
    CK(cudaMalloc(&C->row_ptr, sizeof(int64_t) * (size_t)(dC.n + 1)));
    CK(convert_rowptr_to64(dC.rp, C->row_ptr, dC.n + 1, s));
    CK(cudaStreamSynchronize(s));
    C->nrow = dC.n;
    C->ncol = ncolB;
    C->nnz = dC.nnz;
    C->col = dC.ci;
    C->val = dC.v;
    dC.ci = nullptr;
    dC.v = nullptr;
done:
    cudaFree(bad); cudaFree(rp64);
    cudaFree(dA.rp); cudaFree(dA.ci); cudaFree(dA.v);
    cudaFree(dB.rp); cudaFree(dB.ci); cudaFree(dB.v);
    cudaFree(dC.rp); cudaFree(dC.ci); cudaFree(dC.v);
    if (st != AMG_OK) amg_csr_release(C);
    return st;
}

}  // extern "C"
