// batch.cu -- many independent systems solved together: one set of kernel launches per
// V-cycle step and PCG update for the whole batch (no counterpart in the paper, which solves
// one system at a time; each system's arithmetic is that of §1.1, Algorithm 1 and §3.1).
//
// Layout.  Systems are ordered by decreasing number of levels, so the systems that have a
// level L form a prefix of that order, and among them the ones for which L is not the
// coarsest ("intermediate") form a prefix again.  Level L of the batch concatenates level L of
// those systems: block-diagonal A_L and P_L over the intermediate rows, R_L onto all rows of
// level L+1 (column indices shifted by each system's row offset), vectors over every system
// that has level L, and the dense inverses of the systems whose coarsest level is L.  Every
// smoother step, residual and transfer of the V-cycle is one SpMV launch over the whole batch
// (the tile kernel of solve.cu; Chebyshev coefficients per row through a row -> system map);
// the coarse solves are one launch with a block per system.
//
// PCG scalars are per system.  Every vector kernel runs over "chunks" (at most kChunkRows rows
// of one system); a chunk's partial sum goes to its slot, and the last chunk of a system to
// finish (atomic ticket) adds the system's partials in chunk order, so every per-system scalar
// is bitwise reproducible.  One PCG iteration of the whole batch is replayed as a CUDA graph.
// Systems that have converged (or reached max_iter) are masked out of the PCG updates; their
// V-cycle rows are still computed.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "hierarchy.cuh"

namespace amgk {
namespace {

constexpr unsigned kBAll = 0xffffffffu;
constexpr int kBThreads = 256;
constexpr int kChunkRows = 4096;

// ------------------------------------------------------------------------------------ gathers
struct CsrSeg {          // one system's matrix moved into the batch matrix
    const int *rp;
    const int *ci;
    const double *v;
    int n;               // rows
    int row_off;         // first row in the batch matrix
    int nnz_off;         // first entry in the batch matrix
    int col_shift;       // added to every column index
    int sys;             // batch position (row -> system map)
};
struct VecSeg {
    const void *src;
    long long n;
    long long off;
};

template <typename TV>
__global__ void gather_csr_kernel(const CsrSeg *segs, int *rp, int *ci, TV *v, int *rowsys)
{
    const CsrSeg sg = segs[blockIdx.y];
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = t0; i < sg.n; i += stride) {
        rp[sg.row_off + i] = sg.rp[i] + sg.nnz_off;
        if (rowsys) rowsys[sg.row_off + i] = sg.sys;
    }
    const int nnz = sg.n > 0 ? sg.rp[sg.n] : 0;
    for (int e = t0; e < nnz; e += stride) {
        ci[sg.nnz_off + e] = sg.ci[e] + sg.col_shift;
        v[sg.nnz_off + e] = (TV)sg.v[e];
    }
}

template <typename TS, typename TD>
__global__ void gather_vec_kernel(const VecSeg *segs, TD *dst)
{
    const VecSeg sg = segs[blockIdx.y];
    const TS *src = (const TS *)sg.src;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < sg.n;
         i += (long long)gridDim.x * blockDim.x)
        dst[sg.off + i] = (TD)src[i];
}

__global__ void set_int_kernel(int *p, int value) { *p = value; }

struct SysSeg {
    int off, n, sys;     // rows [off, off + n) of a level belong to batch position sys
};
__global__ void fill_rowsys_kernel(const SysSeg *segs, int *rowsys)
{
    const SysSeg sg = segs[blockIdx.y];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < sg.n; i += gridDim.x * blockDim.x)
        rowsys[sg.off + i] = sg.sys;
}

// ------------------------------------------------------------------------------------ V-cycle pieces
// First Chebyshev step from x = 0 with the row's own 1/theta: d = D^-1 f / theta, x = d
template <typename T>
__global__ void bcheb_zero_kernel(int n, const T *f, const T *invd, const int *rowsys, const double *coef,
                                  int cstride, const int *active, T *d, T *x)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!active[rowsys[i]]) continue;
        const T di = (invd[i] * f[i]) * (T)coef[(size_t)rowsys[i] * cstride];
        d[i] = di;
        x[i] = di;
    }
}

struct CoarseSeg {
    int off;             // first row in the level
    int n;               // rows
    int sys;             // batch position
    long long inv_off;   // first entry of the system's n x n inverse
};

// dense coarse solves x = Ainv f, one block per system, one warp per row (FP64 accumulation)
template <typename T>
__global__ void bcoarse_kernel(const CoarseSeg *segs, const int *active, const double *inv, const T *f, T *x)
{
    const CoarseSeg sg = segs[blockIdx.x];
    if (!active[sg.sys]) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double *a = inv + sg.inv_off;
    for (int i = w; i < sg.n; i += nw) {
        double acc = 0.0;
        for (int k = lane; k < sg.n; k += 32) acc += a[(size_t)i * sg.n + k] * (double)f[sg.off + k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kBAll, acc, o);
        if (lane == 0) x[sg.off + i] = (T)acc;
    }
}

template <typename A, typename B>
__global__ void convert_kernel(int n, const A *in, B *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = (B)in[i];
}
template <typename A, typename B>
__global__ void convert_active_kernel(int n, const int *rowsys, const int *active, const A *in, B *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (active[rowsys[i]]) out[i] = (B)in[i];
}

// ------------------------------------------------------------------------------------ PCG pieces
struct Chunk {
    int sys;             // batch position of the system
    int begin, end;      // rows [begin, end) of the batch vectors
    int first, count;    // the system's chunks are [first, first + count)
};

struct BScal {           // per system, on the device
    double rz;           // r . z of the current search direction
    double rz_new;       // r . z after the latest V-cycle
    double cross;        // r . z_prev (flexible form)
    double alpha;
    double pq, rr, tt, bb;
};

// fixed-order block sum; every thread gets the total
__device__ __forceinline__ double block_total(double v)
{
    __shared__ double sh[kBThreads / 32];
    __shared__ double tot;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kBAll, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kBThreads / 32; ++k) t += sh[k];
        tot = t;
    }
    __syncthreads();
    const double r = tot;
    __syncthreads();
    return r;
}

// Stores this chunk's partial; the system's last chunk (ticket) returns true in every thread
// of its block with *total = the system's sum in chunk order, and resets the ticket.
__device__ __forceinline__ bool chunk_finish(const Chunk &c, double part, double *partial, unsigned *ticket,
                                             double *total)
{
    __shared__ bool last;
    __shared__ double tot;
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = part;
        __threadfence();
        last = atomicAdd(&ticket[c.sys], 1u) == (unsigned)c.count - 1u;
    }
    __syncthreads();
    if (!last) return false;
    if (threadIdx.x == 0) {
        __threadfence();
        double t = 0.0;
        for (int k = 0; k < c.count; ++k) t += ((volatile const double *)partial)[c.first + k];
        tot = t;
        ticket[c.sys] = 0u;
    }
    __syncthreads();
    *total = tot;
    return true;
}

// per-system sums over the chunks (systems with mask[sys] = 0 skipped; mask may be null):
// which = 0: a.a -> bb;  1: a.a -> tt;  2: a.b -> rz_new, and p_copy = b
__global__ void __launch_bounds__(kBThreads) bdot_kernel(const Chunk *chunks, const int *mask, const double *a,
                                                        const double *b, double *p_copy, double *partial,
                                                        unsigned *ticket, BScal *sc, int which)
{
    const Chunk c = chunks[blockIdx.x];
    if (mask && !mask[c.sys]) return;
    double acc = 0.0;
    for (int i = c.begin + threadIdx.x; i < c.end; i += kBThreads) {
        const double ai = a[i];
        if (which == 2) {
            const double bi = b[i];
            acc += ai * bi;
            if (p_copy) p_copy[i] = bi;
        } else {
            acc += ai * ai;
        }
    }
    acc = block_total(acc);
    double tot;
    if (chunk_finish(c, acc, partial, ticket, &tot) && threadIdx.x == 0) {
        if (which == 0) sc[c.sys].bb = tot;
        else if (which == 1) sc[c.sys].tt = tot;
        else sc[c.sys].rz_new = tot;
    }
}

// p . q per system; the last chunk sets alpha = rz_new / (p . q) and rz = rz_new
__global__ void __launch_bounds__(kBThreads) bpq_kernel(const Chunk *chunks, const int *active, const double *p,
                                                       const double *q, double *partial, unsigned *ticket, BScal *sc)
{
    const Chunk c = chunks[blockIdx.x];
    if (!active[c.sys]) return;
    double acc = 0.0;
    for (int i = c.begin + threadIdx.x; i < c.end; i += kBThreads) acc += p[i] * q[i];
    acc = block_total(acc);
    double tot;
    if (chunk_finish(c, acc, partial, ticket, &tot) && threadIdx.x == 0) {
        BScal &s = sc[c.sys];
        s.pq = tot;
        s.alpha = s.rz_new / tot;
        s.rz = s.rz_new;
    }
}

// x += alpha p; r -= alpha q; r . r per system into rr_out[sys]
__global__ void __launch_bounds__(kBThreads) bxr_kernel(const Chunk *chunks, const int *active, const double *p,
                                                       const double *q, double *x, double *r, double *partial,
                                                       unsigned *ticket, BScal *sc, double *rr_out)
{
    const Chunk c = chunks[blockIdx.x];
    if (!active[c.sys]) return;
    const double alpha = sc[c.sys].alpha;
    double acc = 0.0;
    for (int i = c.begin + threadIdx.x; i < c.end; i += kBThreads) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        r[i] = ri;
        acc += ri * ri;
    }
    acc = block_total(acc);
    double tot;
    if (chunk_finish(c, acc, partial, ticket, &tot) && threadIdx.x == 0) {
        sc[c.sys].rr = tot;
        rr_out[c.sys] = tot;
    }
}

// r . z (and r . z_prev) per system
__global__ void __launch_bounds__(kBThreads) brz_kernel(const Chunk *chunks, const int *active, const double *r,
                                                       const double *z, const double *zp, double *partial,
                                                       double *partial2, unsigned *ticket, unsigned *ticket2,
                                                       BScal *sc)
{
    const Chunk c = chunks[blockIdx.x];
    if (!active[c.sys]) return;
    double a = 0.0, b = 0.0;
    for (int i = c.begin + threadIdx.x; i < c.end; i += kBThreads) {
        const double ri = r[i];
        a += ri * z[i];
        if (zp) b += ri * zp[i];
    }
    a = block_total(a);
    double tot;
    if (chunk_finish(c, a, partial, ticket, &tot) && threadIdx.x == 0) sc[c.sys].rz_new = tot;
    if (zp) {
        b = block_total(b);
        if (chunk_finish(c, b, partial2, ticket2, &tot) && threadIdx.x == 0) sc[c.sys].cross = tot;
    }
}

// beta = rz_new / rz (flexible: (rz_new - cross) / rz); p = z + beta p
__global__ void __launch_bounds__(kBThreads) bp_kernel(const Chunk *chunks, const int *active, const double *z,
                                                      double *p, const BScal *sc, int flexible)
{
    const Chunk c = chunks[blockIdx.x];
    if (!active[c.sys]) return;
    const BScal s = sc[c.sys];
    const double beta = (flexible ? s.rz_new - s.cross : s.rz_new) / s.rz;
    for (int i = c.begin + threadIdx.x; i < c.end; i += kBThreads) p[i] = z[i] + beta * p[i];
}

// r = t on the systems whose flag is set (residual replacement)
__global__ void bcopy_flagged_kernel(const Chunk *chunks, const int *flag, const double *t, double *r)
{
    const Chunk c = chunks[blockIdx.x];
    if (!flag[c.sys]) return;
    for (int i = c.begin + threadIdx.x; i < c.end; i += blockDim.x) r[i] = t[i];
}

}  // namespace

// ------------------------------------------------------------------------------------ structure
struct BLevel {
    int nrows = 0, nint = 0;            // rows of all systems / of the intermediate prefix
    int nsys = 0, nsys_int = 0;         // systems having this level / intermediate ones
    int ncoarse = 0;                    // systems whose coarsest level this is
    int *arp = nullptr, *aci = nullptr; // block-diagonal A over the intermediate rows
    int *prp = nullptr, *pci = nullptr; // P: nint x (rows of level L+1)
    int *rrp = nullptr, *rci = nullptr; // R: (rows of level L+1) x nint
    void *av = nullptr, *pv = nullptr, *rv = nullptr, *invd = nullptr;   // working type
    int64_t nnz_a = 0, nnz_p = 0, nnz_r = 0;
    SpmvPlan plan_a, plan_p, plan_r;
    int *rowsys = nullptr;              // batch position of each row's system (all rows)
    double *coef = nullptr;             // nsys_int x cstride Chebyshev coefficients
    CoarseSeg *ctable = nullptr;        // ncoarse entries
    double *cinv = nullptr;             // concatenated dense inverses
    void *f = nullptr, *x = nullptr, *x2 = nullptr, *r = nullptr, *d = nullptr;   // working type
};

}  // namespace amgk

struct amg_batch {
    int count = 0;
    int nlev = 0;
    int mixed = 0;
    int degree = 2, cstride = 5;
    cudaStream_t s = nullptr, cap = nullptr;
    std::vector<void *> allocs;
    std::vector<int> order;             // batch position -> caller's index
    std::vector<int> nlev_sys, max_iter;
    std::vector<int64_t> off0;          // fine-level row offsets (batch order), count + 1
    std::vector<double> opc, setup_ms;
    amgk::BLevel lev[32];
    int total = 0;                      // fine rows of all systems
    int64_t nnz0 = 0;
    int *a0rp = nullptr, *a0ci = nullptr;
    double *a0v = nullptr;              // all fine operators, FP64 (PCG)
    amgk::SpmvPlan plan0;
    int nchunks = 0;
    amgk::Chunk *chunks = nullptr;
    double *partial = nullptr, *partial2 = nullptr;
    unsigned *ticket = nullptr, *ticket2 = nullptr;
    int *active = nullptr, *flag = nullptr;
    amgk::BScal *sc = nullptr;
    double *b = nullptr, *x = nullptr, *r = nullptr, *pv = nullptr, *q = nullptr, *t = nullptr;
    double *zb[2] = {nullptr, nullptr};
    double *rr_dev = nullptr;
    double *rr_host = nullptr;          // pinned, count doubles
    int *host_flags = nullptr;          // pinned, 2 x count ints (active, flag)
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    long long gkernels[2] = {0, 0};
    bool graph_failed = false;
};

namespace amgk {
namespace {

#define CKB(expr)                                                         \
    do {                                                                  \
        cudaError_t _e = (expr);                                          \
        if (_e != cudaSuccess) { st = fail_cuda(_e, #expr); goto done; }  \
    } while (0)

template <typename T>
cudaError_t balloc(amg_batch *B, T **p, size_t count)
{
    *p = nullptr;
    cudaError_t e = cudaMallocAsync((void **)p, (count + 16) * sizeof(T), B->s);
    if (e == cudaSuccess) B->allocs.push_back((void *)*p);
    return e;
}

template <typename T>
cudaError_t upload(amg_batch *B, T **dev, const std::vector<T> &host)
{
    AMG_CUDA_TRY(balloc(B, dev, host.size()));
    if (host.empty()) return cudaSuccess;
    AMG_CUDA_TRY(cudaMemcpyAsync(*dev, host.data(), sizeof(T) * host.size(), cudaMemcpyHostToDevice, B->s));
    return cudaStreamSynchronize(B->s);   // the host vector may go away after return
}

int gather_width(int64_t longest)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>(64, (longest + kBThreads * 8 - 1) / (kBThreads * 8)));
}

// one launch gathering the listed matrices into a batch CSR (row pointer closed with nnz);
// longest: the most rows or entries of one listed matrix
cudaError_t gather_csr(amg_batch *B, const std::vector<CsrSeg> &segs, int64_t longest, int rows, int64_t nnz,
                       int **rp, int **ci, void **v, bool to_float, int **rowsys)
{
    cudaStream_t s = B->s;
    AMG_CUDA_TRY(balloc(B, rp, (size_t)rows + 1));
    AMG_CUDA_TRY(balloc(B, ci, (size_t)nnz));
    if (to_float) AMG_CUDA_TRY(balloc(B, (float **)v, (size_t)nnz));
    else AMG_CUDA_TRY(balloc(B, (double **)v, (size_t)nnz));
    if (rowsys) AMG_CUDA_TRY(balloc(B, rowsys, (size_t)rows));
    set_int_kernel<<<1, 1, 0, s>>>(*rp + rows, (int)nnz); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    if (segs.empty()) return cudaSuccess;
    CsrSeg *dsegs = nullptr;
    AMG_CUDA_TRY(upload(B, &dsegs, segs));
    const dim3 grid((unsigned)gather_width(longest), (unsigned)segs.size());
    if (to_float)
        gather_csr_kernel<float><<<grid, kBThreads, 0, s>>>(dsegs, *rp, *ci, (float *)*v, rowsys ? *rowsys : nullptr);
    else
        gather_csr_kernel<double><<<grid, kBThreads, 0, s>>>(dsegs, *rp, *ci, (double *)*v, rowsys ? *rowsys : nullptr);
    note_launch();
    return cudaGetLastError();
}

template <typename TS, typename TD>
cudaError_t gather_vec(amg_batch *B, const std::vector<VecSeg> &segs, TD *dst)
{
    if (segs.empty()) return cudaSuccess;
    VecSeg *dsegs = nullptr;
    AMG_CUDA_TRY(upload(B, &dsegs, segs));
    long long longest = 1;
    for (const VecSeg &g : segs) longest = std::max(longest, g.n);
    const dim3 grid((unsigned)gather_width(longest), (unsigned)segs.size());
    gather_vec_kernel<TS, TD><<<grid, kBThreads, 0, B->s>>>(dsegs, dst); note_launch();
    return cudaGetLastError();
}

// Chebyshev coefficients of one system on one level, the recurrence of solve.cu's smoother
// on [b lambda / ratio, b lambda] (§3.1's Chebyshev smoothing): [1/theta, then (c1, c2) for
// each step k of a pass that starts from a non-zero iterate (step 0: c1 = 0, c2 = 1/theta)]
void cheb_table(double lambda, const amg_params_t &p, std::vector<double> &out)
{
    const double lmax = p.cheb_boost * lambda, lmin = lmax / p.cheb_ratio;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma1 = theta / delta;
    out.push_back(1.0 / theta);
    out.push_back(0.0);
    out.push_back(1.0 / theta);
    double rho = 1.0 / sigma1;
    for (int k = 1; k < p.cheb_degree; ++k) {
        const double rho_new = 1.0 / (2.0 * sigma1 - rho);
        out.push_back(rho_new * rho);
        out.push_back(2.0 * rho_new / delta);
        rho = rho_new;
    }
}

amg_status_t too_large()
{
    set_last_error("batch too large for 32-bit indices");
    return AMG_ERR_UNSUPPORTED;
}

amg_status_t batch_assemble(amg_batch *Bt, const amg_handle_t *H, int C)
{
    amg_status_t st = AMG_OK;
    cudaStream_t s = Bt->s;
    const bool mixed = Bt->mixed != 0;
    const size_t ts = mixed ? sizeof(float) : sizeof(double);
    std::vector<std::vector<int64_t>> off;
    Bt->count = C;
    Bt->order.resize(C);
    for (int i = 0; i < C; ++i) Bt->order[i] = i;
    std::stable_sort(Bt->order.begin(), Bt->order.end(), [&](int a, int b) { return H[a]->nlev > H[b]->nlev; });
    Bt->nlev = C ? H[Bt->order[0]]->nlev : 0;
    Bt->nlev_sys.resize(C);
    Bt->max_iter.resize(C);
    Bt->opc.resize(C);
    Bt->setup_ms.resize(C);
    for (int k = 0; k < C; ++k) {
        const amg_hierarchy *h = H[Bt->order[k]];
        Bt->nlev_sys[k] = h->nlev;
        Bt->max_iter[k] = h->p.max_iter;
        Bt->setup_ms[k] = h->setup_ms;
        double tot = 0.0;
        for (int L = 0; L < h->nlev; ++L) tot += (double)h->lev[L].A.nnz;
        Bt->opc[k] = h->fine_nnz ? tot / (double)h->fine_nnz : 0.0;
    }
    // row offsets and sizes per level (int32 indices throughout)
    off.resize(Bt->nlev);
    for (int L = 0; L < Bt->nlev; ++L) {
        BLevel &bl = Bt->lev[L];
        std::vector<int64_t> &o = off[L];
        o.push_back(0);
        int64_t nint = 0;
        for (int k = 0; k < C; ++k) {
            const amg_hierarchy *h = H[Bt->order[k]];
            if (h->nlev <= L) break;
            o.push_back(o.back() + h->lev[L].A.n);
            bl.nsys++;
            if (h->nlev > L + 1) { bl.nsys_int++; nint = o.back(); }
        }
        if (o.back() > 0x7ffffff0LL) return too_large();
        bl.nrows = (int)o.back();
        bl.nint = (int)nint;
        bl.ncoarse = bl.nsys - bl.nsys_int;
    }
    Bt->off0 = C ? off[0] : std::vector<int64_t>(1, 0);
    Bt->total = C ? Bt->lev[0].nrows : 0;
    // ---- all fine operators (FP64) for the PCG; level 0 of the V-cycle uses its first rows
    {
        std::vector<CsrSeg> segs;
        int64_t nnz = 0, longest = 1;
        for (int k = 0; k < C; ++k) {
            const DevCsr &A = H[Bt->order[k]]->lev[0].A;
            segs.push_back(CsrSeg{A.rp, A.ci, A.v, A.n, (int)off[0][k], (int)nnz, (int)off[0][k], k});
            nnz += A.nnz;
            longest = std::max<int64_t>(longest, std::max<int64_t>(A.nnz, A.n));
            if (nnz > 0x7ffffff0LL) return too_large();
        }
        Bt->nnz0 = nnz;
        int *rowsys0 = nullptr;
        CKB(gather_csr(Bt, segs, longest, Bt->total, nnz, &Bt->a0rp, &Bt->a0ci, (void **)&Bt->a0v, false, &rowsys0));
        if (Bt->nlev > 0) {
            BLevel &l0 = Bt->lev[0];
            l0.arp = Bt->a0rp;
            l0.aci = Bt->a0ci;
            l0.rowsys = rowsys0;
            int64_t nnz_int = 0;
            for (int k = 0; k < l0.nsys_int; ++k) nnz_int += H[Bt->order[k]]->lev[0].A.nnz;
            l0.nnz_a = nnz_int;
            if (mixed) {
                CKB(balloc(Bt, (float **)&l0.av, (size_t)nnz));
                if (nnz) {
                    convert_kernel<double, float><<<grid_for(nnz, 256, 16384), 256, 0, s>>>((int)nnz, Bt->a0v,
                                                                                        (float *)l0.av); note_launch();
                    CKB(cudaGetLastError());
                }
            } else {
                l0.av = Bt->a0v;
            }
        }
    }
    // ---- per level: A (L >= 1), P, R, 1/diag, row map, Chebyshev tables, coarse inverses
    for (int L = 0; L < Bt->nlev; ++L) {
        BLevel &bl = Bt->lev[L];
        if (L > 0 && bl.nint > 0) {
            std::vector<CsrSeg> segs;
            int64_t nnz = 0, longest = 1;
            for (int k = 0; k < bl.nsys_int; ++k) {
                const DevCsr &A = H[Bt->order[k]]->lev[L].A;
                segs.push_back(CsrSeg{A.rp, A.ci, A.v, A.n, (int)off[L][k], (int)nnz, (int)off[L][k], k});
                nnz += A.nnz;
                longest = std::max<int64_t>(longest, std::max<int64_t>(A.nnz, A.n));
            }
            if (nnz > 0x7ffffff0LL) return too_large();
            bl.nnz_a = nnz;
            CKB(gather_csr(Bt, segs, longest, bl.nint, nnz, &bl.arp, &bl.aci, &bl.av, mixed, nullptr));
        }
        if (L > 0) {
            std::vector<SysSeg> ss;
            int longest = 1;
            for (int k = 0; k < bl.nsys; ++k) {
                ss.push_back(SysSeg{(int)off[L][k], (int)(off[L][k + 1] - off[L][k]), k});
                longest = std::max(longest, ss.back().n);
            }
            CKB(balloc(Bt, &bl.rowsys, (size_t)bl.nrows));
            SysSeg *dss = nullptr;
            CKB(upload(Bt, &dss, ss));
            fill_rowsys_kernel<<<dim3((unsigned)gather_width(longest), (unsigned)ss.size()), kBThreads, 0, s>>>(dss, bl.rowsys); note_launch();
            CKB(cudaGetLastError());
        }
        if (bl.nint > 0) {
            std::vector<CsrSeg> ps, rs;
            std::vector<VecSeg> ds;
            std::vector<double> coef;
            int64_t np = 0, nr = 0, longest = 1;
            for (int k = 0; k < bl.nsys_int; ++k) {
                const amg_hierarchy *h = H[Bt->order[k]];
                const Level &lv = h->lev[L];
                ps.push_back(CsrSeg{lv.P.rp, lv.P.ci, lv.P.v, lv.P.n, (int)off[L][k], (int)np, (int)off[L + 1][k], k});
                rs.push_back(CsrSeg{lv.R.rp, lv.R.ci, lv.R.v, lv.R.n, (int)off[L + 1][k], (int)nr, (int)off[L][k], k});
                np += lv.P.nnz;
                nr += lv.R.nnz;
                longest = std::max<int64_t>(longest, std::max<int64_t>(lv.P.nnz, lv.P.n));
                ds.push_back(VecSeg{mixed ? (const void *)lv.invdiag_f : (const void *)lv.invdiag, lv.A.n, off[L][k]});
                cheb_table(lv.lambda_cheb, h->p, coef);
            }
            if (np > 0x7ffffff0LL) return too_large();
            bl.nnz_p = np;
            bl.nnz_r = nr;
            CKB(gather_csr(Bt, ps, longest, bl.nint, np, &bl.prp, &bl.pci, &bl.pv, mixed, nullptr));
            CKB(gather_csr(Bt, rs, longest, Bt->lev[L + 1].nrows, nr, &bl.rrp, &bl.rci, &bl.rv, mixed, nullptr));
            if (mixed) {
                CKB(balloc(Bt, (float **)&bl.invd, (size_t)bl.nint));
                CKB((gather_vec<float, float>(Bt, ds, (float *)bl.invd)));
            } else {
                CKB(balloc(Bt, (double **)&bl.invd, (size_t)bl.nint));
                CKB((gather_vec<double, double>(Bt, ds, (double *)bl.invd)));
            }
            CKB(upload(Bt, &bl.coef, coef));
            CKB(spmv_plan(bl.arp, bl.nint, bl.nnz_a, &bl.plan_a, s));
            CKB(spmv_plan(bl.prp, bl.nint, bl.nnz_p, &bl.plan_p, s));
            CKB(spmv_plan(bl.rrp, Bt->lev[L + 1].nrows, bl.nnz_r, &bl.plan_r, s));
        }
        if (bl.ncoarse > 0) {
            std::vector<CoarseSeg> cs;
            std::vector<VecSeg> is;
            long long ioff = 0;
            for (int k = bl.nsys_int; k < bl.nsys; ++k) {
                const amg_hierarchy *h = H[Bt->order[k]];
                const int n = h->lev[L].A.n;
                cs.push_back(CoarseSeg{(int)off[L][k], n, k, ioff});
                is.push_back(VecSeg{h->coarse_inv, (long long)n * n, ioff});
                ioff += (long long)n * n;
            }
            CKB(upload(Bt, &bl.ctable, cs));
            CKB(balloc(Bt, &bl.cinv, (size_t)ioff));
            CKB((gather_vec<double, double>(Bt, is, bl.cinv)));
        }
        // work vectors (x and x2 both hold all rows: the level's result may end in either)
        const size_t nr = (size_t)bl.nrows, ni = (size_t)bl.nint;
        CKB(balloc(Bt, (char **)&bl.f, nr * ts));
        CKB(balloc(Bt, (char **)&bl.x, nr * ts));
        if (ni > 0) {
            CKB(balloc(Bt, (char **)&bl.x2, nr * ts));
            CKB(balloc(Bt, (char **)&bl.r, ni * ts));
            CKB(balloc(Bt, (char **)&bl.d, ni * ts));
        }
    }
    // ---- PCG workspace
    {
        const size_t n = (size_t)Bt->total;
        std::vector<Chunk> ch;
        for (int k = 0; k < C; ++k) {
            const int b0 = (int)Bt->off0[k], b1 = (int)Bt->off0[k + 1];
            const int cnt = b1 > b0 ? (b1 - b0 + kChunkRows - 1) / kChunkRows : 0;
            const int first = (int)ch.size();
            for (int c = 0; c < cnt; ++c)
                ch.push_back(Chunk{k, b0 + c * kChunkRows, std::min(b1, b0 + (c + 1) * kChunkRows), first, cnt});
        }
        Bt->nchunks = (int)ch.size();
        CKB(upload(Bt, &Bt->chunks, ch));
        CKB(balloc(Bt, &Bt->partial, ch.size()));
        CKB(balloc(Bt, &Bt->partial2, ch.size()));
        CKB(balloc(Bt, &Bt->ticket, (size_t)C));
        CKB(balloc(Bt, &Bt->ticket2, (size_t)C));
        CKB(cudaMemsetAsync(Bt->ticket, 0, sizeof(unsigned) * (size_t)C, s));
        CKB(cudaMemsetAsync(Bt->ticket2, 0, sizeof(unsigned) * (size_t)C, s));
        CKB(balloc(Bt, &Bt->active, (size_t)C));
        CKB(balloc(Bt, &Bt->flag, (size_t)C));
        CKB(balloc(Bt, (char **)&Bt->sc, sizeof(BScal) * (size_t)C));
        CKB(balloc(Bt, &Bt->rr_dev, (size_t)C));
        for (double **v : {&Bt->b, &Bt->x, &Bt->r, &Bt->pv, &Bt->q, &Bt->t, &Bt->zb[0]}) CKB(balloc(Bt, v, n));
        if (mixed) CKB(balloc(Bt, &Bt->zb[1], n));
        CKB(cudaMallocHost(&Bt->rr_host, sizeof(double) * (size_t)(C > 0 ? C : 1)));
        CKB(cudaMallocHost(&Bt->host_flags, sizeof(int) * 2 * (size_t)(C > 0 ? C : 1)));
        if (n > 0) CKB(spmv_plan(Bt->a0rp, Bt->total, Bt->nnz0, &Bt->plan0, s));
    }
    CKB(cudaStreamCreateWithFlags(&Bt->cap, cudaStreamNonBlocking));
    CKB(cudaStreamSynchronize(s));
done:
    return st;
}

// V-cycle of the whole batch from level L with x = 0 (Algorithm 1 per system).  f: the
// level's right-hand side; final_out (level 0 only, may be null): where the finest result
// goes; *out: the buffer holding the result.
template <typename T>
cudaError_t bvcycle(amg_batch *Bt, int L, const T *f, T *final_out, T **out, cudaStream_t s)
{
    BLevel &lv = Bt->lev[L];
    T *x = (T *)lv.x, *x2 = (T *)lv.x2;
    // the systems whose coarsest level this is: dense solves into the buffer that holds the
    // level's result (rows [nint, nrows) of it)
    auto coarse = [&](T *dst) -> cudaError_t {
        if (lv.ncoarse == 0) return cudaSuccess;
        bcoarse_kernel<T><<<lv.ncoarse, kBThreads, 0, s>>>(lv.ctable, Bt->active, lv.cinv, f, dst); note_launch();
        return cudaGetLastError();
    };
    if (lv.nint == 0) {
        *out = final_out ? final_out : x;
        return coarse(*out);
    }
    const int ni = lv.nint;
    const T *av = (const T *)lv.av;
    const T *inv = (const T *)lv.invd;
    T *d = (T *)lv.d;
    const int deg = Bt->degree, cs = Bt->cstride;
    // pre-smoothing from x = 0
    const int *act = Bt->active;
    bcheb_zero_kernel<T><<<grid_for(ni, 256, 16384), 256, 0, s>>>(ni, f, inv, lv.rowsys, lv.coef, cs, act, d, x); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    for (int k = 1; k < deg; ++k) {
        AMG_CUDA_TRY(seg_spmv<T>(SEG_CHEB, lv.plan_a, ni, lv.arp, lv.aci, av, x, x2, f, inv, d, lv.rowsys,
                                 lv.coef + 1 + 2 * k, cs, act, s));
        std::swap(x, x2);
    }
    // r = f - A x; f_c = R r; recursion; x += P x_c
    BLevel &cl = Bt->lev[L + 1];
    AMG_CUDA_TRY(seg_spmv<T>(SEG_RESID, lv.plan_a, ni, lv.arp, lv.aci, av, x, (T *)lv.r, f, nullptr, nullptr,
                             lv.rowsys, nullptr, 0, act, s));
    AMG_CUDA_TRY(seg_spmv<T>(SEG_Y, lv.plan_r, cl.nrows, lv.rrp, lv.rci, (const T *)lv.rv, (const T *)lv.r,
                             (T *)cl.f, nullptr, nullptr, nullptr, cl.rowsys, nullptr, 0, act, s));
    T *xc = nullptr;
    AMG_CUDA_TRY(bvcycle<T>(Bt, L + 1, (const T *)cl.f, nullptr, &xc, s));
    AMG_CUDA_TRY(seg_spmv<T>(SEG_PROLONG, lv.plan_p, ni, lv.prp, lv.pci, (const T *)lv.pv, xc, x, nullptr, nullptr,
                             nullptr, lv.rowsys, nullptr, 0, act, s));
    // post-smoothing from the corrected x
    for (int k = 0; k < deg; ++k) {
        T *dst = (final_out && k == deg - 1) ? final_out : x2;
        AMG_CUDA_TRY(seg_spmv<T>(SEG_CHEB, lv.plan_a, ni, lv.arp, lv.aci, av, x, dst, f, inv, d, lv.rowsys,
                                 lv.coef + 1 + 2 * k, cs, act, s));
        x2 = x;
        x = dst;
    }
    *out = x;
    return coarse(x);
}

// z = M^-1 r for every system of the batch (r, z: FP64 over all fine rows)
cudaError_t bprecond(amg_batch *Bt, const double *r, double *z, cudaStream_t s)
{
    if (Bt->nlev == 0 || Bt->total == 0) return cudaSuccess;
    const int n = Bt->total;
    if (Bt->mixed) {
        BLevel &l0 = Bt->lev[0];
        convert_active_kernel<double, float><<<grid_for(n, 256, 16384), 256, 0, s>>>(n, l0.rowsys, Bt->active, r,
                                                                                    (float *)l0.f); note_launch();
        AMG_CUDA_TRY(cudaGetLastError());
        float *out = nullptr;
        AMG_CUDA_TRY(bvcycle<float>(Bt, 0, (const float *)l0.f, nullptr, &out, s));
        convert_active_kernel<float, double><<<grid_for(n, 256, 16384), 256, 0, s>>>(n, l0.rowsys, Bt->active, out,
                                                                                    z); note_launch();
        return cudaGetLastError();
    }
    double *out = nullptr;
    AMG_CUDA_TRY(bvcycle<double>(Bt, 0, r, z, &out, s));
    if (out == z) return cudaSuccess;
    return cudaMemcpyAsync(z, out, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s);
}

// head of an iteration: q = A p, alpha per system, x and r update, r . r to the host
cudaError_t bhead(amg_batch *Bt, cudaStream_t s)
{
    const int nc = Bt->nchunks;
    AMG_CUDA_TRY(seg_spmv<double>(SEG_Y, Bt->plan0, Bt->total, Bt->a0rp, Bt->a0ci, Bt->a0v, Bt->pv, Bt->q, nullptr,
                                  nullptr, nullptr, Bt->lev[0].rowsys, nullptr, 0, Bt->active, s));
    bpq_kernel<<<nc, kBThreads, 0, s>>>(Bt->chunks, Bt->active, Bt->pv, Bt->q, Bt->partial, Bt->ticket, Bt->sc); note_launch();
    bxr_kernel<<<nc, kBThreads, 0, s>>>(Bt->chunks, Bt->active, Bt->pv, Bt->q, Bt->x, Bt->r, Bt->partial, Bt->ticket,
                                        Bt->sc, Bt->rr_dev); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    return cudaMemcpyAsync(Bt->rr_host, Bt->rr_dev, sizeof(double) * (size_t)Bt->count, cudaMemcpyDeviceToHost, s);
}

// tail of an iteration: z = M^-1 r, r . z (and r . z_prev), p = z + beta p
cudaError_t btail(amg_batch *Bt, int parity, cudaStream_t s)
{
    const int nc = Bt->nchunks;
    double *z = Bt->zb[Bt->zb[1] ? parity : 0];
    double *zp = Bt->zb[1] ? Bt->zb[1 - parity] : nullptr;
    AMG_CUDA_TRY(bprecond(Bt, Bt->r, z, s));
    brz_kernel<<<nc, kBThreads, 0, s>>>(Bt->chunks, Bt->active, Bt->r, z, zp, Bt->partial, Bt->partial2, Bt->ticket,
                                        Bt->ticket2, Bt->sc); note_launch();
    bp_kernel<<<nc, kBThreads, 0, s>>>(Bt->chunks, Bt->active, z, Bt->pv, Bt->sc, zp ? 1 : 0); note_launch();
    return cudaGetLastError();
}

cudaGraphExec_t bgraph(amg_batch *Bt, int parity)
{
    if (Bt->graph_failed) return nullptr;
    if (Bt->gexec[parity]) return Bt->gexec[parity];
    cudaGraph_t g = nullptr;
    const long long before = launch_count();
    cudaError_t e = cudaStreamBeginCapture(Bt->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = btail(Bt, parity, Bt->cap);
        cudaError_t e2 = e1 == cudaSuccess ? bhead(Bt, Bt->cap) : e1;
        e = cudaStreamEndCapture(Bt->cap, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&Bt->gexec[parity], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        Bt->graph_failed = true;    // iterations run eagerly from now on
        Bt->gexec[parity] = nullptr;
        return nullptr;
    }
    Bt->gkernels[parity] = launch_count() - before;
    note_launches(-Bt->gkernels[parity]);
    return Bt->gexec[parity];
}

// t = b - A x and |t|^2 into sc[].tt for the systems in mask (null: all)
cudaError_t btrue_residual(amg_batch *Bt, const int *mask, cudaStream_t s)
{
    AMG_CUDA_TRY(seg_spmv<double>(SEG_RESID, Bt->plan0, Bt->total, Bt->a0rp, Bt->a0ci, Bt->a0v, Bt->x, Bt->t, Bt->b,
                                  nullptr, nullptr, Bt->lev[0].rowsys, nullptr, 0, mask, s));
    bdot_kernel<<<Bt->nchunks, kBThreads, 0, s>>>(Bt->chunks, mask, Bt->t, nullptr, nullptr, Bt->partial, Bt->ticket,
                                                  Bt->sc, 1); note_launch();
    return cudaGetLastError();
}

double now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void batch_release(amg_batch *Bt)
{
    for (int k = 0; k < 2; ++k)
        if (Bt->gexec[k]) cudaGraphExecDestroy(Bt->gexec[k]);
    if (Bt->cap) cudaStreamDestroy(Bt->cap);
    for (void *p : Bt->allocs) cudaFreeAsync(p, Bt->s);
    Bt->allocs.clear();
    cudaStreamSynchronize(Bt->s);
    if (Bt->rr_host) cudaFreeHost(Bt->rr_host);
    if (Bt->host_flags) cudaFreeHost(Bt->host_flags);
}

}  // namespace
}  // namespace amgk

using namespace amgk;

extern "C" {

amg_status_t amg_setup_batch(int count, const amg_csr_t *const *A, const double *const *nullspace,
                             const amg_params_t *p, int threads, amg_handle_t *out)
{
    if (count < 0 || (count > 0 && (!A || !p || !out))) return AMG_ERR_INVALID_ARG;
    for (int k = 0; k < count; ++k) out[k] = nullptr;
    for (int k = 0; k < count; ++k)
        if (!A[k]) return AMG_ERR_INVALID_ARG;
    if (count == 0) return AMG_OK;
    if (spmv_error_flag() == nullptr) return fail_cuda(cudaErrorMemoryAllocation, "amg_setup_batch");
    int nt = threads > 0 ? threads : (int)std::min(16u, std::max(1u, std::thread::hardware_concurrency()));
    nt = std::min(nt, count);
    int dev = 0;
    cudaError_t de = cudaGetDevice(&dev);
    if (de != cudaSuccess) return fail_cuda(de, "amg_setup_batch");
    std::atomic<int> next{0};
    std::vector<amg_status_t> status((size_t)count, AMG_OK);
    std::vector<std::string> msg((size_t)count);
    auto worker = [&]() {
        cudaSetDevice(dev);
        cudaStream_t ws = nullptr;
        if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) ws = nullptr;
        for (;;) {
            const int k = next.fetch_add(1);
            if (k >= count) break;
            if (!ws) { status[k] = AMG_ERR_CUDA; msg[k] = "stream creation failed"; continue; }
            amg_params_t pk = *p;
            pk.cuda_stream = ws;
            amg_handle_t h = nullptr;
            status[k] = amg_setup(A[k], nullspace ? nullspace[k] : nullptr, &pk, &h);
            if (status[k] != AMG_OK) { msg[k] = amg_last_error(); continue; }
            // amg_setup synchronised its stream; the handle continues on the caller's stream
            h->s = (cudaStream_t)p->cuda_stream;
            h->p.cuda_stream = p->cuda_stream;
            out[k] = h;
        }
        if (ws) cudaStreamDestroy(ws);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
    worker();
    for (std::thread &t : pool) t.join();
    for (int k = 0; k < count; ++k) {
        if (status[k] != AMG_OK) {
            for (int j = 0; j < count; ++j) {
                amg_free(out[j]);
                out[j] = nullptr;
            }
            set_last_error("system " + std::to_string(k) + ": " + msg[k]);
            return status[k];
        }
    }
    return AMG_OK;
}

amg_status_t amg_batch_create(int count, const amg_handle_t *h, void *cuda_stream, amg_batch_t *out)
{
    if (!out) return AMG_ERR_INVALID_ARG;
    *out = nullptr;
    if (count < 0 || (count > 0 && !h)) return AMG_ERR_INVALID_ARG;
    if (count > 65535) {
        set_last_error("at most 65535 systems per batch");
        return AMG_ERR_UNSUPPORTED;
    }
    for (int k = 0; k < count; ++k) {
        if (!h[k]) return AMG_ERR_INVALID_ARG;
        if (h[k]->p.precision != h[0]->p.precision || h[k]->p.cheb_degree != h[0]->p.cheb_degree) {
            set_last_error("all systems of a batch need the same precision and Chebyshev degree");
            return AMG_ERR_INVALID_ARG;
        }
    }
    amg_batch *Bt = new amg_batch();
    Bt->s = (cudaStream_t)cuda_stream;
    Bt->mixed = count > 0 && h[0]->p.precision == AMG_MIXED;
    Bt->degree = count > 0 ? h[0]->p.cheb_degree : 2;
    Bt->cstride = 1 + 2 * Bt->degree;
    amg_status_t st = batch_assemble(Bt, h, count);
    if (st == AMG_OK) {
        cudaError_t e = cudaStreamSynchronize(Bt->s);
        if (e != cudaSuccess) st = fail_cuda(e, "amg_batch_create");
    }
    if (st != AMG_OK) {
        batch_release(Bt);
        delete Bt;
        return st;
    }
    *out = Bt;
    return AMG_OK;
}

amg_status_t amg_batch_free(amg_batch_t Bt)
{
    if (!Bt) return AMG_OK;
    batch_release(Bt);
    delete Bt;
    return AMG_OK;
}

amg_status_t amg_batch_solve(amg_batch_t Bt, const double *const *b, double *const *x, double tol, amg_info_t *infos)
{
    if (!Bt) return AMG_ERR_INVALID_ARG;
    const int C = Bt->count;
    if (C > 0 && (!b || !x)) return AMG_ERR_INVALID_ARG;
    if (!(tol >= 0.0)) return AMG_ERR_INVALID_ARG;
    for (int k = 0; k < C; ++k) {
        const int u = Bt->order[k];
        if (Bt->off0[k + 1] > Bt->off0[k] && (!b[u] || !x[u])) return AMG_ERR_INVALID_ARG;
    }
    const double t0 = now_ms();
    amg_status_t st = AMG_OK;
    cudaStream_t s = Bt->s;
    const size_t n = (size_t)Bt->total;
    const int nc = Bt->nchunks;
    std::vector<int> iters((size_t)C, 0);
    std::vector<amg_status_t> result((size_t)C, AMG_ERR_NOT_CONVERGED);
    std::vector<double> nb((size_t)C, 0.0), relres((size_t)C, 0.0);
    std::vector<BScal> hs((size_t)C);
    int *act = Bt->host_flags, *flg = Bt->host_flags + C;
    const double *hrr = Bt->rr_host;
    int it = 0, live = 0;
    auto push_flags = [&](const int *src, int *dst) -> cudaError_t {
        return cudaMemcpyAsync(dst, src, sizeof(int) * (size_t)C, cudaMemcpyHostToDevice, s);
    };
    auto pull_scalars = [&]() -> cudaError_t {
        AMG_CUDA_TRY(cudaMemcpyAsync(hs.data(), Bt->sc, sizeof(BScal) * (size_t)C, cudaMemcpyDeviceToHost, s));
        return cudaStreamSynchronize(s);
    };
    if (C == 0) goto finish;
    CKB(cudaMemsetAsync(Bt->sc, 0, sizeof(BScal) * (size_t)C, s));
    // right-hand sides into batch order
    for (int k = 0; k < C; ++k) {
        const size_t len = (size_t)(Bt->off0[k + 1] - Bt->off0[k]);
        if (len) CKB(cudaMemcpyAsync(Bt->b + Bt->off0[k], b[Bt->order[k]], sizeof(double) * len, cudaMemcpyDefault, s));
    }
    if (n > 0) {
        CKB(cudaMemsetAsync(Bt->x, 0, sizeof(double) * n, s));
        CKB(cudaMemcpyAsync(Bt->r, Bt->b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        bdot_kernel<<<nc, kBThreads, 0, s>>>(Bt->chunks, nullptr, Bt->b, nullptr, nullptr, Bt->partial, Bt->ticket,
                                             Bt->sc, 0); note_launch();
        CKB(cudaGetLastError());
    }
    CKB(pull_scalars());
    for (int k = 0; k < C; ++k) {
        nb[k] = std::sqrt(hs[k].bb);
        act[k] = nb[k] > 0.0 && Bt->max_iter[k] > 0 ? 1 : 0;
        flg[k] = 0;
        if (nb[k] == 0.0) result[k] = AMG_OK;
        live += act[k];
    }
    CKB(push_flags(act, Bt->active));
    if (live == 0) goto finish;
    // z = M^-1 r, p = z, r . z; then the first head
    CKB(bprecond(Bt, Bt->r, Bt->zb[0], s));
    bdot_kernel<<<nc, kBThreads, 0, s>>>(Bt->chunks, Bt->active, Bt->r, Bt->zb[0], Bt->pv, Bt->partial, Bt->ticket,
                                         Bt->sc, 2); note_launch();
    CKB(cudaGetLastError());
    CKB(bhead(Bt, s));
    it = 1;
    for (int k = 0; k < C; ++k) iters[k] += act[k];
    for (;;) {
        CKB(cudaStreamSynchronize(s));
        bool any_flag = false, changed = false;
        for (int k = 0; k < C; ++k) {
            flg[k] = act[k] && std::sqrt(hrr[k]) / nb[k] <= tol ? 1 : 0;
            any_flag |= flg[k] != 0;
        }
        if (any_flag) {
            // the recursive residual says converged: check b - A x of those systems
            CKB(push_flags(flg, Bt->flag));
            CKB(btrue_residual(Bt, Bt->flag, s));
            CKB(pull_scalars());
            bool replace = false;
            for (int k = 0; k < C; ++k) {
                if (!flg[k]) continue;
                if (std::sqrt(hs[k].tt) / nb[k] <= tol) {
                    act[k] = 0;
                    flg[k] = 0;
                    result[k] = AMG_OK;
                    changed = true;
                } else {
                    replace = true;     // flg[k] stays set: r = b - A x for this system
                }
            }
            if (replace) {
                CKB(push_flags(flg, Bt->flag));
                bcopy_flagged_kernel<<<nc, kBThreads, 0, s>>>(Bt->chunks, Bt->flag, Bt->t, Bt->r); note_launch();
                CKB(cudaGetLastError());
            }
        }
        live = 0;
        for (int k = 0; k < C; ++k) {
            if (act[k] && iters[k] >= Bt->max_iter[k]) { act[k] = 0; changed = true; }
            live += act[k];
        }
        if (live == 0) break;
        if (changed) CKB(push_flags(act, Bt->active));
        const int parity = Bt->zb[1] ? (it & 1) : 0;
        cudaGraphExec_t gx = bgraph(Bt, parity);
        if (gx) {
            CKB(cudaGraphLaunch(gx, s));
            note_launches(Bt->gkernels[parity]);
        } else {
            CKB(btail(Bt, parity, s));
            CKB(bhead(Bt, s));
        }
        ++it;
        for (int k = 0; k < C; ++k) iters[k] += act[k];
    }
finish:
    if (C > 0 && n > 0) {
        CKB(btrue_residual(Bt, nullptr, s));
        for (int k = 0; k < C; ++k) {
            const size_t len = (size_t)(Bt->off0[k + 1] - Bt->off0[k]);
            if (len)
                CKB(cudaMemcpyAsync(x[Bt->order[k]], Bt->x + Bt->off0[k], sizeof(double) * len, cudaMemcpyDefault, s));
        }
        CKB(pull_scalars());
        for (int k = 0; k < C; ++k) relres[k] = nb[k] > 0.0 ? std::sqrt(hs[k].tt) / nb[k] : 0.0;
    }
    st = AMG_OK;
    for (int k = 0; k < C; ++k)
        if (result[k] != AMG_OK) st = AMG_ERR_NOT_CONVERGED;
    if (spmv_take_errors(s) != 0) {
        set_last_error("a bulk copy into shared memory did not complete in time");
        st = AMG_ERR_INTERNAL;
        for (int k = 0; k < C; ++k) result[k] = AMG_ERR_INTERNAL;
    }
done:
    if (infos) {
        const double ms = now_ms() - t0;
        const bool per_system = st == AMG_OK || st == AMG_ERR_NOT_CONVERGED || st == AMG_ERR_INTERNAL;
        for (int k = 0; k < C; ++k) {
            amg_info_t &in = infos[Bt->order[k]];
            in.iters = iters[k];
            in.status = per_system ? result[k] : st;
            in.relres_true = relres[k];
            in.setup_ms = Bt->setup_ms[k];
            in.solve_ms = ms;
            in.levels = Bt->nlev_sys[k];
            in.op_complexity = Bt->opc[k];
        }
    }
    return st;
}

amg_status_t amg_solve_batch(int count, const amg_handle_t *h, const double *const *b, double *const *x, double tol,
                             amg_info_t *infos)
{
    if (count < 0 || (count > 0 && !h)) return AMG_ERR_INVALID_ARG;
    for (int k = 0; k < count; ++k)
        if (!h[k]) return AMG_ERR_INVALID_ARG;
    amg_batch_t Bt = nullptr;
    amg_status_t st = amg_batch_create(count, h, count > 0 ? h[0]->p.cuda_stream : nullptr, &Bt);
    if (st != AMG_OK) return st;
    st = amg_batch_solve(Bt, b, x, tol, infos);
    amg_batch_free(Bt);
    return st;
}

amg_status_t amg_batch_info(amg_batch_t Bt, int *count, int *levels, int64_t *rows, int64_t *graph_kernels)
{
    if (!Bt) return AMG_ERR_INVALID_ARG;
    if (count) *count = Bt->count;
    if (levels) *levels = Bt->nlev;
    if (rows) *rows = Bt->total;
    if (graph_kernels) *graph_kernels = Bt->gkernels[0];
    return AMG_OK;
}

}  // extern "C"
