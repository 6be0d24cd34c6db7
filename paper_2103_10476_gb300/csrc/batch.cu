// batch.cu -- the segment-indexed engine (engine.cuh) and the batch ABI on top of it: many
// independent systems solved together (no counterpart in the paper, which treats one system;
// each member's arithmetic is that of §1.1, Algorithm 1 and §3.1, as in amg_solve).
//
// Per-member state is a slot: its hierarchy, the offsets of its vectors in the arenas, its
// PCG scalars and stopping test.  A member joins a running engine at the top of an
// iteration: with x = 0, r = b, p = 0, z_prev = 0 and r.z "= 1", the next iteration's
// p = z + beta p is p = z, i.e. exactly the first step of PCG, so starting and joining are
// the same code path.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "engine.cuh"
#include "tma.cuh"

namespace amgk {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kET = 256;            // threads per block of every engine kernel
constexpr int kEngChunk = 4096;     // fine rows per PCG chunk
constexpr int kEngMaxTile = 6144;   // shared-memory tile entries at most
constexpr int kLprs[5] = {2, 4, 8, 16, 32};
enum { SK_Y = 0, SK_RESID = 1, SK_CHEB = 2, SK_PROLONG = 3 };

// ------------------------------------------------------------------------------------ SpMV tiles
// Persistent: block b takes tiles b, b + grid, ... of the list.  Each tile's values and
// column indices are staged in shared memory by two bulk copies completed on one mbarrier
// (its phase advances once per staged tile), then LPR lanes per row gather x.
// records the first violation; every later one only counts
__device__ void guard_hit(EngGuard *g, int kind, int slot, int where, const int *info = nullptr, int ninfo = 0)
{
    if (atomicAdd(&g->count, 1) == 0) {
        g->kind = kind;
        g->slot = slot;
        g->where = where;
        for (int k = 0; k < ninfo && k < 12; ++k) g->info[k] = info[k];
    }
}

// the tile's rows, its entries and the vector ranges it touches all lie inside their arrays
__device__ __forceinline__ bool tile_ok(const SegTile &tl, const SegOp &op, int nslots, int xcap, int ycap,
                                        EngGuard *g)
{
    bool ok = tl.slot >= 0 && tl.slot < nslots && tl.row0 >= 0 && tl.rows > 0 && tl.row0 + tl.rows <= op.n &&
              op.xoff >= 0 && op.yoff >= 0 && (int64_t)op.xoff + op.ncol <= xcap &&
              (int64_t)op.yoff + op.n <= ycap;
    int k0 = -1, k1 = -1;
    if (ok) {
        k0 = op.rp[tl.row0];
        k1 = op.rp[tl.row0 + tl.rows];
        ok = k0 >= 0 && k0 <= k1 && k1 <= op.nnz;
    }
    if (!ok && threadIdx.x == 0) {
        const int info[12] = {tl.row0, tl.rows, op.n, op.ncol, op.nnz, k0, k1, op.xoff, op.yoff, xcap, ycap,
                              op.rp ? op.rp[0] : -7};
        guard_hit(g, 1, tl.slot, tl.row0, info, 12);
    }
    return ok;
}

template <typename T, int LPR, int MODE>
__global__ void __launch_bounds__(kET) segtile_kernel(const SegTile *__restrict__ tiles, const int *__restrict__ count,
                                                      const SegOp *__restrict__ ops, const T *__restrict__ x, T *y,
                                                      const T *__restrict__ f, T *d, int coef_idx, int cap, int *err,
                                                      int nslots, int xcap, int ycap, EngGuard *guard)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    constexpr int VA = 16 / (int)sizeof(T);
    T *sv = (T *)smem;
    int *sci = (int *)(smem + tile_values_bytes<T>(cap));
    const int ntiles = *count;
    if ((int)blockIdx.x >= ntiles) return;
    if (cap > 0) {
        if (threadIdx.x == 0) mbar_init(&bar, 1);
        __syncthreads();
    }
    unsigned phase = 0;
    const int lrow = threadIdx.x / LPR, lane = threadIdx.x % LPR;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const SegTile tl = tiles[t];
        if (tl.slot < 0 || tl.slot >= nslots) {
            if (threadIdx.x == 0) guard_hit(guard, 1, tl.slot, t);
            continue;
        }
        const SegOp op = ops[tl.slot];
        if (!tile_ok(tl, op, nslots, xcap, ycap, guard)) continue;     // uniform over the block
        const T *v = (const T *)op.v;
        const int r0 = tl.row0, r1 = tl.row0 + tl.rows;
        const int k0 = op.rp[r0], k1 = op.rp[r1];
        const int k0v = k0 & ~(VA - 1), k1v = (k1 + VA - 1) & ~(VA - 1);
        const int k0i = k0 & ~3, k1i = (k1 + 3) & ~3;
        const bool staged = cap > 0 && (k1v - k0v) <= cap + 2 * VA && (k1i - k0i) <= cap + 8 && k1 > k0;
        if (staged) {
            if (threadIdx.x == 0) {
                const unsigned bv = (unsigned)((k1v - k0v) * (int)sizeof(T)), bi = (unsigned)((k1i - k0i) * 4);
                mbar_expect_tx(&bar, bv + bi);
                bulk_g2s(sv, v + k0v, bv, &bar);
                bulk_g2s(sci, op.ci + k0i, bi, &bar);
            }
            const bool ok = __syncthreads_and(mbar_wait_bounded(&bar, phase & 1u, err));
            ++phase;
            if (!ok) return;    // error recorded; nothing more is written by this block
        }
        const int row = r0 + lrow;
        const T *xs = x + op.xoff;
        T sum = T(0);
        if (row < r1) {
            const int b = op.rp[row], e = op.rp[row + 1];
            if (staged) {
                for (int k = b + lane; k < e; k += LPR) sum += sv[k - k0v] * xs[sci[k - k0i]];
            } else {
                for (int k = b + lane; k < e; k += LPR) sum += v[k] * xs[op.ci[k]];
            }
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o, LPR);
        if (row < r1 && lane == 0) {
            const int yi = op.yoff + row;
            if (MODE == SK_Y) {
                y[yi] = sum;
            } else if (MODE == SK_RESID) {
                y[yi] = f[yi] - sum;
            } else if (MODE == SK_CHEB) {
                const double *cs = op.coef + coef_idx;
                const T c1 = (T)cs[0], c2 = (T)cs[1];
                const T rr = f[yi] - sum;
                const T dn = c1 * d[yi] + c2 * (((const T *)op.invd)[row] * rr);
                d[yi] = dn;
                y[yi] = x[yi] + dn;     // square operator: x is row-indexed at the same offset
            } else {
                y[yi] += sum;
            }
        }
        __syncthreads();                // the next tile overwrites the shared tile
    }
}

// first Chebyshev step from x = 0 over the rows of the A tiles: d = D^-1 f / theta, x = d
template <typename T>
__global__ void __launch_bounds__(kET) segcheb0_kernel(const SegTile *tiles, const int *count, const SegOp *ops,
                                                       const T *f, T *d, T *x, int nslots, int cap, EngGuard *guard)
{
    const int ntiles = *count;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const SegTile tl = tiles[t];
        if (tl.slot < 0 || tl.slot >= nslots) {
            if (threadIdx.x == 0) guard_hit(guard, 2, tl.slot, t);
            continue;
        }
        const SegOp op = ops[tl.slot];
        if (tl.row0 < 0 || tl.row0 + tl.rows > op.n || op.yoff < 0 || (int64_t)op.yoff + op.n > cap) {
            if (threadIdx.x == 0) guard_hit(guard, 2, tl.slot, tl.row0);
            continue;
        }
        const T inv_theta = (T)op.coef[0];
        const T *invd = (const T *)op.invd;
        for (int i = threadIdx.x; i < tl.rows; i += kET) {
            const int row = tl.row0 + i, yi = op.yoff + row;
            const T di = (invd[row] * f[yi]) * inv_theta;
            d[yi] = di;
            x[yi] = di;
        }
    }
}

// dense coarsest-level solves x = Ainv f: a block per item (kCoarseRows rows of one slot's
// solve), a warp per row (FP64 sums over the row in lane-strided order)
template <typename T>
__global__ void __launch_bounds__(kET) segcoarse_kernel(const SegCoarse *list, const int *count, const T *f, T *x,
                                                        int nslots, int cap, EngGuard *guard)
{
    const int n_items = *count;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < n_items; t += gridDim.x) {
        const SegCoarse c = list[t];
        if (c.slot < 0 || c.slot >= nslots || c.n < 0 || c.off < 0 || (int64_t)c.off + c.n > cap || !c.inv ||
            c.row0 < 0 || c.row0 >= c.n) {
            if (threadIdx.x == 0) guard_hit(guard, 3, c.slot, c.off);
            continue;
        }
        const int r1 = min(c.n, c.row0 + kCoarseRows);
        for (int i = c.row0 + w; i < r1; i += kET / 32) {
            double acc = 0.0;
            for (int k = lane; k < c.n; k += 32) acc += c.inv[(size_t)i * c.n + k] * (double)f[c.off + k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
            if (lane == 0) x[c.off + i] = (T)acc;
        }
    }
}

// ------------------------------------------------------------------------------------ PCG chunks
__device__ __forceinline__ double block_total(double v)
{
    __shared__ double sh[kET / 32];
    __shared__ double tot;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kET / 32; ++k) t += sh[k];
        tot = t;
    }
    __syncthreads();
    const double r = tot;
    __syncthreads();
    return r;
}

// Stores the chunk's partial at its id; the slot's last chunk to arrive (ticket) returns
// true with *total = the slot's partials added in chunk order, and resets the ticket.
__device__ __forceinline__ bool chunk_finish(const SegChunk &c, double part, double *partial, unsigned *ticket,
                                             double *total)
{
    __shared__ bool last;
    __shared__ double tot;
    if (threadIdx.x == 0) {
        partial[c.id] = part;
        __threadfence();
        last = atomicAdd(&ticket[c.slot], 1u) == (unsigned)c.count - 1u;
    }
    __syncthreads();
    if (!last) return false;
    if (threadIdx.x == 0) {
        __threadfence();
        double t = 0.0;
        for (int k = 0; k < c.count; ++k) t += ((volatile const double *)partial)[c.first + k];
        tot = t;
        ticket[c.slot] = 0u;
    }
    __syncthreads();
    *total = tot;
    return true;
}

// a chunk inside the fine arena and the slot table (uniform over the block)
__device__ __forceinline__ bool chunk_ok(const SegChunk &c, int nslots, int cap, EngGuard *g)
{
    const bool ok = c.slot >= 0 && c.slot < nslots && c.begin >= 0 && c.begin <= c.end && c.end <= cap &&
                    c.first >= 0 && c.id >= c.first && c.id < c.first + c.count;
    if (!ok && threadIdx.x == 0) guard_hit(g, 4, c.slot, c.begin);
    return ok;
}

// start of a solve: x = 0, r = b, p = 0, z_prev = 0, r.z = 1
__global__ void __launch_bounds__(kET) eng_init_kernel(const SegChunk *chunks, const int *count, const double *b,
                                                       double *x, double *r, double *p, double *zp, EngScal *sc,
        int nslots, int cap, EngGuard *guard)
{
    const int n = *count;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const SegChunk c = chunks[t];
        if (!chunk_ok(c, nslots, cap, guard)) continue;
        for (int i = c.begin + threadIdx.x; i < c.end; i += kET) {
            x[i] = 0.0;
            r[i] = b[i];
            p[i] = 0.0;
            if (zp) zp[i] = 0.0;
        }
        if (threadIdx.x == 0 && c.id == c.first) sc[c.slot].rz = 1.0;
    }
}

// a . a per slot: which = 0 -> bb, 1 -> tt
__global__ void __launch_bounds__(kET) eng_norm_kernel(const SegChunk *chunks, const int *count, const double *a,
                                                       double *partial, unsigned *ticket, EngScal *sc, int which,
        int nslots, int cap, EngGuard *guard)
{
    const int n = *count;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const SegChunk c = chunks[t];
        if (!chunk_ok(c, nslots, cap, guard)) continue;
        double acc = 0.0;
        for (int i = c.begin + threadIdx.x; i < c.end; i += kET) acc += a[i] * a[i];
        acc = block_total(acc);
        double tot;
        if (chunk_finish(c, acc, partial, ticket, &tot) && threadIdx.x == 0) {
            if (which == 0) sc[c.slot].bb = tot;
            else sc[c.slot].tt = tot;
        }
    }
}

// p . q per slot; the slot's last chunk sets alpha = rz_new / (p . q) and rz = rz_new
__global__ void __launch_bounds__(kET) eng_pq_kernel(const SegChunk *chunks, const int *count, const double *p,
                                                     const double *q, double *partial, unsigned *ticket, EngScal *sc,
        int nslots, int cap, EngGuard *guard)
{
    const int n = *count;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const SegChunk c = chunks[t];
        if (!chunk_ok(c, nslots, cap, guard)) continue;
        double acc = 0.0;
        for (int i = c.begin + threadIdx.x; i < c.end; i += kET) acc += p[i] * q[i];
        acc = block_total(acc);
        double tot;
        if (chunk_finish(c, acc, partial, ticket, &tot) && threadIdx.x == 0) {
            EngScal &s = sc[c.slot];
            s.pq = tot;
            s.alpha = s.rz_new / tot;
            s.rz = s.rz_new;
        }
    }
}

// x += alpha p; r -= alpha q; r . r per slot into rr[slot]
__global__ void __launch_bounds__(kET) eng_xr_kernel(const SegChunk *chunks, const int *count, const double *p,
                                                     const double *q, double *x, double *r, double *partial,
                                                     unsigned *ticket, EngScal *sc, double *rr,
        int nslots, int cap, EngGuard *guard)
{
    const int n = *count;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const SegChunk c = chunks[t];
        if (!chunk_ok(c, nslots, cap, guard)) continue;
        const double alpha = sc[c.slot].alpha;
        double acc = 0.0;
        for (int i = c.begin + threadIdx.x; i < c.end; i += kET) {
            x[i] += alpha * p[i];
            const double ri = r[i] - alpha * q[i];
            r[i] = ri;
            acc += ri * ri;
        }
        acc = block_total(acc);
        double tot;
        if (chunk_finish(c, acc, partial, ticket, &tot) && threadIdx.x == 0) {
            sc[c.slot].rr = tot;
            rr[c.slot] = tot;
        }
    }
}

// r . z -> rz_new and r . z_prev -> cross (flexible form) per slot
__global__ void __launch_bounds__(kET) eng_rz_kernel(const SegChunk *chunks, const int *count, const double *r,
                                                     const double *z, const double *zp, double *partial,
                                                     double *partial2, unsigned *ticket, unsigned *ticket2,
                                                     EngScal *sc,
        int nslots, int cap, EngGuard *guard)
{
    const int n = *count;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const SegChunk c = chunks[t];
        if (!chunk_ok(c, nslots, cap, guard)) continue;
        double a = 0.0, b = 0.0;
        for (int i = c.begin + threadIdx.x; i < c.end; i += kET) {
            const double ri = r[i];
            a += ri * z[i];
            if (zp) b += ri * zp[i];
        }
        a = block_total(a);
        double tot;
        if (chunk_finish(c, a, partial, ticket, &tot) && threadIdx.x == 0) sc[c.slot].rz_new = tot;
        if (zp) {
            b = block_total(b);
            if (chunk_finish(c, b, partial2, ticket2, &tot) && threadIdx.x == 0) sc[c.slot].cross = tot;
        }
    }
}

// beta = rz_new / rz (flexible: (rz_new - cross) / rz); p = z + beta p
__global__ void __launch_bounds__(kET) eng_p_kernel(const SegChunk *chunks, const int *count, const double *z,
                                                    double *p, const EngScal *sc, int flexible,
        int nslots, int cap, EngGuard *guard)
{
    const int n = *count;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const SegChunk c = chunks[t];
        if (!chunk_ok(c, nslots, cap, guard)) continue;
        const EngScal s = sc[c.slot];
        const double beta = (flexible ? s.rz_new - s.cross : s.rz_new) / s.rz;
        for (int i = c.begin + threadIdx.x; i < c.end; i += kET) p[i] = z[i] + beta * p[i];
    }
}

__global__ void __launch_bounds__(kET) eng_copy_kernel(const SegChunk *chunks, const int *count, const double *src,
                                                       double *dst,
        int nslots, int cap, EngGuard *guard)
{
    const int n = *count;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const SegChunk c = chunks[t];
        if (!chunk_ok(c, nslots, cap, guard)) continue;
        for (int i = c.begin + threadIdx.x; i < c.end; i += kET) dst[i] = src[i];
    }
}

template <typename A, typename B>
__global__ void __launch_bounds__(kET) eng_convert_kernel(const SegChunk *chunks, const int *count, const A *src,
                                                          B *dst,
        int nslots, int cap, EngGuard *guard)
{
    const int n = *count;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const SegChunk c = chunks[t];
        if (!chunk_ok(c, nslots, cap, guard)) continue;
        for (int i = c.begin + threadIdx.x; i < c.end; i += kET) dst[i] = (B)src[i];
    }
}

// ------------------------------------------------------------------------------------ lists
// out = the items of `full` whose slot has mask[slot] != 0 (order of arrival: every item is
// independent work, and every reduction is ordered by chunk id, not by list position)
template <typename E>
__global__ void compact_kernel(const E *full, int n, const int *mask, E *out, int *count)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const E e = full[i];
        if (mask[e.slot]) out[atomicAdd(count, 1)] = e;
    }
}

// largest number of stored entries of one tile of the list
__global__ void span_kernel(const SegTile *tiles, int n, const SegOp *ops, int *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const SegTile t = tiles[i];
        const SegOp op = ops[t.slot];
        atomicMax(out, op.rp[t.row0 + t.rows] - op.rp[t.row0]);
    }
}

__global__ void set_count_kernel(int *count, int value) { *count = value; }

// ------------------------------------------------------------------------------------ launch helpers
// Persistent grid: as many blocks as can be resident at once (the occupancy of this
// instantiation with this shared-memory tile), capped by `grid` (the list's length bound).
template <typename T, int LPR, int MODE>
cudaError_t seg_launch_lpr(const SegTile *tiles, const int *count, const SegOp *ops, const T *x, T *y, const T *f,
                           T *d, int coef_idx, int cap, int grid, const SegCtx &cx, cudaStream_t s)
{
    static std::once_flag once;
    static cudaError_t cfg = cudaSuccess;
    static int sms = 0;
    std::call_once(once, [] {
        cfg = cudaFuncSetAttribute(segtile_kernel<T, LPR, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   tile_bytes<T>(kEngMaxTile));
        int dev = 0;
        if (cfg == cudaSuccess) cfg = cudaGetDevice(&dev);
        if (cfg == cudaSuccess) cfg = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    });
    AMG_CUDA_TRY(cfg);
    const int smem = tile_bytes<T>(cap);
    int per_sm = 0;
    AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, segtile_kernel<T, LPR, MODE>, kET, smem));
    const int g = std::max(1, std::min(grid, std::max(1, per_sm) * sms));
    segtile_kernel<T, LPR, MODE><<<g, kET, smem, s>>>(tiles, count, ops, x, y, f, d, coef_idx, cap,
                                                      &cx.guard->waits, cx.nslots, cx.xcap, cx.ycap, cx.guard); note_launch();
    return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t seg_launch(int lpr, const SegTile *tiles, const int *count, const SegOp *ops, const T *x, T *y,
                       const T *f, T *d, int coef_idx, int cap, int grid, const SegCtx &cx, cudaStream_t s)
{
    switch (lpr) {
    case 2: return seg_launch_lpr<T, 2, MODE>(tiles, count, ops, x, y, f, d, coef_idx, cap, grid, cx, s);
    case 4: return seg_launch_lpr<T, 4, MODE>(tiles, count, ops, x, y, f, d, coef_idx, cap, grid, cx, s);
    case 8: return seg_launch_lpr<T, 8, MODE>(tiles, count, ops, x, y, f, d, coef_idx, cap, grid, cx, s);
    case 16: return seg_launch_lpr<T, 16, MODE>(tiles, count, ops, x, y, f, d, coef_idx, cap, grid, cx, s);
    default: return seg_launch_lpr<T, 32, MODE>(tiles, count, ops, x, y, f, d, coef_idx, cap, grid, cx, s);
    }
}

// Chebyshev coefficients of one level of one system, the recurrence of solve.cu's smoother on
// [b lambda / ratio, b lambda] (§3.1's Chebyshev smoothing): [1/theta, then (c1, c2) for each
// step k of a pass that starts from a non-zero iterate (step 0: c1 = 0, c2 = 1/theta)]
void cheb_table(double lambda, const amg_params_t &p, double *out)
{
    const double lmax = p.cheb_boost * lambda, lmin = lmax / p.cheb_ratio;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma1 = theta / delta;
    int k = 0;
    out[k++] = 1.0 / theta;
    out[k++] = 0.0;
    out[k++] = 1.0 / theta;
    double rho = 1.0 / sigma1;
    for (int j = 1; j < p.cheb_degree; ++j) {
        const double rho_new = 1.0 / (2.0 * sigma1 - rho);
        out[k++] = rho_new * rho;
        out[k++] = 2.0 * rho_new / delta;
        rho = rho_new;
    }
}

void cut_tiles(std::vector<SegTile> &out, int slot, int rows, int rpb)
{
    for (int r = 0; r < rows; r += rpb) out.push_back(SegTile{slot, r, std::min(rpb, rows - r), 0});
}

double now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// (re)allocates a list's device arrays when the host list outgrew them; *moved if it did
template <typename E>
cudaError_t upload_list(EngList<E> &l, std::vector<void *> &allocs, size_t &bytes, cudaStream_t s, bool *moved)
{
    l.nfull = (int)l.host.size();
    if (!l.full || (size_t)l.nfull > l.capacity) {
        // the old arrays stay in the owner's allocation list until it is destroyed
        const size_t cap = std::max<size_t>(64, (size_t)l.nfull + l.nfull / 4);
        for (E **p : {&l.full, &l.act, &l.flg}) {
            AMG_CUDA_TRY(cudaMallocAsync((void **)p, sizeof(E) * (cap + 16), s));
            allocs.push_back((void *)*p);
            bytes += sizeof(E) * (cap + 16);
        }
        if (!l.count) {
            AMG_CUDA_TRY(cudaMallocAsync((void **)&l.count, sizeof(int) * 16, s));
            allocs.push_back((void *)l.count);
            AMG_CUDA_TRY(cudaMemsetAsync(l.count, 0, sizeof(int) * 16, s));
        }
        l.capacity = cap;
        *moved = true;
    }
    if (l.nfull > 0)
        AMG_CUDA_TRY(cudaMemcpyAsync(l.full, l.host.data(), sizeof(E) * (size_t)l.nfull, cudaMemcpyHostToDevice, s));
    return cudaSuccess;
}

}  // namespace

// ------------------------------------------------------------------------------------ Engine
template <typename T>
cudaError_t Engine::alloc(T **p, size_t count)
{
    *p = nullptr;
    const size_t bytes = (count + 16) * sizeof(T);
    cudaError_t e = cudaMallocAsync((void **)p, bytes, s_);
    if (e == cudaSuccess) {
        allocs_.push_back((void *)*p);
        bytes_ += bytes;
    }
    return e;
}

Engine::~Engine()
{
    drop_graphs();
    if (cap_) cudaStreamDestroy(cap_);
    for (void *p : allocs_) cudaFreeAsync(p, s_);
    cudaStreamSynchronize(s_);
    if (rr_host_) cudaFreeHost(rr_host_);
    if (hflags_) cudaFreeHost(hflags_);
    for (cudaEvent_t e : flag_ev_)
        if (e) cudaEventDestroy(e);
}

void Engine::drop_graphs()
{
    for (int k = 0; k < 2; ++k) {
        if (gexec_[k]) cudaGraphExecDestroy(gexec_[k]);
        gexec_[k] = nullptr;
    }
}

#define EK(expr)                                                           \
    do {                                                                   \
        cudaError_t _e = (expr);                                           \
        if (_e != cudaSuccess) return fail_cuda(_e, #expr);                \
    } while (0)

amg_status_t Engine::init(const Config &c, cudaStream_t s)
{
    cfg_ = c;
    s_ = s;
    cstride_ = 1 + 2 * c.degree;
    const int S = c.slots > 0 ? c.slots : 1;
    const size_t ts = c.mixed ? sizeof(float) : sizeof(double);
    const size_t n0 = (size_t)std::max<int64_t>(c.cap0, 1), nc = (size_t)std::max<int64_t>(c.capc, 1);
    slots_.assign((size_t)S, Slot());
    hA_.assign((size_t)kEngLevels * S, SegOp{});
    hP_ = hA_;
    hR_ = hA_;
    h0_.assign((size_t)S, SegOp{});
    hC_.assign((size_t)kEngLevels * S, SegCoarse{});
    hcoef_.assign((size_t)S * kEngLevels * cstride_, 0.0);
    free0_.assign(1, {0, c.cap0});
    freec_.assign(1, {0, c.capc});
    EK(alloc(&opA_, hA_.size()));
    EK(alloc(&opP_, hA_.size()));
    EK(alloc(&opR_, hA_.size()));
    EK(alloc(&op0_, h0_.size()));
    EK(alloc(&opC_, hC_.size()));
    EK(alloc(&coef_, hcoef_.size()));
    EK(alloc(&active_, (size_t)S));
    EK(alloc(&flag_, (size_t)S));
    EK(cudaMemsetAsync(active_, 0, sizeof(int) * S, s_));
    EK(cudaMemsetAsync(flag_, 0, sizeof(int) * S, s_));
    EK(alloc((char **)&sc_, sizeof(EngScal) * (size_t)S));
    EK(cudaMemsetAsync(sc_, 0, sizeof(EngScal) * S, s_));
    EK(alloc(&rr_dev_, (size_t)S));
    EK(alloc(&ticket_, (size_t)S));
    EK(alloc(&ticket2_, (size_t)S));
    EK(cudaMemsetAsync(ticket_, 0, sizeof(unsigned) * S, s_));
    EK(cudaMemsetAsync(ticket2_, 0, sizeof(unsigned) * S, s_));
    EK(alloc(&caps_dev_, (size_t)(3 * kEngLevels + 1)));
    EK(alloc(&guard_, 1));
    EK(cudaMemsetAsync(guard_, 0, sizeof(EngGuard), s_));
    EK(cudaMallocHost(&rr_host_, sizeof(double) * S));
    EK(cudaMallocHost(&hflags_, sizeof(int) * 2 * S));
    for (cudaEvent_t &e : flag_ev_) EK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    std::memset(hflags_, 0, sizeof(int) * 2 * S);
    for (double **v : {&b_, &x_, &r_, &p_, &q_, &t_, &zb_[0]}) EK(alloc(v, n0));
    if (c.mixed) EK(alloc(&zb_[1], n0));
    for (void **v : {&x0_, &x20_, &r0_, &d0_}) EK(alloc((char **)v, n0 * ts));
    for (void **v : {&fc_, &xc_, &x2c_, &rc_, &dc_}) EK(alloc((char **)v, nc * ts));
    if (c.mixed) EK(alloc((char **)&f0_, n0 * ts));
    EK(cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking));
    {
        int dev = 0, sms = 0;
        EK(cudaGetDevice(&dev));
        EK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        grid_tiles_ = sms * 8;      // persistent grids of the elementwise and coarse kernels
        grid_chunks_ = sms * 8;
    }
    EK(cudaStreamSynchronize(s_));
    return AMG_OK;
}

int64_t Engine::arena_take(std::vector<std::pair<int64_t, int64_t>> &fl, int64_t n)
{
    if (n == 0) return 0;
    for (size_t i = 0; i < fl.size(); ++i) {
        if (fl[i].second >= n) {
            const int64_t off = fl[i].first;
            fl[i].first += n;
            fl[i].second -= n;
            if (fl[i].second == 0) fl.erase(fl.begin() + (long)i);
            return off;
        }
    }
    return -1;
}

void Engine::arena_give(std::vector<std::pair<int64_t, int64_t>> &fl, int64_t off, int64_t n)
{
    if (n == 0) return;
    fl.push_back({off, n});
    std::sort(fl.begin(), fl.end());
    std::vector<std::pair<int64_t, int64_t>> m;
    for (auto &h : fl) {
        if (!m.empty() && m.back().first + m.back().second == h.first) m.back().second += h.second;
        else m.push_back(h);
    }
    fl.swap(m);
}

int Engine::add(amg_hierarchy *h)
{
    if (!h || h->nlev < 1 || h->nlev > kEngLevels || !h->coarse_inv) return -1;
    if ((h->p.precision == AMG_MIXED) != (cfg_.mixed != 0) || h->p.cheb_degree != cfg_.degree) return -1;
    int k = -1;
    for (int i = 0; i < (int)slots_.size(); ++i)
        if (!slots_[i].used) { k = i; break; }
    if (k < 0) return -1;
    Slot sl;
    sl.h = h;
    sl.nlev = h->nlev;
    sl.n0 = h->lev[0].A.n;
    for (int L = 1; L < h->nlev; ++L) sl.csize += h->lev[L].A.n;
    sl.o0 = arena_take(free0_, sl.n0);
    if (sl.o0 < 0) return -1;
    sl.oc = arena_take(freec_, sl.csize);
    if (sl.oc < 0) {
        arena_give(free0_, sl.o0, sl.n0);
        return -1;
    }
    sl.off[0] = sl.o0;
    int64_t o = sl.oc;
    for (int L = 1; L < h->nlev; ++L) {
        sl.off[L] = o;
        o += h->lev[L].A.n;
    }
    sl.used = true;
    const int S = (int)slots_.size();
    const bool mixed = cfg_.mixed != 0;
    for (int L = 0; L + 1 < h->nlev; ++L) {
        const Level &lv = h->lev[L];
        const size_t i = (size_t)L * S + k;
        const size_t ci = ((size_t)k * kEngLevels + L) * cstride_;
        cheb_table(lv.lambda_cheb, h->p, &hcoef_[ci]);
        hA_[i] = SegOp{lv.A.rp, lv.A.ci, mixed ? (const void *)lv.Af : (const void *)lv.A.v,
                       mixed ? (const void *)lv.invdiag_f : (const void *)lv.invdiag, coef_ + ci, (int)sl.off[L],
                       (int)sl.off[L], lv.A.n, lv.A.n, (int)lv.A.nnz, 0};
        hP_[i] = SegOp{lv.P.rp, lv.P.ci, mixed ? (const void *)lv.Pf : (const void *)lv.P.v, nullptr, nullptr,
                       (int)sl.off[L + 1], (int)sl.off[L], lv.P.n, lv.P.ncol, (int)lv.P.nnz, 0};
        hR_[i] = SegOp{lv.R.rp, lv.R.ci, mixed ? (const void *)lv.Rf : (const void *)lv.R.v, nullptr, nullptr,
                       (int)sl.off[L], (int)sl.off[L + 1], lv.R.n, lv.R.ncol, (int)lv.R.nnz, 0};
    }
    {
        const int L = h->nlev - 1;
        hC_[(size_t)L * S + k] = SegCoarse{h->coarse_inv, h->lev[L].A.n, (int)sl.off[L], k, 0};
    }
    const Level &l0 = h->lev[0];
    h0_[k] = SegOp{l0.A.rp, l0.A.ci, l0.A.v, nullptr, nullptr, (int)sl.o0, (int)sl.o0, l0.A.n, l0.A.n,
                   (int)l0.A.nnz, 0};
    slots_[k] = sl;
    members_changed_ = true;
    return k;
}

void Engine::remove(int k)
{
    if (k < 0 || k >= (int)slots_.size() || !slots_[k].used) return;
    Slot &sl = slots_[k];
    arena_give(free0_, sl.o0, sl.n0);
    arena_give(freec_, sl.oc, sl.csize);
    if (sl.active) --live_;
    sl = Slot();
    members_changed_ = true;
}

void Engine::load(int k, const double *b, double tol, int max_iter)
{
    if (k < 0 || k >= (int)slots_.size() || !slots_[k].used) return;
    Slot &sl = slots_[k];
    sl.pending = true;
    sl.b = b;
    sl.tol = tol;
    sl.max_iter = max_iter;
}

// host lists of every used slot, in slot order, with each list's current lanes per row
void Engine::build_lists()
{
    for (int L = 0; L < kEngLevels; ++L) {
        lA_[L].host.clear();
        lP_[L].host.clear();
        lR_[L].host.clear();
        lC_[L].host.clear();
    }
    l0_.host.clear();
    lch_.host.clear();
    nlev_ = 0;
    const size_t S = slots_.size();
    for (int k = 0; k < (int)S; ++k) {
        const Slot &sl = slots_[k];
        if (!sl.used) continue;
        const amg_hierarchy *h = sl.h;
        nlev_ = std::max(nlev_, sl.nlev);
        for (int L = 0; L + 1 < sl.nlev; ++L) {
            cut_tiles(lA_[L].host, k, h->lev[L].A.n, kET / lA_[L].lpr);
            cut_tiles(lP_[L].host, k, h->lev[L].A.n, kET / lP_[L].lpr);
            cut_tiles(lR_[L].host, k, h->lev[L + 1].A.n, kET / lR_[L].lpr);
        }
        {
            SegCoarse c = hC_[(size_t)(sl.nlev - 1) * S + k];
            for (c.row0 = 0; c.row0 < c.n; c.row0 += kCoarseRows) lC_[sl.nlev - 1].host.push_back(c);
        }
        cut_tiles(l0_.host, k, sl.n0, kET / l0_.lpr);
        const int cnt = (sl.n0 + kEngChunk - 1) / kEngChunk;
        const int first = (int)lch_.host.size();
        for (int c = 0; c < cnt; ++c) {
            const int b0 = (int)sl.o0 + c * kEngChunk;
            lch_.host.push_back(SegChunk{k, b0, (int)std::min<int64_t>(sl.o0 + sl.n0, b0 + kEngChunk), first, cnt,
                                         first + c});
        }
    }
}

cudaError_t Engine::upload_lists()
{
    bool moved = false;
    for (int L = 0; L < kEngLevels; ++L) {
        AMG_CUDA_TRY(upload_list(lA_[L], allocs_, bytes_, s_, &moved));
        AMG_CUDA_TRY(upload_list(lP_[L], allocs_, bytes_, s_, &moved));
        AMG_CUDA_TRY(upload_list(lR_[L], allocs_, bytes_, s_, &moved));
        AMG_CUDA_TRY(upload_list(lC_[L], allocs_, bytes_, s_, &moved));
    }
    AMG_CUDA_TRY(upload_list(l0_, allocs_, bytes_, s_, &moved));
    const size_t old_cap = lch_.capacity;
    AMG_CUDA_TRY(upload_list(lch_, allocs_, bytes_, s_, &moved));
    if (!partial_ || lch_.capacity != old_cap) {
        // chunk partial sums follow the chunk list's capacity (indexed by chunk id)
        AMG_CUDA_TRY(alloc(&partial_, lch_.capacity));
        AMG_CUDA_TRY(alloc(&partial2_, lch_.capacity));
        moved = true;
    }
    if (moved) drop_graphs();
    return cudaStreamSynchronize(s_);   // the host vectors may change after return
}

cudaError_t Engine::compute_caps()
{
    const int S = (int)slots_.size();
    AMG_CUDA_TRY(cudaMemsetAsync(caps_dev_, 0, sizeof(int) * (3 * kEngLevels + 1), s_));
    auto span = [&](EngList<SegTile> &l, const SegOp *ops, int idx) -> cudaError_t {
        if (l.nfull == 0) return cudaSuccess;
        span_kernel<<<grid_for(l.nfull, 256, 4096), 256, 0, s_>>>(l.full, l.nfull, ops, caps_dev_ + idx); note_launch();
        return cudaGetLastError();
    };
    for (int L = 0; L < nlev_; ++L) {
        AMG_CUDA_TRY(span(lA_[L], opA_ + (size_t)L * S, 3 * L));
        AMG_CUDA_TRY(span(lP_[L], opP_ + (size_t)L * S, 3 * L + 1));
        AMG_CUDA_TRY(span(lR_[L], opR_ + (size_t)L * S, 3 * L + 2));
    }
    AMG_CUDA_TRY(span(l0_, op0_, 3 * kEngLevels));
    int h[3 * kEngLevels + 1];
    AMG_CUDA_TRY(cudaMemcpyAsync(h, caps_dev_, sizeof h, cudaMemcpyDeviceToHost, s_));
    AMG_CUDA_TRY(cudaStreamSynchronize(s_));
    bool changed = false;
    auto setcap = [&](EngList<SegTile> &l, int span_entries) {
        const int c = span_entries > 0 ? std::min(kEngMaxTile, span_entries + 8) : 0;
        if (c != l.cap) changed = true;
        l.cap = c;
    };
    for (int L = 0; L < nlev_; ++L) {
        setcap(lA_[L], h[3 * L]);
        setcap(lP_[L], h[3 * L + 1]);
        setcap(lR_[L], h[3 * L + 2]);
    }
    setcap(l0_, h[3 * kEngLevels]);
    if (changed) drop_graphs();
    return cudaSuccess;
}

// active = true: every list by the active mask; false: the fine lists by the flag mask
cudaError_t Engine::compact(bool active)
{
    const int *mask = active ? active_ : flag_;
    const int ci = active ? 0 : 1;
    auto one = [&](auto &l) -> cudaError_t {
        if (!l.count) return cudaSuccess;
        AMG_CUDA_TRY(cudaMemsetAsync(l.count + ci, 0, sizeof(int), s_));
        if (l.nfull == 0) return cudaSuccess;
        compact_kernel<<<grid_for(l.nfull, 256, 2048), 256, 0, s_>>>(l.full, l.nfull, mask, active ? l.act : l.flg,
                                                                     l.count + ci); note_launch();
        return cudaGetLastError();
    };
    if (active) {
        for (int L = 0; L < nlev_; ++L) {
            AMG_CUDA_TRY(one(lA_[L]));
            AMG_CUDA_TRY(one(lP_[L]));
            AMG_CUDA_TRY(one(lR_[L]));
            AMG_CUDA_TRY(one(lC_[L]));
        }
    }
    AMG_CUDA_TRY(one(l0_));
    AMG_CUDA_TRY(one(lch_));
    return cudaSuccess;
}

cudaError_t Engine::push_flags(const std::vector<int> &v, int *dst)
{
    const int half = dst == active_ ? 0 : 1;
    int *h = hflags_ + (half ? slots_.size() : 0);
    // the previous upload from this half must have read it before it is rewritten
    AMG_CUDA_TRY(cudaEventSynchronize(flag_ev_[half]));
    for (size_t i = 0; i < v.size(); ++i) h[i] = v[i];
    AMG_CUDA_TRY(cudaMemcpyAsync(dst, h, sizeof(int) * v.size(), cudaMemcpyHostToDevice, s_));
    return cudaEventRecord(flag_ev_[half], s_);
}

// Lanes per row of every tile list, chosen by timing each candidate on the current members
// (y = A x into the list's own scratch vectors); the winners are kept.
cudaError_t Engine::autotune()
{
    const int S = (int)slots_.size();
    cudaEvent_t e0, e1;
    AMG_CUDA_TRY(cudaEventCreate(&e0));
    AMG_CUDA_TRY(cudaEventCreate(&e1));
    cudaError_t err = cudaSuccess;
    build_lists();
    const int nl = nlev_;
    for (int li = 0; li <= 3 * nl && err == cudaSuccess; ++li) {
        const bool fine = li == 3 * nl;
        const int L = fine ? 0 : li / 3, kind = fine ? 3 : li % 3;
        if (!fine && L + 1 >= nl) continue;
        EngList<SegTile> &l = fine ? l0_ : (kind == 0 ? lA_[L] : (kind == 1 ? lP_[L] : lR_[L]));
        const SegOp *ops = fine ? op0_ : (kind == 0 ? opA_ : (kind == 1 ? opP_ : opR_)) + (size_t)L * S;
        double best = 1e300;
        int best_lpr = l.lpr;
        for (int lpr : kLprs) {
            l.lpr = lpr;
            build_lists();
            if (l.host.empty()) break;
            if ((err = upload_lists()) != cudaSuccess) break;
            if ((err = compute_caps()) != cudaSuccess) break;
            set_count_kernel<<<1, 1, 0, s_>>>(l.count + 2, l.nfull); note_launch();
            // x: the level's (or, for P, the next level's) iterate; y: a scratch vector
            const bool coarse_cols = kind == 1 || L > 0;
            const SegCtx cx = fine ? ctx(0, 0) : ctx(kind == 1 || L > 0 ? 1 : 0, kind == 2 || L > 0 ? 1 : 0);
            auto run = [&]() -> cudaError_t {
                if (fine)
                    return seg_launch<double, SK_Y>(lpr, l.full, l.count + 2, ops, x_, q_, nullptr, nullptr, 0, l.cap,
                                                    1 << 30, cx, s_);
                void *xs = (kind == 2) ? (L == 0 ? r0_ : rc_) : (coarse_cols ? xc_ : x0_);
                void *ys = (kind == 2) ? fc_ : (L == 0 ? x20_ : x2c_);
                if (cfg_.mixed)
                    return seg_launch<float, SK_Y>(lpr, l.full, l.count + 2, ops, (const float *)xs, (float *)ys,
                                                   nullptr, nullptr, 0, l.cap, 1 << 30, cx, s_);
                return seg_launch<double, SK_Y>(lpr, l.full, l.count + 2, ops, (const double *)xs, (double *)ys,
                                                nullptr, nullptr, 0, l.cap, 1 << 30, cx, s_);
            };
            if ((err = run()) != cudaSuccess) break;
            if ((err = cudaEventRecord(e0, s_)) != cudaSuccess) break;
            for (int r = 0; r < 3 && err == cudaSuccess; ++r) err = run();
            if (err != cudaSuccess || (err = cudaEventRecord(e1, s_)) != cudaSuccess) break;
            if ((err = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float ms = 0.f;
            if ((err = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
            if (ms < best) { best = ms; best_lpr = lpr; }
        }
        l.lpr = best_lpr;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return err;
}

// lanes per row from each list's mean row length (deterministic; the autotuner's fallback)
void Engine::heuristic_lanes()
{
    double rows[3][kEngLevels] = {}, nnz[3][kEngLevels] = {}, r0 = 0, z0 = 0;
    for (const Slot &sl : slots_) {
        if (!sl.used) continue;
        const amg_hierarchy *h = sl.h;
        r0 += h->lev[0].A.n;
        z0 += (double)h->lev[0].A.nnz;
        for (int L = 0; L + 1 < sl.nlev; ++L) {
            const Level &lv = h->lev[L];
            rows[0][L] += lv.A.n; nnz[0][L] += (double)lv.A.nnz;
            rows[1][L] += lv.P.n; nnz[1][L] += (double)lv.P.nnz;
            rows[2][L] += lv.R.n; nnz[2][L] += (double)lv.R.nnz;
        }
    }
    auto pick = [](double z, double r) { return pick_lanes(r > 0 ? z / r : 1.0); };
    l0_.lpr = pick(z0, r0);
    for (int L = 0; L < kEngLevels; ++L) {
        lA_[L].lpr = pick(nnz[0][L], rows[0][L]);
        lP_[L].lpr = pick(nnz[1][L], rows[1][L]);
        lR_[L].lpr = pick(nnz[2][L], rows[2][L]);
    }
}

SegCtx Engine::ctx(int xl, int yl) const
{
    const int c0 = (int)std::max<int64_t>(cfg_.cap0, 1), cc = (int)std::max<int64_t>(cfg_.capc, 1);
    return SegCtx{(int)slots_.size(), xl ? cc : c0, yl ? cc : c0, guard_};
}

std::string Engine::take_guard(int *slot)
{
    EngGuard g{};
    if (cudaMemcpyAsync(&g, guard_, sizeof g, cudaMemcpyDeviceToHost, s_) != cudaSuccess ||
        cudaStreamSynchronize(s_) != cudaSuccess)
        return "guard unreadable";
    if (g.count == 0 && g.waits == 0) return std::string();
    cudaMemsetAsync(guard_, 0, sizeof(EngGuard), s_);
    if (g.count == 0)
        return std::to_string(g.waits) + " blocks gave up waiting for a bulk copy into shared memory";
    static const char *kinds[] = {"?", "spmv tile", "chebyshev start", "coarse solve", "pcg chunk"};
    if (slot) *slot = g.slot;
    std::string info;
    if (g.kind == 1) {
        static const char *names[12] = {"row0", "rows", "n", "ncol", "nnz", "k0", "k1", "xoff", "yoff", "xcap",
                                        "ycap", "rp0"};
        for (int k = 0; k < 12; ++k) info += std::string(k ? " " : " (") + names[k] + "=" + std::to_string(g.info[k]);
        info += ")";
    }
    return std::to_string(g.count) + " work items outside their arrays; first: " +
           kinds[(g.kind >= 1 && g.kind <= 4) ? g.kind : 0] + " of slot " + std::to_string(g.slot) + " at " +
           std::to_string(g.where) + info;
}

std::string Engine::describe() const
{
    std::string s = "fine:" + std::to_string(l0_.lpr);
    for (int L = 0; L + 1 < nlev_; ++L)
        s += " L" + std::to_string(L) + ":A" + std::to_string(lA_[L].lpr) + "/P" + std::to_string(lP_[L].lpr) + "/R" +
             std::to_string(lR_[L].lpr);
    return s;
}

amg_status_t Engine::commit()
{
    const int S = (int)slots_.size();
    if (members_changed_) {
        EK(cudaMemcpyAsync(opA_, hA_.data(), sizeof(SegOp) * hA_.size(), cudaMemcpyHostToDevice, s_));
        EK(cudaMemcpyAsync(opP_, hP_.data(), sizeof(SegOp) * hP_.size(), cudaMemcpyHostToDevice, s_));
        EK(cudaMemcpyAsync(opR_, hR_.data(), sizeof(SegOp) * hR_.size(), cudaMemcpyHostToDevice, s_));
        EK(cudaMemcpyAsync(op0_, h0_.data(), sizeof(SegOp) * h0_.size(), cudaMemcpyHostToDevice, s_));
        EK(cudaMemcpyAsync(opC_, hC_.data(), sizeof(SegCoarse) * hC_.size(), cudaMemcpyHostToDevice, s_));
        EK(cudaMemcpyAsync(coef_, hcoef_.data(), sizeof(double) * hcoef_.size(), cudaMemcpyHostToDevice, s_));
        const int old_nlev = nlev_;
        build_lists();
        if (!tuned_ && !l0_.host.empty()) {
            if (cfg_.tune) EK(autotune());
            else heuristic_lanes();
            tuned_ = true;
            build_lists();
        }
        EK(upload_lists());
        EK(compute_caps());
        if (old_nlev != nlev_) drop_graphs();
        // a graph launches the dense solves only of the levels that held coarsest levels when
        // it was captured
        unsigned cm = 0;
        for (int L = 0; L < kEngLevels; ++L)
            if (lC_[L].nfull > 0) cm |= 1u << L;
        if (cm != coarse_mask_) {
            drop_graphs();
            coarse_mask_ = cm;
        }
        members_changed_ = false;
    }
    // solves to start
    std::vector<int> flags((size_t)S, 0);
    bool any = false;
    for (int k = 0; k < S; ++k) {
        Slot &sl = slots_[k];
        if (!sl.used || !sl.pending) continue;
        flags[k] = 1;
        any = true;
        if (sl.n0 > 0) EK(copy_to_device(b_ + sl.o0, sl.b, sizeof(double) * (size_t)sl.n0, s_));
        if (sl.active) {
            sl.active = 0;
            --live_;
        }
    }
    if (!any) {
        std::vector<int> act((size_t)S, 0);
        for (int k = 0; k < S; ++k) act[k] = slots_[k].active;
        EK(push_flags(act, active_));
        EK(compact(true));
        return AMG_OK;
    }
    EK(push_flags(flags, flag_));
    EK(compact(false));
    {
        const int parity_next = cfg_.mixed ? (it_ & 1) : 0;
        double *zp = cfg_.mixed ? zb_[1 - parity_next] : nullptr;
        const SegCtx cx = ctx(0, 0);
        eng_init_kernel<<<grid_chunks_, kET, 0, s_>>>(lch_.flg, lch_.count + 1, b_, x_, r_, p_, zp, sc_, cx.nslots,
                                                      cx.ycap, cx.guard); note_launch();
        eng_norm_kernel<<<grid_chunks_, kET, 0, s_>>>(lch_.flg, lch_.count + 1, b_, partial_, ticket_, sc_, 0,
                                                      cx.nslots, cx.ycap, cx.guard); note_launch();
        EK(cudaGetLastError());
    }
    std::vector<EngScal> hs((size_t)S);
    EK(cudaMemcpyAsync(hs.data(), sc_, sizeof(EngScal) * S, cudaMemcpyDeviceToHost, s_));
    EK(cudaStreamSynchronize(s_));
    {
        const std::string g = take_guard();
        if (!g.empty()) {
            set_last_error("engine guard: " + g);
            return AMG_ERR_INTERNAL;
        }
    }
    std::vector<int> act((size_t)S, 0);
    for (int k = 0; k < S; ++k) {
        Slot &sl = slots_[k];
        act[k] = sl.active;
        if (!flags[k]) continue;
        sl.pending = false;
        sl.iters = 0;
        sl.nb = sl.n0 > 0 ? std::sqrt(hs[k].bb) : 0.0;
        sl.relres = 0.0;
        sl.result = sl.nb == 0.0 ? AMG_OK : AMG_ERR_NOT_CONVERGED;
        sl.active = sl.nb > 0.0 && sl.max_iter > 0 ? 1 : 0;
        act[k] = sl.active;
        live_ += sl.active;
    }
    EK(push_flags(act, active_));
    EK(compact(true));
    return AMG_OK;
}

template <typename T>
cudaError_t Engine::vcycle(int L, const T *f, T *final_out, T **out, cudaStream_t s)
{
    const int S = (int)slots_.size();
    T *x = (T *)(L == 0 ? x0_ : xc_), *x2 = (T *)(L == 0 ? x20_ : x2c_);
    T *rv = (T *)(L == 0 ? r0_ : rc_), *d = (T *)(L == 0 ? d0_ : dc_);
    auto coarse = [&](T *dst) -> cudaError_t {
        if (lC_[L].nfull == 0) return cudaSuccess;
        const SegCtx cx = ctx(L > 0, L > 0);
        segcoarse_kernel<T><<<grid_tiles_, kET, 0, s>>>(lC_[L].act, lC_[L].count, f, dst, cx.nslots, cx.ycap,
                                                        cx.guard); note_launch();
        return cudaGetLastError();
    };
    if (L == nlev_ - 1) {
        *out = final_out ? final_out : x;
        return coarse(*out);
    }
    const SegOp *opA = opA_ + (size_t)L * S, *opP = opP_ + (size_t)L * S, *opR = opR_ + (size_t)L * S;
    EngList<SegTile> &la = lA_[L], &lp = lP_[L], &lr = lR_[L];
    const int deg = cfg_.degree;
    const SegCtx ca = ctx(L > 0, L > 0), cp = ctx(1, L > 0), cr = ctx(L > 0, 1);
    segcheb0_kernel<T><<<grid_tiles_, kET, 0, s>>>(la.act, la.count, opA, f, d, x, ca.nslots, ca.ycap, ca.guard); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    for (int k = 1; k < deg; ++k) {
        AMG_CUDA_TRY((seg_launch<T, SK_CHEB>(la.lpr, la.act, la.count, opA, x, x2, f, d, 1 + 2 * k, la.cap,
                                             1 << 30, ca, s)));
        std::swap(x, x2);
    }
    T *fc = (T *)fc_;
    AMG_CUDA_TRY((seg_launch<T, SK_RESID>(la.lpr, la.act, la.count, opA, x, rv, f, nullptr, 0, la.cap, 1 << 30, ca,
                                          s)));
    AMG_CUDA_TRY((seg_launch<T, SK_Y>(lr.lpr, lr.act, lr.count, opR, rv, fc, nullptr, nullptr, 0, lr.cap, grid_tiles_,
                                      cr, s)));
    T *xcv = nullptr;
    AMG_CUDA_TRY(vcycle<T>(L + 1, fc, nullptr, &xcv, s));
    AMG_CUDA_TRY((seg_launch<T, SK_PROLONG>(lp.lpr, lp.act, lp.count, opP, xcv, x, nullptr, nullptr, 0, lp.cap,
                                            1 << 30, cp, s)));
    for (int k = 0; k < deg; ++k) {
        T *dst = (final_out && k == deg - 1) ? final_out : x2;
        AMG_CUDA_TRY((seg_launch<T, SK_CHEB>(la.lpr, la.act, la.count, opA, x, dst, f, d, 1 + 2 * k, la.cap,
                                             1 << 30, ca, s)));
        x2 = x;
        x = dst;
    }
    *out = x;
    return coarse(x);
}

cudaError_t Engine::tail(int parity, cudaStream_t s)
{
    const SegCtx c0 = ctx(0, 0);
    double *z = zb_[cfg_.mixed ? parity : 0];
    double *zp = cfg_.mixed ? zb_[1 - parity] : nullptr;
    if (nlev_ > 0) {
        if (cfg_.mixed) {
            eng_convert_kernel<double, float><<<grid_chunks_, kET, 0, s>>>(lch_.act, lch_.count, r_, (float *)f0_,
                                                                          c0.nslots, c0.ycap, c0.guard); note_launch();
            AMG_CUDA_TRY(cudaGetLastError());
            float *out = nullptr;
            AMG_CUDA_TRY(vcycle<float>(0, (const float *)f0_, nullptr, &out, s));
            eng_convert_kernel<float, double><<<grid_chunks_, kET, 0, s>>>(lch_.act, lch_.count, out, z, c0.nslots,
                                                                          c0.ycap, c0.guard); note_launch();
            AMG_CUDA_TRY(cudaGetLastError());
        } else {
            double *out = nullptr;
            AMG_CUDA_TRY(vcycle<double>(0, r_, z, &out, s));
            if (out != z) {
                eng_copy_kernel<<<grid_chunks_, kET, 0, s>>>(lch_.act, lch_.count, out, z, c0.nslots, c0.ycap,
                                                             c0.guard); note_launch();
                AMG_CUDA_TRY(cudaGetLastError());
            }
        }
    }
    eng_rz_kernel<<<grid_chunks_, kET, 0, s>>>(lch_.act, lch_.count, r_, z, zp, partial_, partial2_, ticket_, ticket2_,
                                               sc_, c0.nslots, c0.ycap, c0.guard); note_launch();
    eng_p_kernel<<<grid_chunks_, kET, 0, s>>>(lch_.act, lch_.count, z, p_, sc_, zp ? 1 : 0, c0.nslots, c0.ycap,
                                              c0.guard); note_launch();
    return cudaGetLastError();
}

cudaError_t Engine::head(cudaStream_t s)
{
    const SegCtx c0 = ctx(0, 0);
    AMG_CUDA_TRY((seg_launch<double, SK_Y>(l0_.lpr, l0_.act, l0_.count, op0_, p_, q_, nullptr, nullptr, 0, l0_.cap,
                                           1 << 30, c0, s)));
    eng_pq_kernel<<<grid_chunks_, kET, 0, s>>>(lch_.act, lch_.count, p_, q_, partial_, ticket_, sc_, c0.nslots, c0.ycap,
                                               c0.guard); note_launch();
    eng_xr_kernel<<<grid_chunks_, kET, 0, s>>>(lch_.act, lch_.count, p_, q_, x_, r_, partial_, ticket_, sc_, rr_dev_,
                                               c0.nslots, c0.ycap, c0.guard); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    return cudaMemcpyAsync(rr_host_, rr_dev_, sizeof(double) * slots_.size(), cudaMemcpyDeviceToHost, s);
}

cudaError_t Engine::true_residual(cudaStream_t s)
{
    const SegCtx c0 = ctx(0, 0);
    AMG_CUDA_TRY((seg_launch<double, SK_RESID>(l0_.lpr, l0_.flg, l0_.count + 1, op0_, x_, t_, b_, nullptr, 0, l0_.cap,
                                               1 << 30, c0, s)));
    eng_norm_kernel<<<grid_chunks_, kET, 0, s>>>(lch_.flg, lch_.count + 1, t_, partial_, ticket_, sc_, 1, c0.nslots,
                                                 c0.ycap, c0.guard); note_launch();
    return cudaGetLastError();
}

cudaGraphExec_t Engine::graph(int parity)
{
    if (graph_failed_) return nullptr;
    if (gexec_[parity]) return gexec_[parity];
    cudaGraph_t g = nullptr;
    const long long before = launch_count();
    cudaError_t e = cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = tail(parity, cap_);
        cudaError_t e2 = e1 == cudaSuccess ? head(cap_) : e1;
        e = cudaStreamEndCapture(cap_, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec_[parity], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        graph_failed_ = true;       // iterations run eagerly from now on
        gexec_[parity] = nullptr;
        return nullptr;
    }
    gkernels_[parity] = launch_count() - before;
    note_launches(-gkernels_[parity]);
    return gexec_[parity];
}

amg_status_t Engine::step(std::vector<int> *finished)
{
    if (finished) finished->clear();
    if (live_ == 0) return AMG_OK;
    const int S = (int)slots_.size();
    const int parity = cfg_.mixed ? (it_ & 1) : 0;
    cudaGraphExec_t gx = graph(parity);
    if (gx) {
        EK(cudaGraphLaunch(gx, s_));
        note_launches(gkernels_[parity]);
    } else {
        EK(tail(parity, s_));
        EK(head(s_));
    }
    ++it_;
    for (auto &sl : slots_)
        if (sl.used && sl.active) ++sl.iters;
    EK(cudaStreamSynchronize(s_));
    {
        int gslot = -1;
        const std::string g = take_guard(&gslot);
        if (!g.empty()) {
            // is the slot's hierarchy itself still intact?
            std::string what = "; hierarchy of the slot ";
            if (gslot >= 0 && gslot < S && slots_[gslot].used) {
                std::string detail;
                const int f = hierarchy_check(slots_[gslot].h, s_, &detail);
                what += f == 0 ? "intact" : (f < 0 ? "not checkable" : "damaged: " + detail);
            } else {
                what += "not in use";
            }
            set_last_error("engine guard: " + g + what);
            return AMG_ERR_INTERNAL;
        }
    }
    std::vector<int> flags((size_t)S, 0), act((size_t)S, 0);
    std::vector<int> stopped;
    bool any = false;
    for (int k = 0; k < S; ++k) {
        const Slot &sl = slots_[k];
        act[k] = sl.active;
        if (sl.active && std::sqrt(rr_host_[k]) / sl.nb <= sl.tol) { flags[k] = 1; any = true; }
    }
    std::vector<EngScal> hs((size_t)S);
    if (any) {
        // the recurrence says converged: check b - A x of those slots
        EK(push_flags(flags, flag_));
        EK(compact(false));
        EK(true_residual(s_));
        EK(cudaMemcpyAsync(hs.data(), sc_, sizeof(EngScal) * S, cudaMemcpyDeviceToHost, s_));
        EK(cudaStreamSynchronize(s_));
        bool replace = false;
        for (int k = 0; k < S; ++k) {
            if (!flags[k]) continue;
            Slot &sl = slots_[k];
            const double rel = std::sqrt(hs[k].tt) / sl.nb;
            if (rel <= sl.tol) {
                sl.active = 0;
                act[k] = 0;
                sl.result = AMG_OK;
                sl.relres = rel;
                flags[k] = 0;
                stopped.push_back(k);
            } else {
                replace = true;     // flags[k] stays set: r = b - A x for this slot
            }
        }
        if (replace) {
            EK(push_flags(flags, flag_));
            EK(compact(false));
            const SegCtx c0 = ctx(0, 0);
            eng_copy_kernel<<<grid_chunks_, kET, 0, s_>>>(lch_.flg, lch_.count + 1, t_, r_, c0.nslots, c0.ycap,
                                                          c0.guard); note_launch();
            EK(cudaGetLastError());
        }
    }
    // iteration limits: stop, with the true residual of the last iterate
    std::fill(flags.begin(), flags.end(), 0);
    bool limit = false;
    for (int k = 0; k < S; ++k) {
        Slot &sl = slots_[k];
        if (sl.active && sl.iters >= sl.max_iter) {
            sl.active = 0;
            act[k] = 0;
            sl.result = AMG_ERR_NOT_CONVERGED;
            flags[k] = 1;
            limit = true;
            stopped.push_back(k);
        }
    }
    if (limit) {
        EK(push_flags(flags, flag_));
        EK(compact(false));
        EK(true_residual(s_));
        EK(cudaMemcpyAsync(hs.data(), sc_, sizeof(EngScal) * S, cudaMemcpyDeviceToHost, s_));
        EK(cudaStreamSynchronize(s_));
        for (int k = 0; k < S; ++k)
            if (flags[k]) slots_[k].relres = std::sqrt(hs[k].tt) / slots_[k].nb;
    }
    if (!stopped.empty()) {
        live_ -= (int)stopped.size();
        EK(push_flags(act, active_));
        EK(compact(true));
        if (finished) *finished = stopped;
    }
    return AMG_OK;
}

amg_status_t Engine::download(int k, double *x)
{
    const Slot &sl = slots_[k];
    if (sl.n0 == 0) return AMG_OK;
    EK(copy_to_host(x, x_ + sl.o0, sizeof(double) * (size_t)sl.n0, s_));
    return AMG_OK;
}

#undef EK

}  // namespace amgk

// ====================================================================================== batch ABI

struct amg_batch {
    amgk::Engine eng;
    std::vector<int> slot;              // caller's index -> engine slot
    std::vector<amg_hierarchy *> h;
};

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
            pk.coarse_solve = AMG_COARSE_INVERSE;      // the engine applies the dense inverse
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

amg_status_t amg_batch_create(int count, const amg_handle_t *h, void *cuda_stream, int tune, amg_batch_t *out)
{
    if (!out) return AMG_ERR_INVALID_ARG;
    *out = nullptr;
    if (count < 0 || (count > 0 && !h)) return AMG_ERR_INVALID_ARG;
    for (int k = 0; k < count; ++k) {
        if (!h[k]) return AMG_ERR_INVALID_ARG;
        if (h[k]->p.precision != h[0]->p.precision || h[k]->p.cheb_degree != h[0]->p.cheb_degree) {
            set_last_error("all systems of a batch need the same precision and Chebyshev degree");
            return AMG_ERR_INVALID_ARG;
        }
        if (h[k]->p.krylov != AMG_KRYLOV_CG) {
            set_last_error("the batch engine runs PCG only");
            return AMG_ERR_UNSUPPORTED;
        }
        if (h[k]->nlev > kEngLevels) {
            set_last_error("a hierarchy deeper than the batch engine's level limit");
            return AMG_ERR_UNSUPPORTED;
        }
        // the engine applies the coarsest level's dense inverse
        const amg_status_t ci = ensure_coarse_inverse(h[k]);
        if (ci != AMG_OK) return ci;
    }
    Engine::Config cfg;
    cfg.mixed = count > 0 && h[0]->p.precision == AMG_MIXED;
    cfg.degree = count > 0 ? h[0]->p.cheb_degree : 2;
    cfg.slots = count;
    cfg.tune = tune != 0;
    for (int k = 0; k < count; ++k) {
        cfg.cap0 += h[k]->lev[0].A.n;
        for (int L = 1; L < h[k]->nlev; ++L) cfg.capc += h[k]->lev[L].A.n;
    }
    if (cfg.cap0 > 0x7ffffff0LL || cfg.capc > 0x7ffffff0LL) {
        set_last_error("batch too large for 32-bit vector offsets");
        return AMG_ERR_UNSUPPORTED;
    }
    amg_batch *Bt = new amg_batch();
    amg_status_t st = Bt->eng.init(cfg, (cudaStream_t)cuda_stream);
    for (int k = 0; k < count && st == AMG_OK; ++k) {
        const int s = Bt->eng.add(h[k]);
        if (s < 0) {
            set_last_error("batch engine has no room for a system");
            st = AMG_ERR_INTERNAL;
        }
        Bt->slot.push_back(s);
        Bt->h.push_back(h[k]);
    }
    if (st != AMG_OK) {
        delete Bt;
        return st;
    }
    *out = Bt;
    return AMG_OK;
}

amg_status_t amg_batch_free(amg_batch_t Bt)
{
    delete Bt;
    return AMG_OK;
}

amg_status_t amg_batch_solve(amg_batch_t Bt, const double *const *b, double *const *x, double tol, amg_info_t *infos)
{
    if (!Bt) return AMG_ERR_INVALID_ARG;
    const int C = (int)Bt->slot.size();
    if (C > 0 && (!b || !x)) return AMG_ERR_INVALID_ARG;
    if (!(tol >= 0.0)) return AMG_ERR_INVALID_ARG;
    for (int k = 0; k < C; ++k)
        if (Bt->eng.slot(Bt->slot[k]).n0 > 0 && (!b[k] || !x[k])) return AMG_ERR_INVALID_ARG;
    const double t0 = now_ms();
    Engine &E = Bt->eng;
    for (int k = 0; k < C; ++k) E.load(Bt->slot[k], b[k], tol, Bt->h[k]->p.max_iter);
    amg_status_t st = E.commit();
    while (st == AMG_OK && E.live() > 0) st = E.step(nullptr);
    for (int k = 0; k < C && st == AMG_OK; ++k) st = E.download(Bt->slot[k], x[k]);
    amg_status_t overall = st;
    if (st == AMG_OK) {
        for (int k = 0; k < C; ++k)
            if (E.slot(Bt->slot[k]).result != AMG_OK) overall = AMG_ERR_NOT_CONVERGED;
        if (spmv_take_errors(nullptr) != 0) {
            set_last_error("a bulk copy into shared memory did not complete in time");
            overall = AMG_ERR_INTERNAL;
        }
    }
    if (infos) {
        const double ms = now_ms() - t0;
        for (int k = 0; k < C; ++k) {
            const Engine::Slot &sl = E.slot(Bt->slot[k]);
            const amg_hierarchy *h = Bt->h[k];
            amg_info_t &in = infos[k];
            in.iters = sl.iters;
            in.status = (st == AMG_OK && overall != AMG_ERR_INTERNAL) ? sl.result : overall;
            in.relres_true = sl.relres;
            in.setup_ms = h->setup_ms;
            in.solve_ms = ms;
            in.levels = h->nlev;
            double tot = 0.0;
            for (int L = 0; L < h->nlev; ++L) tot += (double)h->lev[L].A.nnz;
            in.op_complexity = h->fine_nnz > 0 ? tot / (double)h->fine_nnz : 0.0;
        }
    }
    return overall;
}

amg_status_t amg_solve_batch(int count, const amg_handle_t *h, const double *const *b, double *const *x, double tol,
                             amg_info_t *infos)
{
    if (count < 0 || (count > 0 && !h)) return AMG_ERR_INVALID_ARG;
    for (int k = 0; k < count; ++k)
        if (!h[k]) return AMG_ERR_INVALID_ARG;
    amg_batch_t Bt = nullptr;
    amg_status_t st = amg_batch_create(count, h, count > 0 ? h[0]->p.cuda_stream : nullptr, 0, &Bt);
    if (st != AMG_OK) return st;
    st = amg_batch_solve(Bt, b, x, tol, infos);
    amg_batch_free(Bt);
    return st;
}

amg_status_t amg_batch_info(amg_batch_t Bt, int *count, int *levels, int64_t *rows, int64_t *graph_kernels)
{
    if (!Bt) return AMG_ERR_INVALID_ARG;
    int64_t tot = 0;
    for (int k = 0; k < (int)Bt->slot.size(); ++k) tot += Bt->eng.slot(Bt->slot[k]).n0;
    if (count) *count = (int)Bt->slot.size();
    if (levels) *levels = Bt->eng.levels();
    if (rows) *rows = tot;
    if (graph_kernels) *graph_kernels = Bt->eng.kernels_per_iteration();
    return AMG_OK;
}

}  // extern "C"
