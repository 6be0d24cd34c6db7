// solve.cu -- solve-phase kernels: CSR SpMV with fused epilogues (residual, Chebyshev step,
// prolongation, dot products), the V-cycle of Algorithm 1 with degree-k Chebyshev smoothing,
// the coarsest-level dense solve and the PCG vector updates.
//
// SpMV layout (one design for every level and both precisions): a block of 256 threads owns
// 256/LPR consecutive rows, LPR lanes per row (LPR from the mean row length: 2 for the
// 27-point fine operators, wider for the denser coarse operators).  One thread of the block
// copies the block's contiguous range of values and column indices into shared memory with
// two bulk asynchronous copies (cp.async.bulk + mbarrier), widened to 16-byte boundaries;
// the lanes then walk their row from shared memory and gather x from global memory (L2).
// Blocks whose range exceeds the shared tile read their rows directly from global memory.
// Few lanes per row keep the cross-lane FP64 additions (issued on GB300's narrow FP64 pipe)
// to log2(LPR) per row.  The working type T is double (FP64 path) or float (the mixed
// path's V-cycle); accumulation is in T.  Partial dot products are per block, in a fixed
// order, so every reduction is bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <mutex>

#include <vector>

#include "amg_internal.cuh"
#include "tma.cuh"

namespace amgk {

constexpr unsigned kAll = 0xffffffffu;
constexpr int kSpmvThreads = 256;
constexpr int kMaxTile = 6144;            // entries staged per block at most

enum SpmvMode {
    MODE_Y = 0,          // y = A x
    MODE_RESID = 1,      // y = f - A x
    MODE_CHEB = 2,       // r = f - A x; d = c1 d + c2 D^-1 r; y = x + d
    MODE_PROLONG = 3,    // y += A x
    MODE_DOT = 4,        // y = A x; partial[block] = sum of x_i y_i
    MODE_SCALEDOT = 5,   // y = (A x) / D; partial[block] = sum of x_i y_i
    MODE_POWER = 6,      // power-method sweep on an unnormalised x with f[0] = x . x, f[1] = 1 / sqrt(x . x),
                         // aux = D^-1: y = (D^-1 A x) f[1]; result[0] = (x . y) f[1]; d[0] = y . y and
                         // d[1] = 1 / sqrt(y . y) (the next sweep's f)
};


// partial[i] over i = threadIdx.x, + blockDim.x, ... < n, added in that order from 0; the loads
// of four steps are issued before their additions (thousands of partials: the last block's
// tail).  L2 loads: the other blocks' partials are visible there after their fences and the
// ticket.
__device__ __forceinline__ double ordered_strided_sum(const double *p, int n)
{
    const int bd = (int)blockDim.x;
    double acc = 0.0;
    int i = (int)threadIdx.x;
    for (; i + 3 * bd < n; i += 4 * bd) {
        const double v0 = __ldcg(p + i), v1 = __ldcg(p + i + bd), v2 = __ldcg(p + i + 2 * bd),
                     v3 = __ldcg(p + i + 3 * bd);
        acc += v0;
        acc += v1;
        acc += v2;
        acc += v3;
    }
    for (; i < n; i += bd) acc += __ldcg(p + i);
    return acc;
}

// Fixed-order completion of a two-stage sum: the block that arrives last (atomic ticket)
// adds every block's partial in index order -- the same order whichever block is last -- and
// stores the total; it then returns the ticket counter to zero for the next launch.
__device__ __forceinline__ void last_block_total(const double *partial, int nblocks, unsigned *counter,
                                                 double *result)
{
    __shared__ bool last;
    __shared__ double wsum[32];
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)nblocks - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double acc = ordered_strided_sum(partial, nblocks);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kAll, acc, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
        *result = t;
        *counter = 0u;
    }
}

// Two fixed-order sums at once (partial[0, nblocks) and partial[nblocks, 2 nblocks)); the last
// block to arrive (of narrive; nblocks when not given) stores *r1 = scale * (first total) and
// *r2 = second total.
__device__ __forceinline__ void last_block_total2(const double *partial, int nblocks, unsigned *counter, double *r1,
                                                  double *r2, double scale, int narrive = -1, bool r2_rsqrt = false)
{
    __shared__ bool last;
    __shared__ double w1[32], w2[32];
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)(narrive < 0 ? nblocks : narrive) - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = ordered_strided_sum(partial, nblocks), b = ordered_strided_sum(partial + nblocks, nblocks);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(kAll, a, o);
        b += __shfl_down_sync(kAll, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        w1[threadIdx.x >> 5] = a;
        w2[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t1 += w1[w];
            t2 += w2[w];
        }
        *r1 = scale * t1;
        *r2 = t2;
        if (r2_rsqrt) r2[1] = 1.0 / __dsqrt_rn(t2);    // the next sweep's 1 / ||y||
        *counter = 0u;
    }
}

// The update of one row whose sum sr was formed outside the row tiles (long and split rows).
// DOT and SCALEDOT store the row's y only (the tile kernel adds its share of the dot products
// in its block's fixed order); POWER reads q = x . x from f[0].
template <typename T, int MODE>
__device__ __forceinline__ void outside_row_update(int row, T sr, const T *x, T *y, const T *f, const T *aux, T *d,
                                                   T c1, T c2)
{
    if (MODE == MODE_Y || MODE == MODE_DOT) {
        y[row] = sr;
    } else if (MODE == MODE_RESID) {
        y[row] = f[row] - sr;
    } else if (MODE == MODE_CHEB) {
        T r = f[row] - sr;
        T dn = c1 * d[row] + c2 * (aux[row] * r);
        d[row] = dn;
        y[row] = x[row] + dn;
    } else if (MODE == MODE_PROLONG) {
        y[row] += sr;
    } else if (MODE == MODE_SCALEDOT) {
        y[row] = sr / aux[row];
    } else {
        const double rq = (double)f[1];
        y[row] = (T)(((double)sr * (double)aux[row]) * rq);
    }
}

// sum of v[k] x[ci[k]] over k = k, k + stride, ... < e in four independent partial sums: four
// gathers of x in flight per thread (the rows summed outside the row tiles are few and long, and
// their time is the latency of these loads, not the arithmetic)
template <typename T>
__device__ __forceinline__ T strided_sum4(int k, int e, int stride, const int *__restrict__ ci,
                                          const T *__restrict__ v, const T *x)
{
    T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
    for (; (int64_t)k + 3 * stride < (int64_t)e; k += 4 * stride) {
        const int c0 = ci[k], c1 = ci[k + stride], c2 = ci[k + 2 * stride], c3 = ci[k + 3 * stride];
        const T a0 = v[k], a1 = v[k + stride], a2 = v[k + 2 * stride], a3 = v[k + 3 * stride];
        s0 += a0 * x[c0];
        s1 += a1 * x[c1];
        s2 += a2 * x[c2];
        s3 += a3 * x[c3];
    }
    for (; k < e; k += stride) s0 += v[k] * x[ci[k]];
    return (s0 + s1) + (s2 + s3);
}

// A row's sum by every thread of the block (four strided partial sums per thread, a shuffle
// tree per warp, the warps in order); thread 0 applies the update
template <typename T, int MODE>
__device__ __forceinline__ void block_row(int row, const int *__restrict__ rp, const int *__restrict__ ci,
                                          const T *__restrict__ v, const T *x, T *y, const T *f, const T *aux,
                                          T *d, T c1, T c2)
{
    __shared__ T ws[kSpmvThreads / 32];
    const int b = rp[row], e = rp[row + 1];
    T sum = strided_sum4<T>(b + (int)threadIdx.x, e, kSpmvThreads, ci, v, x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kAll, sum, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x != 0) return;
    T sr = T(0);
    for (int w = 0; w < kSpmvThreads / 32; ++w) sr += ws[w];
    outside_row_update<T, MODE>(row, sr, x, y, f, aux, d, c1, c2);
}

// Block b of a plan's split rows (SplitRows): the segment blocks first (a segment's sum by the
// whole block; the row's last segment block to finish, by an arrival ticket, adds the row's
// segment sums in segment order and applies the update, then resets the ticket), then a block
// per row of the block rows, then the warp rows eight to a block.
constexpr int kSplitRowsPerBlock = kSpmvThreads / 32;
__host__ __device__ __forceinline__ int split_blocks(const SplitRows &sr)
{
    return sr.nsegb + sr.nblock + (sr.nwarp + kSplitRowsPerBlock - 1) / kSplitRowsPerBlock;
}
template <typename T, int MODE>
__device__ __forceinline__ void split_rows_block(int b, const SplitRows &sr, const int *__restrict__ rp,
                                                 const int *__restrict__ ci, const T *__restrict__ v, const T *x,
                                                 T *y, const T *f, const T *aux, T *d, T c1, T c2)
{
    if (b < sr.nsegb) {
        __shared__ T ws[kSpmvThreads / 32];
        const int *g = sr.seg + 5 * b;
        const int row = g[0], k0 = g[1], k1 = g[2], first = g[3], nseg = g[4];
        T sum = strided_sum4<T>(k0 + (int)threadIdx.x, k1, kSpmvThreads, ci, v, x);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kAll, sum, o);
        if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = sum;
        __syncthreads();
        if (threadIdx.x != 0) return;
        T t = T(0);
        for (int w = 0; w < kSpmvThreads / 32; ++w) t += ws[w];
        sr.part[b] = (double)t;
        __threadfence();
        if (atomicAdd(&sr.tick[first], 1u) != (unsigned)nseg - 1u) return;
        __threadfence();
        double acc = 0.0;
        for (int q = 0; q < nseg; ++q) acc += ((volatile const double *)sr.part)[first + q];
        sr.tick[first] = 0u;
        outside_row_update<T, MODE>(row, (T)acc, x, y, f, aux, d, c1, c2);
        return;
    }
    b -= sr.nsegb;
    if (b < sr.nblock) {
        block_row<T, MODE>(sr.rows[sr.nseg_rows + b], rp, ci, v, x, y, f, aux, d, c1, c2);
        return;
    }
    b -= sr.nblock;
    const int m = b * kSplitRowsPerBlock + (int)(threadIdx.x >> 5);
    if (m >= sr.nwarp) return;
    const int row = sr.rows[sr.nseg_rows + sr.nblock + m];
    const int lane = threadIdx.x & 31;
    T sum = strided_sum4<T>(rp[row] + lane, rp[row + 1], 32, ci, v, x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kAll, sum, o);
    if (lane == 0) outside_row_update<T, MODE>(row, sum, x, y, f, aux, d, c1, c2);
}

// the split rows of a product with dot products, summed before its tile kernel
template <typename T, int MODE>
__global__ void __launch_bounds__(kSpmvThreads) spmv_split_kernel(SplitRows sr, const int *__restrict__ rp,
                                                                  const int *__restrict__ ci,
                                                                  const T *__restrict__ v, const T *__restrict__ x,
                                                                  T *y, const T *__restrict__ f,
                                                                  const T *__restrict__ aux, T *d, T c1, T c2)
{
    split_rows_block<T, MODE>(blockIdx.x, sr, rp, ci, v, x, y, f, aux, d, c1, c2);
}

// Short rows (a prolongator's: a few entries each) by one thread per row, without staging: the
// rows of a warp are contiguous in memory, so their loads are as coalesced as the tile's.  The
// arithmetic of the two-lanes-per-row tile kernel (even and odd entries summed apart, then
// added), so both give the same bits.  Update modes only.
template <typename T, int MODE>
__global__ void __launch_bounds__(kSpmvThreads) spmv_rows_kernel(int n, const int *__restrict__ rp,
                                                                 const int *__restrict__ ci,
                                                                 const T *__restrict__ v, const T *__restrict__ x,
                                                                 T *y, const T *__restrict__ f,
                                                                 const T *__restrict__ aux, T *d, T c1, T c2)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const int b = rp[row], e = rp[row + 1];
    T s0 = T(0), s1 = T(0);
    int k = b;
    for (; k + 1 < e; k += 2) {
        s0 += v[k] * x[ci[k]];
        s1 += v[k + 1] * x[ci[k + 1]];
    }
    if (k < e) s0 += v[k] * x[ci[k]];
    const T sr = s0 + s1;
    if (MODE == MODE_Y) {
        y[row] = sr;
    } else if (MODE == MODE_RESID) {
        y[row] = f[row] - sr;
    } else if (MODE == MODE_CHEB) {
        T r = f[row] - sr;
        T dn = c1 * d[row] + c2 * (aux[row] * r);
        d[row] = dn;
        y[row] = x[row] + dn;
    } else {
        y[row] += sr;
    }
}

// the longest row of each of count matrices into out[k]
__global__ void max_row_kernel(int n, const int *rp, int *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicMax(out, rp[i + 1] - rp[i]);
}

template <typename T, int LPR, int MODE>
__global__ void __launch_bounds__(kSpmvThreads) spmv_tile_kernel(int n, const int *__restrict__ rp,
                                                                 const int *__restrict__ ci,
                                                                 const T *__restrict__ v, const T *__restrict__ x,
                                                                 T *y, const T *__restrict__ f,
                                                                 const T *__restrict__ aux, T *d, T c1, T c2,
                                                                 int cap, double *partial, double *result,
                                                                 unsigned *counter, int *err, int long_len,
                                                                 SplitRows sr)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    constexpr int RPB = kSpmvThreads / LPR;
    constexpr int VA = 16 / (int)sizeof(T);
    // the first blocks of an update-only product sum the plan's split rows (none given to the
    // products with dot products, whose split rows a separate launch sums first)
    int bx = blockIdx.x, nbx = gridDim.x;
    {
        const int extra = split_blocks(sr);
        if (bx < extra) {
            split_rows_block<T, MODE>(bx, sr, rp, ci, v, x, y, f, aux, d, c1, c2);
            return;
        }
        bx -= extra;
        nbx -= extra;
    }
    const int r0 = bx * RPB;
    const int r1 = min(n, r0 + RPB);
    const int k0 = rp[r0], k1 = rp[r1];
    const int k0v = k0 & ~(VA - 1), k1v = (k1 + VA - 1) & ~(VA - 1);
    const int k0i = k0 & ~3, k1i = (k1 + 3) & ~3;
    const bool staged = cap > 0 && (k1v - k0v) <= cap + 2 * VA && (k1i - k0i) <= cap + 8 && k1 > k0;
    T *sv = (T *)smem;
    int *sc = (int *)(smem + tile_values_bytes<T>(cap));
    bool tile_ok = true;   // a bulk copy that did not arrive in time: no row is written
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
    T sum = T(0);
    // rows longer than long_len are summed elsewhere: by spmv_long_kernel or spmv_split_kernel,
    // launched before this kernel, or by this kernel's first blocks (split rows, above)
    const bool is_long = row < r1 && rp[row + 1] - rp[row] > long_len;
    if (row < r1 && tile_ok && !is_long) {
        const int b = rp[row], e = rp[row + 1];
        // (unrolled: the gathers of x of four iterations are issued before their additions,
        // which stay in order)
        if (staged) {
#pragma unroll 4
            for (int k = b + lane; k < e; k += LPR) sum += sv[k - k0v] * x[sc[k - k0i]];
        } else {
#pragma unroll 4
            for (int k = b + lane; k < e; k += LPR) sum += v[k] * x[ci[k]];
        }
    }
    if (MODE == MODE_Y || MODE == MODE_RESID || MODE == MODE_CHEB || MODE == MODE_PROLONG) {
        // The row's sum and its update are formed by thread r < RPB for row r of the block, every
        // lane of those warps busy, instead of by the first of each row's LPR lanes: a warp's FP64
        // instruction takes the FP64 pipe whether one lane in LPR or all lanes are active, and the
        // update is up to five of them per row.  Same sums: with two lanes, partial 0 + partial 1
        // as the shuffle gives; with more, the shuffle tree first.
        __shared__ T ps[kSpmvThreads];
        if (LPR == 2) {
            ps[lane * RPB + threadIdx.x / LPR] = sum;
        } else {
#pragma unroll
            for (int o = LPR / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(kAll, sum, o, LPR);
            if (lane == 0) ps[threadIdx.x / LPR] = sum;
        }
        __syncthreads();
        const int rw = r0 + (int)threadIdx.x;
        if ((int)threadIdx.x < RPB && rw < r1 && tile_ok && rp[rw + 1] - rp[rw] <= long_len) {
            const T sr = LPR == 2 ? ps[threadIdx.x] + ps[RPB + threadIdx.x] : ps[threadIdx.x];
            if (MODE == MODE_Y) {
                y[rw] = sr;
            } else if (MODE == MODE_RESID) {
                y[rw] = f[rw] - sr;
            } else if (MODE == MODE_CHEB) {
                T r = f[rw] - sr;
                T dn = c1 * d[rw] + c2 * (aux[rw] * r);
                d[rw] = dn;
                y[rw] = x[rw] + dn;
            } else {
                y[rw] += sr;
            }
        }
        return;
    }
    if (MODE == MODE_DOT) {
        // As for the update modes: row r's y and x_r y_r by thread r < RPB, then the dot
        // product's trees over those warps only (a row a lane; the other warps would hold zeros)
        __shared__ T pd[kSpmvThreads];
        if (LPR == 2) {
            pd[lane * RPB + threadIdx.x / LPR] = sum;
        } else {
#pragma unroll
            for (int o = LPR / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(kAll, sum, o, LPR);
            if (lane == 0) pd[threadIdx.x / LPR] = sum;
        }
        __syncthreads();
        constexpr int kActive = (RPB + 31) / 32;
        __shared__ double sd[kActive];
        const int rw = r0 + (int)threadIdx.x;
        double c = 0.0;
        if ((int)threadIdx.x < RPB && rw < r1 && tile_ok) {
            if (rp[rw + 1] - rp[rw] > long_len) {
                c = (double)x[rw] * (double)y[rw];     // summed outside the tiles, in y already
            } else {
                const T sr = LPR == 2 ? pd[threadIdx.x] + pd[RPB + threadIdx.x] : pd[threadIdx.x];
                y[rw] = sr;
                c = (double)x[rw] * (double)sr;
            }
        }
        const int wp = (int)threadIdx.x >> 5;
        if (wp < kActive) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(kAll, c, o);
            if ((threadIdx.x & 31) == 0) sd[wp] = c;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kActive; ++w) t += sd[w];
            partial[bx] = t;
        }
        if (result) last_block_total(partial, nbx, counter, result);
        return;
    }
    if (MODE == MODE_POWER) {
        // As for the update modes: row r's update by thread r < RPB (full warps; y_i takes three
        // FP64 products), D^-1 from aux, 1 / sqrt(x . x) formed once per block (a square root
        // and a division are long FP64 sequences); then the block's two dot-product partials.
        __shared__ double pps[kSpmvThreads];
        __shared__ double rq_s;
        if (LPR == 2) {
            pps[lane * RPB + threadIdx.x / LPR] = (double)sum;
        } else {
#pragma unroll
            for (int o = LPR / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(kAll, sum, o, LPR);
            if (lane == 0) pps[threadIdx.x / LPR] = (double)sum;
        }
        if (threadIdx.x == 0) rq_s = (double)f[1];
        __syncthreads();
        const double rq = rq_s;
        double c1v = 0.0, c2v = 0.0;
        const int rw = r0 + (int)threadIdx.x;
        if ((int)threadIdx.x < RPB && rw < r1 && tile_ok) {
            double yi;
            if (rp[rw + 1] - rp[rw] > long_len) {
                yi = (double)y[rw];                 // summed outside the tiles, in y already
            } else {
                const double sr = LPR == 2 ? pps[threadIdx.x] + pps[RPB + threadIdx.x] : pps[threadIdx.x];
                yi = (sr * (double)aux[rw]) * rq;
                y[rw] = (T)yi;
            }
            if (c1 != T(0)) c1v = (double)x[rw] * yi;
            c2v = yi * yi;
        }
        // Only the first kActive warps hold rows' updates (the rest hold zeros, whose sums would
        // add exact zeros to sums that start from +0 and so never become -0): their trees alone,
        // each FP64 step a full pipe slot on GB300 whatever the lanes hold
        constexpr int kActive = (RPB + 31) / 32;
        __shared__ double sp1[kActive], sp2[kActive];
        const int wp = (int)threadIdx.x >> 5;
        if (wp < kActive) {
            // x . y only when asked (c1 != 0: the last sweep's, the estimate); y . y every sweep
            if (c1 != T(0)) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) c1v += __shfl_down_sync(kAll, c1v, o);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c2v += __shfl_down_sync(kAll, c2v, o);
            if ((threadIdx.x & 31) == 0) {
                sp1[wp] = c1 != T(0) ? c1v : 0.0;
                sp2[wp] = c2v;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t1 = 0.0, t2 = 0.0;
            for (int w = 0; w < kActive; ++w) {
                if (c1 != T(0)) t1 += sp1[w];
                t2 += sp2[w];
            }
            partial[bx] = t1;
            partial[nbx + bx] = t2;
        }
        last_block_total2(partial, nbx, counter, result, (double *)d, rq, -1, true);
        return;
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(kAll, sum, o, LPR);
    double contrib = 0.0;
    if (row < r1 && lane == 0 && tile_ok && is_long) {
        // the long row's value is in y already: only its share of the dot product here
        contrib = (double)x[row] * (double)y[row];
    } else if (row < r1 && lane == 0 && tile_ok) {
        if (MODE == MODE_Y) {
            y[row] = sum;
        } else if (MODE == MODE_RESID) {
            y[row] = f[row] - sum;
        } else if (MODE == MODE_CHEB) {
            T r = f[row] - sum;
            T dn = c1 * d[row] + c2 * (aux[row] * r);
            d[row] = dn;
            y[row] = x[row] + dn;
        } else if (MODE == MODE_PROLONG) {
            y[row] += sum;
        } else if (MODE == MODE_SCALEDOT) {
            T yi = sum / aux[row];
            y[row] = yi;
            contrib = (double)x[row] * (double)yi;
        }
    }
    if (MODE == MODE_SCALEDOT) {
        __shared__ double sh[kSpmvThreads / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) contrib += __shfl_down_sync(kAll, contrib, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = contrib;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kSpmvThreads / 32; ++w) t += sh[w];
            partial[bx] = t;
        }
        if (result) last_block_total(partial, nbx, counter, result);
    }
}

// One block per long row (the plan's list, by value): the row's sum by every thread of the
// block in a fixed order (strided partial sums, a shuffle tree per warp, the warps in order),
// then the same update as spmv_tile_kernel's for that row.  DOT, SCALEDOT and POWER store the
// row's y only; spmv_tile_kernel, launched after this kernel, adds the row's share of the dot
// products in its block's fixed order.
template <typename T, int MODE>
__global__ void __launch_bounds__(kSpmvThreads) spmv_long_kernel(LongRows lr, const int *__restrict__ rp,
                                                                 const int *__restrict__ ci,
                                                                 const T *__restrict__ v, const T *__restrict__ x,
                                                                 T *y, const T *__restrict__ f,
                                                                 const T *__restrict__ aux, T *d, T c1, T c2)
{
    if ((int)blockIdx.x >= lr.count) return;
    block_row<T, MODE>(lr.rows[blockIdx.x], rp, ci, v, x, y, f, aux, d, c1, c2);
}

// rows longer than len: count (cnt[0]) and the first kMaxLongRows of them (order of arrival;
// sorted on the host)
__global__ void long_rows_kernel(int n, const int *rp, int len, int *cnt, int *rows)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || rp[i + 1] - rp[i] <= len) return;
    const int k = atomicAdd(cnt, 1);
    if (k < kMaxLongRows) rows[k] = i;
}

// per threshold t = 0..7: rows longer than base << t
__global__ void long_hist_kernel(int n, const int *rp, int base, int *hist)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int len = rp[i + 1] - rp[i];
    for (int t = 0; t < 8; ++t)
        if (len > (base << t)) atomicAdd(&hist[t], 1);
}

// Lanes per row of a product from its mean row length.  Rows of 40-80 entries take 8 lanes, not
// 4: on the first coarse level of the 128^3 random-coefficient cube (58.6 a row) the shorter
// chains of dependent gathers beat the extra shuffle level (solve 23.5 → 22.9 ms).
int pick_lpr(double avg_row)
{
    if (avg_row <= 40.0) return 2;
    if (avg_row <= 160.0) return 8;
    if (avg_row <= 320.0) return 16;
    return 32;
}

// the batch engine's lanes per row (its segment tiles keep four lanes for rows of 40-80)
int pick_lanes(double avg_row)
{
    if (avg_row <= 40.0) return 2;
    if (avg_row <= 80.0) return 4;
    return pick_lpr(avg_row);
}

int spmv_blocks(int n, int lpr) { return n > 0 ? (n + kSpmvThreads / lpr - 1) / (kSpmvThreads / lpr) : 0; }

// Lanes per row of a level operator's products: the row-length rule, then doubled while the grid
// would hold fewer than two blocks per SM and every lane still keeps four entries or more (a
// small level with long rows otherwise runs on a fraction of the SMs, latency-bound).
int pick_lpr_rows(double avg_row, int n)
{
    int lpr = pick_lpr(avg_row);
    while (lpr < 32 && spmv_blocks(n, lpr) < kReduceBlocks && avg_row >= 8.0 * lpr) lpr *= 2;
    return lpr;
}

// the largest block range of a plan, over the blocks without a long row (a block holding one is
// not staged: its range exceeds the tile, and its short rows read global memory)
// (a warp per block range, its lanes over the range's rows)
__global__ void span_max_kernel(int n, const int *rp, int rpb, int long_len, int *out)
{
    const int lane = threadIdx.x & 31;
    const int b = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int r0 = b * rpb;
    if (r0 >= n) return;             // the whole warp: r0 is the same for its lanes
    const int r1 = min(n, r0 + rpb);
    bool has_long = false;
    for (int r = r0 + lane; r < r1; r += 32) has_long |= rp[r + 1] - rp[r] > long_len;
    if (__any_sync(kAll, has_long)) return;
    if (lane == 0) atomicMax(out, rp[r1] - rp[r0]);
}

// The long rows of a plan: more than max(512, 8 x the mean row) entries, the threshold doubled
// (up to 7 times) until at most kMaxLongRows rows exceed it.  One synchronisation per call.
// lr.len stays "none" when no row qualifies.
cudaError_t long_rows_plan(int count, SpmvPlan *const *plans, const int *const *rps, const int *ns,
                           const int64_t *nnzs, cudaStream_t s)
{
    std::vector<int> base((size_t)count, 0);
    int *d = nullptr;
    AMG_CUDA_TRY(cudaMallocAsync(&d, sizeof(int) * (size_t)count * (9 + kMaxLongRows), s));
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int) * (size_t)count * (9 + kMaxLongRows), s);
    std::vector<int> h((size_t)count * (9 + kMaxLongRows), 0);
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        plans[k]->lr = LongRows();
        const int n = ns[k];
        if (n == 0 || nnzs[k] == 0) continue;
        const double avg = (double)nnzs[k] / n;
        base[(size_t)k] = (int)std::min(1.0e9, std::max(512.0, 8.0 * avg));
        long_hist_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, rps[k], base[(size_t)k], d + (size_t)k * (9 + kMaxLongRows));
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    bool any = false;
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        const int *hist = h.data() + (size_t)k * (9 + kMaxLongRows);
        int t = 0;
        while (t < 8 && hist[t] > kMaxLongRows) ++t;
        if (t == 8 || hist[t] == 0) continue;
        plans[k]->lr.len = base[(size_t)k] << t;
        int *slot = d + (size_t)k * (9 + kMaxLongRows);
        e = cudaMemsetAsync(slot + 8, 0, sizeof(int), s);
        if (e == cudaSuccess) {
            long_rows_kernel<<<grid_for(ns[k], 256), 256, 0, s>>>(ns[k], rps[k], plans[k]->lr.len, slot + 8, slot + 9);
            note_launch();
            e = cudaGetLastError();
        }
        any = true;
    }
    if (any && e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, s);
    if (any && e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(d, s);
    for (int k = 0; any && e == cudaSuccess && k < count; ++k) {
        if (plans[k]->lr.len == 0x7fffffff) continue;
        const int *slot = h.data() + (size_t)k * (9 + kMaxLongRows);
        LongRows &lr = plans[k]->lr;
        lr.count = std::min(slot[8], kMaxLongRows);
        std::copy(slot + 9, slot + 9 + lr.count, lr.rows);
        std::sort(lr.rows, lr.rows + lr.count);
    }
    return e;
}

// Plans of several matrices with one synchronisation: every span kernel is queued first,
// then one copy of all maxima to the host.
cudaError_t spmv_plans(int count, SpmvPlan *const *plans, const int *const *rps, const int *ns, const int64_t *nnzs,
                       cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    AMG_CUDA_TRY(long_rows_plan(count, plans, rps, ns, nnzs, s));
    int *d = nullptr;
    std::vector<int> h((size_t)count, 0);
    AMG_CUDA_TRY(cudaMallocAsync(&d, sizeof(int) * (size_t)count, s));
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int) * (size_t)count, s);
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        SpmvPlan *pl = plans[k];
        const int n = ns[k];
        pl->lpr = pick_lpr_rows(n ? (double)nnzs[k] / n : 1.0, n);
        pl->cap = 0;
        if (n == 0 || nnzs[k] == 0) continue;
        const int nb = spmv_blocks(n, pl->lpr);
        span_max_kernel<<<grid_for((int64_t)nb * 32, 256), 256, 0, s>>>(n, rps[k], kSpmvThreads / pl->lpr,
                                                                          pl->lr.len, d + k);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, sizeof(int) * (size_t)count, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int k = 0; k < count; ++k)
        if (ns[k] > 0 && nnzs[k] > 0) plans[k]->cap = h[(size_t)k] + 8 < kMaxTile ? h[(size_t)k] + 8 : kMaxTile;
    return e;
}

cudaError_t spmv_plan(const int *rp, int n, int64_t nnz, SpmvPlan *plan, cudaStream_t s)
{
    SpmvPlan *pls[1] = {plan};
    const int *rps[1] = {rp};
    const int ns[1] = {n};
    const int64_t nz[1] = {nnz};
    return spmv_plans(1, pls, rps, ns, nz, s);
}

// rows with more than len entries, by class: cnt[0] more than kSegRowLen entries, cnt[1] more
// than kBlockRowLen, cnt[2] the others
__device__ __forceinline__ int split_class(int l) { return l > kSegRowLen ? 0 : l > kBlockRowLen ? 1 : 2; }
__global__ void split_count_kernel(int n, const int *rp, int len, int *cnt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = rp[i + 1] - rp[i];
    if (l > len) atomicAdd(&cnt[split_class(l)], 1);
}

// the same rows into list, class after class (order of arrival within a class: a row's sum does
// not depend on which block or warp forms it)
__global__ void split_fill_kernel(int n, const int *rp, int len, int n0, int n1, int *cnt, int *list)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = rp[i + 1] - rp[i];
    if (l <= len) return;
    const int c = split_class(l);
    list[(c == 0 ? 0 : c == 1 ? n0 : n0 + n1) + atomicAdd(&cnt[c], 1)] = i;
}

// segment block b's row: entry 0 of its table row holds the row's index in the list
__global__ void split_seg_rows_kernel(int nsegb, const int *list, int *seg)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nsegb) seg[5 * b] = list[seg[5 * b]];
}

// first and end entry of each of the m listed rows
__global__ void split_ranges_kernel(int m, const int *list, const int *rp, int *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    out[2 * t] = rp[list[t]];
    out[2 * t + 1] = rp[list[t] + 1];
}

// A solve plan's row-tile limit: a row of more than 16 entries a lane (and more than 4 x its
// operator's mean, and more than 32) leaves the tiles, whose lanes would walk it as one serial
// chain of FP64 additions while the rest of the block waits.
int split_threshold(int lpr, double avg)
{
    const double t = std::max(std::max(32.0, 16.0 * lpr), 4.0 * avg);
    return t < 1.0e9 ? (int)t : 1000000000;
}

// Per plan, one allocation of ints: the segment sums (2 ints each, first: 8-byte aligned), the
// tickets, the segment table (5 ints each), the row list.
cudaError_t spmv_split_rows(int count, SpmvPlan *const *plans, const int *const *rps, const int *ns,
                            const int64_t *nnzs, const std::function<cudaError_t(int **, size_t)> &alloc,
                            cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    constexpr int W = 8;     // counter ints per plan: 3 to count, 3 to fill
    int *d = nullptr;
    AMG_CUDA_TRY(cudaMallocAsync(&d, sizeof(int) * W * (size_t)count, s));
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int) * W * (size_t)count, s);
    std::vector<int> len((size_t)count, 0x7fffffff);
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        SpmvPlan *pl = plans[k];
        pl->sr = SplitRows();
        pl->split_len = 0x7fffffff;
        if (ns[k] == 0 || nnzs[k] == 0) continue;
        len[(size_t)k] = split_threshold(pl->lpr, (double)nnzs[k] / ns[k]);
        split_count_kernel<<<grid_for(ns[k], 256), 256, 0, s>>>(ns[k], rps[k], len[(size_t)k], d + W * k);
        note_launch();
        e = cudaGetLastError();
    }
    std::vector<int> h((size_t)count * W, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    // the row lists, and the ranges of the rows to be segmented
    std::vector<int *> base((size_t)count, nullptr);
    std::vector<size_t> rng_off((size_t)count, 0);
    size_t rng_total = 0;
    for (int k = 0; k < count; ++k) {
        rng_off[(size_t)k] = rng_total;
        rng_total += 2 * (size_t)h[(size_t)W * k];
    }
    int *rng = nullptr;
    if (e == cudaSuccess && rng_total) e = cudaMallocAsync(&rng, sizeof(int) * rng_total, s);
    std::vector<int *> lists((size_t)count, nullptr);
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        const int n0 = h[(size_t)W * k], n1 = h[(size_t)W * k + 1], n2 = h[(size_t)W * k + 2];
        if (n0 + n1 + n2 == 0) continue;
        e = cudaMallocAsync(&lists[(size_t)k], sizeof(int) * ((size_t)n0 + n1 + n2), s);
        if (e != cudaSuccess) break;
        split_fill_kernel<<<grid_for(ns[k], 256), 256, 0, s>>>(ns[k], rps[k], len[(size_t)k], n0, n1, d + W * k + 3,
                                                               lists[(size_t)k]);
        note_launch();
        if (n0) {
            split_ranges_kernel<<<grid_for(n0, 256), 256, 0, s>>>(n0, lists[(size_t)k], rps[k],
                                                                  rng + rng_off[(size_t)k]);
            note_launch();
        }
        e = cudaGetLastError();
    }
    std::vector<int> hr(rng_total);
    if (e == cudaSuccess && rng_total)
        e = cudaMemcpyAsync(hr.data(), rng, sizeof(int) * rng_total, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    // per plan: the segment table on the host, then one allocation for everything
    std::vector<std::vector<int>> tables((size_t)count);
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        const int n0 = h[(size_t)W * k], n1 = h[(size_t)W * k + 1], n2 = h[(size_t)W * k + 2];
        const int nl = n0 + n1 + n2;
        if (nl == 0) continue;
        std::vector<int> &seg = tables[(size_t)k];
        for (int t = 0; t < n0; ++t) {
            const int k0 = hr[rng_off[(size_t)k] + 2 * t], k1 = hr[rng_off[(size_t)k] + 2 * t + 1];
            const int first = (int)(seg.size() / 5), nseg = (k1 - k0 + kSegRowLen - 1) / kSegRowLen;
            for (int q = 0; q < nseg; ++q) {
                seg.push_back(-1);                          // the row, from the device list below
                seg.push_back(k0 + q * kSegRowLen);
                seg.push_back(std::min(k1, k0 + (q + 1) * kSegRowLen));
                seg.push_back(first);
                seg.push_back(nseg);
            }
        }
        const size_t nsegb = seg.size() / 5;
        int *buf = nullptr;
        e = alloc(&buf, 2 * nsegb + nsegb + 5 * nsegb + (size_t)nl);
        if (e != cudaSuccess) break;
        SplitRows &sr = plans[k]->sr;
        sr.part = (double *)buf;
        sr.tick = (unsigned *)(buf + 2 * nsegb);
        int *dseg = buf + 3 * nsegb;       // filled below, once each segment's row is known
        int *drows = dseg + 5 * nsegb;
        sr.seg = dseg;
        sr.rows = drows;
        sr.nseg_rows = n0;
        sr.nblock = n1;
        sr.nwarp = n2;
        sr.nsegb = (int)nsegb;
        plans[k]->split_len = len[(size_t)k];
        if (nsegb) e = cudaMemsetAsync(sr.tick, 0, sizeof(unsigned) * nsegb, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(drows, lists[(size_t)k], sizeof(int) * (size_t)nl, cudaMemcpyDeviceToDevice, s);
        // each segment's row: the segmented rows in list order
        if (e == cudaSuccess && nsegb) {
            int t = 0;
            for (size_t b = 0; b < nsegb; ++b) {
                if (b > 0 && seg[5 * b + 3] != seg[5 * (b - 1) + 3]) ++t;
                seg[5 * b] = t;            // index into the list for now
            }
        }
    }
    // the row of each segment block from the list (a device gather: the list order is the
    // device's), then the tables
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        SplitRows &sr = plans[k]->sr;
        if (!sr.nsegb) continue;
        e = cudaMemcpyAsync((void *)sr.seg, tables[(size_t)k].data(), sizeof(int) * tables[(size_t)k].size(),
                            cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            split_seg_rows_kernel<<<grid_for(sr.nsegb, 256), 256, 0, s>>>(sr.nsegb, sr.rows, (int *)sr.seg);
            note_launch();
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);       // the host tables go out of scope
    for (int *p : lists)
        if (p) cudaFreeAsync(p, s);
    if (rng) cudaFreeAsync(rng, s);
    cudaFreeAsync(d, s);
    return e;
}

// Plans of short rows (two lanes per row in the tiles, at most 8 entries a row on average and
// 16 at most) take spmv_rows_kernel: one synchronisation for all.
cudaError_t spmv_short_rows(int count, SpmvPlan *const *plans, const int *const *rps, const int *ns,
                            const int64_t *nnzs, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    int *d = nullptr;
    AMG_CUDA_TRY(cudaMallocAsync(&d, sizeof(int) * (size_t)count, s));
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int) * (size_t)count, s);
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        plans[k]->rowk = 0;
        if (ns[k] == 0 || plans[k]->lpr != 2 || nnzs[k] > 8 * (int64_t)ns[k]) continue;
        max_row_kernel<<<grid_for(ns[k], 256), 256, 0, s>>>(ns[k], rps[k], d + k);
        note_launch();
        e = cudaGetLastError();
    }
    std::vector<int> h((size_t)count, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, sizeof(int) * (size_t)count, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(d, s);
    for (int k = 0; k < count && e == cudaSuccess; ++k)
        if (ns[k] > 0 && plans[k]->lpr == 2 && nnzs[k] <= 8 * (int64_t)ns[k] && h[(size_t)k] <= 16)
            plans[k]->rowk = 1;
    return e;
}

static int *g_spmv_err = nullptr;   // device error flag of the bounded waits (allocated once)
static std::once_flag g_spmv_err_once;

int *spmv_error_flag()
{
    std::call_once(g_spmv_err_once, [] {
        if (cudaMalloc(&g_spmv_err, sizeof(int)) != cudaSuccess) { g_spmv_err = nullptr; return; }
        cudaMemset(g_spmv_err, 0, sizeof(int));
    });
    return g_spmv_err;
}

// number of blocks whose bounded wait for a bulk copy ran out since the last call (resets it)
int spmv_take_errors(cudaStream_t s)
{
    if (!g_spmv_err) return 0;
    int h = 0;
    if (cudaMemcpyAsync(&h, g_spmv_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    if (h) cudaMemsetAsync(g_spmv_err, 0, sizeof(int), s);
    return h;
}

// ------------------------------------------------------------------------------------ sliced ELL
// The solve's products with A on levels of short rows read a sliced-ELL copy of A: slices of
// kSliceRows consecutive rows, each as wide as its longest row, stored column-major (entry k
// of the slice's row t at sp[slice] + kSliceRows k + t).  Padding has value 0 and the row's own
// column (the last row's for rows past n).  One lane per row, so the loads of values, columns
// and x are coalesced across the warp.  A row is summed in two parts, entries 0, 2, 4, ... and
// 1, 3, 5, ..., added at the end: the arithmetic of the CSR kernel with two lanes per row, so
// both forms give the same bits (a padding entry adds an exact 0).
constexpr int kSliceRows = 32;
constexpr int kSellThreads = 256;

__device__ __forceinline__ double ld_stream(const double *p)
{
    double v;
    asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream(const float *p)
{
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int ld_stream(const int *p)
{
    int v;
    asm volatile("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// MODE_Y, MODE_RESID, MODE_CHEB, MODE_DOT (partials only) and MODE_POWER as in
// spmv_tile_kernel.  MODE_DOT and MODE_POWER write the partials of the two-lanes-per-row CSR
// kernel: one per 128 rows (nparts), each summed by the same shuffle tree and the same order of
// warps; MODE_POWER then completes its two sums as the CSR kernel does (result, counter).
template <typename T, int MODE>
__global__ void __launch_bounds__(kSellThreads) spmv_sell_kernel(int n, const int *__restrict__ sp,
                                                                 const int *__restrict__ sw,
                                                                 const int *__restrict__ sci,
                                                                 const T *__restrict__ sv, const T *__restrict__ x,
                                                                 T *y, const T *__restrict__ f,
                                                                 const T *__restrict__ aux, T *d, T c1, T c2,
                                                                 double *partial, int nparts, double *result,
                                                                 unsigned *counter)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double rq = MODE == MODE_POWER ? (double)f[1] : 0.0;
    const int slice = blockIdx.x * (kSellThreads / kSliceRows) + warp;
    const int row = slice * kSliceRows + lane;
    T sum = T(0);
    if (slice * kSliceRows < n) {
        const int base = sp[slice] + lane, w = sw[slice];
        const T *vv = sv + base;
        const int *cc = sci + base;
        T s0 = T(0), s1 = T(0);
        int k = 0;
#pragma unroll 2
        for (; k + 1 < w; k += 2) {
            s0 += ld_stream(vv + kSliceRows * k) * x[ld_stream(cc + kSliceRows * k)];
            s1 += ld_stream(vv + kSliceRows * (k + 1)) * x[ld_stream(cc + kSliceRows * (k + 1))];
        }
        if (k < w) s0 += ld_stream(vv + kSliceRows * k) * x[ld_stream(cc + kSliceRows * k)];
        sum = s0 + s1;
    }
    double contrib = 0.0, contrib2 = 0.0;
    if (row < n) {
        if (MODE == MODE_Y) {
            y[row] = sum;
        } else if (MODE == MODE_RESID) {
            y[row] = f[row] - sum;
        } else if (MODE == MODE_CHEB) {
            T r = f[row] - sum;
            T dn = c1 * d[row] + c2 * (aux[row] * r);
            d[row] = dn;
            y[row] = x[row] + dn;
        } else if (MODE == MODE_POWER) {
            const double yi = ((double)sum * (double)aux[row]) * rq;
            y[row] = (T)yi;
            if (c1 != T(0)) contrib = (double)x[row] * yi;
            contrib2 = yi * yi;
        } else {
            y[row] = sum;
            contrib = (double)x[row] * (double)sum;
        }
    }
    if (MODE == MODE_POWER) {
        // CSR block b = rows 128 b .. 128 b + 127 = this block's warps 4 hh .. 4 hh + 3 (rows of
        // the CSR block's warp w' on its lanes, in order); the CSR block's warps 4-7 hold zeros,
        // which it does not add
        __shared__ double q1[kSellThreads / 32], q2[kSellThreads / 32];
        if (c1 != T(0)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) contrib += __shfl_down_sync(kAll, contrib, o);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) contrib2 += __shfl_down_sync(kAll, contrib2, o);
        if (lane == 0) {
            q1[warp] = c1 != T(0) ? contrib : 0.0;
            q2[warp] = contrib2;
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            const int part = 2 * blockIdx.x + threadIdx.x;
            if (part < nparts) {
                double t1 = 0.0, t2 = 0.0;
                for (int w = 0; w < 4; ++w) {
                    if (c1 != T(0)) t1 += q1[4 * threadIdx.x + w];
                    t2 += q2[4 * threadIdx.x + w];
                }
                partial[part] = t1;
                partial[nparts + part] = t2;
            }
        }
        last_block_total2(partial, nparts, counter, result, (double *)d, rq, (int)gridDim.x, true);
        return;
    }
    if (MODE == MODE_DOT) {
        // CSR block b = rows 128 b .. 128 b + 127 = this block's warps 4 hh .. 4 hh + 3, row r of
        // a CSR warp on lane r of the same warp here: the same trees, the same partials
        __shared__ double qd[kSellThreads / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) contrib += __shfl_down_sync(kAll, contrib, o);
        if (lane == 0) qd[warp] = contrib;
        __syncthreads();
        if (threadIdx.x < 2) {
            const int part = 2 * blockIdx.x + threadIdx.x;
            if (part < nparts) {
                double t = 0.0;
                for (int w = 0; w < 4; ++w) t += qd[4 * threadIdx.x + w];
                partial[part] = t;
            }
        }
    }
}

// slice s: sw[s] = its width, size[s] = kSliceRows sw[s]; *total64 += size[s] (the int offsets
// are used only when this 64-bit total fits an int)
__global__ void sell_width_kernel(int n, const int *rp, int ns, int *sw, int *size, unsigned long long *total64)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const int r0 = s * kSliceRows, r1 = min(n, r0 + kSliceRows);
    int w = 0;
    for (int r = r0; r < r1; ++r) w = max(w, rp[r + 1] - rp[r]);
    sw[s] = w;
    size[s] = kSliceRows * w;
    atomicAdd(total64, (unsigned long long)kSliceRows * (unsigned long long)w);
}

// one thread per row slot of every slice: its columns (sci non-null) and values (sv non-null).
// A block of kFillRows rows first copies their CSR entries into shared memory with coalesced
// loads (when they fit kFillCap), so that the threads' walks along their own rows read shared
// memory instead of 32 scattered rows of global memory at a time.
constexpr int kFillRows = 128;     // four slices a block
constexpr int kFillCap = 3584;     // staged entries a block (43 KB with FP64 values)
template <typename T>
__global__ void __launch_bounds__(kFillRows) sell_fill_kernel(int n, const int *rp, const int *ci, const T *v, int ns,
                                                              const int *sp, const int *sw, int *sci, T *sv)
{
    __shared__ int stc[kFillCap];
    __shared__ T stv[kFillCap];
    const int r0 = blockIdx.x * kFillRows;
    const int t = r0 + (int)threadIdx.x;
    const int k0 = rp[min(r0, n)], k1 = rp[min(r0 + kFillRows, n)];
    const bool staged = k1 - k0 <= kFillCap;
    if (staged) {
        for (int e = k0 + (int)threadIdx.x; e < k1; e += kFillRows) {
            if (sci) stc[e - k0] = ci[e];
            if (sv) stv[e - k0] = v[e];
        }
    }
    __syncthreads();
    if (t >= ns * kSliceRows) return;
    const int s = t / kSliceRows, lane = t % kSliceRows;
    const int w = sw[s], base = sp[s] + lane;
    const int b = t < n ? rp[t] : 0, len = t < n ? rp[t + 1] - b : 0;
    const int pad = t < n ? t : n - 1;
    for (int k = 0; k < w; ++k) {
        if (sci) sci[base + kSliceRows * k] = k < len ? (staged ? stc[b - k0 + k] : ci[b + k]) : pad;
        if (sv) sv[base + kSliceRows * k] = k < len ? (staged ? stv[b - k0 + k] : v[b + k]) : T(0);
    }
}

template <typename T>
const T *sell_values(const SpmvPlan &pl);
template <>
const double *sell_values<double>(const SpmvPlan &pl) { return pl.sv64; }
template <>
const float *sell_values<float>(const SpmvPlan &pl) { return pl.sv32; }

template <typename T, int MODE>
cudaError_t launch_sell(const SpmvPlan &pl, int n, const T *sv, const T *x, T *y, const T *f, const T *aux, T *d,
                        T c1, T c2, double *partial, cudaStream_t s, double *result = nullptr,
                        unsigned *counter = nullptr)
{
    const int blocks = (pl.ns + kSellThreads / kSliceRows - 1) / (kSellThreads / kSliceRows);
    spmv_sell_kernel<T, MODE><<<blocks, kSellThreads, 0, s>>>(n, pl.sp, pl.sw, pl.sci, sv, x, y, f, aux, d, c1, c2,
                                                              partial, spmv_blocks(n, 2), result, counter);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t sell_fill_t(int n, const int *rp, const int *ci, const T *v, int ns, const int *sp, const int *sw,
                        int *sci, T *sv, cudaStream_t s)
{
    if (ns == 0) return cudaSuccess;
    const int64_t slots = (int64_t)ns * kSliceRows;
    sell_fill_kernel<T><<<(int)((slots + kFillRows - 1) / kFillRows), kFillRows, 0, s>>>(n, rp, ci, v, ns, sp, sw,
                                                                                       sci, sv); note_launch();
    return cudaGetLastError();
}

template <typename T, int LPR, int MODE>
cudaError_t launch_tile(int n, const int *rp, const int *ci, const T *v, const T *x, T *y, const T *f, const T *aux,
                        T *d, T c1, T c2, int cap, double *partial, double *result, unsigned *counter,
                        cudaStream_t s, int long_len, const SplitRows &sr)
{
    const int extra = split_blocks(sr);
    const int smem = tile_bytes<T>(cap);
    // the attribute is set once per instantiation (any thread may get here first)
    static std::once_flag configured;
    static cudaError_t cfg_err = cudaSuccess;
    std::call_once(configured, [] {
        cfg_err = cudaFuncSetAttribute(spmv_tile_kernel<T, LPR, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       tile_bytes<T>(kMaxTile));
    });
    AMG_CUDA_TRY(cfg_err);
    spmv_tile_kernel<T, LPR, MODE><<<spmv_blocks(n, LPR) + extra, kSpmvThreads, smem, s>>>(
        n, rp, ci, v, x, y, f, aux, d, c1, c2, cap, partial, result, counter, spmv_error_flag(), long_len, sr);
    note_launch();
    return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t spmv_mode(const SpmvPlan &pl, int n, const int *rp, const int *ci, const T *v, const T *x, T *y,
                      const T *f, const T *aux, T *d, T c1, T c2, double *partial, cudaStream_t s,
                      double *result = nullptr, unsigned *counter = nullptr)
{
    if (n == 0) return cudaSuccess;
    if ((MODE == MODE_Y || MODE == MODE_RESID || MODE == MODE_CHEB || (MODE == MODE_DOT && result == nullptr) ||
         MODE == MODE_POWER) &&
        pl.ns > 0 && pl.lpr == 2 && pl.lr.count == 0 && pl.sr.rows == nullptr) {
        const T *sv = sell_values<T>(pl);
        if (sv) return launch_sell<T, MODE>(pl, n, sv, x, y, f, aux, d, c1, c2, partial, s, result, counter);
    }
    if ((MODE == MODE_Y || MODE == MODE_RESID || MODE == MODE_CHEB || MODE == MODE_PROLONG) && pl.rowk &&
        pl.sr.rows == nullptr && pl.lr.count == 0) {
        spmv_rows_kernel<T, MODE><<<(n + kSpmvThreads - 1) / kSpmvThreads, kSpmvThreads, 0, s>>>(n, rp, ci, v, x, y,
                                                                                              f, aux, d, c1, c2);
        note_launch();
        return cudaGetLastError();
    }
    int long_len = 0x7fffffff;
    SplitRows sr;
    if (pl.sr.rows) {
        long_len = pl.split_len;
        if (MODE == MODE_DOT || MODE == MODE_SCALEDOT || MODE == MODE_POWER) {
            // the tile kernel's dot products read the split rows' y: they go first
            spmv_split_kernel<T, MODE><<<split_blocks(pl.sr), kSpmvThreads, 0, s>>>(pl.sr, rp, ci, v, x, y, f, aux, d,
                                                                                    c1, c2);
            note_launch();
            AMG_CUDA_TRY(cudaGetLastError());
        } else {
            sr = pl.sr;
        }
    } else if (pl.lr.count > 0) {
        spmv_long_kernel<T, MODE><<<pl.lr.count, kSpmvThreads, 0, s>>>(pl.lr, rp, ci, v, x, y, f, aux, d, c1, c2);
        note_launch();
        AMG_CUDA_TRY(cudaGetLastError());
        long_len = pl.lr.len;
    }
    switch (pl.lpr) {
    case 2:
        return launch_tile<T, 2, MODE>(n, rp, ci, v, x, y, f, aux, d, c1, c2, pl.cap, partial, result, counter, s,
                                       long_len, sr);
    case 4:
        return launch_tile<T, 4, MODE>(n, rp, ci, v, x, y, f, aux, d, c1, c2, pl.cap, partial, result, counter, s,
                                       long_len, sr);
    case 8:
        return launch_tile<T, 8, MODE>(n, rp, ci, v, x, y, f, aux, d, c1, c2, pl.cap, partial, result, counter, s,
                                       long_len, sr);
    case 16:
        return launch_tile<T, 16, MODE>(n, rp, ci, v, x, y, f, aux, d, c1, c2, pl.cap, partial, result, counter, s,
                                        long_len, sr);
    default:
        return launch_tile<T, 32, MODE>(n, rp, ci, v, x, y, f, aux, d, c1, c2, pl.cap, partial, result, counter, s,
                                        long_len, sr);
    }
}

// ------------------------------------------------------------------------------------ FP64 entry points
cudaError_t spmv_d(const DevCsr &A, const SpmvPlan &pl, const double *x, double *y, cudaStream_t s)
{
    return spmv_mode<double, MODE_Y>(pl, A.n, A.rp, A.ci, A.v, x, y, nullptr, nullptr, nullptr, 0.0, 0.0, nullptr, s);
}

cudaError_t residual_d(const DevCsr &A, const SpmvPlan &pl, const double *b, const double *x, double *r,
                       cudaStream_t s)
{
    return spmv_mode<double, MODE_RESID>(pl, A.n, A.rp, A.ci, A.v, x, r, b, nullptr, nullptr, 0.0, 0.0, nullptr, s);
}

// q = A p and p . q into *result (fixed-order two-stage sum)
cudaError_t spmv_dot(const DevCsr &A, const SpmvPlan &pl, const double *p, double *q, double *partial,
                     double *result, unsigned *counter, cudaStream_t s)
{
    return spmv_mode<double, MODE_DOT>(pl, A.n, A.rp, A.ci, A.v, p, q, nullptr, nullptr, nullptr, 0.0, 0.0, partial,
                                       s, result, counter);
}

// y = (A x) / D and x . y into *result
cudaError_t spmv_scaled_dot(const DevCsr &A, const SpmvPlan &pl, const double *D, const double *x, double *y,
                            double *partial, double *result, unsigned *counter, cudaStream_t s)
{
    return spmv_mode<double, MODE_SCALEDOT>(pl, A.n, A.rp, A.ci, A.v, x, y, nullptr, D, nullptr, 0.0, 0.0, partial,
                                            s, result, counter);
}

// one sweep of the power method on D^-1 A (invD = D^-1) from the unnormalised x with
// xx[0] = x . x and xx[1] = 1 / sqrt(x . x): y = (D^-1 A x) xx[1], *lambda = (x . y) xx[1] (the
// Rayleigh quotient of the unit vector; only with_lambda, else 0), yy[0] = y . y,
// yy[1] = 1 / sqrt(y . y).  partial holds 2 x the plan's blocks.
cudaError_t spmv_power(const DevCsr &A, const SpmvPlan &pl, const double *invD, const double *x, const double *xx,
                       double *y, double *yy, double *partial, double *lambda, unsigned *counter, cudaStream_t s,
                       bool with_lambda)
{
    return spmv_mode<double, MODE_POWER>(pl, A.n, A.rp, A.ci, A.v, x, y, xx, invD, yy, with_lambda ? 1.0 : 0.0, 0.0,
                                         partial, s, lambda, counter);
}

// per-block partial sums of a product over n rows: as many as blocks at the most lanes per row
// (fewest rows per block) any plan chooses, plus one
int spmv_partials_needed(int n) { return spmv_blocks(n, 32) + 1; }

int sell_slices(int n) { return n > 0 ? (n + kSliceRows - 1) / kSliceRows : 0; }

cudaError_t sell_layout(int n, const int *rp, int *sw, int *sp, unsigned long long *total64, cudaStream_t s)
{
    const int ns = sell_slices(n);
    AMG_CUDA_TRY(cudaMemsetAsync(total64, 0, sizeof(unsigned long long), s));
    if (ns == 0) return cudaMemsetAsync(sp, 0, sizeof(int), s);
    sell_width_kernel<<<(ns + 255) / 256, 256, 0, s>>>(n, rp, ns, sw, sp, total64); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    return scan_exclusive(sp, sp, ns, s);
}

cudaError_t sell_fill_d(int n, const int *rp, const int *ci, const double *v, int ns, const int *sp, const int *sw,
                        int *sci, double *sv, cudaStream_t s)
{
    return sell_fill_t<double>(n, rp, ci, v, ns, sp, sw, sci, sv, s);
}

cudaError_t sell_fill_f(int n, const int *rp, const float *v, int ns, const int *sp, const int *sw, float *sv,
                        cudaStream_t s)
{
    return sell_fill_t<float>(n, rp, nullptr, v, ns, sp, sw, nullptr, sv, s);
}
int spmv_block_count(int n, const SpmvPlan &pl) { return spmv_blocks(n, pl.lpr); }

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

// Every block sums the same partials in the same fixed order, so every block holds the
// same scalar and no separate scalar kernel (and launch) is needed.
__device__ __forceinline__ double block_sum_all(double v)
{
    __shared__ double sh[kReduceThreads / 32];
    __shared__ double total;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kAll, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kReduceThreads / 32; ++w) t += sh[w];
        total = t;
    }
    __syncthreads();
    return total;
}

__device__ __forceinline__ double sum_partials_all(const double *partial, int count)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < count; i += kReduceThreads) acc += partial[i];
    return block_sum_all(acc);
}

// alpha = rz / (p . q); x += alpha p; r -= alpha q; partial sums of r . r (read back by the
// host for the stopping test)
// (the vector loops below are unrolled with their arrays marked unaliased, so a thread's loads of
// several iterations are in flight at once; the sums still add in iteration order)
__global__ void __launch_bounds__(kReduceThreads) pcg_xr_kernel(int n, double *__restrict__ x,
                                                                double *__restrict__ r,
                                                                const double *__restrict__ p,
                                                                const double *__restrict__ q, PcgScalars *sc,
                                                                const double *pq_partial, int pq_count,
                                                                double *rr_partial)
{
    // p . q from the SpMV's per-block partial sums, the same fixed order in every block
    const double pq = sum_partials_all(pq_partial, pq_count);
    const double alpha = sc->rz_next / pq;
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->pq = pq;
    // rz_next (this iteration's r . z) becomes rz, read by the next p update; this kernel
    // reads only rz_next, so the write races with nothing
    if (blockIdx.x == 0 && threadIdx.x == 0) { sc->alpha = alpha; sc->rz = sc->rz_next; }
    double acc = 0.0;
#pragma unroll 4
    for (int i = blockIdx.x * kReduceThreads + threadIdx.x; i < n; i += kReduceBlocks * kReduceThreads) {
        x[i] += alpha * p[i];
        double ri = r[i] - alpha * q[i];
        r[i] = ri;
        acc += ri * ri;
    }
    double t = block_sum_all(acc);
    if (threadIdx.x == 0) rr_partial[blockIdx.x] = t;
}

cudaError_t pcg_update_xr(int n, double *x, double *r, const double *p, const double *q, PcgScalars *sc,
                          const double *pq_partial, int pq_count, double *rr_partial, cudaStream_t s)
{
    pcg_xr_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, x, r, p, q, sc, pq_partial, pq_count, rr_partial); note_launch();
    return cudaGetLastError();
}

// r . z (and r . z_prev for the flexible form) into scalars, fixed-order two-stage sums
__global__ void __launch_bounds__(kReduceThreads) dot_rz_kernel(int n, const double *__restrict__ r,
                                                                const double *__restrict__ z,
                                                                const double *__restrict__ zp, double *pa,
                                                                double *pb, PcgScalars *sc, unsigned *counters)
{
    double a = 0.0, b = 0.0;
#pragma unroll 4
    for (int i = blockIdx.x * kReduceThreads + threadIdx.x; i < n; i += kReduceBlocks * kReduceThreads) {
        const double ri = r[i];
        a += ri * z[i];
        if (zp) b += ri * zp[i];
    }
    const double ta = block_sum_all(a);
    if (threadIdx.x == 0) pa[blockIdx.x] = ta;
    last_block_total(pa, gridDim.x, counters, &sc->rz_new);
    if (zp) {
        const double tb = block_sum_all(b);
        if (threadIdx.x == 0) pb[blockIdx.x] = tb;
        last_block_total(pb, gridDim.x, counters + 1, &sc->rz_cross);
    }
}

// beta = rz_new / rz (flexible: (rz_new - rz_cross) / rz); p = z + beta p.  rz_new goes to
// rz_next, which the next alpha reads (no block overwrites what another still reads).
__global__ void __launch_bounds__(kReduceThreads) pcg_p_kernel(int n, double *__restrict__ p,
                                                               const double *__restrict__ z, PcgScalars *sc,
                                                               int flexible)
{
    const double rz_new = sc->rz_new;
    const double beta = (flexible ? rz_new - sc->rz_cross : rz_new) / sc->rz;
#pragma unroll 4
    for (int i = blockIdx.x * kReduceThreads + threadIdx.x; i < n; i += kReduceBlocks * kReduceThreads)
        p[i] = z[i] + beta * p[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) { sc->beta = beta; sc->rz_next = rz_new; }
}

cudaError_t pcg_update_p(int n, double *p, const double *r, const double *z, const double *z_prev, PcgScalars *sc,
                         double *pa, double *pb, unsigned *counters, cudaStream_t s)
{
    dot_rz_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, r, z, z_prev, pa, pb, sc, counters); note_launch();
    pcg_p_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, p, z, sc, z_prev ? 1 : 0); note_launch();
    return cudaGetLastError();
}

__device__ __forceinline__ double sum_partials(const double *partial, int count)
{
    return sum_partials_all(partial, count);
}

__global__ void __launch_bounds__(kReduceThreads) pcg_store_kernel(const double *partial, int count,
                                                                   double *dst)
{
    double t = sum_partials(partial, count);
    if (threadIdx.x == 0) *dst = t;
}

cudaError_t pcg_store(const double *partial, int count, double *dst, cudaStream_t s)
{
    pcg_store_kernel<<<1, kReduceThreads, 0, s>>>(partial, count, dst); note_launch();
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

// ------------------------------------------------------------------------------------ coarse polynomial solve
// A large, sparse coarsest operator whose Jacobi-scaled form is well conditioned (what stalled
// aggregation leaves: 7,004 rows with scaled condition number 1.2 on the 128^3 random-
// coefficient cube) is solved in every V-cycle by a Chebyshev iteration of fixed degree m on an
// interval [lo, hi] holding the spectrum of D^-1 A, instead of a product with a dense inverse.
// m steps from x = 0 apply a fixed polynomial in D^-1 A, so the coarse solve stays one linear
// operator (as the exact inverse is); m is the least degree whose bound 2 rho^m on the error,
// rho = (sqrt(hi/lo) - 1) / (sqrt(hi/lo) + 1), is below kCoarseChebTol.
//
// The interval: m_L = 16 steps of Jacobi-preconditioned CG on A x = b for a pseudo-random b are m_L
// steps of the Lanczos process on D^-1 A (the tridiagonal matrix follows from the CG
// coefficients alpha_j = rz_j / pq_j and beta_j = rz_{j+1} / rz_j).  Its extreme eigenvalues
// lie inside the spectrum; widened by a fifth of their distance each way they bound it, and a
// solve of a second pseudo-random right-hand side checks the result.
constexpr int kLanczosSteps = 16;
constexpr int kCoarseChebMax = 40;
constexpr double kCoarseChebTol = 1e-16;

__device__ __forceinline__ double coarse_rand(int i, uint64_t stream)
{
    uint64_t z = stream + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-52 - 1.0;       // uniform in [-1, 1)
}

// b pseudo-random (stream); r = b, p = D^-1 b, *rz0 = r . D^-1 r (fixed-order two-stage sum)
__global__ void __launch_bounds__(kReduceThreads) lz_start_kernel(int n, uint64_t stream, const double *invdiag,
                                                                  double *r, double *p, double *partial,
                                                                  unsigned *counter, double *rz0)
{
    double acc = 0.0;
    for (int i = blockIdx.x * kReduceThreads + threadIdx.x; i < n; i += gridDim.x * kReduceThreads) {
        const double b = coarse_rand(i, stream);
        const double z = invdiag[i] * b;
        r[i] = b;
        p[i] = z;
        acc += b * z;
    }
    const double t = block_sum_all(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
    last_block_total(partial, gridDim.x, counter, rz0);
}

// CG step j after q = A p, pq[j] = p . q: r -= alpha q, rz[j + 1] = r . D^-1 r
__global__ void __launch_bounds__(kReduceThreads) lz_update_kernel(int n, const double *invdiag, double *r,
                                                                   const double *q, double *rz, const double *pq,
                                                                   int j, double *partial, unsigned *counter)
{
    const double a = (pq[j] > 0.0 && rz[j] > 0.0) ? rz[j] / pq[j] : 0.0;
    double acc = 0.0;
    for (int i = blockIdx.x * kReduceThreads + threadIdx.x; i < n; i += gridDim.x * kReduceThreads) {
        const double ri = r[i] - a * q[i];
        r[i] = ri;
        acc += ri * (invdiag[i] * ri);
    }
    const double t = block_sum_all(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
    last_block_total(partial, gridDim.x, counter, rz + j + 1);
}

// p = D^-1 r + beta p, beta = rz[j + 1] / rz[j]
__global__ void __launch_bounds__(kReduceThreads) lz_direction_kernel(int n, const double *invdiag, const double *r,
                                                                      double *p, const double *rz, int j)
{
    const double b = rz[j] > 0.0 ? rz[j + 1] / rz[j] : 0.0;
    for (int i = blockIdx.x * kReduceThreads + threadIdx.x; i < n; i += gridDim.x * kReduceThreads)
        p[i] = invdiag[i] * r[i] + b * p[i];
}

// out[0] = r . D^-1 r, out[1] = f . D^-1 f (the check's residual and right-hand side norms)
__global__ void __launch_bounds__(kReduceThreads) dnorm2_kernel(int n, const double *invdiag, const double *r,
                                                                const double *f, double *partial, unsigned *counter,
                                                                double *out)
{
    double a = 0.0, b = 0.0;
    for (int i = blockIdx.x * kReduceThreads + threadIdx.x; i < n; i += gridDim.x * kReduceThreads) {
        a += r[i] * (invdiag[i] * r[i]);
        b += f[i] * (invdiag[i] * f[i]);
    }
    const double ta = block_sum_all(a);
    if (threadIdx.x == 0) partial[blockIdx.x] = ta;
    const double tb = block_sum_all(b);
    if (threadIdx.x == 0) partial[gridDim.x + blockIdx.x] = tb;
    last_block_total2(partial, gridDim.x, counter, out, out + 1, 1.0);
}

__global__ void rand_fill_kernel(int n, uint64_t stream, double *f)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) f[i] = coarse_rand(i, stream);
}

// Sturm count: eigenvalues of the symmetric tridiagonal (a diagonal, b off-diagonal) below t
static int sturm_below(const std::vector<double> &a, const std::vector<double> &b, double t)
{
    int count = 0;
    double q = 1.0;
    for (size_t i = 0; i < a.size(); ++i) {
        const double off = i ? b[i - 1] * b[i - 1] : 0.0;
        q = (a[i] - t) - (i ? off / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++count;
    }
    return count;
}

// the k-th smallest eigenvalue (k = 0 .. size-1) by bisection inside the Gershgorin bounds
static double tridiag_eig(const std::vector<double> &a, const std::vector<double> &b, int k)
{
    double lo = 1e300, hi = -1e300;
    for (size_t i = 0; i < a.size(); ++i) {
        const double rad = (i ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < a.size() ? std::fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - rad);
        hi = std::max(hi, a[i] + rad);
    }
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_below(a, b, mid) > k) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// x = p_m(D^-1 A) D^-1 f: m Chebyshev steps on [theta - delta, theta + delta] from x = 0; x2
// and d are work vectors.  Returns the buffer holding the result (x or x2).
template <typename T>
T *coarse_cheb_apply(const SpmvPlan &pl, int n, const int *rp, const int *ci, const T *v, const T *invdiag,
                     const T *f, T *x, T *x2, T *d, double theta, double delta, int degree, cudaStream_t s,
                     cudaError_t *err)
{
    const double sigma1 = theta / delta;
    double rho = 1.0 / sigma1;
    cheb_first_zero_kernel<T><<<grid_for(n, 256, 8192), 256, 0, s>>>(n, f, invdiag, (T)(1.0 / theta), d, x);
    note_launch();
    *err = cudaGetLastError();
    for (int k = 1; k < degree && *err == cudaSuccess; ++k) {
        const double rho_new = 1.0 / (2.0 * sigma1 - rho);
        const double c1 = rho_new * rho, c2 = 2.0 * rho_new / delta;
        *err = spmv_mode<T, MODE_CHEB>(pl, n, rp, ci, v, x, x2, f, invdiag, d, (T)c1, (T)c2, nullptr, s);
        T *t = x; x = x2; x2 = t;
        rho = rho_new;
    }
    return x;
}

cudaError_t coarse_cheb_setup(const DevCsr &A, const SpmvPlan &pl, const double *invdiag, int *degree,
                              double *theta, double *delta, double *check, cudaStream_t s)
{
    *degree = 0;
    *check = -1.0;
    const int n = A.n;
    if (n == 0) return cudaSuccess;
    const int np = std::max(spmv_partials_needed(n), 2 * kReduceBlocks);
    const size_t vec = (size_t)n + 16;
    double *w = nullptr;
    const size_t total = 5 * vec + (size_t)np + 2 * kLanczosSteps + 8;
    AMG_CUDA_TRY(cudaMallocAsync(&w, sizeof(double) * total + 64, s));
    struct Release {
        double *p; cudaStream_t s;
        ~Release() { cudaFreeAsync(p, s); }
    } release{w, s};
    double *r = w, *p = r + vec, *q = p + vec, *x2 = q + vec, *d = x2 + vec, *partial = d + vec;
    double *rz = partial + np, *pq = rz + kLanczosSteps + 1, *out = pq + kLanczosSteps;
    unsigned *counter = (unsigned *)(out + 4);
    AMG_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
    AMG_CUDA_TRY(cudaMemsetAsync(rz, 0, sizeof(double) * (2 * kLanczosSteps + 1), s));
    lz_start_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, 0x243F6A8885A308D3ULL, invdiag, r, p, partial,
                                                             counter, rz);
    note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    for (int j = 0; j < kLanczosSteps; ++j) {
        AMG_CUDA_TRY(spmv_dot(A, pl, p, q, partial, pq + j, counter, s));
        lz_update_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, invdiag, r, q, rz, pq, j, partial, counter);
        note_launch();
        lz_direction_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, invdiag, r, p, rz, j);
        note_launch();
        AMG_CUDA_TRY(cudaGetLastError());
    }
    std::vector<double> h(2 * kLanczosSteps + 1);
    AMG_CUDA_TRY(cudaMemcpyAsync(h.data(), rz, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    const double *hrz = h.data(), *hpq = h.data() + kLanczosSteps + 1;
    if (!(hrz[0] > 0.0) || !std::isfinite(hrz[0])) return cudaSuccess;
    // the steps before the residual fell to 1e-13 of its start (later coefficients are noise)
    int J = 0;
    while (J < kLanczosSteps && hpq[J] > 0.0 && std::isfinite(hpq[J]) && hrz[J] > 1e-26 * hrz[0]) ++J;
    if (J == 0) return cudaSuccess;
    std::vector<double> a((size_t)J), b((size_t)(J > 1 ? J - 1 : 0));
    for (int j = 0; j < J; ++j) {
        const double alpha = hrz[j] / hpq[j];
        a[(size_t)j] = 1.0 / alpha;
        if (j > 0) {
            const double alpha_prev = hrz[j - 1] / hpq[j - 1], beta_prev = hrz[j] / hrz[j - 1];
            a[(size_t)j] += beta_prev / alpha_prev;
            b[(size_t)j - 1] = std::sqrt(beta_prev) / alpha_prev;
        }
    }
    const double tmin = tridiag_eig(a, b, 0), tmax = tridiag_eig(a, b, J - 1);
    if (!(tmin > 0.0) || !(tmax >= tmin) || !std::isfinite(tmax)) return cudaSuccess;
    const double margin = 0.2 * (tmax - tmin) + 1e-3 * tmax;
    const double lo = tmin - margin, hi = tmax + margin;
    if (!(lo > 0.0)) return cudaSuccess;
    const double sk = std::sqrt(hi / lo), rho = (sk - 1.0) / (sk + 1.0);
    int m = rho > 0.0 ? (int)std::ceil(std::log(kCoarseChebTol / 2.0) / std::log(rho)) : 1;
    m = std::max(m, 2);
    if (m > kCoarseChebMax) return cudaSuccess;
    // the check: a solve of another pseudo-random right-hand side, its residual in the D^-1 norm
    double *f = p;
    rand_fill_kernel<<<grid_for(n, 256, 8192), 256, 0, s>>>(n, 0x13198A2E03707344ULL, f);
    note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    cudaError_t e = cudaSuccess;
    double *x = coarse_cheb_apply<double>(pl, n, A.rp, A.ci, A.v, invdiag, f, q, x2, d, 0.5 * (hi + lo),
                                          0.5 * (hi - lo), m, s, &e);
    AMG_CUDA_TRY(e);
    AMG_CUDA_TRY(residual_d(A, pl, f, x, r, s));
    dnorm2_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, invdiag, r, f, partial, counter, out);
    note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    double hn[2] = {0.0, 0.0};
    AMG_CUDA_TRY(cudaMemcpyAsync(hn, out, sizeof hn, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (!(hn[1] > 0.0)) return cudaSuccess;
    *check = std::sqrt(hn[0] / hn[1]);
    if (!(*check <= 1e-12)) return cudaSuccess;
    *degree = m;
    *theta = 0.5 * (hi + lo);
    *delta = 0.5 * (hi - lo);
    return cudaSuccess;
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

ChebCoef cheb_coef(double lambda, double ratio, double boost)
{
    // interval [b lambda / ratio, b lambda]: b lifts the power-method estimate (a lower bound)
    double lmax = boost * lambda, lmin = lmax / ratio;
    ChebCoef c;
    c.theta = 0.5 * (lmax + lmin);
    c.delta = 0.5 * (lmax - lmin);
    c.sigma1 = c.theta / c.delta;
    return c;
}

// Chebyshev smoothing of degree m on level L; x holds the iterate (x_is_zero: it is 0).
// Returns the buffer that holds the result (x or x2).
template <typename T>
cudaError_t chebyshev(const SolveCtx &c, int L, T *&x, T *&x2, bool x_is_zero, cudaStream_t s,
                      T *final_out = nullptr)
{
    const LevelView &lv = c.lev[L];
    const ChebCoef cc = cheb_coef(lv.lambda, c.cheb_ratio, c.cheb_boost);
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
        T *dst = (final_out && c.cheb_degree == 1) ? final_out : x2;
        AMG_CUDA_TRY((spmv_mode<T, MODE_CHEB>(lv.plan_a, lv.n, lv.arp, lv.aci, av, x, dst, f, inv, d, (T)0,
                                              (T)(1.0 / cc.theta), nullptr, s)));
        x2 = dst;
        T *t = x; x = x2; x2 = t;
    }
    for (int k = 1; k < c.cheb_degree; ++k) {
        double rho_new = 1.0 / (2.0 * cc.sigma1 - rho);
        double c1 = rho_new * rho, c2 = 2.0 * rho_new / cc.delta;
        ProfScope ps(L == 0 ? KC_VCYCLE_SPMV : KC_COUNT, s, spmv_bytes<T>(lv, 6));
        T *dst = (final_out && k == c.cheb_degree - 1) ? final_out : x2;
        AMG_CUDA_TRY((spmv_mode<T, MODE_CHEB>(lv.plan_a, lv.n, lv.arp, lv.aci, av, x, dst, f, inv, d, (T)c1, (T)c2,
                                              nullptr, s)));
        x2 = dst;
        T *t = x; x = x2; x2 = t;
        rho = rho_new;
    }
    return cudaSuccess;
}

// Algorithm 1 from level L with x = 0; on return *out points at the level's solution buffer.
template <typename T>
cudaError_t vcycle_level(const SolveCtx &c, int L, T **out, cudaStream_t s, T *final_out = nullptr)
{
    const LevelView &lv = c.lev[L];
    T *x = (T *)lv.x, *x2 = (T *)lv.x2;
    if (L == c.nlev - 1) {
        if (c.coarse_degree > 0 && lv.n > 0) {
            cudaError_t e = cudaSuccess;
            *out = coarse_cheb_apply<T>(lv.plan_a, lv.n, lv.arp, lv.aci, (const T *)lv.av, (const T *)lv.invdiag,
                                        (const T *)lv.f, x, x2, (T *)lv.d, c.coarse_theta, c.coarse_delta,
                                        c.coarse_degree, s, &e);
            return e;
        }
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
    AMG_CUDA_TRY((spmv_mode<T, MODE_RESID>(lv.plan_a, lv.n, lv.arp, lv.aci, (const T *)lv.av, x, (T *)lv.r,
                                           (const T *)lv.f, nullptr, nullptr, (T)0, (T)0, nullptr, s)));
    }
    AMG_CUDA_TRY((spmv_mode<T, MODE_Y>(lv.plan_r, cl.n, lv.rrp, lv.rci, (const T *)lv.rv, (const T *)lv.r, (T *)cl.f,
                                       nullptr, nullptr, nullptr, (T)0, (T)0, nullptr, s)));
    T *xc = nullptr;
    AMG_CUDA_TRY(vcycle_level<T>(c, L + 1, &xc, s));
    // x += P x_c
    AMG_CUDA_TRY((spmv_mode<T, MODE_PROLONG>(lv.plan_p, lv.n, lv.prp, lv.pci, (const T *)lv.pv, xc, x, nullptr,
                                             nullptr, nullptr, (T)0, (T)0, nullptr, s)));
    AMG_CUDA_TRY(chebyshev<T>(c, L, x, x2, false, s, final_out));
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
        AMG_CUDA_TRY(vcycle_level<double>(cc, 0, &out, s, c.nlev > 1 ? z : nullptr));
        if (out == z) return cudaSuccess;
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
