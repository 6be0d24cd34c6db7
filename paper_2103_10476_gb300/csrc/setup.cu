// setup.cu -- hierarchy-setup kernels: strength of connection, filtering and lumping,
// aggregation, tentative and smoothed prolongator with the four adaptations, transpose and
// eigenvalue estimates.
//
// Compiled with --fmad=false: every product and sum is rounded as written, and every
// per-row sum runs in ascending column order, so the values match a sequential evaluation
// of the same formulas bit for bit (decisions taken on them are then identical too).
#include <math.h>

#include <algorithm>
#include <utility>

#include "amg_internal.cuh"

namespace amgk {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------------------------ helpers
__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Aggregation priority: top 30 bits of the SplitMix64 finaliser of seed ^ (level << 40) ^ i,
// then the index; distinct for distinct i.
__device__ __forceinline__ uint64_t agg_priority(uint64_t seed, int level, int i)
{
    uint64_t h = splitmix_mix(seed ^ ((uint64_t)level << 40) ^ (uint64_t)(uint32_t)i);
    return ((h >> 34) << 32) | (uint64_t)(uint32_t)i;
}

// ------------------------------------------------------------------------------------ diagonal
__global__ void diag_kernel(int n, const int *rp, const int *ci, const double *v, int *pos, double *d)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = rp[i], hi = rp[i + 1] - 1, found = -1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int c = ci[mid];
        if (c == i) { found = mid; break; }
        if (c < i) lo = mid + 1; else hi = mid - 1;
    }
    if (pos) pos[i] = found;
    if (d) d[i] = found >= 0 ? v[found] : 0.0;
}

cudaError_t diag_extract(const DevCsr &A, int *diagpos, double *d, cudaStream_t s)
{
    if (A.n == 0) return cudaSuccess;
    diag_kernel<<<grid_for(A.n, 256), 256, 0, s>>>(A.n, A.rp, A.ci, A.v, diagpos, d); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ strength, Eq. (7)
// One warp per row.  theta = 0 makes every stored off-diagonal strong (the filtered matrix is
// then A); otherwise |a_ij| >= theta * sqrt(a_ii * a_jj) with each operation rounded, and a
// negative product (sqrt = NaN) makes the entry weak.
// The FP64 test costs a square root (about ten FP64 instructions) per entry, and most entries
// lie far from the threshold, so the test is first taken without FP64 instructions: the row's
// and column's diagonals come in FP32 (converted once per row, NaN when outside [1e-18, 1e18]),
// t32 = theta sqrt(d_i d_j) in FP32 with every operation rounded to nearest (this file is
// compiled without contraction) lies within 4.5 units of 2^-24 (2.7e-7) of the exact value, and
// the FP64 threshold within 4e-16 of it.  The bounds hi = t32 (1 + 2e-6) and lo = t32 (1 - 2e-6)
// (FP32, normal) are turned into the bit patterns of the same values in FP64 by integer
// arithmetic and compared with |a_ij|'s bit pattern (positive doubles order as their bits):
// above hi proves the FP64 test true, below lo proves it false.  Entries in between, NaN
// entries, diagonals outside the range and theta below 1e-6 take the FP64 test itself.  The
// decisions are the FP64 test's, bit for bit.
__device__ __forceinline__ unsigned long long f32_to_f64_bits(float x)      // x positive, normal
{
    const unsigned u = __float_as_uint(x);
    const unsigned long long e = (unsigned long long)(((u >> 23) & 0xffu) - 127u + 1023u);
    return (e << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
}

__global__ void diag_f32_kernel(int n, const double *d, float *df)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = d[i];
    df[i] = (x >= 1e-18 && x <= 1e18) ? (float)x : __int_as_float(0x7fc00000);
}

// Eq. 7 for entry e = (i, j), j != i: the FP32 bounds decide it unless |a_ij| is within a
// relative 2e-6 of the FP32 threshold (compared as bit patterns: FP64-pipe work avoided); then
// the literal FP64 test, every operation rounded (the oracle's arithmetic, R1)
__device__ __forceinline__ bool strong_entry(double vij, const double *d, int i, int j, float dfi, float dfj,
                                             double theta, float thf)
{
    if (theta == 0.0) return true;
    const unsigned long long ab = (unsigned long long)__double_as_longlong(vij) & 0x7fffffffffffffffull;
    const float t32 = __fmul_rn(thf, __fsqrt_rn(__fmul_rn(dfi, dfj)));
    if (thf >= 1e-6f && t32 >= 1e-30f && t32 <= 1e30f && ab < 0x7ff0000000000000ull) {
        if (ab > f32_to_f64_bits(__fmul_rn(t32, 1.000002f))) return true;
        if (ab < f32_to_f64_bits(__fmul_rn(t32, 0.999998f))) return false;
    }
    const double prod = __dmul_rn(d[i], d[j]);
    const double thr = __dmul_rn(theta, __dsqrt_rn(prod));
    return fabs(vij) >= thr;
}

// A block per tile of consecutive rows (tile_rows: about kStrEntries entries, at most kStrRows
// rows): its threads stride over the rows' entries (contiguous),
// each entry's row found by binary search in the block's row pointers (shared memory), so loads
// and the flag stores are coalesced however long or short the rows; kept counts per row by
// shared-memory atomics.
constexpr int kStrRows = 256;         // rows of a tile at most
constexpr int kStrEntries = 4096;     // entries a tile aims at (16 a thread)

// rows per tile for a matrix of n rows and nnz entries (and at least kStrBlocks tiles: the
// stalled coarse levels' few thousand rows would otherwise fill a fifth of the multiprocessors)
constexpr int kStrBlocks = 608;
int tile_rows(int n, int64_t nnz)
{
    const double avg = n > 0 ? (double)nnz / n : 1.0;
    const int spread = (int)(((int64_t)n + kStrBlocks - 1) / kStrBlocks);
    return std::max(1, std::min(std::min(kStrRows, spread), (int)(kStrEntries / std::max(avg, 1.0))));
}
// (scnt, when given: each row's count of strong entries, the strong graph's row lengths)
__global__ void __launch_bounds__(256) strength_kernel(int n, const int *rp, const int *ci, const double *v,
                                                       const double *d, const float *df, double theta, float thf,
                                                       uint8_t *strong, uint8_t *removed, int *kept, int rpb,
                                                       int *scnt)
{
    __shared__ int srp[kStrRows + 1];
    __shared__ float sdf[kStrRows];
    __shared__ int skept[kStrRows], sstr[kStrRows];
    const int r0 = blockIdx.x * rpb;
    if (r0 >= n) return;
    const int nr = min(n - r0, rpb);
    for (int t = threadIdx.x; t <= nr; t += blockDim.x) srp[t] = rp[r0 + t];
    for (int t = threadIdx.x; t < nr; t += blockDim.x) {
        sdf[t] = df[r0 + t];
        skept[t] = 0;
        sstr[t] = 0;
    }
    __syncthreads();
    const int k0 = srp[0], k1 = srp[nr];
    for (int e = k0 + (int)threadIdx.x; e < k1; e += blockDim.x) {
        // the row of e: the last t with srp[t] <= e (an empty row shares its start with the next)
        int lo = 0, hi = nr - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (srp[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        const int i = r0 + lo;
        const int j = ci[e];
        bool st = false, rem = false;
        if (j != i) {
            st = strong_entry(v[e], d, i, j, sdf[lo], df[j], theta, thf);
            rem = !st;
        }
        strong[e] = st ? 1 : 0;
        removed[e] = rem ? 1 : 0;
        if (!rem) atomicAdd(&skept[lo], 1);
        if (st) atomicAdd(&sstr[lo], 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nr; t += blockDim.x) {
        kept[r0 + t] = skept[t];
        if (scnt) scnt[r0 + t] = sstr[t];
    }
}

cudaError_t strength(const DevCsr &A, const double *d, double theta, uint8_t *strong, uint8_t *removed,
                     int *kept, cudaStream_t s, int *strong_cnt)
{
    if (A.n == 0) return cudaSuccess;
    float *df = nullptr;
    AMG_CUDA_TRY(cudaMallocAsync(&df, sizeof(float) * (size_t)A.n, s));
    diag_f32_kernel<<<grid_for(A.n, 256), 256, 0, s>>>(A.n, d, df); note_launch();
    const int rpb = tile_rows(A.n, A.nnz);
    strength_kernel<<<(A.n + rpb - 1) / rpb, 256, 0, s>>>(A.n, A.rp, A.ci, A.v, d, df, theta, (float)theta, strong,
                                                          removed, kept, rpb, strong_cnt);
    note_launch();
    cudaError_t e = cudaGetLastError();
    cudaError_t e2 = cudaFreeAsync(df, s);
    return e != cudaSuccess ? e : e2;
}

// ------------------------------------------------------------------------------------ nonsymmetric operators
// Thread per row: entry (i, j) is strong when its own test or that of (j, i) (found by binary
// search in row j) passed; removed and the kept count follow.
__global__ void symmetrize_kernel(int n, const int *rp, const int *ci, const uint8_t *own, uint8_t *strong,
                                  uint8_t *removed, int *kept)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int nk = 0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const int j = ci[e];
        bool st = false;
        if (j != i) {
            st = own[e] != 0;
            if (!st) {
                int lo = rp[j], hi = rp[j + 1] - 1;
                while (lo <= hi) {
                    const int mid = (lo + hi) >> 1;
                    const int c = ci[mid];
                    if (c == i) { st = own[mid] != 0; break; }
                    if (c < i) lo = mid + 1; else hi = mid - 1;
                }
            }
        }
        strong[e] = st ? 1 : 0;
        const bool rem = j != i && !st;
        removed[e] = rem ? 1 : 0;
        nk += rem ? 0 : 1;
    }
    kept[i] = nk;
}

cudaError_t symmetrize_strength(const DevCsr &A, const uint8_t *own, uint8_t *strong, uint8_t *removed, int *kept,
                                cudaStream_t s)
{
    if (A.n == 0) return cudaSuccess;
    symmetrize_kernel<<<grid_for(A.n, 128), 128, 0, s>>>(A.n, A.rp, A.ci, own, strong, removed, kept); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ distance Laplacian, §3.1
// Thread per row, entries in ascending column order: off the diagonal L_ij = -1 / |x_i - x_j|
// (the distance from the squared coordinate differences summed in coordinate order), on it
// the sum of the 1 / |x_i - x_j|, so every row sums to zero.  Each operation is rounded.
__global__ void dlap_kernel(int n, const int *rp, const int *ci, const double *X, int dim, double *L, double *Ld,
                            int *bad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double diag = 0.0;
    int dpos = -1;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const int j = ci[e];
        if (j == i) {
            dpos = e;
            continue;
        }
        double d2 = 0.0;
        for (int c = 0; c < dim; ++c) {
            const double dx = __dsub_rn(X[(size_t)i * dim + c], X[(size_t)j * dim + c]);
            d2 = __dadd_rn(d2, __dmul_rn(dx, dx));
        }
        const double dist = __dsqrt_rn(d2);
        if (!(dist > 0.0)) atomicAdd(bad, 1);
        const double w = __ddiv_rn(1.0, dist);
        L[e] = -w;
        diag = __dadd_rn(diag, w);
    }
    if (dpos >= 0) L[dpos] = diag;
    Ld[i] = diag;
}

cudaError_t distance_laplacian(const DevCsr &A, const double *X, int dim, double *L, double *Ld, int *bad,
                               cudaStream_t s)
{
    if (A.n == 0) return cudaSuccess;
    dlap_kernel<<<grid_for(A.n, 128), 128, 0, s>>>(A.n, A.rp, A.ci, X, dim, L, Ld, bad); note_launch();
    return cudaGetLastError();
}

// thread per aggregate: members in ascending order, sum then divide by the member count
__global__ void coarse_coords_kernel(int nagg, const int *mstart, const int *members, const double *X, int dim,
                                     double *Xc)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nagg) return;
    const int b = mstart[a], e = mstart[a + 1];
    for (int c = 0; c < dim; ++c) {
        double sum = 0.0;
        for (int t = b; t < e; ++t) sum = __dadd_rn(sum, X[(size_t)members[t] * dim + c]);
        Xc[(size_t)a * dim + c] = __ddiv_rn(sum, (double)(e - b));
    }
}

cudaError_t coarse_coords(int nagg, const int *mstart, const int *members, const double *X, int dim, double *Xc,
                          cudaStream_t s)
{
    if (nagg == 0) return cudaSuccess;
    coarse_coords_kernel<<<grid_for(nagg, 128), 128, 0, s>>>(nagg, mstart, members, X, dim, Xc); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ strong graph
// Row tiles as in strength_kernel: a block per tile of rows, threads strided over the rows'
// entries (coalesced however short the rows), each entry's row by binary search in the block's
// row pointers in shared memory.
__device__ __forceinline__ int tile_row(int e, const int *srp, int nr)
{
    int lo = 0, hi = nr - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (srp[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// cnt[i] = strong entries of row i
__global__ void __launch_bounds__(256) sg_count_kernel(int n, const int *rp, const uint8_t *strong, int *cnt, int rpb)
{
    __shared__ int srp[kStrRows + 1];
    __shared__ int sc[kStrRows];
    const int r0 = blockIdx.x * rpb;
    if (r0 >= n) return;
    const int nr = min(n - r0, rpb);
    for (int t = threadIdx.x; t <= nr; t += blockDim.x) srp[t] = rp[r0 + t];
    for (int t = threadIdx.x; t < nr; t += blockDim.x) sc[t] = 0;
    __syncthreads();
    for (int e = srp[0] + (int)threadIdx.x; e < srp[nr]; e += blockDim.x)
        if (strong[e]) atomicAdd(&sc[tile_row(e, srp, nr)], 1);
    __syncthreads();
    for (int t = threadIdx.x; t < nr; t += blockDim.x) cnt[r0 + t] = sc[t];
}

// gci[grp[i] ...]: row i's strong columns in ascending order.  The block's entries go in chunks
// of four a thread (consecutive); a block-wide scan of the threads' strong counts gives each
// entry its rank among the strong entries of the block so far, and the rank of its row's first
// entry (recorded when that entry's chunk was scanned) turns it into the rank within the row.
constexpr int kFillPer = 4;
__global__ void __launch_bounds__(256) sg_fill_kernel(int n, const int *rp, const int *ci, const uint8_t *strong,
                                                      const int *grp, int *gci, int rpb)
{
    __shared__ int srp[kStrRows + 1];
    __shared__ int rowbase[kStrRows];
    __shared__ int wsum[8];
    __shared__ int chunk_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = blockIdx.x * rpb;
    if (r0 >= n) return;
    const int nr = min(n - r0, rpb);
    for (int t = threadIdx.x; t <= nr; t += blockDim.x) srp[t] = rp[r0 + t];
    if (threadIdx.x == 0) chunk_base = 0;
    __syncthreads();
    const int k0 = srp[0], k1 = srp[nr];
    for (int c0 = k0; c0 < k1; c0 += kFillPer * (int)blockDim.x) {
        const int e0 = c0 + kFillPer * (int)threadIdx.x;
        int lo = e0 < k1 ? tile_row(e0, srp, nr) : 0;
        bool st[kFillPer];
        int rows_of[kFillPer], mine = 0;
#pragma unroll
        for (int u = 0; u < kFillPer; ++u) {
            const int e = e0 + u;
            st[u] = false;
            rows_of[u] = lo;
            if (e < k1) {
                while (srp[lo + 1] <= e) ++lo;     // rows advance with e (empty rows skipped)
                rows_of[u] = lo;
                st[u] = strong[e] != 0;
            }
            mine += st[u];
        }
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int rank = chunk_base + incl - mine;
        for (int w = 0; w < warp; ++w) rank += wsum[w];
        // the first entry of a row records the block's strong count before it
        {
            int r = rank;
#pragma unroll
            for (int u = 0; u < kFillPer; ++u) {
                const int e = e0 + u;
                if (e < k1 && e == srp[rows_of[u]]) rowbase[rows_of[u]] = r;
                r += st[u];
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kFillPer; ++u) {
            if (st[u]) {
                gci[grp[r0 + rows_of[u]] + rank - rowbase[rows_of[u]]] = ci[e0 + u];
                ++rank;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < 8; ++w) t += wsum[w];
            chunk_base += t;
        }
        __syncthreads();
    }
}

cudaError_t strong_graph_counts(const DevCsr &A, const uint8_t *strong, int *cnt, cudaStream_t s)
{
    if (A.n == 0) return cudaSuccess;
    const int rpb = tile_rows(A.n, A.nnz);
    sg_count_kernel<<<(A.n + rpb - 1) / rpb, 256, 0, s>>>(A.n, A.rp, strong, cnt, rpb); note_launch();
    return cudaGetLastError();
}

cudaError_t strong_graph_fill(const DevCsr &A, const uint8_t *strong, const int *grp, int *gci, cudaStream_t s)
{
    if (A.n == 0) return cudaSuccess;
    const int rpb = tile_rows(A.n, A.nnz);
    sg_fill_kernel<<<(A.n + rpb - 1) / rpb, 256, 0, s>>>(A.n, A.rp, A.ci, strong, grp, gci, rpb); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ aggregation
// Roots: the greedy maximal independent set of the distance-2 strong graph in decreasing
// priority.  Computed by synchronous rounds on 64-bit tuples (state << 62 | priority) with
// state OUT = 0 < UNDECIDED = 1 < ROOT = 2: two rounds of max-propagation over the strong
// graph give each vertex the largest tuple within distance 2; an undecided vertex whose own
// tuple is that maximum becomes a root, one that sees a root becomes OUT.  A vertex joins
// only when every higher-priority vertex within distance 2 is OUT, and leaves only next to a
// root, so the result is the sequential greedy set.
constexpr unsigned long long kStUndec = 1ULL << 62;
constexpr unsigned long long kStRoot = 2ULL << 62;
constexpr unsigned long long kPrioMask = (1ULL << 62) - 1ULL;

__global__ void mis_init_kernel(int n, uint64_t seed, int level, unsigned long long *t0)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) t0[i] = kStUndec | agg_priority(seed, level, i);
}

// one sub-warp of 8 lanes per vertex (no early exit: the shuffles use the full warp).  Only the
// vertices flagged in act: the ones an undecided vertex reads (itself and its neighbours).
__global__ void mis_max_kernel(int n, const int *grp, const int *gci, const unsigned long long *in,
                               unsigned long long *out, const uint8_t *act)
{
    const int sub = threadIdx.x & 7;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const bool valid = i < n && act[i];
    unsigned long long m = (valid && sub == 0) ? in[i] : 0ULL;
    if (valid) {
        for (int e = grp[i] + sub; e < grp[i + 1]; e += 8) {
            unsigned long long t = in[gci[e]];
            m = t > m ? t : m;
        }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        unsigned long long t = __shfl_down_sync(kFull, m, o, 8);
        m = t > m ? t : m;
    }
    if (valid && sub == 0) out[i] = m;
}

// (a vertex still undecided flags itself and its neighbours in act_next: the next round's max
// is needed there only)
__global__ void mis_decide_kernel(int n, const int *grp, const int *gci, const unsigned long long *t1,
                                  unsigned long long *t0, int *undecided, uint8_t *act_next)
{
    const int sub = threadIdx.x & 7;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const bool valid = i < n;
    int und = 0;
    // a decided vertex (root or out) never changes again: no need for its neighbourhood
    const unsigned long long own0 = valid ? t0[i] : 0ULL;
    const bool open = valid && (own0 >> 62) == 1ULL;
    unsigned long long m = (open && sub == 0) ? t1[i] : 0ULL;
    if (open) {
        for (int e = grp[i] + sub; e < grp[i + 1]; e += 8) {
            unsigned long long t = t1[gci[e]];
            m = t > m ? t : m;
        }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        unsigned long long t = __shfl_down_sync(kFull, m, o, 8);
        m = t > m ? t : m;
    }
    if (open && sub == 0) {
        const unsigned long long own = own0;
        if (m == own) t0[i] = kStRoot | (own & kPrioMask);
        else if ((m >> 62) == 2ULL) t0[i] = own & kPrioMask;
        else und = 1;
    }
    const int still = __shfl_sync(kFull, und, 0, 8);
    if (still) {
        if (sub == 0) act_next[i] = 1;
        for (int e = grp[i] + sub; e < grp[i + 1]; e += 8) act_next[gci[e]] = 1;
    }
    // block-level count of still-undecided vertices
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    if (und) atomicAdd(&cnt, 1);
    __syncthreads();
    if (threadIdx.x == 0 && cnt) atomicAdd(undecided, cnt);
}

__global__ void mis_roots_kernel(int n, const unsigned long long *t0, uint8_t *root, int *rootflag_int)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = (t0[i] >> 62) == 2ULL;
    root[i] = (uint8_t)r;
    rootflag_int[i] = r;
}

// Join 1: a non-root adjacent to roots joins the adjacent root of largest priority.
__global__ void join1_kernel(int n, const int *grp, const int *gci, const uint8_t *root, uint64_t seed, int level,
                             int *join1)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (root[i]) { join1[i] = i; return; }
    int best = -1;
    uint64_t bk = 0;
    for (int e = grp[i]; e < grp[i + 1]; ++e) {
        int u = gci[e];
        if (root[u]) {
            uint64_t k = agg_priority(seed, level, u);
            if (best < 0 || k > bk) { best = u; bk = k; }
        }
    }
    join1[i] = best;
}

// Join 2: a vertex not yet assigned joins through the step-1 neighbour whose root has the
// largest priority (reads only step-1 results).
__global__ void join2_kernel(int n, const int *grp, const int *gci, const uint8_t *root, const int *join1,
                             uint64_t seed, int level, int *rootof)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = join1[i];
    if (r < 0) {
        uint64_t bk = 0;
        for (int e = grp[i]; e < grp[i + 1]; ++e) {
            int u = gci[e];
            int ru = join1[u];
            if (!root[u] && ru >= 0) {
                uint64_t k = agg_priority(seed, level, ru);
                if (r < 0 || k > bk) { r = ru; bk = k; }
            }
        }
    }
    rootof[i] = r;
}

__global__ void agg_ids_kernel(int n, const int *rootof, const int *rootid, int *agg, int *bad)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = rootof[i];
    if (r < 0) { agg[i] = -1; atomicAdd(bad, 1); }
    else agg[i] = rootid[r];
}

cudaError_t aggregate_mis2(int n, const int *grp, const int *gci, uint64_t seed, int level, AggWork w, int *agg,
                           uint8_t *root, int *nagg_host, int *rounds_host, cudaStream_t s)
{
    *nagg_host = 0;
    *rounds_host = 0;
    if (n == 0) return cudaSuccess;
    const int tb = 256;
    mis_init_kernel<<<grid_for(n, tb), tb, 0, s>>>(n, seed, level, w.t0); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    // rounds go in pairs between looks at the undecided count (a round after the last decision
    // changes nothing), which halves the host round trips
    // which vertices need the next round's max (every vertex in the first round)
    uint8_t *act = nullptr;
    AMG_CUDA_TRY(cudaMallocAsync(&act, 2 * (size_t)n, s));
    struct Release {
        uint8_t *p; cudaStream_t s;
        ~Release() { cudaFreeAsync(p, s); }
    } release{act, s};
    uint8_t *act_cur = act, *act_next = act + n;
    AMG_CUDA_TRY(cudaMemsetAsync(act_cur, 1, (size_t)n, s));
    int h_und = 1, rounds = 0;
    while (h_und > 0) {
        if (rounds >= 10000) return cudaErrorLaunchFailure;   // cannot happen: each round decides >= 1 vertex
        for (int q = 0; q < 2; ++q) {
            if (q == 1) AMG_CUDA_TRY(cudaMemsetAsync(w.counter, 0, sizeof(int), s));
            AMG_CUDA_TRY(cudaMemsetAsync(act_next, 0, (size_t)n, s));
            mis_max_kernel<<<grid_for((int64_t)n * 8, tb), tb, 0, s>>>(n, grp, gci, w.t0, w.t1, act_cur); note_launch();
            mis_decide_kernel<<<grid_for((int64_t)n * 8, tb), tb, 0, s>>>(n, grp, gci, w.t1, w.t0, w.counter,
                                                                          act_next); note_launch();
            std::swap(act_cur, act_next);
        }
        AMG_CUDA_TRY(cudaGetLastError());
        AMG_CUDA_TRY(cudaMemcpyAsync(&h_und, w.counter, sizeof(int), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        rounds += 2;
    }
    *rounds_host = rounds;
    // root flags and ids (exclusive scan of root flags -> aggregate numbers by increasing root index)
    int *rootid = w.rootof;           // n+1 ints of scratch (rootof reused below after ids)
    mis_roots_kernel<<<grid_for(n, tb), tb, 0, s>>>(n, w.t0, root, rootid); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    AMG_CUDA_TRY(scan_exclusive(rootid, rootid, n, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(nagg_host, rootid + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    join1_kernel<<<grid_for(n, tb), tb, 0, s>>>(n, grp, gci, root, seed, level, w.join1); note_launch();
    // agg[] temporarily holds the root of each vertex
    join2_kernel<<<grid_for(n, tb), tb, 0, s>>>(n, grp, gci, root, w.join1, seed, level, agg); note_launch();
    AMG_CUDA_TRY(cudaMemsetAsync(w.counter + 1, 0, sizeof(int), s));
    // agg_ids reads rootof (in agg) and writes agg: use join1 as the staging copy
    AMG_CUDA_TRY(cudaMemcpyAsync(w.join1, agg, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    agg_ids_kernel<<<grid_for(n, tb), tb, 0, s>>>(n, w.join1, rootid, agg, w.counter + 1); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    int bad = 0;
    AMG_CUDA_TRY(cudaMemcpyAsync(&bad, w.counter + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (bad) return cudaErrorInvalidValue;
    return cudaSuccess;
}

// ------------------------------------------------------------------------------------ aggregate members
__global__ void member_count_kernel(int n, const int *agg, int *cnt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[agg[i]], 1);
}
__global__ void member_scatter_kernel(int n, const int *agg, const int *mstart, int *fill, int *tmp)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        int a = agg[i];
        int p = mstart[a] + atomicAdd(&fill[a], 1);
        tmp[p] = i;
    }
}
// one warp per aggregate: place each member at its rank (members are distinct)
__global__ void member_sort_kernel(int nagg, const int *mstart, const int *tmp, int *members)
{
    const int lane = threadIdx.x & 31;
    const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (a >= nagg) return;
    const int b = mstart[a], m = mstart[a + 1] - b;
    for (int t = lane; t < m; t += 32) {
        int v = tmp[b + t], rank = 0;
        for (int u = 0; u < m; ++u) rank += tmp[b + u] < v;
        members[b + rank] = v;
    }
}

cudaError_t aggregate_members(int n, int nagg, const int *agg, int *mstart, int *members, int *fill, cudaStream_t s)
{
    AMG_CUDA_TRY(cudaMemsetAsync(mstart, 0, sizeof(int) * (size_t)(nagg + 1), s));
    if (n == 0) return cudaSuccess;
    member_count_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, agg, mstart); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    AMG_CUDA_TRY(scan_exclusive(mstart, mstart, nagg, s));
    AMG_CUDA_TRY(cudaMemsetAsync(fill, 0, sizeof(int) * (size_t)nagg, s));
    int *tmp = nullptr;
    AMG_CUDA_TRY(cudaMallocAsync(&tmp, sizeof(int) * (size_t)n, s));
    member_scatter_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, agg, mstart, fill, tmp); note_launch();
    member_sort_kernel<<<grid_for((int64_t)nagg * 32, 256), 256, 0, s>>>(nagg, mstart, tmp, members); note_launch();
    cudaError_t e = cudaGetLastError();
    cudaError_t e2 = cudaFreeAsync(tmp, s);
    return e != cudaSuccess ? e : e2;
}

// sum of B^2 over members in ascending order, then sqrt
__global__ void agg_norm_kernel(int nagg, const int *mstart, const int *members, const double *B, double *nrm,
                                int *bad)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nagg) return;
    double ss = 0.0;
    for (int t = mstart[a]; t < mstart[a + 1]; ++t) {
        double b = B[members[t]];
        ss = ss + b * b;
    }
    if (!(ss > 0.0)) atomicAdd(bad, 1);
    nrm[a] = __dsqrt_rn(ss);
}

cudaError_t aggregate_norms(int nagg, const int *mstart, const int *members, const double *B, double *nrm,
                            int *bad, cudaStream_t s)
{
    if (nagg == 0) return cudaSuccess;
    agg_norm_kernel<<<grid_for(nagg, 128), 128, 0, s>>>(nagg, mstart, members, B, nrm, bad); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ §2.5 sparsification
// One warp per aggregate a with root rho.  For each distinct aggregate c != a reached by a
// weak entry of rho's row and holding no strong neighbour of rho, count the strong links
// from a's non-root members into c; a single link is marked for dropping.
__global__ void sprsfy_kernel(int nagg, const int *rp, const int *ci, const uint8_t *strong, const int *agg,
                              const int *mstart, const int *members, const uint8_t *root, uint8_t *drop)
{
    const int lane = threadIdx.x & 31;
    const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (a >= nagg) return;
    const int mb = mstart[a], me = mstart[a + 1];
    // the root of aggregate a
    int rho = -1;
    for (int t = mb + lane; t < me; t += 32)
        if (root[members[t]]) rho = members[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rho = max(rho, __shfl_xor_sync(kFull, rho, o));
    if (rho < 0) return;
    const int rb = rp[rho], re = rp[rho + 1];
    for (int e = rb; e < re; ++e) {
        int j = ci[e];
        if (j == rho || strong[e]) continue;
        int c = agg[j];
        if (c == a) continue;
        // first weak entry of rho's row reaching c, and no strong neighbour of rho in c
        int skip = 0;
        for (int f = rb + lane; f < re; f += 32) {
            int jf = ci[f];
            if (jf == rho) continue;
            if (agg[jf] != c) continue;
            if (strong[f]) skip = 1;
            else if (f < e) skip = 1;
        }
        if (__any_sync(kFull, skip)) continue;
        int cnt = 0, link = -1;
        for (int t = mb + lane; t < me; t += 32) {
            int v = members[t];
            if (v == rho) continue;
            for (int f = rp[v]; f < rp[v + 1]; ++f) {
                int w = ci[f];
                if (w != v && strong[f] && agg[w] == c) { ++cnt; link = f; }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cnt += __shfl_xor_sync(kFull, cnt, o);
            link = max(link, __shfl_xor_sync(kFull, link, o));
        }
        if (cnt == 1 && lane == 0) drop[link] = 1;
    }
}

// removed |= drop on (v, w) and on (w, v); kept counts recomputed afterwards
__global__ void sprsfy_symm_kernel(int n, const int *rp, const int *ci, const uint8_t *drop, uint8_t *removed)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    for (int e = rp[v]; e < rp[v + 1]; ++e) {
        if (!drop[e]) continue;
        removed[e] = 1;
        int w = ci[e];
        int lo = rp[w], hi = rp[w + 1] - 1;
        while (lo <= hi) {
            int mid = (lo + hi) >> 1;
            int c = ci[mid];
            if (c == v) { removed[mid] = 1; break; }
            if (c < v) lo = mid + 1; else hi = mid - 1;
        }
    }
}

__global__ void kept_count_kernel(int n, const int *rp, const int *ci, const uint8_t *removed, int *kept)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = 0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) k += (ci[e] == i) || !removed[e];
    kept[i] = k;
}

cudaError_t sprsfy(const DevCsr &A, const uint8_t *strong, const int *agg, const uint8_t *root, int nagg,
                   const int *mstart, const int *members, uint8_t *drop, uint8_t *removed, int *kept,
                   cudaStream_t s)
{
    if (A.n == 0) return cudaSuccess;
    AMG_CUDA_TRY(cudaMemsetAsync(drop, 0, (size_t)A.nnz, s));
    sprsfy_kernel<<<grid_for((int64_t)nagg * 32, 128), 128, 0, s>>>(nagg, A.rp, A.ci, strong, agg, mstart,
                                                                     members, root, drop); note_launch();
    sprsfy_symm_kernel<<<grid_for(A.n, 256), 256, 0, s>>>(A.n, A.rp, A.ci, drop, removed); note_launch();
    kept_count_kernel<<<grid_for(A.n, 256), 256, 0, s>>>(A.n, A.rp, A.ci, removed, kept); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ filtered matrix
// One warp per row.  Standard (Eq. 6): removed entries summed in ascending column order and
// added to a_ii.  OffLmp: Algorithm 2 with these readings -- r = 0 takes the diagonal branch;
// D(A_i) counts every off-diagonal of A; a_ii <= 0 falls back to Eq. (6); with K- empty all of
// r goes to K+ if K+ is not empty, else the row is left unlumped; the diagonal share is the
// largest r in [0, |rhat|] keeping (N - r)/(a_ii - r) <= t (N = -kappa- - rhat,
// t = tau D(A_i)): |rhat| if N <= a_ii, min(|rhat|, (t a_ii - N)/(t - 1)) if a_ii < N <= t a_ii,
// and 0 if N > t a_ii.
// The smoothing diagonal: Dbar_ii, or (1Norm) Dtilde_ii = sum_j |Abar_ij| raised to
// 4 s_i / (3 (1 - sigma)) (2 s_i for sigma = 1/3) and set to 1 for an all-zero row (Eq. 9-11).
enum { LUMP_DIAG = 0, LUMP_KPLUS = 1, LUMP_DIAG_KMINUS = 2, LUMP_KPLUS_NEG = 3, LUMP_SKIPPED = 4,
       LUMP_FALLBACK = 5 };

// Every sum runs in ascending column order: left to right from 0 over a row of at most
// kFilterLong stored positions, one thread per row (the per-row FP64 work is a handful of
// additions per stored entry, and GB300's FP64 pipe makes redundant per-lane sums expensive).
// A longer row (a stalled coarse level holds rows of thousands) is summed by segments of
// kFilterLong positions, each left to right from 0, the segment sums then added left to right
// (the oracle's reading for long rows): one warp per row, lane q summing segment q, so the row's
// time is one segment's chain of dependent additions instead of the whole row's.
constexpr int kFilterLong = 256;

// x > 0 and x < 0 decided on the bit pattern with integer instructions instead of FP64
// comparisons (GB300's FP64 pipe is the filter's bound); the same answers for every double,
// zeros, infinities and NaN included
__device__ __forceinline__ bool dpos(double x)
{
    const long long b = __double_as_longlong(x);
    return b > 0 && b <= 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool dneg(double x)
{
    const long long b = __double_as_longlong(x);
    const long long m = b & 0x7fffffffffffffffLL;
    return b < 0 && m != 0 && m <= 0x7ff0000000000000LL;
}

// The row's outcome from its sums (Eq. 6, or Algorithm 2 with offlmp)
struct FilterOutcome {
    int flag = LUMP_DIAG;
    double new_diag = 0.0, fplus = 1.0, fminus = 1.0;
    bool zero_plus = false;
};

__device__ __forceinline__ FilterOutcome filter_outcome(double aii, double r, double kp, double km, double offabs,
                                                        int nkp, int nkm, int offlmp, double tau)
{
    FilterOutcome o;
    o.new_diag = aii + r;     // Eq. (6)
    if (!offlmp) return o;
    if (!(aii > 0.0)) {
        o.flag = LUMP_FALLBACK;
    } else if (r >= 0.0) {
        o.flag = LUMP_DIAG;
    } else if (fabs(r) <= kp) {
        o.flag = LUMP_KPLUS;
        o.new_diag = aii;
        o.fplus = 1.0 + r / kp;
    } else if (nkm == 0) {
        o.new_diag = aii;
        if (nkp > 0) {
            o.flag = LUMP_KPLUS_NEG;
            o.fplus = 1.0 + r / kp;
        } else {
            o.flag = LUMP_SKIPPED;
        }
    } else {
        o.flag = LUMP_DIAG_KMINUS;
        o.zero_plus = true;
        double rhat = r + kp;
        double t_bound = tau * (offabs / fabs(aii));
        double N = -km - rhat;
        double mag = -rhat;
        double rstar;
        if (N <= aii) {
            rstar = mag;
        } else if (N <= t_bound * aii) {
            double rmax = (t_bound * aii - N) / (t_bound - 1.0);
            rstar = rmax < mag ? rmax : mag;
        } else {
            rstar = 0.0;
        }
        o.new_diag = aii - rstar;
        o.fminus = 1.0 + (rhat + rstar) / km;
    }
    return o;
}

// a kept entry's new value (j != i): the factor chosen first, then one multiply (the lanes of a
// warp take different sign branches; one FP64 instruction instead of one per branch)
__device__ __forceinline__ double filter_kept_value(double val, const FilterOutcome &o, int offlmp)
{
    if (!offlmp || o.flag == LUMP_FALLBACK) return val;
    const bool pos = dpos(val);
    const bool scale_p = pos && !o.zero_plus && (o.flag == LUMP_KPLUS || o.flag == LUMP_KPLUS_NEG);
    const bool scale_m = !pos && o.flag == LUMP_DIAG_KMINUS && dneg(val);
    const double prod = val * (scale_p ? o.fplus : o.fminus);
    return pos && o.zero_plus ? 0.0 : (scale_p || scale_m) ? prod : val;
}

// Adds val to the one of r (removed entries), kp (kept positive) and km (kept negative) that
// takes it, through a single FP64 addition on the selected sum
__device__ __forceinline__ void filter_accumulate(double val, bool rem, int offlmp, double &r, double &kp, double &km,
                                                  int &nkp, int &nkm)
{
    const bool p = !rem && offlmp && dpos(val);
    const bool m = !rem && offlmp && !p && dneg(val);
    const double nx = (rem ? r : p ? kp : km) + val;
    r = rem ? nx : r;
    kp = p ? nx : kp;
    km = m ? nx : km;
    nkp += p;
    nkm += m;
}

// the smoothing diagonal from the row's sums
__device__ __forceinline__ double filter_dsm(int onenorm, double sigma, double dsum, double ssum, int has_diag,
                                             double new_diag, int *zero_diag)
{
    double dd;
    if (onenorm) {
        double f = (sigma == 1.0 / 3.0) ? 2.0 : 4.0 / (3.0 * (1.0 - sigma));
        dd = dsum;
        if (dd == 0.0) dd = 1.0;
        if (dd < f * ssum) dd = f * ssum;
    } else {
        dd = has_diag ? new_diag : 0.0;
        if (dd == 0.0) atomicAdd(zero_diag, 1);
    }
    return dd;
}

__device__ __forceinline__ void filter_row(int i, int b, int e_end, const int *ci, const double *v,
                                           const uint8_t *removed, int offlmp, double tau, int onenorm, double sigma,
                                           const int *brp, int *bci, double *bv, double *Dsm, uint8_t *lumpflag,
                                           int *zero_diag)
{
    // pass 1: row sums in ascending order
    double r = 0.0, kp = 0.0, km = 0.0, offabs = 0.0, aii = 0.0;
    int nkp = 0, nkm = 0, has_diag = 0;
    // (unrolled: eight entries' loads in flight at once; the sums stay in order)
#pragma unroll 8
    for (int e = b; e < e_end; ++e) {
        const int j = ci[e];
        const double val = v[e];
        if (j == i) {
            aii = val;
            has_diag = 1;
            continue;
        }
        if (offlmp) offabs = offabs + fabs(val);
        filter_accumulate(val, removed[e] != 0, offlmp, r, kp, km, nkp, nkm);
    }
    const FilterOutcome o = filter_outcome(aii, r, kp, km, offabs, nkp, nkm, offlmp, tau);
    // pass 2: the kept entries, and the 1-norm sums over them in ascending order
    int out = brp[i];
    double dsum = 0.0, ssum = 0.0;
#pragma unroll 8
    for (int e = b; e < e_end; ++e) {
        const int j = ci[e];
        double nv;
        if (j == i) nv = o.new_diag;
        else if (!removed[e]) nv = filter_kept_value(v[e], o, offlmp);
        else continue;
        bci[out] = j;
        bv[out] = nv;
        ++out;
        if (onenorm) {
            dsum = dsum + fabs(nv);
            ssum = ssum + nv;
        }
    }
    lumpflag[i] = (uint8_t)o.flag;
    Dsm[i] = filter_dsm(onenorm, sigma, dsum, ssum, has_diag, o.new_diag, zero_diag);
}

// Row i of more than kFilterLong entries, by one warp: segment q (positions q kFilterLong ..
// (q + 1) kFilterLong - 1 of A's row in pass 1, of Abar's row for the 1-norm sums) on lane
// q mod 32; every lane folds the segment sums of each group of 32 in segment order (shuffles),
// so all lanes hold the row's sums.
__device__ void filter_long_row(int i, int b, int e_end, const int *ci, const double *v, const uint8_t *removed,
                                int offlmp, double tau, int onenorm, double sigma, const int *brp, int *bci,
                                double *bv, double *Dsm, uint8_t *lumpflag, int *zero_diag)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nseg = (e_end - b + kFilterLong - 1) / kFilterLong;
    double r = 0.0, kp = 0.0, km = 0.0, offabs = 0.0, aii = 0.0;
    int nkp = 0, nkm = 0, has_diag = 0;
    for (int q0 = 0; q0 < nseg; q0 += 32) {
        const int q = q0 + lane;
        double sr = 0.0, skp = 0.0, skm = 0.0, soff = 0.0, da = 0.0;
        int cp = 0, cm = 0, hd = 0;
        if (q < nseg) {
            const int e0 = b + q * kFilterLong, e1 = min(e_end, e0 + kFilterLong);
            // (unrolled: a lane's loads of eight entries in flight at once; the sums stay in order)
#pragma unroll 8
            for (int e = e0; e < e1; ++e) {
                const int j = ci[e];
                const double val = v[e];
                if (j == i) {
                    da = val;
                    hd = 1;
                    continue;
                }
                if (offlmp) soff = soff + fabs(val);
                filter_accumulate(val, removed[e] != 0, offlmp, sr, skp, skm, cp, cm);
            }
        }
        const int last = min(32, nseg - q0);
        for (int t = 0; t < last; ++t) {
            const double a1 = __shfl_sync(full, sr, t), a2 = __shfl_sync(full, skp, t);
            const double a3 = __shfl_sync(full, skm, t), a4 = __shfl_sync(full, soff, t);
            if (q0 + t == 0) {
                r = a1; kp = a2; km = a3; offabs = a4;
            } else {
                r = r + a1; kp = kp + a2; km = km + a3; offabs = offabs + a4;
            }
        }
        nkp += __reduce_add_sync(full, cp);
        nkm += __reduce_add_sync(full, cm);
        const unsigned dm = __ballot_sync(full, hd);
        if (dm) {
            aii = __shfl_sync(full, da, __ffs(dm) - 1);
            has_diag = 1;
        }
    }
    const FilterOutcome o = filter_outcome(aii, r, kp, km, offabs, nkp, nkm, offlmp, tau);
    // pass 2: each lane writes the kept entries of its segments at their places in Abar's row
    int base = brp[i];
    for (int q0 = 0; q0 < nseg; q0 += 32) {
        const int q = q0 + lane;
        const int e0 = b + q * kFilterLong, e1 = q < nseg ? min(e_end, e0 + kFilterLong) : e0;
        int kept = 0;
#pragma unroll 8
        for (int e = e0; e < e1; ++e) kept += (ci[e] == i || !removed[e]);
        int incl = kept;
#pragma unroll
        for (int o2 = 1; o2 < 32; o2 <<= 1) {
            const int y = __shfl_up_sync(full, incl, o2);
            if (lane >= o2) incl += y;
        }
        int out = base + incl - kept;
#pragma unroll 8
        for (int e = e0; e < e1; ++e) {
            const int j = ci[e];
            double nv;
            if (j == i) nv = o.new_diag;
            else if (!removed[e]) nv = filter_kept_value(v[e], o, offlmp);
            else continue;
            bci[out] = j;
            bv[out] = nv;
            ++out;
        }
        base += __shfl_sync(full, incl, 31);
    }
    // the 1-norm sums over Abar's row, by segments of its positions
    double dsum = 0.0, ssum = 0.0;
    if (onenorm) {
        __threadfence_block();
        __syncwarp();
        const int ab = brp[i], ae = base;
        const int nseg2 = (ae - ab + kFilterLong - 1) / kFilterLong;
        for (int q0 = 0; q0 < nseg2; q0 += 32) {
            const int q = q0 + lane;
            double sd = 0.0, ss = 0.0;
            if (q < nseg2) {
                const int e0 = ab + q * kFilterLong, e1 = min(ae, e0 + kFilterLong);
#pragma unroll 8
                for (int e = e0; e < e1; ++e) {
                    const double nv = bv[e];
                    sd = sd + fabs(nv);
                    ss = ss + nv;
                }
            }
            const int last = min(32, nseg2 - q0);
            for (int t = 0; t < last; ++t) {
                const double a1 = __shfl_sync(full, sd, t), a2 = __shfl_sync(full, ss, t);
                if (q0 + t == 0) {
                    dsum = a1; ssum = a2;
                } else {
                    dsum = dsum + a1; ssum = ssum + a2;
                }
            }
        }
    }
    if (lane == 0) {
        lumpflag[i] = (uint8_t)o.flag;
        Dsm[i] = filter_dsm(onenorm, sigma, dsum, ssum, has_diag, o.new_diag, zero_diag);
    }
}

__global__ void filter_kernel(int n, const int *rp, const int *ci, const double *v, const uint8_t *removed,
                              int offlmp, double tau, int onenorm, double sigma, const int *brp, int *bci,
                              double *bv, double *Dsm, uint8_t *lumpflag, int *zero_diag, int *long_rows,
                              int *nlong)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = rp[i], e_end = rp[i + 1];
    if (e_end - b > kFilterLong) {
        long_rows[atomicAdd(nlong, 1)] = i;
        return;
    }
    filter_row(i, b, e_end, ci, v, removed, offlmp, tau, onenorm, sigma, brp, bci, bv, Dsm, lumpflag, zero_diag);
}

__global__ void filter_long_kernel(const int *rp, const int *ci, const double *v, const uint8_t *removed, int offlmp,
                                   double tau, int onenorm, double sigma, const int *brp, int *bci, double *bv,
                                   double *Dsm, uint8_t *lumpflag, int *zero_diag, const int *long_rows,
                                   const int *nlong)
{
    const int warps = (int)((gridDim.x * (size_t)blockDim.x) >> 5);
    for (int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5); w < *nlong; w += warps) {
        const int i = long_rows[w];
        filter_long_row(i, rp[i], rp[i + 1], ci, v, removed, offlmp, tau, onenorm, sigma, brp, bci, bv, Dsm, lumpflag,
                        zero_diag);
    }
}

cudaError_t filter(const DevCsr &A, const uint8_t *removed, int offlmp, double tau, int onenorm, double sigma,
                   DevCsr &Abar, double *Dsm, uint8_t *lumpflag, int *zero_diag, cudaStream_t s)
{
    if (A.n == 0) return cudaSuccess;
    int *lr = nullptr;
    AMG_CUDA_TRY(cudaMallocAsync(&lr, sizeof(int) * ((size_t)A.n + 1), s));
    cudaError_t e = cudaMemsetAsync(lr, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        filter_kernel<<<grid_for(A.n, 128), 128, 0, s>>>(A.n, A.rp, A.ci, A.v, removed, offlmp, tau, onenorm, sigma,
                                                         Abar.rp, Abar.ci, Abar.v, Dsm, lumpflag, zero_diag, lr + 1,
                                                         lr); note_launch();
        filter_long_kernel<<<2 * kReduceBlocks, 128, 0, s>>>(A.rp, A.ci, A.v, removed, offlmp, tau, onenorm, sigma,
                                                             Abar.rp, Abar.ci, Abar.v, Dsm, lumpflag, zero_diag, lr + 1,
                                                             lr); note_launch();
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaFreeAsync(lr, s);
    return e != cudaSuccess ? e : e2;
}

// ------------------------------------------------------------------------------------ smoothed prolongator
// Row i of P = (I - omega D^-1 Abar) Pt has the aggregates of Abar's row-i columns, sorted;
// (Abar Pt)_ic sums Abar_ik B_k over those k (ascending) with agg(k) = c.
constexpr int kSmoothLocal = 64;    // distinct columns a thread keeps locally

// distinct aggregates of the row's columns (thread per row; integer work only)
__global__ void smooth_count_kernel(int n, const int *rp, const int *ci, const int *agg, int *cnt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = rp[i], m = rp[i + 1] - b;
    int distinct = 0;
    for (int t = 0; t < m; ++t) {
        const int c = agg[ci[b + t]];
        bool first = true;
        for (int u = 0; u < t; ++u)
            if (agg[ci[b + u]] == c) { first = false; break; }
        distinct += first;
    }
    cnt[i] = distinct;
}

// Thread per row: the terms Abar_ik B_k are accumulated (one fused multiply-add each) in
// ascending k into the slot of agg(k)
// (a local list in first-seen order), then the list is sorted by column and written as
// P_ic = Pt_ic - (omega / D_i) (Abar Pt)_ic.  Rows with more than kSmoothLocal distinct
// columns are listed for the warp kernel below.
__global__ void smooth_fill_kernel(int n, const int *rp, const int *ci, const double *v, const int *agg,
                                   const double *B, const double *Dsm, const double *omega_dev, const int *prp,
                                   int *pci, double *pv, int *wide_rows, int *nwide)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nd = prp[i + 1] - prp[i];
    if (nd > kSmoothLocal) {
        wide_rows[atomicAdd(nwide, 1)] = i;
        return;
    }
    int cols[kSmoothLocal];
    double acc[kSmoothLocal];
    int cnt = 0;
    const int b = rp[i], e = rp[i + 1];
    for (int t = b; t < e; ++t) {
        const int k = ci[t];
        const int c = agg[k];
        int p = 0;
        while (p < cnt && cols[p] != c) ++p;
        if (p == cnt) { cols[cnt] = c; acc[cnt] = 0.0; ++cnt; }
        acc[p] = __fma_rn(v[t], B[k], acc[p]);
    }
    // insertion sort by column
    for (int a = 1; a < cnt; ++a) {
        int c = cols[a];
        double x = acc[a];
        int q = a - 1;
        while (q >= 0 && cols[q] > c) { cols[q + 1] = cols[q]; acc[q + 1] = acc[q]; --q; }
        cols[q + 1] = c;
        acc[q + 1] = x;
    }
    const double scale = *omega_dev / Dsm[i];
    const int ai = agg[i];
    const double bi = B[i];
    const int o = prp[i];
    for (int a = 0; a < cnt; ++a) {
        const double pt = (cols[a] == ai) ? bi : 0.0;
        pci[o + a] = cols[a];
        pv[o + a] = pt - scale * acc[a];
    }
}

// one warp per wide row (listed by smooth_fill_kernel): each distinct column's sum runs
// sequentially over the row in ascending order
__global__ void smooth_fill_wide_kernel(const int *rows, const int *nrows, const int *rp, const int *ci,
                                        const double *v, const int *agg, const double *B, const double *Dsm,
                                        const double *omega_dev, const int *prp, int *pci, double *pv)
{
    const int lane = threadIdx.x & 31;
    const int total = *nrows;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += (gridDim.x * blockDim.x) >> 5) {
    const int i = rows[w];
    const int b = rp[i], m = rp[i + 1] - b;
    const double scale = *omega_dev / Dsm[i];
    const int ai = agg[i];
    const double bi = B[i];
    for (int t = lane; t < m; t += 32) {
        int c = agg[ci[b + t]];
        bool first = true;
        for (int u = 0; u < t; ++u)
            if (agg[ci[b + u]] == c) { first = false; break; }
        if (!first) continue;
        int rank = 0;
        double acc = 0.0;
        for (int u = 0; u < m; ++u) {
            int k = ci[b + u];
            int cu = agg[k];
            if (cu == c) {
                acc = __fma_rn(v[b + u], B[k], acc);
            } else if (cu < c) {
                bool fu = true;
                for (int q = 0; q < u; ++q)
                    if (agg[ci[b + q]] == cu) { fu = false; break; }
                rank += fu;
            }
        }
        double pt = (c == ai) ? bi : 0.0;
        int p = prp[i] + rank;
        pci[p] = c;
        pv[p] = pt - scale * acc;
    }
    }
}

cudaError_t smooth_counts(const DevCsr &Abar, const int *agg, int *cnt, cudaStream_t s)
{
    if (Abar.n == 0) return cudaSuccess;
    smooth_count_kernel<<<grid_for(Abar.n, 128), 128, 0, s>>>(Abar.n, Abar.rp, Abar.ci, agg, cnt); note_launch();
    return cudaGetLastError();
}

cudaError_t smooth_fill(const DevCsr &Abar, const int *agg, const double *B, const double *Dsm,
                        const double *omega_dev, DevCsr &P, cudaStream_t s)
{
    if (Abar.n == 0) return cudaSuccess;
    int *wide = nullptr;
    AMG_CUDA_TRY(cudaMallocAsync(&wide, sizeof(int) * ((size_t)Abar.n + 1), s));
    int *nwide = wide + Abar.n;
    cudaError_t e = cudaMemsetAsync(nwide, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        smooth_fill_kernel<<<grid_for(Abar.n, 128), 128, 0, s>>>(Abar.n, Abar.rp, Abar.ci, Abar.v, agg, B, Dsm,
                                                                 omega_dev, P.rp, P.ci, P.v, wide, nwide); note_launch();
        // the wide rows (normally none): one warp each, grid-stride over the list
        smooth_fill_wide_kernel<<<grid_for((int64_t)Abar.n * 32, 256, 608), 256, 0, s>>>(
            wide, nwide, Abar.rp, Abar.ci, Abar.v, agg, B, Dsm, omega_dev, P.rp, P.ci, P.v); note_launch();
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaFreeAsync(wide, s);
    return e != cudaSuccess ? e : e2;
}

// ------------------------------------------------------------------------------------ Algorithm 3
// One thread per row of the unit-basis P.  The working set w starts as the nonzero entries
// (inw, one byte per stored entry); each pass pins the smallest entry if negative and then
// the largest if above one (ties to the lowest position) and shares the pinned excess
// equally over w; the loop runs while any entry is below 0 or above 1, at most m + 1 passes.
// A negative row sum, a row sum above |w|, or w emptying with a nonzero excess give the
// tentative row; a zero row sum gives the zero row.
// Outcome: 0 kept or clipped, 1 zero row, 2 tentative row.
__global__ void constrain_kernel(int n, const int *rp, const int *ci, double *pv, const int *agg, const double *B,
                                 uint8_t *inw_all, uint8_t *cflag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = rp[i], m = rp[i + 1] - b;
    double *p = pv + b;
    uint8_t *inw = inw_all + b;
    double s = 0.0;
    int nw = 0;
    for (int k = 0; k < m; ++k) {
        s = s + p[k];
        inw[k] = p[k] != 0.0;
        nw += inw[k];
    }
    int outcome = 0;
    if (s < 0.0 || s > (double)nw) {
        outcome = 2;
    } else if (s == 0.0) {
        for (int k = 0; k < m; ++k) p[k] = 0.0;
        cflag[i] = 1;
        return;
    } else {
        for (int pass = 0; pass <= m; ++pass) {
            int kmin = 0, kmax = 0;
            for (int k = 1; k < m; ++k) {
                if (p[k] < p[kmin]) kmin = k;
                if (p[k] > p[kmax]) kmax = k;
            }
            if (!(p[kmin] < 0.0 || p[kmax] > 1.0)) break;
            double delta = 0.0;
            if (p[kmin] < 0.0) {
                delta = delta + p[kmin];
                p[kmin] = 0.0;
                if (inw[kmin]) { inw[kmin] = 0; --nw; }
            }
            if (p[kmax] > 1.0) {
                delta = delta + (p[kmax] - 1.0);
                p[kmax] = 1.0;
                if (inw[kmax]) { inw[kmax] = 0; --nw; }
            }
            if (nw == 0) {
                if (delta != 0.0) outcome = 2;
                break;
            }
            double share = delta / (double)nw;
            for (int k = 0; k < m; ++k)
                if (inw[k]) p[k] = p[k] + share;
        }
    }
    if (outcome == 2) {
        for (int k = 0; k < m; ++k) p[k] = (ci[b + k] == agg[i]) ? B[i] : 0.0;
    }
    cflag[i] = (uint8_t)outcome;
}

cudaError_t constrain(DevCsr &P, const int *agg, const double *B, uint8_t *cflag, cudaStream_t s)
{
    if (P.n == 0) return cudaSuccess;
    uint8_t *inw = nullptr;
    AMG_CUDA_TRY(cudaMallocAsync(&inw, (size_t)(P.nnz > 0 ? P.nnz : 1), s));
    constrain_kernel<<<grid_for(P.n, 128), 128, 0, s>>>(P.n, P.rp, P.ci, P.v, agg, B, inw, cflag); note_launch();
    cudaError_t e = cudaGetLastError();
    cudaError_t e2 = cudaFreeAsync(inw, s);
    return e != cudaSuccess ? e : e2;
}

__global__ void scale_columns_kernel(int64_t nnz, const int *ci, double *v, const double *nrm)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        v[e] = v[e] / nrm[ci[e]];
}

cudaError_t scale_columns(DevCsr &P, const double *nrm, cudaStream_t s)
{
    if (P.nnz == 0) return cudaSuccess;
    scale_columns_kernel<<<grid_for(P.nnz, 256, 8192), 256, 0, s>>>(P.nnz, P.ci, P.v, nrm); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ transpose
__global__ void tr_count_kernel(int64_t nnz, const int *ci, int *cnt)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[ci[e]], 1);
}
__global__ void tr_scatter_kernel(int n, const int *rp, const int *ci, const double *v, const int *trp, int *fill,
                                  int *tci, double *tv)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        int c = ci[e];
        int p = trp[c] + atomicAdd(&fill[c], 1);
        tci[p] = i;
        tv[p] = v[e];
    }
}
// one warp per row of the transpose: each entry goes to its rank (row indices are distinct)
__global__ void tr_sort_kernel(int nrow, const int *trp, const int *tci, const double *tv, int *oci, double *ov)
{
    const int lane = threadIdx.x & 31;
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= nrow) return;
    const int b = trp[r], m = trp[r + 1] - b;
    for (int t = lane; t < m; t += 32) {
        int key = tci[b + t], rank = 0;
        for (int u = 0; u < m; ++u) rank += tci[b + u] < key;
        oci[b + rank] = key;
        ov[b + rank] = tv[b + t];
    }
}

cudaError_t transpose_counts(const DevCsr &P, int *cnt, cudaStream_t s)
{
    AMG_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)(P.ncol + 1), s));
    if (P.nnz == 0) return cudaSuccess;
    tr_count_kernel<<<grid_for(P.nnz, 256, 8192), 256, 0, s>>>(P.nnz, P.ci, cnt); note_launch();
    return cudaGetLastError();
}

cudaError_t transpose_fill(const DevCsr &P, DevCsr &R, int *fill, cudaStream_t s)
{
    if (P.nnz == 0) return cudaSuccess;
    AMG_CUDA_TRY(cudaMemsetAsync(fill, 0, sizeof(int) * (size_t)R.n, s));
    int *tci = nullptr;
    double *tv = nullptr;
    AMG_CUDA_TRY(cudaMallocAsync(&tci, sizeof(int) * (size_t)P.nnz, s));
    cudaError_t e = cudaMallocAsync(&tv, sizeof(double) * (size_t)P.nnz, s);
    if (e == cudaSuccess) {
        tr_scatter_kernel<<<grid_for(P.n, 256), 256, 0, s>>>(P.n, P.rp, P.ci, P.v, R.rp, fill, tci, tv); note_launch();
        tr_sort_kernel<<<grid_for((int64_t)R.n * 32, 256), 256, 0, s>>>(R.n, R.rp, tci, tv, R.ci, R.v); note_launch();
        e = cudaGetLastError();
        cudaError_t e2 = cudaFreeAsync(tv, s);
        if (e == cudaSuccess) e = e2;
    }
    cudaError_t e3 = cudaFreeAsync(tci, s);
    return e != cudaSuccess ? e : e3;
}

// ------------------------------------------------------------------------------------ power method
// x0_i = 2 u_i - 1, u_i the i-th output of the SplitMix64 stream started at stream_seed;
// x = x0 / ||x0||; each sweep y = D^-1 A x, lambda = x . y; between sweeps x = y / ||y||.
// (The sweeps multiply by 1/D_i where the oracle divides by D_i: the estimate agrees to
// rounding.)
uint64_t power_stream_seed(uint64_t seed, int level, int purpose)
{
    return seed ^ ((uint64_t)(level + 1) << 48) ^ ((uint64_t)purpose << 56);
}

__global__ void power_init_kernel(int n, uint64_t s0, double *x)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t z = splitmix_mix(s0 + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ULL);
    double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    x[i] = 2.0 * u - 1.0;
}

// q[1] = 1 / sqrt(q[0])
__global__ void rsqrt_slot_kernel(double *q) { q[1] = 1.0 / __dsqrt_rn(q[0]); }

__global__ void reciprocal_kernel(int n, const double *D, double *inv)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) inv[i] = 1.0 / D[i];
}

cudaError_t power_lambda(const DevCsr &A, const SpmvPlan &plan, const double *D, int sweeps, uint64_t stream_seed,
                         double *x, double *y, double *partial, double *scal, double *lambda_dev, cudaStream_t s)
{
    const int n = A.n;
    if (n == 0) return cudaMemsetAsync(lambda_dev, 0, sizeof(double), s);
    // D^-1 once (the sweeps multiply by it: an FP64 division per row and sweep is a long
    // instruction sequence on this GPU)
    double *invD = nullptr;
    AMG_CUDA_TRY(cudaMallocAsync(&invD, sizeof(double) * (size_t)n, s));
    struct Release {
        double *p; cudaStream_t s;
        ~Release() { cudaFreeAsync(p, s); }
    } release{invD, s};
    reciprocal_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, D, invD); note_launch();
    // x0 and x0 . x0; each sweep then works on the unnormalised iterate, its squared norm and
    // the reciprocal of its norm (scal[3..4] and scal[5..6] alternate), which equals
    // normalising before every sweep
    power_init_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, stream_seed, x); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    AMG_CUDA_TRY(dot(x, x, n, partial, scal + 3, s));
    rsqrt_slot_kernel<<<1, 1, 0, s>>>(scal + 3); note_launch();
    // ticket counter of the SpMV's fixed-order reduction (scal[7], zero)
    unsigned *counter = reinterpret_cast<unsigned *>(scal + 7);
    AMG_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(double), s));
    double *a = x, *b = y;
    for (int k = 0; k < sweeps; ++k) {
        AMG_CUDA_TRY(spmv_power(A, plan, invD, a, scal + 3 + 2 * (k & 1), b, scal + 5 - 2 * (k & 1), partial,
                                lambda_dev, counter, s, k + 1 == sweeps));
        std::swap(a, b);
    }
    return cudaGetLastError();
}

__global__ void omega_kernel(const double *lambda, double *omega)
{
    *omega = 4.0 / (3.0 * *lambda);
}

cudaError_t omega_from_lambda(const double *lambda_dev, double *omega_dev, cudaStream_t s)
{
    omega_kernel<<<1, 1, 0, s>>>(lambda_dev, omega_dev); note_launch();
    return cudaGetLastError();
}

__global__ void invert_diag_kernel(const double *d, double *inv, float *invf, int n, int *zero)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double di = d[i];
    if (di == 0.0) atomicAdd(zero, 1);
    double r = 1.0 / di;
    inv[i] = r;
    if (invf) invf[i] = (float)r;
}

cudaError_t invert_diag(const double *d, double *inv, float *invf, int n, int *zero, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    invert_diag_kernel<<<grid_for(n, 256), 256, 0, s>>>(d, inv, invf, n, zero); note_launch();
    return cudaGetLastError();
}

}  // namespace amgk
