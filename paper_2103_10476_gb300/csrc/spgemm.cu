// spgemm.cu -- two-phase (symbolic count, numeric fill) hash SpGEMM C = A B, one warp per
// row of A, hash tables in shared memory (global memory for rows whose table does not fit).
//
// Numeric order: the products of a row are taken 32 at a time in (k, j) order; the terms that
// land in one slot are applied in that order, each as c = fma(a_ik, b_kj, c), so every c_ij is
// accumulated over ascending k from 0 with one rounding per term, independent of the hash
// layout (the same arithmetic as a sequential Gustavson product with fma).
//
// Rows are binned by table size so each launch uses one size: the symbolic phase by an
// upper bound (min(products, columns)), the numeric phase by the exact count.
#include <algorithm>
#include <climits>
#include <functional>
#include <mutex>
#include <stdio.h>
#include <string>

#include <vector>

#include "amg_internal.cuh"

namespace amgk {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kMinTable = 32;
constexpr int kMaxSharedSym = 8192;     // symbolic: 4 bytes per slot
constexpr int kMaxSharedNum = 4096;     // numeric: 12 bytes per slot
constexpr int kCapTable = 1024;         // symbolic: the first table of a row whose bound asks more
constexpr int kCapRows = 32768;         // ... in products of at least this many rows (a second round
                                        // costs a host round trip that small products do not repay)
constexpr int kNumBins = 11;            // 32 .. 8192, the global bin and the segmented rows
constexpr int kGlobalBin = 9;
constexpr int kSegBin = 10;             // numeric phase: rows of A of more than kSegLen entries
constexpr int kSegLen = 256;
constexpr int kChainProducts = 32768;      // rows with more products take the chain path (B wide) ...
constexpr int kSegProducts = 4096;         // ... or with more than these, the segment kernels (B narrow)
constexpr int kSmemBudget = 96 * 1024;

__device__ __forceinline__ unsigned hash_col(int j) { return (unsigned)j * 2654435761u; }

// Insert key j into keys[0..S); returns the slot, and whether it was new.  Bounded probing.
__device__ __forceinline__ int hash_insert(int *keys, int S, int j, bool &fresh, int *overflow)
{
    unsigned slot = hash_col(j) & (unsigned)(S - 1);
    fresh = false;
    for (int probe = 0; probe < S; ++probe) {
        int cur = keys[slot];
        if (cur == j) return (int)slot;
        if (cur == -1) {
            int old = atomicCAS(&keys[slot], -1, j);
            if (old == -1) { fresh = true; return (int)slot; }
            if (old == j) return (int)slot;
        }
        slot = (slot + 1) & (unsigned)(S - 1);
    }
    atomicAdd(overflow, 1);
    return -1;
}

__device__ __forceinline__ int bin_of_table(int S)
{
    int b = 0;
    while ((kMinTable << b) < S) ++b;
    return b;
}

__device__ __forceinline__ int table_for(int64_t need)
{
    int S = kMinTable;
    while ((int64_t)S < 2 * need && S < (1 << 28)) S <<= 1;
    return S;
}

// ------------------------------------------------------------------------------------ bounds and bins
// per-block histogram of bins, one global atomic per (block, bin)
__device__ __forceinline__ void bin_count_block(int b, bool valid, int *binCount)
{
    __shared__ int hist[kNumBins];
    if (threadIdx.x < kNumBins) hist[threadIdx.x] = 0;
    __syncthreads();
    if (valid) atomicAdd(&hist[b], 1);
    __syncthreads();
    if (threadIdx.x < kNumBins && hist[threadIdx.x]) atomicAdd(&binCount[threadIdx.x], hist[threadIdx.x]);
}

// Row i's product count (an upper bound of its entries), one thread per row; a row of more than
// 64 entries (stalled levels hold rows of thousands) is counted by its whole warp instead, the
// warp taking its long rows one after another.  (ubstats, when given: [0] the most products of a
// row, [1] all products, warp-reduced first.)
// dense_above: rows of more products go to the global bin (whose symbolic kernel is then a
// block per row with dense counters over B's columns; B narrow enough for them)
// cap_table > 0: a row whose bound asks for a larger table goes to the bin of cap_table slots
// first (tsize keeps the bound's size; ubstats[2] counts such rows): the symbolic phase counts
// it there unless it holds more than cap_table / 2 columns, and sends it back to its own bin then
__global__ void ub_kernel(int n, const int *arp, const int *aci, const int *brp, int ncolB, int *bin, int *binCount,
                          int *tsize, unsigned long long *ubstats = nullptr, long long dense_above = LLONG_MAX,
                          int cap_table = 0)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = i < n;
    const int r0 = valid ? arp[i] : 0, r1 = valid ? arp[i + 1] : 0;
    const bool longrow = r1 - r0 > 64;
    long long ub = 0;
    if (valid && !longrow)
        for (int e = r0; e < r1; ++e) {
            const int k = aci[e];
            ub += brp[k + 1] - brp[k];
        }
    unsigned m = __ballot_sync(kFullMask, longrow);
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const int sb = __shfl_sync(kFullMask, r0, src), se = __shfl_sync(kFullMask, r1, src);
        long long part = 0;
        for (int e = sb + lane; e < se; e += 32) {
            const int k = aci[e];
            part += brp[k + 1] - brp[k];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFullMask, part, o);
        if (lane == src) ub = part;
    }
    int b = 0;
    bool capped = false;
    if (valid) {
        const int64_t need = ub < ncolB ? ub : ncolB;
        const int S = table_for(need);
        if (ub > dense_above) {
            b = kGlobalBin;
        } else if (cap_table > 0 && S > cap_table) {
            b = bin_of_table(cap_table);
            capped = true;
        } else {
            b = S > kMaxSharedSym ? kGlobalBin : bin_of_table(S);
        }
        bin[i] = b;
        tsize[i] = S;
    }
    if (ubstats && cap_table > 0) {
        const unsigned cm = __ballot_sync(kFullMask, capped);
        if (lane == 0 && cm) atomicAdd(&ubstats[2], (unsigned long long)__popc(cm));
    }
    if (ubstats) {
        unsigned long long mx = (unsigned long long)ub, sm = (unsigned long long)ub;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(kFullMask, mx, o);
            mx = y > mx ? y : mx;
            sm += __shfl_xor_sync(kFullMask, sm, o);
        }
        if (lane == 0 && sm) {
            atomicMax(&ubstats[0], mx);
            atomicAdd(&ubstats[1], sm);
        }
    }
    bin_count_block(b, valid, binCount);
}

// numeric bins by the exact row counts.  kSegBin takes the rows of A with more than kSegLen
// entries and, with seg_wide (B narrow enough for the segment kernels' dense accumulator), the
// rows too long for a shared-memory table as well (*segmax: the longest row of A among them).
__global__ void exact_bin_kernel(int n, const int *crp, const int *arp, int *bin, int *binCount, int *tsize,
                                 int *segmax, int seg_wide, const int *aci = nullptr, const int *brp = nullptr)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int b = 0;
    if (i < n) {
        const int alen = arp[i + 1] - arp[i];
        const int64_t cnt = crp[i + 1] - crp[i];
        const int S = table_for(cnt);
        // (with aci and brp: also the rows of more than kSegProducts products, which a warp on a
        // hash table would walk 32 products at a time)
        bool many = false;
        if (seg_wide && aci && alen <= kSegLen) {
            int64_t prod = 0;
            for (int e = arp[i]; e < arp[i + 1]; ++e) prod += brp[aci[e] + 1] - brp[aci[e]];
            many = prod > kSegProducts;
        }
        if (alen > kSegLen || (seg_wide && (S > kMaxSharedNum || many))) {
            b = kSegBin;
            tsize[i] = 0;
            atomicMax(segmax, alen);
        } else {
            b = S > kMaxSharedNum ? kGlobalBin : bin_of_table(S);
            tsize[i] = S;
        }
        bin[i] = b;
    }
    bin_count_block(b, i < n, binCount);
}

// The symbolic phase's second round: a capped row that stopped (count -1) to the bin of its
// own table size; every other row to kSegBin, which the symbolic phase does not run
__global__ void retry_bin_kernel(int n, const int *ccnt, const int *tsize, int *bin, int *binCount)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int b = kSegBin;
    if (i < n) {
        if (ccnt[i] < 0) {
            const int S = tsize[i];
            b = S > kMaxSharedSym ? kGlobalBin : bin_of_table(S);
        }
        bin[i] = b;
    }
    bin_count_block(b, i < n, binCount);
}

// rows to their bin's segment: block-local ranks, one global atomic per (block, bin)
__global__ void bin_scatter_kernel(int n, const int *bin, const int *binStart, int *binFill, int *perm)
{
    __shared__ int hist[kNumBins], base[kNumBins];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (threadIdx.x < kNumBins) hist[threadIdx.x] = 0;
    __syncthreads();
    int b = 0, local = 0;
    if (i < n) {
        b = bin[i];
        local = atomicAdd(&hist[b], 1);
    }
    __syncthreads();
    if (threadIdx.x < kNumBins && hist[threadIdx.x])
        base[threadIdx.x] = binStart[threadIdx.x] + atomicAdd(&binFill[threadIdx.x], hist[threadIdx.x]);
    __syncthreads();
    if (i < n) perm[base[b] + local] = i;
}

// global-bin table offsets: tsize of listed rows, scanned on the host side of the launch
__global__ void gather_tsize_kernel(int cnt, const int *rows, const int *tsize, int *out)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < cnt) out[t] = tsize[rows[t]];
}

// ------------------------------------------------------------------------------------ symbolic
// The products of row i, a_ik b_kj for k ascending and j ascending within B's row k, are
// enumerated 32 at a time: lane l of a batch holds product number base + l.  For a chunk of
// up to 32 entries of A's row, each lane holds one entry and the running (inclusive) count
// of B-row lengths; a product's entry is found by binary search over those counts.
struct ProductBatch {
    int j;          // column of the product (valid lanes)
    double a, b;    // a_ik and b_kj
    bool valid;
};

template <bool WITH_VALUES>
__device__ __forceinline__ ProductBatch product_at(int q, int total, int incl, int excl, int fb, double a,
                                                   const int *bci, const double *bv)
{
    ProductBatch pb;
    pb.valid = q < total;
    int lo = 0, hi = 31;
#pragma unroll
    for (int step = 0; step < 5; ++step) {
        int mid = (lo + hi) >> 1;
        int v = __shfl_sync(kFullMask, incl, mid);
        if (v > q) hi = mid; else lo = mid + 1;
    }
    const int owner = lo;
    const int off = q - __shfl_sync(kFullMask, excl, owner);
    const int f = __shfl_sync(kFullMask, fb, owner) + off;
    const double ao = WITH_VALUES ? __shfl_sync(kFullMask, a, owner) : 0.0;
    pb.j = pb.valid ? bci[f] : -1;
    pb.a = ao;
    pb.b = (WITH_VALUES && pb.valid) ? bv[f] : 0.0;
    return pb;
}

// capped: the row's bound asked for a larger table; it stops, with ccnt[i] = -1, once it holds
// more than S / 2 columns (a batch adds at most 32, so the table never fills)
__device__ void symbolic_row(int i, const int *arp, const int *aci, const int *brp, const int *bci, int *keys, int S,
                             int *ccnt, int *overflow, bool capped = false)
{
    const int lane = threadIdx.x & 31;
    for (int t = lane; t < S; t += 32) keys[t] = -1;
    __syncwarp();
    int mine = 0, held = 0;
    const int ae = arp[i + 1];
    for (int eb = arp[i]; eb < ae; eb += 32) {
        const int e = eb + lane;
        int len = 0, fb = 0;
        if (e < ae) {
            const int k = aci[e];
            fb = brp[k];
            len = brp[k + 1] - fb;
        }
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFullMask, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(kFullMask, incl, 31);
        const int excl = incl - len;
        for (int qb = 0; qb < total; qb += 32) {
            ProductBatch pb = product_at<false>(qb + lane, total, incl, excl, fb, 0.0, bci, nullptr);
            bool fresh = false;
            if (pb.valid) {
                hash_insert(keys, S, pb.j, fresh, overflow);
                mine += fresh;
            }
            if (capped) {
                held += __popc(__ballot_sync(kFullMask, fresh));
                if (held > S / 2) {
                    if (lane == 0) ccnt[i] = -1;
                    __syncwarp();
                    return;
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(kFullMask, mine, o);
    if (lane == 0) ccnt[i] = mine;
    __syncwarp();
}

// tsize (when given): the rows' own table sizes; a row of a larger one is capped here
template <int S>
__global__ void symbolic_shared_kernel(int cnt, const int *rows, const int *arp, const int *aci, const int *brp,
                                       const int *bci, int *ccnt, int *overflow, const int *tsize)
{
    extern __shared__ int smem_keys[];
    const int w = threadIdx.x >> 5;
    const int row_slot = blockIdx.x * (blockDim.x >> 5) + w;
    if (row_slot >= cnt) return;
    const int i = rows[row_slot];
    symbolic_row(i, arp, aci, brp, bci, smem_keys + w * S, S, ccnt, overflow, tsize && tsize[i] > S);
}

__global__ void symbolic_global_kernel(int cnt, const int *rows, const int *toff, const int *tsize, int *gkeys,
                                       const int *arp, const int *aci, const int *brp, const int *bci, int *ccnt,
                                       int *overflow)
{
    const int row_slot = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row_slot >= cnt) return;
    int i = rows[row_slot];
    symbolic_row(i, arp, aci, brp, bci, gkeys + toff[row_slot], tsize[i], ccnt, overflow);
}

// ------------------------------------------------------------------------------------ numeric
// The row's entries of C from the occupied slots of its table, in ascending column order: each
// column's rank is the number of occupied columns below it, read from a bitmap over B's columns
// (bm: `words` words, then as many exclusive prefix counts of the words).  Two passes over the
// table instead of a compaction and a sort.  Returns false (and counts an overflow) when the
// number of columns differs from the symbolic phase's.
__device__ bool emit_by_bitmap(const int *keys, const double *vals, int S, unsigned *bm, int words, int out, int nc,
                               int *cci, double *cv, int *overflow)
{
    const int lane = threadIdx.x & 31;
    int *pre = reinterpret_cast<int *>(bm + words);
    for (int w = lane; w < words; w += 32) bm[w] = 0u;
    __syncwarp();
    for (int t = lane; t < S; t += 32) {
        const int key = keys[t];
        if (key != -1) atomicOr(&bm[key >> 5], 1u << (key & 31));
    }
    __syncwarp();
    const int per = (words + 31) >> 5;
    const int w0 = lane * per, w1 = min(words, w0 + per);
    int c = 0;
    for (int w = w0; w < w1; ++w) c += __popc(bm[w]);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFullMask, incl, o);
        if (lane >= o) incl += y;
    }
    int run = incl - c;
    for (int w = w0; w < w1; ++w) {
        pre[w] = run;
        run += __popc(bm[w]);
    }
    const int total = __shfl_sync(kFullMask, incl, 31);
    __syncwarp();
    if (total != nc) {
        if (lane == 0) atomicAdd(overflow, 1);
        return false;
    }
    for (int t = lane; t < S; t += 32) {
        const int key = keys[t];
        if (key != -1) {
            const int w = key >> 5;
            const int rank = pre[w] + __popc(bm[w] & ((1u << (key & 31)) - 1u));
            cci[out + rank] = key;
            cv[out + rank] = vals[t];
        }
    }
    return true;
}

// bm: nullptr, or the warp's bitmap over B's columns (words words + words prefix counts), which
// then orders the row's entries (emit_by_bitmap)
__device__ void numeric_row(int i, const int *arp, const int *aci, const double *av, const int *brp, const int *bci,
                            const double *bv, int *keys, double *vals, int S, const int *crp, int *cci, double *cv,
                            int *overflow, unsigned *bm = nullptr, int words = 0)
{
    const int lane = threadIdx.x & 31;
    for (int t = lane; t < S; t += 32) { keys[t] = -1; vals[t] = 0.0; }
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    const int ae = arp[i + 1];
    for (int eb = arp[i]; eb < ae; eb += 32) {
        const int e = eb + lane;
        int len = 0, fb = 0;
        double a = 0.0;
        if (e < ae) {
            const int k = aci[e];
            a = av[e];
            fb = brp[k];
            len = brp[k + 1] - fb;
        }
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFullMask, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(kFullMask, incl, 31);
        const int excl = incl - len;
        for (int qb = 0; qb < total; qb += 32) {
            ProductBatch pb = product_at<true>(qb + lane, total, incl, excl, fb, a, bci, bv);
            int slot = -1;
            if (pb.valid) {
                bool fresh;
                slot = hash_insert(keys, S, pb.j, fresh, overflow);
            }
            // products of one column inside the batch are added in lane (= product) order
            const bool act = pb.valid && slot >= 0;
            const unsigned same = __match_any_sync(kFullMask, act ? slot : -1 - lane);
            const unsigned rank = act ? (unsigned)__popc(same & lt) : 0u;
            const unsigned maxrank = __reduce_max_sync(kFullMask, rank);
            for (unsigned r = 0; r <= maxrank; ++r) {
                if (act && rank == r) vals[slot] = __fma_rn(pb.a, pb.b, vals[slot]);
                __syncwarp();
            }
        }
    }
    if (bm) {
        emit_by_bitmap(keys, vals, S, bm, words, crp[i], crp[i + 1] - crp[i], cci, cv, overflow);
        return;
    }
    // compact occupied slots to the front, in slot order
    int base = 0;
    for (int t0 = 0; t0 < S; t0 += 32) {
        int t = t0 + lane;
        int key = keys[t];
        double val = vals[t];
        bool occ = key != -1;
        unsigned m = __ballot_sync(kFullMask, occ);
        __syncwarp();
        if (occ) {
            int p = base + __popc(m & ((1u << lane) - 1u));
            keys[p] = key;
            vals[p] = val;
        }
        base += __popc(m);
        __syncwarp();
    }
    const int cnt = base;
    const int out = crp[i];
    if (cnt != crp[i + 1] - out) {
        if (lane == 0) atomicAdd(overflow, 1);
        return;
    }
    if (cnt <= 512) {
        // each entry to its rank (columns are distinct)
        for (int t = lane; t < cnt; t += 32) {
            int key = keys[t], rank = 0;
            for (int u = 0; u < cnt; ++u) rank += keys[u] < key;
            cci[out + rank] = key;
            cv[out + rank] = vals[t];
        }
        return;
    }
    // bitonic sort of the first P2 slots (padding keys above every column)
    int P2 = 1;
    while (P2 < cnt) P2 <<= 1;
    for (int t = cnt + lane; t < P2; t += 32) { keys[t] = 0x7fffffff; vals[t] = 0.0; }
    __syncwarp();
    for (int kk = 2; kk <= P2; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int t = lane; t < P2; t += 32) {
                int ixj = t ^ jj;
                if (ixj > t) {
                    bool asc = (t & kk) == 0;
                    int a = keys[t], b = keys[ixj];
                    if ((a > b) == asc) {
                        keys[t] = b; keys[ixj] = a;
                        double va = vals[t];
                        vals[t] = vals[ixj]; vals[ixj] = va;
                    }
                }
            }
            __syncwarp();
        }
    }
    for (int t = lane; t < cnt; t += 32) {
        cci[out + t] = keys[t];
        cv[out + t] = vals[t];
    }
}

// words > 0: each warp also holds a bitmap of `words` words over B's columns (and their prefix
// counts) after the tables, which orders its rows' entries
template <int S>
__global__ void numeric_shared_kernel(int cnt, const int *rows, const int *arp, const int *aci, const double *av,
                                      const int *brp, const int *bci, const double *bv, const int *crp, int *cci,
                                      double *cv, int *overflow, int words)
{
    extern __shared__ double smem_num[];
    const int warps = blockDim.x >> 5;
    const int w = threadIdx.x >> 5;
    double *vals = smem_num + w * S;
    int *keys = reinterpret_cast<int *>(smem_num + warps * S) + w * S;
    unsigned *bm = words > 0 ? reinterpret_cast<unsigned *>(smem_num + warps * S) + warps * S + 2 * w * words
                             : nullptr;
    const int row_slot = blockIdx.x * warps + w;
    if (row_slot >= cnt) return;
    numeric_row(rows[row_slot], arp, aci, av, brp, bci, bv, keys, vals, S, crp, cci, cv, overflow, bm, words);
}

__global__ void numeric_global_kernel(int cnt, const int *rows, const int *toff, const int *tsize, int *gkeys,
                                      double *gvals, const int *arp, const int *aci, const double *av, const int *brp,
                                      const int *bci, const double *bv, const int *crp, int *cci, double *cv,
                                      int *overflow)
{
    const int row_slot = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row_slot >= cnt) return;
    int i = rows[row_slot];
    numeric_row(i, arp, aci, av, brp, bci, bv, gkeys + toff[row_slot], gvals + toff[row_slot], tsize[i], crp, cci, cv,
                overflow);
}

// ------------------------------------------------------------------------------------ numeric by chains
// The numeric phase of the allocating product runs in three passes instead of numeric_row's one:
//   pattern  C's sorted columns per row and, per entry c_ij, its number of terms (how many
//            a_ik b_kj reach it) -- integer work only;
//   place    every product's (a_ik, b_kj) into the chain of its entry, in the row's product
//            order (k ascending), so chain q holds c_q's terms in the order they are summed;
//   chain    each lane of a warp sums whole chains, c = fma(a, b, c) from 0 in chain order,
//            taking the next chain of the warp's range when it finishes one.
// The sums are numeric_row's, bit for bit; but every FP64 instruction of the chain pass has
// all 32 lanes busy (until the last chains of a range), where numeric_row issues one FP64
// instruction per distinct column per batch of 32 products, most of its lanes idle.  Rows of
// more than 2048 entries count their columns in a dense array in shared memory (one block
// per row) when B has at most kDenseCols columns, instead of one warp on a global hash table.
constexpr int kDenseCols = 49152;          // 192 KB of int counters in shared memory
constexpr int kChainOutputs = 256;         // entries of C per warp of the chain pass
constexpr long long kChainTotal = 16 << 20;  // ... when the whole product has at most this many

// visit(j) for the column of every product of row i, block-wide, in no particular order: one
// thread per entry of A's row walks a row of B of up to 32 entries; the longer rows of B (a
// stalled level's dense rows) are deferred to whole warps, so no thread walks a long chain of
// dependent loads alone.  blockDim.x <= kDenseThreads.
constexpr int kDenseThreads = 512;
constexpr long long kDenseSymProducts = 2048;   // symbolic: rows of more products by dense counters
template <typename F>
__device__ __forceinline__ void row_products(int i, const int *arp, const int *aci, const int *brp, const int *bci,
                                             F visit)
{
    __shared__ int dk[kDenseThreads];
    __shared__ int nd;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ae = arp[i + 1];
    for (int e0 = arp[i]; e0 < ae; e0 += blockDim.x) {
        if (threadIdx.x == 0) nd = 0;
        __syncthreads();
        const int e = e0 + (int)threadIdx.x;
        if (e < ae) {
            const int k = aci[e];
            const int b0 = brp[k], b1 = brp[k + 1];
            if (b1 - b0 <= 32) {
                for (int f = b0; f < b1; ++f) visit(bci[f]);
            } else {
                dk[atomicAdd(&nd, 1)] = k;
            }
        }
        __syncthreads();
        for (int d = warp; d < nd; d += nw) {
            const int k = dk[d];
            for (int f = brp[k] + lane; f < brp[k + 1]; f += 32) visit(bci[f]);
        }
        __syncthreads();
    }
}

// counts[ncolB] of row i's products per column (block-wide, any order)
__device__ __forceinline__ void dense_count_row(int i, const int *arp, const int *aci, const int *brp, const int *bci,
                                                int ncolB, int *cnt)
{
    for (int j = threadIdx.x; j < ncolB; j += blockDim.x) cnt[j] = 0;
    __syncthreads();
    row_products(i, arp, aci, brp, bci, [cnt](int j) { atomicAdd(&cnt[j], 1); });
}

__global__ void __launch_bounds__(kDenseThreads) dense_symbolic_kernel(int cnt_rows, const int *rows, const int *arp,
                                                                       const int *aci, const int *brp, const int *bci,
                                                                       int ncolB, int *ccnt)
{
    extern __shared__ int dcnt[];
    __shared__ int wsum[kDenseThreads / 32];
    if ((int)blockIdx.x >= cnt_rows) return;
    const int i = rows[blockIdx.x];
    dense_count_row(i, arp, aci, brp, bci, ncolB, dcnt);
    int mine = 0;
    for (int j = threadIdx.x; j < ncolB; j += blockDim.x) mine += dcnt[j] > 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(kFullMask, mine, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
        ccnt[i] = t;
    }
}

// columns of row i in ascending order and their term counts, from the dense counters: thread
// t owns the contiguous column range [t cpt, (t + 1) cpt)
__global__ void __launch_bounds__(kDenseThreads) dense_pattern_kernel(int cnt_rows, const int *rows, const int *arp,
                                                                      const int *aci, const int *brp, const int *bci,
                                                                      int ncolB, const int *crp, int *cci,
                                                                      int *ccount, int *overflow, int zero_counts)
{
    extern __shared__ int dcnt[];
    __shared__ int wsum[kDenseThreads / 32];
    if ((int)blockIdx.x >= cnt_rows) return;
    const int i = rows[blockIdx.x];
    dense_count_row(i, arp, aci, brp, bci, ncolB, dcnt);
    const int cpt = (ncolB + (int)blockDim.x - 1) / (int)blockDim.x;
    const int j0 = threadIdx.x * cpt, j1 = min(ncolB, j0 + cpt);
    int mine = 0;
    for (int j = j0; j < j1; ++j) mine += dcnt[j] > 0;
    // exclusive scan of the per-thread counts, threads in order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFullMask, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        if (w < warp) before += wsum[w];
        total += wsum[w];
    }
    const int out = crp[i];
    if (total != crp[i + 1] - out) {
        if (threadIdx.x == 0) atomicAdd(overflow, 1);
        return;
    }
    int p = out + before + incl - mine;
    for (int j = j0; j < j1; ++j) {
        const int c = dcnt[j];
        if (c > 0) {
            cci[p] = j;
            ccount[p] = zero_counts ? 0 : c;     // zero: the row's values come from dense_direct_kernel
            ++p;
        }
    }
}

// hash-table form (one warp per row): columns and their term counts, sorted by column
__device__ void pattern_row(int i, const int *arp, const int *aci, const int *brp, const int *bci, int *keys, int *cnts,
                            int S, const int *crp, int *cci, int *ccount, int *overflow)
{
    const int lane = threadIdx.x & 31;
    for (int t = lane; t < S; t += 32) { keys[t] = -1; cnts[t] = 0; }
    __syncwarp();
    const int ae = arp[i + 1];
    for (int eb = arp[i]; eb < ae; eb += 32) {
        const int e = eb + lane;
        int len = 0, fb = 0;
        if (e < ae) {
            const int k = aci[e];
            fb = brp[k];
            len = brp[k + 1] - fb;
        }
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFullMask, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(kFullMask, incl, 31);
        const int excl = incl - len;
        for (int qb = 0; qb < total; qb += 32) {
            ProductBatch pb = product_at<false>(qb + lane, total, incl, excl, fb, 0.0, bci, nullptr);
            if (pb.valid) {
                bool fresh;
                const int slot = hash_insert(keys, S, pb.j, fresh, overflow);
                if (slot >= 0) atomicAdd(&cnts[slot], 1);
            }
        }
    }
    __syncwarp();
    // compact occupied slots to the front, in slot order
    int base = 0;
    for (int t0 = 0; t0 < S; t0 += 32) {
        const int t = t0 + lane;
        const int key = keys[t], c = cnts[t];
        const bool occ = key != -1;
        const unsigned m = __ballot_sync(kFullMask, occ);
        __syncwarp();
        if (occ) {
            const int p = base + __popc(m & ((1u << lane) - 1u));
            keys[p] = key;
            cnts[p] = c;
        }
        base += __popc(m);
        __syncwarp();
    }
    const int cnt = base;
    const int out = crp[i];
    if (cnt != crp[i + 1] - out) {
        if (lane == 0) atomicAdd(overflow, 1);
        return;
    }
    if (cnt <= 512) {
        for (int t = lane; t < cnt; t += 32) {
            const int key = keys[t];
            int rank = 0;
            for (int u = 0; u < cnt; ++u) rank += keys[u] < key;
            cci[out + rank] = key;
            ccount[out + rank] = cnts[t];
        }
        return;
    }
    int P2 = 1;
    while (P2 < cnt) P2 <<= 1;
    for (int t = cnt + lane; t < P2; t += 32) { keys[t] = 0x7fffffff; cnts[t] = 0; }
    __syncwarp();
    for (int kk = 2; kk <= P2; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int t = lane; t < P2; t += 32) {
                const int ixj = t ^ jj;
                if (ixj > t) {
                    const bool asc = (t & kk) == 0;
                    const int a = keys[t], b = keys[ixj];
                    if ((a > b) == asc) {
                        keys[t] = b; keys[ixj] = a;
                        const int ca = cnts[t];
                        cnts[t] = cnts[ixj]; cnts[ixj] = ca;
                    }
                }
            }
            __syncwarp();
        }
    }
    for (int t = lane; t < cnt; t += 32) {
        cci[out + t] = keys[t];
        ccount[out + t] = cnts[t];
    }
}

template <int S>
__global__ void pattern_shared_kernel(int cnt, const int *rows, const int *arp, const int *aci, const int *brp,
                                      const int *bci, const int *crp, int *cci, int *ccount, int *overflow)
{
    extern __shared__ int smem_pat[];
    const int warps = blockDim.x >> 5;
    const int w = threadIdx.x >> 5;
    const int row_slot = blockIdx.x * warps + w;
    if (row_slot >= cnt) return;
    pattern_row(rows[row_slot], arp, aci, brp, bci, smem_pat + 2 * w * S, smem_pat + (2 * w + 1) * S, S, crp, cci,
                ccount, overflow);
}

__global__ void pattern_global_kernel(int cnt, const int *rows, const int *toff, const int *tsize, int *gkeys,
                                      int *gcnts, const int *arp, const int *aci, const int *brp, const int *bci,
                                      const int *crp, int *cci, int *ccount, int *overflow)
{
    const int row_slot = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row_slot >= cnt) return;
    const int i = rows[row_slot];
    pattern_row(i, arp, aci, brp, bci, gkeys + toff[row_slot], gcnts + toff[row_slot], tsize[i], crp, cci, ccount,
                overflow);
}

// Every product of row i (warp per row, k ascending, then B's row order) to its chain:
// position off[q] + (terms of q already placed) for the entry q of its column, found by binary
// search in the row's sorted columns.  Rows are taken from the end of `rows` first (the bins
// of the longest rows come last there), so that the longest start first.
// Rows of more than skip_above entries are placed by place_dense_kernel instead.
__device__ __forceinline__ void place_row(int i, const int *arp, const int *aci, const double *av, const int *brp,
                                          const int *bci, const double *bv, const int *crp, const int *cci,
                                          const int *rank_map, const int *off, int *run, double *sa, double *sb)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int rb = crp[i], nc = crp[i + 1] - rb;
    const int *cols = cci + rb;
    const int ae = arp[i + 1];
    for (int eb = arp[i]; eb < ae; eb += 32) {
        const int e = eb + lane;
        int len = 0, fb = 0;
        double a = 0.0;
        if (e < ae) {
            const int k = aci[e];
            a = av[e];
            fb = brp[k];
            len = brp[k + 1] - fb;
        }
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFullMask, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(kFullMask, incl, 31);
        const int excl = incl - len;
        for (int qb = 0; qb < total; qb += 32) {
            ProductBatch pb = product_at<true>(qb + lane, total, incl, excl, fb, a, bci, bv);
            int q = -1 - lane;
            if (pb.valid) {
                if (rank_map) {
                    q = rb + rank_map[pb.j];
                } else {
                    int lo = 0, hi = nc;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (cols[mid] < pb.j) lo = mid + 1; else hi = mid;
                    }
                    q = rb + lo;
                }
            }
            const unsigned same = __match_any_sync(kFullMask, q);
            const int rib = __popc(same & lt), grp = __popc(same);
            const int base = pb.valid ? run[q] : 0;
            if (pb.valid) {
                const int pos = off[q] + base + rib;
                sa[pos] = pb.a;
                sb[pos] = pb.b;
            }
            __syncwarp();
            if (pb.valid && rib == grp - 1) run[q] = base + grp;
            __syncwarp();
        }
    }
}

__global__ void place_kernel(int cnt, const int *rows, const int *arp, const int *aci, const double *av, const int *brp,
                             const int *bci, const double *bv, const int *crp, const int *cci, const int *off, int *run,
                             double *sa, double *sb, int skip_above)
{
    const int slot = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (slot >= cnt) return;
    const int i = rows[cnt - 1 - slot];
    if (crp[i + 1] - crp[i] > skip_above) return;
    place_row(i, arp, aci, av, brp, bci, bv, crp, cci, nullptr, off, run, sa, sb);
}

// Rows of thousands of entries against at most kDenseCols columns: the block writes each column's
// position in the row into a dense map in shared memory, then its first warp places the products
// (a lookup per product instead of a binary search over thousands of columns).
__global__ void __launch_bounds__(kDenseThreads) place_dense_kernel(int cnt_rows, const int *rows, const int *arp,
                                                                    const int *aci, const double *av, const int *brp,
                                                                    const int *bci, const double *bv, const int *crp,
                                                                    const int *cci, const int *off, int *run,
                                                                    double *sa, double *sb)
{
    extern __shared__ int rank_map[];
    if ((int)blockIdx.x >= cnt_rows) return;
    const int i = rows[blockIdx.x];
    const int rb = crp[i], nc = crp[i + 1] - rb;
    for (int t = threadIdx.x; t < nc; t += blockDim.x) rank_map[cci[rb + t]] = t;
    __syncthreads();
    if (threadIdx.x >= 32) return;
    place_row(i, arp, aci, av, brp, bci, bv, crp, cci, rank_map, off, run, sa, sb);
}

// B^T in CSR for dense_direct_kernel (B with at most kDenseCols rows): counts, scan, an unordered
// scatter (a warp per row of B), then each row of B^T sorted by its (distinct) keys -- by rank
// counting in a warp when short, by a dense marker array over B's rows in shared memory when long.
constexpr int kTrShort = 64;
__global__ void trw_count_kernel(int64_t nnz, const int *ci, int *cnt)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[ci[e]], 1);
}
__global__ void trw_scatter_kernel(int n, const int *rp, const int *ci, const double *v, const int *trp, int *fill,
                                   int *tci, double *tv)
{
    const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    for (int e = rp[i] + lane; e < rp[i + 1]; e += 32) {
        const int c = ci[e];
        const int p = trp[c] + atomicAdd(&fill[c], 1);
        tci[p] = i;
        tv[p] = v[e];
    }
}
__global__ void trw_sort_short_kernel(int nrow, const int *trp, const int *tci, const double *tv, int *oci, double *ov,
                                      int *long_rows, int *nlong)
{
    const int lane = threadIdx.x & 31;
    const int r = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (r >= nrow) return;
    const int b = trp[r], m = trp[r + 1] - b;
    if (m > kTrShort) {
        if (lane == 0) long_rows[atomicAdd(nlong, 1)] = r;
        return;
    }
    for (int t = lane; t < m; t += 32) {
        const int key = tci[b + t];
        int rank = 0;
        for (int u = 0; u < m; ++u) rank += tci[b + u] < key;
        oci[b + rank] = key;
        ov[b + rank] = tv[b + t];
    }
}
__global__ void __launch_bounds__(kDenseThreads) trw_sort_long_kernel(int nkeys, const int *trp, const int *tci,
                                                                      const double *tv, int *oci, double *ov,
                                                                      const int *long_rows, const int *nlong)
{
    extern __shared__ int where[];
    __shared__ int wsum[kDenseThreads / 32];
    for (int w = blockIdx.x; w < *nlong; w += gridDim.x) {
        const int r = long_rows[w];
        const int b = trp[r], m = trp[r + 1] - b;
        for (int k = threadIdx.x; k < nkeys; k += blockDim.x) where[k] = -1;
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += blockDim.x) where[tci[b + t]] = t;
        __syncthreads();
        // keys in ascending order: thread t owns keys [t kpt, (t + 1) kpt)
        const int kpt = (nkeys + (int)blockDim.x - 1) / (int)blockDim.x;
        const int k0 = threadIdx.x * kpt, k1 = min(nkeys, k0 + kpt);
        int mine = 0;
        for (int k = k0; k < k1; ++k) mine += where[k] >= 0;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFullMask, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int p = 0;
        for (int q = 0; q < warp; ++q) p += wsum[q];
        p += incl - mine;
        for (int k = k0; k < k1; ++k) {
            const int t = where[k];
            if (t >= 0) {
                oci[b + p] = k;
                ov[b + p] = tv[b + t];
                ++p;
            }
        }
        __syncthreads();
    }
}

// Rows of thousands of entries when B has at most kDenseCols rows and columns: c_ij directly from
// column j of B (Bt = B^T in CSR: its row j lists the k with b_kj != 0, ascending).  The block
// maps each k of A's row i to its entry (or -1) in shared memory; each thread walks the columns
// of some of the row's entries and sums c_ij = fma(a_ik, b_kj, c_ij) over the k of the column
// that row i holds, ascending -- the order of every other path -- with no staging at all.
__global__ void __launch_bounds__(kDenseThreads) dense_direct_kernel(int cnt_rows, const int *rows, int nB,
                                                                     const int *arp, const int *aci, const double *av,
                                                                     const int *btrp, const int *btci,
                                                                     const double *btv, const int *crp, const int *cci,
                                                                     double *cv)
{
    extern __shared__ int pos_of_k[];
    if ((int)blockIdx.x >= cnt_rows) return;
    const int i = rows[blockIdx.x];
    for (int k = threadIdx.x; k < nB; k += blockDim.x) pos_of_k[k] = -1;
    __syncthreads();
    for (int e = arp[i] + threadIdx.x; e < arp[i + 1]; e += blockDim.x) pos_of_k[aci[e]] = e;
    __syncthreads();
    const int rb = crp[i], nc = crp[i + 1] - rb;
    for (int t = threadIdx.x; t < nc; t += blockDim.x) {
        const int j = cci[rb + t];
        double acc = 0.0;
        for (int f = btrp[j]; f < btrp[j + 1]; ++f) {
            const int e = pos_of_k[btci[f]];
            if (e >= 0) acc = __fma_rn(av[e], btv[f], acc);
        }
        cv[rb + t] = acc;
    }
}

// c_q = sum of its chain, fma from 0 in chain order; warp w owns entries [w K, (w + 1) K), each
// lane sums one chain at a time and takes the warp's next chain when it finishes
__global__ void __launch_bounds__(256) chain_kernel(int nnz, const int *off, const double *sa, const double *sb,
                                                    double *cv)
{
    const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int q0 = warp * kChainOutputs;
    if (q0 >= nnz) return;
    const int q1 = min(nnz, q0 + kChainOutputs);
    int q = q0 + lane, next = q0 + 32;
    int pos = 0, end = 0;
    double acc = 0.0;
    if (q < q1) { pos = off[q]; end = off[q + 1]; }
    for (;;) {
        const bool act = q < q1;
        if (!__any_sync(kFullMask, act)) break;
        if (act && pos < end) {
            acc = __fma_rn(sa[pos], sb[pos], acc);
            ++pos;
        }
        const bool fin = act && pos >= end;
        const unsigned fm = __ballot_sync(kFullMask, fin);
        if (fin) {
            cv[q] = acc;
            acc = 0.0;
            q = next + __popc(fm & lt);
            if (q < q1) { pos = off[q]; end = off[q + 1]; }
        }
        next += __popc(fm);
    }
}

// ------------------------------------------------------------------------------------ segmented rows
// Rows of A with more than kSegLen stored entries (stalled coarse levels hold rows of thousands)
// follow the segmented reading of the sums: the row's positions fall in segments of kSegLen;
// c_ij is summed with fma over each segment's terms in ascending k from 0, and the sums of all
// the row's segments (0 where a segment has no term for j) are added in segment order.  The
// segments are independent, so a block per (row, segment) forms its segment's sums: the
// segment's rows of B staged in shared memory, then one k after another (a barrier per k) into
// an accumulator over B's columns in shared memory (over the row's entries in a scratch slice,
// found by binary search, when B has more than kSegCols columns); the sums go to a scratch
// array, and one pass adds each entry's segment sums in order.  The row's columns come from a
// flag array over B's columns, one block per row.  When B has at most kSegCols columns, the rows
// of C too long for a shared-memory hash table (rows of A of at most kSegLen entries: a single
// segment, the plain ascending-k sums) take this path as well: a k at a time into the dense
// accumulator instead of a global hash table or a walk of every column of B.
constexpr int kSegCols = 8192;          // B columns of the shared accumulator (64 KB)
constexpr int kSegStage = 6144;         // staged entries of B per pass (72 KB)
constexpr int kSegThreads = 512;

// size[r] = segments x entries of segmented row r (its scratch slice)
__global__ void seg_size_kernel(int cnt, const int *rows, const int *arp, const int *crp, int *size)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= cnt) return;
    const int i = rows[r];
    const int nseg = (arp[i + 1] - arp[i] + kSegLen - 1) / kSegLen;
    size[r] = nseg * (crp[i + 1] - crp[i]);
}

// C's sorted columns of segmented row r = blockIdx.x (flags over B's columns: shared memory, or
// the block's slice of gflags); *ovf += 1 when the count differs from the symbolic phase's
__global__ void __launch_bounds__(kSegThreads) seg_pattern_kernel(int cnt, const int *rows, const int *arp,
                                                                   const int *aci, const int *brp, const int *bci,
                                                                   int ncolB, const int *crp, int *cci, int *ovf,
                                                                   int *gflags)
{
    extern __shared__ int seg_flag_s[];
    __shared__ int wsum[kSegThreads / 32];
    __shared__ int base_s;
    if ((int)blockIdx.x >= cnt) return;
    int *flag = gflags ? gflags + (size_t)blockIdx.x * (size_t)ncolB : seg_flag_s;
    const int i = rows[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = threadIdx.x; j < ncolB; j += blockDim.x) flag[j] = 0;
    if (threadIdx.x == 0) base_s = 0;
    __syncthreads();
    row_products(i, arp, aci, brp, bci, [flag](int j) { flag[j] = 1; });
    const int out0 = crp[i], nc = crp[i + 1] - out0;
    for (int j0 = 0; j0 < ncolB; j0 += blockDim.x) {
        const int j = j0 + (int)threadIdx.x;
        const int fl = j < ncolB ? flag[j] : 0;
        const unsigned m = __ballot_sync(kFullMask, fl);
        if (lane == 0) wsum[warp] = __popc(m);
        __syncthreads();
        int p = base_s + __popc(m & ((1u << lane) - 1u));
        for (int w = 0; w < warp; ++w) p += wsum[w];
        if (fl && p < nc) cci[out0 + p] = j;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < nw; ++w) t += wsum[w];
            base_s += t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && base_s != nc) atomicAdd(ovf, 1);
}

// position of column j among the n sorted columns c (present by construction)
__device__ __forceinline__ int seg_find(const int *c, int n, int j)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (c[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// exclusive prefix sum of one int per thread over a block of kSegThreads threads
__device__ __forceinline__ int seg_block_scan(int v, int *wsum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFullMask, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int x = lane < kSegThreads / 32 ? wsum[lane] : 0;
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFullMask, xi, o);
            if (lane >= o) xi += y;
        }
        if (lane < kSegThreads / 32) wsum[lane] = xi - x;
    }
    __syncthreads();
    return incl - v + wsum[warp];
}

// dynamic shared memory of seg_numeric_kernel: the dense accumulator (DENSE), then the staged
// columns (int), values (double), bucket lists (uint16) and k indices (uint8) of kSegStage entries
constexpr size_t kSegStageBytes = (size_t)kSegStage * (4 + 8 + 2 + 1);
constexpr size_t seg_numeric_smem(bool dense) { return (dense ? sizeof(double) * kSegCols : 0) + kSegStageBytes; }

// segment q = blockIdx.y of segmented row r = blockIdx.x: S[soff[r] + q nc + t] = the sum over
// the segment's terms of entry t, fma in ascending k from 0 (DENSE: accumulator over B's
// columns in shared memory; else in the scratch slice itself, positions by binary search).
// The segment's k's go in chunks whose rows of B fit the stage together.  A staged chunk's
// products fall in kSegThreads buckets by their accumulator position; each thread sorts its
// bucket by product index (products are staged in ascending k, and a row of B holds a column
// once, so this is ascending k within every position) and applies its fma's in that order:
// the sums of a per-k sweep with a barrier after every k, without the barriers.  Chunks of k's
// with many terms each keep the per-k sweep (a few barriers, and buckets of one position's many
// terms would be long serial sorts).  A k whose row of B alone exceeds the stage is swept
// straight from global memory (its columns are distinct).
template <bool DENSE>
__global__ void __launch_bounds__(kSegThreads) seg_numeric_kernel(int cnt, const int *rows, const int *arp,
                                                                   const int *aci, const double *av, const int *brp,
                                                                   const int *bci, const double *bv, const int *crp,
                                                                   const int *cci, const int *soff, double *S)
{
    extern __shared__ __align__(16) unsigned char seg_num_s[];
    __shared__ int sk[kSegLen], spre[kSegLen + 1];
    __shared__ double sa[kSegLen];
    __shared__ int bfill[kSegThreads], wsum[kSegThreads / 32];
    __shared__ int chunk_end;
    const int r = blockIdx.x, q = blockIdx.y;
    if (r >= cnt) return;
    const int i = rows[r];
    const int a0 = arp[i], alen = arp[i + 1] - a0;
    const int nseg = (alen + kSegLen - 1) / kSegLen;
    const int out0 = crp[i], nc = crp[i + 1] - out0;
    if (q >= nseg || nc == 0) return;
    double *slice = S + soff[r] + (size_t)q * (size_t)nc;
    double *acc = DENSE ? (double *)seg_num_s : slice;
    int *scol = (int *)(seg_num_s + (DENSE ? sizeof(double) * kSegCols : 0));
    double *sval = (double *)(scol + kSegStage);
    unsigned short *bucket = (unsigned short *)(sval + kSegStage);
    unsigned char *st = (unsigned char *)(bucket + kSegStage);
    const int *rc = cci + out0;
    const int tid = threadIdx.x;
    for (int t = tid; t < nc; t += blockDim.x) {
        if (DENSE) acc[rc[t]] = 0.0;
        else acc[t] = 0.0;
    }
    const int m = min(kSegLen, alen - q * kSegLen);
    for (int t = tid; t < m; t += blockDim.x) {
        const int k = aci[a0 + q * kSegLen + t];
        sk[t] = k;
        sa[t] = av[a0 + q * kSegLen + t];
        spre[t + 1] = brp[k + 1] - brp[k];
    }
    if (tid == 0) spre[0] = 0;
    __syncthreads();
    if (tid == 0)
        for (int t = 0; t < m; ++t) spre[t + 1] += spre[t];
    __syncthreads();
    int kk = 0;
    while (kk < m) {
        // the next k's whose rows of B fit the stage together (at least one)
        if (tid == 0) {
            int ke = kk + 1;
            while (ke < m && spre[ke + 1] - spre[kk] <= kSegStage) ++ke;
            chunk_end = ke;
        }
        __syncthreads();
        const int ke = chunk_end;
        const int base = spre[kk], total = spre[ke] - base;
        if (total > kSegStage) {
            // one k (ke == kk + 1): its columns are distinct, every term at once
            const double a = sa[kk];
            const int fb = brp[sk[kk]];
            for (int u = tid; u < total; u += blockDim.x) {
                const int j = bci[fb + u];
                const int pos = DENSE ? j : seg_find(rc, nc, j);
                acc[pos] = __fma_rn(a, bv[fb + u], acc[pos]);
            }
            __syncthreads();
            kk = ke;
            continue;
        }
        // buckets when the chunk's k's average fewer than 16 terms (a barrier per k would leave
        // most threads idle); else one k after another, a barrier after each
        const bool bucketed = total < 16 * (ke - kk);
        if (bucketed) bfill[tid] = 0;
        __syncthreads();
        for (int p = tid; p < total; p += blockDim.x) {
            // the k of staged entry p: the last t in [kk, ke) with spre[t] - base <= p
            int lo = kk, hi = ke - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (spre[mid] - base <= p) lo = mid;
                else hi = mid - 1;
            }
            const int f = brp[sk[lo]] + (p - (spre[lo] - base));
            const int j = bci[f];
            const int pos = DENSE ? j : seg_find(rc, nc, j);
            scol[p] = pos;
            sval[p] = bv[f];
            st[p] = (unsigned char)lo;
            if (bucketed) atomicAdd(&bfill[pos & (kSegThreads - 1)], 1);
        }
        __syncthreads();
        if (!bucketed) {
            for (int t = kk; t < ke; ++t) {
                const double a = sa[t];
                const int p0 = spre[t] - base, len = spre[t + 1] - spre[t];
                for (int u = tid; u < len; u += blockDim.x) {
                    const int pos = scol[p0 + u];
                    acc[pos] = __fma_rn(a, sval[p0 + u], acc[pos]);
                }
                __syncthreads();
            }
            kk = ke;
            continue;
        }
        const int mine = bfill[tid];
        const int b0 = seg_block_scan(mine, wsum);
        bfill[tid] = b0;
        __syncthreads();
        for (int p = tid; p < total; p += blockDim.x)
            bucket[atomicAdd(&bfill[scol[p] & (kSegThreads - 1)], 1)] = (unsigned short)p;
        __syncthreads();
        // this thread's bucket: insertion sort by product index, then its fma's in that order
        unsigned short *bk = bucket + b0;
        for (int x = 1; x < mine; ++x) {
            const unsigned short v = bk[x];
            int y = x - 1;
            while (y >= 0 && bk[y] > v) {
                bk[y + 1] = bk[y];
                --y;
            }
            bk[y + 1] = v;
        }
        for (int x = 0; x < mine; ++x) {
            const int p = bk[x];
            const int pos = scol[p];
            acc[pos] = __fma_rn(sa[st[p]], sval[p], acc[pos]);
        }
        __syncthreads();
        kk = ke;
    }
    if (DENSE)
        for (int t = tid; t < nc; t += blockDim.x) slice[t] = acc[rc[t]];
}

// C's values of segmented row r = blockIdx.x: each entry's segment sums added in order (the
// row's entries strided over the blockIdx.y blocks of the row)
__global__ void seg_combine_kernel(int cnt, const int *rows, const int *arp, const int *crp, const int *soff,
                                   const double *S, double *cv)
{
    const int r = blockIdx.x;
    if (r >= cnt) return;
    const int i = rows[r];
    const int nseg = (arp[i + 1] - arp[i] + kSegLen - 1) / kSegLen;
    const int out0 = crp[i], nc = crp[i + 1] - out0;
    const double *sl = S + soff[r];
    for (int t = blockIdx.y * blockDim.x + threadIdx.x; t < nc; t += gridDim.y * blockDim.x) {
        double c = sl[t];
        for (int q = 1; q < nseg; ++q) c = c + sl[(size_t)q * nc + t];
        cv[out0 + t] = c;
    }
}

// 64-bit sum of n non-negative ints (a total an int32 scan is about to form)
__global__ void sum64_kernel(const int *v, int n, unsigned long long *out)
{
    unsigned long long acc = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x = v[i];
        acc += x > 0 ? (unsigned long long)x : 0ull;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFullMask, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// ------------------------------------------------------------------------------------ host side
namespace {

struct Bins {
    int count[kNumBins] = {0};
    int start[kNumBins + 1] = {0};
};

cudaError_t make_bins(int n, int *d_bin, int *d_binCount, int *d_binFill, int *d_binStart, int *d_perm, Bins &hb,
                      cudaStream_t s)
{
    AMG_CUDA_TRY(cudaMemcpyAsync(hb.count, d_binCount, sizeof(int) * kNumBins, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    hb.start[0] = 0;
    for (int b = 0; b < kNumBins; ++b) hb.start[b + 1] = hb.start[b] + hb.count[b];
    AMG_CUDA_TRY(cudaMemcpyAsync(d_binStart, hb.start, sizeof(int) * (kNumBins + 1), cudaMemcpyHostToDevice, s));
    AMG_CUDA_TRY(cudaMemsetAsync(d_binFill, 0, sizeof(int) * kNumBins, s));
    if (n > 0) {
        bin_scatter_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, d_bin, d_binStart, d_binFill, d_perm);
        note_launch();
    }
    return cudaGetLastError();
}

template <int S>
cudaError_t launch_symbolic(int cnt, const int *rows, const DevCsr &A, const DevCsr &B, int *ccnt, int *ovf,
                            const int *tsize, cudaStream_t s)
{
    int warps = kSmemBudget / (S * 4);
    if (warps > 8) warps = 8;
    if (warps < 1) warps = 1;
    size_t smem = (size_t)warps * S * 4;
    AMG_CUDA_TRY(cudaFuncSetAttribute(symbolic_shared_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    symbolic_shared_kernel<S><<<(cnt + warps - 1) / warps, warps * 32, smem, s>>>(cnt, rows, A.rp, A.ci, B.rp, B.ci,
                                                                                 ccnt, ovf, tsize); note_launch();
    return cudaGetLastError();
}

// Rows of more than 256 entries of C (tables of 1024 slots and up) order their entries by a
// bitmap over B's columns when B has at most kBitmapCols columns: a warp's sort of 512-2048
// entries (rank counting or a bitonic network, thousands of dependent shared-memory steps) was
// the long pole of the stalled coarse levels' Galerkin products.
constexpr int kBitmapCols = 8192;       // 2 KB a warp: two blocks of 1024-slot tables still fit an SM
constexpr int kBitmapMinTable = 1024;

template <int S>
cudaError_t launch_numeric(int cnt, const int *rows, const DevCsr &A, const DevCsr &B, DevCsr &C, int *ovf,
                           cudaStream_t s)
{
    int warps = kSmemBudget / (S * 12);
    if (warps > 8) warps = 8;
    if (warps < 1) warps = 1;
    const int words = S >= kBitmapMinTable && B.ncol <= kBitmapCols ? (B.ncol + 31) / 32 : 0;
    size_t smem = (size_t)warps * ((size_t)S * 12 + (size_t)words * 8);
    AMG_CUDA_TRY(cudaFuncSetAttribute(numeric_shared_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    numeric_shared_kernel<S><<<(cnt + warps - 1) / warps, warps * 32, smem, s>>>(cnt, rows, A.rp, A.ci, A.v, B.rp,
                                                                                B.ci, B.v, C.rp, C.ci, C.v, ovf,
                                                                                words); note_launch();
    return cudaGetLastError();
}

cudaError_t symbolic_bin(int b, int cnt, const int *rows, const DevCsr &A, const DevCsr &B, int *ccnt, int *ovf,
                         cudaStream_t s, const int *tsize = nullptr)
{
    switch (b) {
    case 0: return launch_symbolic<32>(cnt, rows, A, B, ccnt, ovf, tsize, s);
    case 1: return launch_symbolic<64>(cnt, rows, A, B, ccnt, ovf, tsize, s);
    case 2: return launch_symbolic<128>(cnt, rows, A, B, ccnt, ovf, tsize, s);
    case 3: return launch_symbolic<256>(cnt, rows, A, B, ccnt, ovf, tsize, s);
    case 4: return launch_symbolic<512>(cnt, rows, A, B, ccnt, ovf, tsize, s);
    case 5: return launch_symbolic<1024>(cnt, rows, A, B, ccnt, ovf, tsize, s);
    case 6: return launch_symbolic<2048>(cnt, rows, A, B, ccnt, ovf, tsize, s);
    case 7: return launch_symbolic<4096>(cnt, rows, A, B, ccnt, ovf, tsize, s);
    case 8: return launch_symbolic<8192>(cnt, rows, A, B, ccnt, ovf, tsize, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t numeric_bin(int b, int cnt, const int *rows, const DevCsr &A, const DevCsr &B, DevCsr &C, int *ovf,
                        cudaStream_t s)
{
    switch (b) {
    case 0: return launch_numeric<32>(cnt, rows, A, B, C, ovf, s);
    case 1: return launch_numeric<64>(cnt, rows, A, B, C, ovf, s);
    case 2: return launch_numeric<128>(cnt, rows, A, B, C, ovf, s);
    case 3: return launch_numeric<256>(cnt, rows, A, B, C, ovf, s);
    case 4: return launch_numeric<512>(cnt, rows, A, B, C, ovf, s);
    case 5: return launch_numeric<1024>(cnt, rows, A, B, C, ovf, s);
    case 6: return launch_numeric<2048>(cnt, rows, A, B, C, ovf, s);
    case 7: return launch_numeric<4096>(cnt, rows, A, B, C, ovf, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int S>
cudaError_t launch_pattern(int cnt, const int *rows, const DevCsr &A, const DevCsr &B, const int *crp, int *cci,
                           int *ccount, int *ovf, cudaStream_t s)
{
    int warps = kSmemBudget / (S * 8);
    if (warps > 8) warps = 8;
    if (warps < 1) warps = 1;
    const size_t smem = (size_t)warps * S * 8;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [smem] {
        attr = cudaFuncSetAttribute(pattern_shared_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)std::max<size_t>(smem, (size_t)kSmemBudget));
    });
    AMG_CUDA_TRY(attr);
    pattern_shared_kernel<S><<<(cnt + warps - 1) / warps, warps * 32, smem, s>>>(cnt, rows, A.rp, A.ci, B.rp, B.ci, crp,
                                                                                cci, ccount, ovf); note_launch();
    return cudaGetLastError();
}

cudaError_t pattern_bin(int b, int cnt, const int *rows, const DevCsr &A, const DevCsr &B, const int *crp, int *cci,
                        int *ccount, int *ovf, cudaStream_t s)
{
    switch (b) {
    case 0: return launch_pattern<32>(cnt, rows, A, B, crp, cci, ccount, ovf, s);
    case 1: return launch_pattern<64>(cnt, rows, A, B, crp, cci, ccount, ovf, s);
    case 2: return launch_pattern<128>(cnt, rows, A, B, crp, cci, ccount, ovf, s);
    case 3: return launch_pattern<256>(cnt, rows, A, B, crp, cci, ccount, ovf, s);
    case 4: return launch_pattern<512>(cnt, rows, A, B, crp, cci, ccount, ovf, s);
    case 5: return launch_pattern<1024>(cnt, rows, A, B, crp, cci, ccount, ovf, s);
    case 6: return launch_pattern<2048>(cnt, rows, A, B, crp, cci, ccount, ovf, s);
    case 7: return launch_pattern<4096>(cnt, rows, A, B, crp, cci, ccount, ovf, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t dense_attr()
{
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(dense_symbolic_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kDenseCols * (int)sizeof(int));
        if (attr == cudaSuccess)
            attr = cudaFuncSetAttribute(dense_pattern_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kDenseCols * (int)sizeof(int));
        if (attr == cudaSuccess)
            attr = cudaFuncSetAttribute(place_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kDenseCols * (int)sizeof(int));
        if (attr == cudaSuccess)
            attr = cudaFuncSetAttribute(dense_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kDenseCols * (int)sizeof(int));
        if (attr == cudaSuccess)
            attr = cudaFuncSetAttribute(trw_sort_long_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kDenseCols * (int)sizeof(int));
    });
    return attr;
}

// table offsets (int) for the rows of the global bin; returns total slots
cudaError_t global_tables(int cnt, const int *rows, const int *tsize, int **toff, int64_t *total, cudaStream_t s)
{
    AMG_CUDA_TRY(cudaMallocAsync(toff, sizeof(int) * (size_t)(cnt + 1), s));
    gather_tsize_kernel<<<grid_for(cnt, 256), 256, 0, s>>>(cnt, rows, tsize, *toff); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    // the int offsets must not wrap: the sizes are summed in 64 bits before the int scan
    std::vector<int> sizes((size_t)cnt);
    AMG_CUDA_TRY(cudaMemcpyAsync(sizes.data(), *toff, sizeof(int) * (size_t)cnt, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t sum = 0;
    for (int v : sizes) sum += v;
    if (sum > 0x7fffffffLL) return cudaErrorMemoryAllocation;
    AMG_CUDA_TRY(scan_exclusive(*toff, *toff, cnt, s));
    *total = sum;
    return cudaSuccess;
}

// The numeric phase by chains.  *done = false (nothing written, no error) when the products of
// the whole row set do not fit the int32 chain offsets; the caller then runs numeric_row.
cudaError_t numeric_chains(int n, const DevCsr &A, const DevCsr &B, DevCsr &C, const Bins &hb, const int *d_perm,
                           const int *d_tsize, int *d_ovf, bool *done, cudaStream_t s)
{
    *done = false;
    const int nnz = (int)C.nnz;
    int *off = nullptr, *run = nullptr, *toff = nullptr, *gkeys = nullptr;
    unsigned long long *d_sum = nullptr;
    double *sa = nullptr, *sb = nullptr;
    cudaError_t e = cudaSuccess;
    // the longest rows straight from B's columns when B is small enough for the dense maps
    const bool direct = hb.count[kGlobalBin] > 0 && B.ncol <= kDenseCols && B.n <= kDenseCols;
    DevCsr Bt;
    int *tfill = nullptr, *tci = nullptr;
    double *tv = nullptr;
    do {
        if (direct) {
            Bt.n = B.ncol;
            Bt.ncol = B.n;
            Bt.nnz = B.nnz;
            if ((e = cudaMallocAsync(&Bt.rp, sizeof(int) * ((size_t)B.ncol + 1), s))) break;
            if ((e = cudaMallocAsync(&Bt.ci, sizeof(int) * ((size_t)B.nnz + 1), s))) break;
            if ((e = cudaMallocAsync(&Bt.v, sizeof(double) * ((size_t)B.nnz + 1), s))) break;
            if ((e = cudaMallocAsync(&tfill, sizeof(int) * (2 * (size_t)B.ncol + 2), s))) break;
            if ((e = cudaMallocAsync(&tci, sizeof(int) * ((size_t)B.nnz + 1), s))) break;
            if ((e = cudaMallocAsync(&tv, sizeof(double) * ((size_t)B.nnz + 1), s))) break;
            if ((e = cudaMemsetAsync(Bt.rp, 0, sizeof(int) * ((size_t)B.ncol + 1), s))) break;
            if ((e = cudaMemsetAsync(tfill, 0, sizeof(int) * (2 * (size_t)B.ncol + 2), s))) break;
            if ((e = dense_attr())) break;
            if (B.nnz > 0) {
                trw_count_kernel<<<grid_for(B.nnz, 256, 8192), 256, 0, s>>>(B.nnz, B.ci, Bt.rp); note_launch();
            }
            if ((e = scan_exclusive(Bt.rp, Bt.rp, B.ncol, s))) break;
            int *nlong = tfill + B.ncol, *lrows = nlong + 1;
            trw_scatter_kernel<<<grid_for((int64_t)B.n * 32, 256), 256, 0, s>>>(B.n, B.rp, B.ci, B.v, Bt.rp, tfill,
                                                                                 tci, tv); note_launch();
            trw_sort_short_kernel<<<grid_for((int64_t)B.ncol * 32, 256), 256, 0, s>>>(B.ncol, Bt.rp, tci, tv, Bt.ci,
                                                                                     Bt.v, lrows, nlong); note_launch();
            trw_sort_long_kernel<<<2 * kReduceBlocks, kDenseThreads, sizeof(int) * (size_t)B.n, s>>>(
                B.n, Bt.rp, tci, tv, Bt.ci, Bt.v, lrows, nlong); note_launch();
            if ((e = cudaGetLastError())) break;
        }
        if ((e = cudaMallocAsync(&off, sizeof(int) * ((size_t)nnz + 1), s))) break;
        // zero: the segmented rows' entries get no terms here (their own path fills them)
        if ((e = cudaMemsetAsync(off, 0, sizeof(int) * ((size_t)nnz + 1), s))) break;
        if ((e = cudaMallocAsync(&run, sizeof(int) * (size_t)nnz, s))) break;
        if ((e = cudaMallocAsync(&d_sum, sizeof(unsigned long long), s))) break;
        if ((e = cudaMemsetAsync(run, 0, sizeof(int) * (size_t)nnz, s))) break;
        if ((e = cudaMemsetAsync(d_sum, 0, sizeof(unsigned long long), s))) break;
        // pattern: C's columns (sorted) and each entry's term count (into off)
        for (int b = 0; b < kGlobalBin && !e; ++b)
            if (hb.count[b]) e = pattern_bin(b, hb.count[b], d_perm + hb.start[b], A, B, C.rp, C.ci, off, d_ovf, s);
        if (e) break;
        if (hb.count[kGlobalBin]) {
            const int cnt = hb.count[kGlobalBin];
            const int *rows = d_perm + hb.start[kGlobalBin];
            if (B.ncol <= kDenseCols) {
                if ((e = dense_attr())) break;
                dense_pattern_kernel<<<cnt, kDenseThreads, sizeof(int) * (size_t)B.ncol, s>>>(
                    cnt, rows, A.rp, A.ci, B.rp, B.ci, B.ncol, C.rp, C.ci, off, d_ovf, direct ? 1 : 0); note_launch();
                if ((e = cudaGetLastError())) break;
            } else {
                int64_t total = 0;
                if ((e = global_tables(cnt, rows, d_tsize, &toff, &total, s))) break;
                if ((e = cudaMallocAsync(&gkeys, sizeof(int) * 2 * (size_t)total, s))) break;
                pattern_global_kernel<<<grid_for((int64_t)cnt * 32, 128), 128, 0, s>>>(
                    cnt, rows, toff, d_tsize, gkeys, gkeys + total, A.rp, A.ci, B.rp, B.ci, C.rp, C.ci, off, d_ovf);
                note_launch();
                if ((e = cudaGetLastError())) break;
            }
        }
        // the number of products, in 64 bits, before the int32 scan of the term counts
        sum64_kernel<<<grid_for(nnz, 256, 1024), 256, 0, s>>>(off, nnz, d_sum); note_launch();
        if ((e = cudaGetLastError())) break;
        unsigned long long total = 0;
        if ((e = cudaMemcpyAsync(&total, d_sum, sizeof total, cudaMemcpyDeviceToHost, s))) break;
        if ((e = cudaStreamSynchronize(s))) break;
        if (total > 0x7ffffff0ull) break;                    // too many products: numeric_row instead
        if ((e = scan_exclusive(off, off, nnz, s))) break;
        if ((e = cudaMallocAsync(&sa, sizeof(double) * (size_t)(total + 1), s))) break;
        if ((e = cudaMallocAsync(&sb, sizeof(double) * (size_t)(total + 1), s))) break;
        // the rows of the global bin (more than 2048 entries) by place_dense_kernel when their
        // columns fit the dense map; place_kernel takes the rest
        const bool dense_rows = hb.count[kGlobalBin] > 0 && B.ncol <= kDenseCols;
        if (dense_rows && !direct) {
            place_dense_kernel<<<hb.count[kGlobalBin], kDenseThreads, sizeof(int) * (size_t)B.ncol, s>>>(
                hb.count[kGlobalBin], d_perm + hb.start[kGlobalBin], A.rp, A.ci, A.v, B.rp, B.ci, B.v, C.rp, C.ci,
                off, run, sa, sb); note_launch();
            if ((e = cudaGetLastError())) break;
        }
        // every row but the segmented ones (the last of the bins' order)
        const int nplace = n - hb.count[kSegBin];
        place_kernel<<<grid_for((int64_t)nplace * 32, 128), 128, 0, s>>>(nplace, d_perm, A.rp, A.ci, A.v, B.rp, B.ci,
                                                                        B.v, C.rp, C.ci, off, run, sa, sb,
                                                                        dense_rows ? kMaxSharedNum / 2 : 0x7fffffff);
        note_launch();
        if ((e = cudaGetLastError())) break;
        const int64_t warps = ((int64_t)nnz + kChainOutputs - 1) / kChainOutputs;
        chain_kernel<<<grid_for(warps * 32, 256), 256, 0, s>>>(nnz, off, sa, sb, C.v); note_launch();
        if ((e = cudaGetLastError())) break;
        if (direct) {
            // after the chains: their empty chains of these rows wrote zeros
            dense_direct_kernel<<<hb.count[kGlobalBin], kDenseThreads, sizeof(int) * (size_t)B.n, s>>>(
                hb.count[kGlobalBin], d_perm + hb.start[kGlobalBin], B.n, A.rp, A.ci, A.v, Bt.rp, Bt.ci, Bt.v, C.rp,
                C.ci, C.v); note_launch();
            if ((e = cudaGetLastError())) break;
        }
        *done = true;
    } while (0);
    if (off) cudaFreeAsync(off, s);
    if (run) cudaFreeAsync(run, s);
    if (d_sum) cudaFreeAsync(d_sum, s);
    if (toff) cudaFreeAsync(toff, s);
    if (gkeys) cudaFreeAsync(gkeys, s);
    if (sa) cudaFreeAsync(sa, s);
    if (sb) cudaFreeAsync(sb, s);
    if (Bt.rp) cudaFreeAsync(Bt.rp, s);
    if (Bt.ci) cudaFreeAsync(Bt.ci, s);
    if (Bt.v) cudaFreeAsync(Bt.v, s);
    if (tfill) cudaFreeAsync(tfill, s);
    if (tci) cudaFreeAsync(tci, s);
    if (tv) cudaFreeAsync(tv, s);
    return e;
}

cudaError_t seg_attr()
{
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(seg_pattern_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kDenseCols * (int)sizeof(int));
        if (attr == cudaSuccess)
            attr = cudaFuncSetAttribute(seg_numeric_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)seg_numeric_smem(true));
        if (attr == cudaSuccess)
            attr = cudaFuncSetAttribute(seg_numeric_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)seg_numeric_smem(false));
    });
    return attr;
}

// Device scratch for the segmented rows: take(bytes) gives memory (nullptr when there is none
// left), give(p) returns it.
struct SegScratch {
    std::function<void *(size_t)> take;
    std::function<void(void *)> give;
};

// C's columns and values of the rows of A with more than kSegLen entries (rows[0, cnt), the
// longest segmax entries).  *no_room: the scratch could not hold the segment sums (C untouched).
cudaError_t numeric_segmented(const DevCsr &A, const DevCsr &B, DevCsr &C, const int *rows, int cnt, int segmax,
                              int *d_ovf, const SegScratch &sc, bool *no_room, cudaStream_t s)
{
    *no_room = false;
    if (cnt == 0) return cudaSuccess;
    if ((segmax + kSegLen - 1) / kSegLen > 65535) {     // segments beyond the grid's y extent
        *no_room = true;
        return cudaSuccess;
    }
    AMG_CUDA_TRY(seg_attr());
    int *soff = nullptr, *gflags = nullptr, *ws = nullptr;
    unsigned long long *d_sum = nullptr;
    double *S = nullptr;
    cudaError_t e = cudaSuccess;
    do {
        soff = (int *)sc.take(sizeof(int) * ((size_t)cnt + 1));
        d_sum = (unsigned long long *)sc.take(sizeof(unsigned long long));
        if (!soff || !d_sum) { *no_room = true; break; }
        if ((e = cudaMemsetAsync(d_sum, 0, sizeof(unsigned long long), s))) break;
        seg_size_kernel<<<grid_for(cnt, 256), 256, 0, s>>>(cnt, rows, A.rp, C.rp, soff); note_launch();
        sum64_kernel<<<grid_for(cnt, 256, 1024), 256, 0, s>>>(soff, cnt, d_sum); note_launch();
        if ((e = cudaGetLastError())) break;
        unsigned long long total = 0;
        if ((e = cudaMemcpyAsync(&total, d_sum, sizeof total, cudaMemcpyDeviceToHost, s))) break;
        if ((e = cudaStreamSynchronize(s))) break;
        if (total > 0x7ffffff0ull) { *no_room = true; break; }
        ws = (int *)sc.take(sizeof(int) * (scan_ws_ints(cnt + 1) + 16));
        if (!ws) { *no_room = true; break; }
        if ((e = scan_exclusive_ws(soff, soff, cnt, ws, s))) break;
        S = (double *)sc.take(sizeof(double) * ((size_t)total + 1));
        if (!S) { *no_room = true; break; }
        if (B.ncol > kDenseCols) {
            gflags = (int *)sc.take(sizeof(int) * (size_t)B.ncol * (size_t)cnt);
            if (!gflags) { *no_room = true; break; }
        }
        const size_t psmem = gflags ? 0 : sizeof(int) * (size_t)B.ncol;
        seg_pattern_kernel<<<cnt, kSegThreads, psmem, s>>>(cnt, rows, A.rp, A.ci, B.rp, B.ci, B.ncol, C.rp, C.ci, d_ovf,
                                                            gflags); note_launch();
        const dim3 grid(cnt, std::max(1, (segmax + kSegLen - 1) / kSegLen));
        if (B.ncol <= kSegCols) {
            seg_numeric_kernel<true><<<grid, kSegThreads, seg_numeric_smem(true), s>>>(
                cnt, rows, A.rp, A.ci, A.v, B.rp, B.ci, B.v, C.rp, C.ci, soff, S); note_launch();
        } else {
            seg_numeric_kernel<false><<<grid, kSegThreads, seg_numeric_smem(false), s>>>(
                cnt, rows, A.rp, A.ci, A.v, B.rp, B.ci, B.v, C.rp, C.ci, soff, S); note_launch();
        }
        // about four blocks a multiprocessor over all the rows' entries
        const dim3 cgrid(cnt, std::max(1, std::min(32, 608 / cnt)));
        seg_combine_kernel<<<cgrid, 128, 0, s>>>(cnt, rows, A.rp, C.rp, soff, S, C.v); note_launch();
        e = cudaGetLastError();
    } while (0);
    if (ws) sc.give(ws);
    if (gflags) sc.give(gflags);
    if (S) sc.give(S);
    if (d_sum) sc.give(d_sum);
    if (soff) sc.give(soff);
    return e;
}

}  // namespace

cudaError_t spgemm(const DevCsr &A, const DevCsr &B, DevCsr &C, int *overflow_host, cudaStream_t s)
{
    *overflow_host = 0;
    C = DevCsr();
    C.n = A.n;
    C.ncol = B.ncol;
    const int n = A.n;
    AMG_CUDA_TRY(cudaMallocAsync(&C.rp, sizeof(int) * ((size_t)n + 17), s));
    if (n == 0) {
        AMG_CUDA_TRY(cudaMemsetAsync(C.rp, 0, sizeof(int), s));
        return cudaSuccess;
    }
    int *work = nullptr;   // bin[n] tsize[n] perm[n] binCount binFill binStart overflow segmax
    const size_t nwork = (size_t)3 * n + 3 * (kNumBins + 1) + 2;
    AMG_CUDA_TRY(cudaMallocAsync(&work, sizeof(int) * nwork, s));
    int *d_bin = work, *d_tsize = work + n, *d_perm = work + 2 * n;
    int *d_binCount = work + 3 * n, *d_binFill = d_binCount + kNumBins + 1, *d_binStart = d_binFill + kNumBins + 1;
    int *d_ovf = d_binStart + kNumBins + 1, *d_segmax = d_ovf + 1;
    unsigned long long *d_ubstats = nullptr, h_ubstats[3] = {0, 0, 0};
    cudaError_t e = cudaMallocAsync(&d_ubstats, 3 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        cudaFreeAsync(work, s);
        return e;
    }
    int *gkeys = nullptr, *toff = nullptr;
    double *gvals = nullptr;
    Bins hb;
    do {
        if ((e = cudaMemsetAsync(d_binCount, 0, sizeof(int) * kNumBins, s))) break;
        if ((e = cudaMemsetAsync(d_ovf, 0, sizeof(int), s))) break;
        if ((e = cudaMemsetAsync(d_ubstats, 0, 3 * sizeof(unsigned long long), s))) break;
        // rows of many products: one warp walks a hash table 32 products at a time (thousands
        // of dependent steps on a stalled level's few long rows); a block with dense counters
        // takes them when B is narrow enough.  Rows whose bound asks for more than kCapTable
        // slots (a coarse operator's rows count their products many times over: 600 products
        // for 60 columns on the first coarse level) try a table of kCapTable first, eight warps
        // a block instead of one or two; the few that hold more columns go round again.  (The
        // fine level's R (A P): 3.2 -> 2.3 ms.)
        ub_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp, A.ci, B.rp, B.ncol, d_bin, d_binCount, d_tsize, d_ubstats,
                                                    B.ncol <= kDenseCols ? kDenseSymProducts : LLONG_MAX,
                                                    n >= kCapRows ? kCapTable : 0);
        note_launch();
        if ((e = cudaMemcpyAsync(h_ubstats, d_ubstats, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s))) break;
        if ((e = make_bins(n, d_bin, d_binCount, d_binFill, d_binStart, d_perm, hb, s))) break;
        // symbolic
        auto symbolic_pass = [&]() -> cudaError_t {
            cudaError_t r = cudaSuccess;
            for (int b = 0; b < kGlobalBin && !r; ++b)
                if (hb.count[b]) r = symbolic_bin(b, hb.count[b], d_perm + hb.start[b], A, B, C.rp, d_ovf, s, d_tsize);
            if (r || !hb.count[kGlobalBin]) return r;
            const int cnt = hb.count[kGlobalBin];
            const int *rows = d_perm + hb.start[kGlobalBin];
            if (B.ncol <= kDenseCols) {
                // long rows against few columns: dense counters in shared memory, a block per row
                if ((r = dense_attr())) return r;
                dense_symbolic_kernel<<<cnt, kDenseThreads, sizeof(int) * (size_t)B.ncol, s>>>(
                    cnt, rows, A.rp, A.ci, B.rp, B.ci, B.ncol, C.rp); note_launch();
                return cudaGetLastError();
            }
            int64_t total = 0;
            if ((r = global_tables(cnt, rows, d_tsize, &toff, &total, s))) return r;
            if ((r = cudaMallocAsync(&gkeys, sizeof(int) * (size_t)total, s))) return r;
            symbolic_global_kernel<<<grid_for((int64_t)cnt * 32, 128), 128, 0, s>>>(
                cnt, rows, toff, d_tsize, gkeys, A.rp, A.ci, B.rp, B.ci, C.rp, d_ovf); note_launch();
            if ((r = cudaGetLastError())) return r;
            cudaFreeAsync(gkeys, s); gkeys = nullptr;
            cudaFreeAsync(toff, s); toff = nullptr;
            return cudaSuccess;
        };
        if ((e = symbolic_pass())) break;
        if (h_ubstats[2] > 0) {
            // the capped rows that held more than kCapTable / 2 columns (count -1), in their own bins
            if ((e = cudaMemsetAsync(d_binCount, 0, sizeof(int) * kNumBins, s))) break;
            retry_bin_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, C.rp, d_tsize, d_bin, d_binCount); note_launch();
            if ((e = make_bins(n, d_bin, d_binCount, d_binFill, d_binStart, d_perm, hb, s))) break;
            if ((e = symbolic_pass())) break;
        }
        if ((e = scan_exclusive(C.rp, C.rp, n, s))) break;
        int nnz = 0;
        if ((e = cudaMemcpyAsync(&nnz, C.rp + n, sizeof(int), cudaMemcpyDeviceToHost, s))) break;
        if ((e = cudaMemcpyAsync(overflow_host, d_ovf, sizeof(int), cudaMemcpyDeviceToHost, s))) break;
        if ((e = cudaStreamSynchronize(s))) break;
        if (*overflow_host || nnz < 0) { e = cudaErrorInvalidValue; break; }
        C.nnz = nnz;
        // 16 elements of padding: bulk copies of row ranges widen to 16-byte boundaries
        if ((e = cudaMallocAsync(&C.ci, sizeof(int) * ((size_t)nnz + 16), s))) break;
        if ((e = cudaMallocAsync(&C.v, sizeof(double) * ((size_t)nnz + 16), s))) break;
        // numeric, binned by the exact row counts (rows of A of more than kSegLen entries apart)
        if ((e = cudaMemsetAsync(d_binCount, 0, sizeof(int) * kNumBins, s))) break;
        if ((e = cudaMemsetAsync(d_segmax, 0, sizeof(int), s))) break;
        const bool seg_wide = B.ncol <= kSegCols;
        const bool heavy_rows = h_ubstats[0] > (unsigned long long)kSegProducts;
        const bool long_products = h_ubstats[0] > (unsigned long long)kChainProducts &&
                                   h_ubstats[1] <= (unsigned long long)kChainTotal;
        exact_bin_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, C.rp, A.rp, d_bin, d_binCount, d_tsize, d_segmax,
                                                          seg_wide ? 1 : 0, heavy_rows ? A.ci : nullptr, B.rp);
        note_launch();
        int h_segmax = 0;
        if ((e = cudaMemcpyAsync(&h_segmax, d_segmax, sizeof(int), cudaMemcpyDeviceToHost, s))) break;
        if ((e = make_bins(n, d_bin, d_binCount, d_binFill, d_binStart, d_perm, hb, s))) break;
        // Products with rows of more than 2048 entries (stalled coarse levels): pattern, chain
        // placement and chain sums (see "numeric by chains" above).  Otherwise numeric_row, whose
        // single pass stays cheaper than the chains' staging in global memory on short rows (the
        // 128^3 fine level: 4.1 + 3.0 ms against 5.8 + 6.4 ms for A P and R (A P)); numeric_row also
        // when the products exceed the chains' int32 offsets.
        // Also products with rows of more than kChainProducts products (a stalled level's large
        // aggregates) when the whole product is small enough for the chains' global staging and B
        // is too wide for the segment kernels, which otherwise take those rows (kSegBin).
        bool chained = false;
        if (nnz > 0 && (hb.count[kGlobalBin] > 0 || (long_products && !seg_wide)) &&
            (e = numeric_chains(n, A, B, C, hb, d_perm, d_tsize, d_ovf, &chained, s)))
            break;
        for (int b = 0; b < kGlobalBin && !e && !chained; ++b)
            if (hb.count[b]) e = numeric_bin(b, hb.count[b], d_perm + hb.start[b], A, B, C, d_ovf, s);
        if (e) break;
        if (hb.count[kGlobalBin] && !chained) {
            int cnt = hb.count[kGlobalBin];
            const int *rows = d_perm + hb.start[kGlobalBin];
            int64_t total = 0;
            if ((e = global_tables(cnt, rows, d_tsize, &toff, &total, s))) break;
            if ((e = cudaMallocAsync(&gkeys, sizeof(int) * (size_t)total, s))) break;
            if ((e = cudaMallocAsync(&gvals, sizeof(double) * (size_t)total, s))) break;
            numeric_global_kernel<<<grid_for((int64_t)cnt * 32, 128), 128, 0, s>>>(
                cnt, rows, toff, d_tsize, gkeys, gvals, A.rp, A.ci, A.v, B.rp, B.ci, B.v, C.rp, C.ci, C.v, d_ovf); note_launch();
            if ((e = cudaGetLastError())) break;
        }
        if (hb.count[kSegBin]) {
            SegScratch sc;
            sc.take = [s](size_t bytes) -> void * {
                void *p = nullptr;
                return cudaMallocAsync(&p, bytes, s) == cudaSuccess ? p : nullptr;
            };
            sc.give = [s](void *p) { cudaFreeAsync(p, s); };
            bool no_room = false;
            if ((e = numeric_segmented(A, B, C, d_perm + hb.start[kSegBin], hb.count[kSegBin], h_segmax, d_ovf, sc,
                                       &no_room, s)))
                break;
            if (no_room) {
                cudaGetLastError();
                e = cudaErrorMemoryAllocation;
                break;
            }
        }
        if ((e = cudaMemcpyAsync(overflow_host, d_ovf, sizeof(int), cudaMemcpyDeviceToHost, s))) break;
        if ((e = cudaStreamSynchronize(s))) break;
        if (*overflow_host) e = cudaErrorInvalidValue;
    } while (0);
    if (gkeys) cudaFreeAsync(gkeys, s);
    if (gvals) cudaFreeAsync(gvals, s);
    if (toff) cudaFreeAsync(toff, s);
    cudaFreeAsync(d_ubstats, s);
    cudaFreeAsync(work, s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        if (C.rp) cudaFreeAsync(C.rp, s);
        if (C.ci) cudaFreeAsync(C.ci, s);
        if (C.v) cudaFreeAsync(C.v, s);
        cudaStreamSynchronize(s);
        C.rp = nullptr; C.ci = nullptr; C.v = nullptr; C.nnz = 0;
    }
    return e;
}


// ====================================================================================
// Allocation-free variant of C = A B (used by amg_spgemm_noalloc).
//
// Every temporary of the product lives in one file-scope device array of fixed size instead
// of memory from cudaMalloc: the int32 row pointers of A, B and C, the row bins, the scan
// workspace and the hash tables of long rows.  The array belongs to every device that loads
// this library and stays allocated until the process exits.  Its device address is looked up
// once per device (cudaGetSymbolAddress) by the first call on that device.  All calls share
// the array, so calls that overlap on the GPU (other host threads, or other streams without
// ordering) race on it; the array keeps the previous call's contents, and everything that
// must start at zero is cleared by the call itself.
// ====================================================================================
namespace {

constexpr size_t kNoAllocBytes = (size_t)32 << 20;      // 32 MiB
constexpr int64_t kNoAllocMaxRows = 1000000;             // rows of A and of B, each

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[64] = {nullptr};

struct Arena {
    unsigned char *base = nullptr;
    size_t size = 0, used = 0;
    template <typename T>
    T *take(size_t count)
    {
        size_t off = (used + 255) & ~(size_t)255;
        size_t bytes = count * sizeof(T);
        if (off + bytes > size) return nullptr;
        used = off + bytes;
        return reinterpret_cast<T *>(base + off);
    }
};

}  // namespace

// device address of the scratch array on the current device (looked up on first use)
cudaError_t noalloc_scratch(void **ptr, size_t *bytes)
{
    int dev = 0;
    AMG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *ptr = g_noalloc_addr[dev];
    *bytes = kNoAllocBytes;
    return cudaSuccess;
}

// Input checks of the allocation-free product, run before any kernel walks the rows: *bad
// counts row pointers that do not start at 0 or do not end at nnz, and column indices
// outside [0, ncol).
__global__ void noalloc_ends_kernel(const int64_t *rp, int n, int64_t nnz, int *bad)
{
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rp[0] != 0 || rp[n] != nnz)) atomicAdd(bad, 1);
}
__global__ void noalloc_cols_kernel(const int *ci, int64_t nnz, int ncol, int *bad)
{
    int cnt = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        int c = ci[e];
        cnt += (c < 0 || c >= ncol);
    }
    if (cnt) atomicAdd(bad, cnt);
}
// 64-bit sum of n non-negative ints (the counts an int32 scan is about to add up)
__global__ void noalloc_sum64_kernel(const int *v, int n, unsigned long long *out)
{
    unsigned long long acc = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int x = v[i];
        acc += x > 0 ? (unsigned long long)x : 0ull;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFullMask, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

namespace {
// sum of v[0..n) in 64 bits, read back to the host (synchronises the stream)
cudaError_t noalloc_sum64(const int *v, int n, unsigned long long *d_sum, unsigned long long *sum, cudaStream_t s)
{
    AMG_CUDA_TRY(cudaMemsetAsync(d_sum, 0, sizeof(unsigned long long), s));
    if (n > 0) {
        noalloc_sum64_kernel<<<grid_for(n, 256, 1024), 256, 0, s>>>(v, n, d_sum); note_launch();
        AMG_CUDA_TRY(cudaGetLastError());
    }
    AMG_CUDA_TRY(cudaMemcpyAsync(sum, d_sum, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    return cudaStreamSynchronize(s);
}
}  // namespace

// status: 0 ok, 1 sizes beyond the scratch limits (msg set), 2 output capacity too small
// (*nnz_out = required), 3 invalid row pointers or column indices, 4 hash overflow; CUDA
// errors returned as such.  Every return after the first launch synchronises the stream.
cudaError_t spgemm_noalloc(int nA, int ncolA, const int64_t *arp64, const int *aci, const double *av, int64_t nnzA,
                           int nB, int ncolB, const int64_t *brp64, const int *bci, const double *bv, int64_t nnzB,
                           int64_t *crp64, int *cci, double *cv, int64_t capacity, int64_t *nnz_out, int *status,
                           std::string *msg, cudaStream_t s)
{
    *status = 0;
    *nnz_out = 0;
    if (nA > kNoAllocMaxRows || nB > kNoAllocMaxRows) {
        *status = 1;
        *msg = "amg_spgemm_noalloc: more than 1,000,000 rows in A or B";
        return cudaSuccess;
    }
    void *base = nullptr;
    size_t bytes = 0;
    AMG_CUDA_TRY(noalloc_scratch(&base, &bytes));
    Arena ar{(unsigned char *)base, bytes, 0};
    const int n = nA;
    int *arp = ar.take<int>((size_t)nA + 1);
    int *brp = ar.take<int>((size_t)nB + 1);
    int *crp = ar.take<int>((size_t)nA + 17);
    int *work = ar.take<int>((size_t)3 * n + 3 * (kNumBins + 1) + 8);
    int *scan_ws = ar.take<int>(scan_ws_ints(n + 1) + 16);
    unsigned long long *d_sum = ar.take<unsigned long long>(1);
    if (!arp || !brp || !crp || !work || !scan_ws || !d_sum) {
        *status = 1;
        *msg = "amg_spgemm_noalloc: row arrays do not fit in the 32 MiB scratch";
        return cudaSuccess;
    }
    // from here on kernels may be in flight: every early exit synchronises the stream first
    auto stop = [&](int code, const char *m) -> cudaError_t {
        *status = code;
        *msg = m;
        return cudaStreamSynchronize(s);
    };
    int *d_bin = work, *d_tsize = work + n, *d_perm = work + 2 * n;
    int *d_binCount = work + 3 * n, *d_binFill = d_binCount + kNumBins + 1, *d_binStart = d_binFill + kNumBins + 1;
    int *d_flags = d_binStart + kNumBins + 1;     // [0] bad row pointers, [1] hash overflow, [2] bad columns
    AMG_CUDA_TRY(cudaMemsetAsync(d_flags, 0, 4 * sizeof(int), s));
    AMG_CUDA_TRY(convert_rowptr_to32(arp64, arp, nA + 1, d_flags, s));
    AMG_CUDA_TRY(convert_rowptr_to32(brp64, brp, nB + 1, d_flags, s));
    noalloc_ends_kernel<<<1, 32, 0, s>>>(arp64, nA, nnzA, d_flags); note_launch();
    noalloc_ends_kernel<<<1, 32, 0, s>>>(brp64, nB, nnzB, d_flags); note_launch();
    if (nnzA > 0) { noalloc_cols_kernel<<<grid_for(nnzA, 256, 1024), 256, 0, s>>>(aci, nnzA, nB, d_flags + 2); note_launch(); }
    if (nnzB > 0) { noalloc_cols_kernel<<<grid_for(nnzB, 256, 1024), 256, 0, s>>>(bci, nnzB, ncolB, d_flags + 2); note_launch(); }
    AMG_CUDA_TRY(cudaGetLastError());
    int hflags[3] = {0, 0, 0};
    AMG_CUDA_TRY(cudaMemcpyAsync(hflags, d_flags, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (hflags[0]) return stop(3, "amg_spgemm_noalloc: row pointers must start at 0, never decrease and end at nnz");
    if (hflags[2]) return stop(3, "amg_spgemm_noalloc: column index outside the matrix");
    DevCsr A, B, C;
    A.n = nA; A.ncol = ncolA; A.rp = arp; A.ci = const_cast<int *>(aci); A.v = const_cast<double *>(av);
    B.n = nB; B.ncol = ncolB; B.rp = brp; B.ci = const_cast<int *>(bci); B.v = const_cast<double *>(bv);
    C.n = nA; C.ncol = ncolB; C.rp = crp; C.ci = cci; C.v = cv;
    Bins hb;
    if (n == 0) {
        AMG_CUDA_TRY(cudaMemsetAsync(crp64, 0, sizeof(int64_t), s));
        return cudaStreamSynchronize(s);
    }
    // the long-row tables of the global bin: sizes summed in 64 bits and checked against what
    // is left of the scratch before the int32 scan of their offsets (slot_bytes per slot)
    auto global_tables = [&](int cnt, const int *rows, size_t slot_bytes, int **toff, void **keys,
                             double **vals) -> cudaError_t {
        *toff = ar.take<int>((size_t)cnt + 1);
        int *ws2 = ar.take<int>(scan_ws_ints(cnt + 1) + 16);
        if (!*toff || !ws2) return stop(1, "amg_spgemm_noalloc: long-row tables do not fit in the scratch");
        gather_tsize_kernel<<<grid_for(cnt, 256), 256, 0, s>>>(cnt, rows, d_tsize, *toff); note_launch();
        AMG_CUDA_TRY(cudaGetLastError());
        unsigned long long total = 0;
        AMG_CUDA_TRY(noalloc_sum64(*toff, cnt, d_sum, &total, s));
        if (total > 0x7fffffffull || total * slot_bytes > ar.size - ar.used)
            return stop(1, "amg_spgemm_noalloc: long-row tables do not fit in the scratch");
        AMG_CUDA_TRY(scan_exclusive_ws(*toff, *toff, cnt, ws2, s));
        *keys = ar.take<int>((size_t)total);
        if (vals) *vals = ar.take<double>((size_t)total);
        if (!*keys || (vals && !*vals)) return stop(1, "amg_spgemm_noalloc: long-row tables do not fit in the scratch");
        return cudaSuccess;
    };
    // symbolic
    AMG_CUDA_TRY(cudaMemsetAsync(d_binCount, 0, sizeof(int) * kNumBins, s));
    ub_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp, A.ci, B.rp, B.ncol, d_bin, d_binCount, d_tsize);
    note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    AMG_CUDA_TRY(make_bins(n, d_bin, d_binCount, d_binFill, d_binStart, d_perm, hb, s));
    for (int b = 0; b < kGlobalBin; ++b)
        if (hb.count[b]) AMG_CUDA_TRY(symbolic_bin(b, hb.count[b], d_perm + hb.start[b], A, B, C.rp, d_flags + 1, s));
    const size_t mark = ar.used;
    if (hb.count[kGlobalBin]) {
        int cnt = hb.count[kGlobalBin];
        const int *rows = d_perm + hb.start[kGlobalBin];
        int *toff = nullptr;
        void *gkeys = nullptr;
        AMG_CUDA_TRY(global_tables(cnt, rows, sizeof(int), &toff, &gkeys, nullptr));
        if (*status) return cudaSuccess;
        symbolic_global_kernel<<<grid_for((int64_t)cnt * 32, 128), 128, 0, s>>>(cnt, rows, toff, d_tsize, (int *)gkeys,
                                                                               A.rp, A.ci, B.rp, B.ci, C.rp, d_flags + 1); note_launch();
        AMG_CUDA_TRY(cudaGetLastError());
    }
    ar.used = mark;
    // nnz(C) in 64 bits before the int32 scan of the row counts
    unsigned long long nnz64 = 0;
    AMG_CUDA_TRY(noalloc_sum64(C.rp, n, d_sum, &nnz64, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(hflags, d_flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (hflags[1]) return stop(4, "amg_spgemm_noalloc: hash table overflow");
    *nnz_out = (int64_t)nnz64;
    if (nnz64 > 0x7ffffff0ull) return stop(1, "amg_spgemm_noalloc: more than 2^31 - 16 entries in C");
    if ((int64_t)nnz64 > capacity) return stop(2, "amg_spgemm_noalloc: output capacity smaller than nnz(C)");
    AMG_CUDA_TRY(scan_exclusive_ws(C.rp, C.rp, n, scan_ws, s));
    C.nnz = (int)nnz64;
    // numeric, binned by the exact row counts (rows of A of more than kSegLen entries apart;
    // d_flags[3] holds the longest of them)
    AMG_CUDA_TRY(cudaMemsetAsync(d_binCount, 0, sizeof(int) * kNumBins, s));
    AMG_CUDA_TRY(cudaMemsetAsync(d_flags + 3, 0, sizeof(int), s));
    exact_bin_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, C.rp, A.rp, d_bin, d_binCount, d_tsize, d_flags + 3,
                                                      B.ncol <= kSegCols ? 1 : 0);
    note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    int h_segmax = 0;
    AMG_CUDA_TRY(cudaMemcpyAsync(&h_segmax, d_flags + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(make_bins(n, d_bin, d_binCount, d_binFill, d_binStart, d_perm, hb, s));
    for (int b = 0; b < kGlobalBin; ++b)
        if (hb.count[b]) AMG_CUDA_TRY(numeric_bin(b, hb.count[b], d_perm + hb.start[b], A, B, C, d_flags + 1, s));
    if (hb.count[kGlobalBin]) {
        int cnt = hb.count[kGlobalBin];
        const int *rows = d_perm + hb.start[kGlobalBin];
        int *toff = nullptr;
        void *gkeys = nullptr;
        double *gvals = nullptr;
        AMG_CUDA_TRY(global_tables(cnt, rows, sizeof(int) + sizeof(double), &toff, &gkeys, &gvals));
        if (*status) return cudaSuccess;
        numeric_global_kernel<<<grid_for((int64_t)cnt * 32, 128), 128, 0, s>>>(cnt, rows, toff, d_tsize, (int *)gkeys,
                                                                              gvals, A.rp, A.ci, A.v, B.rp, B.ci, B.v,
                                                                              C.rp, C.ci, C.v, d_flags + 1); note_launch();
        AMG_CUDA_TRY(cudaGetLastError());
    }
    if (hb.count[kSegBin]) {
        SegScratch sc;
        sc.take = [&ar](size_t bytes) -> void * { return ar.take<unsigned char>(bytes); };
        sc.give = [](void *) {};
        bool no_room = false;
        AMG_CUDA_TRY(numeric_segmented(A, B, C, d_perm + hb.start[kSegBin], hb.count[kSegBin], h_segmax, d_flags + 1,
                                       sc, &no_room, s));
        if (no_room) return stop(1, "amg_spgemm_noalloc: the segment sums of long rows do not fit in the scratch");
    }
    AMG_CUDA_TRY(convert_rowptr_to64(C.rp, crp64, n + 1, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(hflags, d_flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (hflags[1]) { *status = 4; *msg = "amg_spgemm_noalloc: hash table overflow"; }
    return cudaSuccess;
}

}  // namespace amgk
