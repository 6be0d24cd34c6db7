// util.cu -- scans, fills, conversions, deterministic reductions, and the launch counter and
// event-based kernel timing used for roofline reports.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "amg_internal.cuh"

namespace amgk {

// ------------------------------------------------------------------------------------ counters
namespace {
std::atomic<long long> g_launches{0};
std::atomic<bool> g_prof_on{false};
std::mutex g_prof_mu;
std::vector<ProfRecord> g_pending;
thread_local ProfList *t_capture = nullptr;   // set while a graph body is being captured
std::vector<cudaEvent_t> g_pool;
long long g_prof_launches[KC_COUNT];
double g_prof_ms[KC_COUNT], g_prof_bytes[KC_COUNT];

cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void drain_locked()
{
    for (auto &r : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.stop) == cudaSuccess && cudaEventElapsedTime(&ms, r.start, r.stop) == cudaSuccess) {
            g_prof_launches[r.cls] += 1;
            g_prof_ms[r.cls] += ms;
            g_prof_bytes[r.cls] += r.bytes;
        } else {
            cudaGetLastError();
        }
        g_pool.push_back(r.start);
        g_pool.push_back(r.stop);
    }
    g_pending.clear();
}
}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
bool profiling_enabled() { return g_prof_on.load(std::memory_order_relaxed); }

ProfScope::ProfScope(int c, cudaStream_t st, double b) : cls(c), s(st), bytes(b)
{
    if (c < 0 || c >= KC_COUNT) return;
    if (!t_capture && !profiling_enabled()) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    start = take_event();
    // inside a capture the record must be an external event node (a plain record would only
    // mark a dependency inside the graph and never set the event)
    if (start) cudaEventRecordWithFlags(start, s, t_capture ? cudaEventRecordExternal : cudaEventRecordDefault);
}

ProfScope::~ProfScope()
{
    if (!start) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t stop = take_event();
    if (!stop) { g_pool.push_back(start); return; }
    cudaEventRecordWithFlags(stop, s, t_capture ? cudaEventRecordExternal : cudaEventRecordDefault);
    if (t_capture) {
        // the events become nodes of the graph being captured; the owner accounts them after
        // each launch of that graph
        t_capture->push_back(ProfRecord{cls, start, stop, bytes});
        return;
    }
    g_pending.push_back(ProfRecord{cls, start, stop, bytes});
    if (g_pending.size() > 4096) drain_locked();
}

void profile_capture_begin(ProfList *list) { t_capture = list; }
void profile_capture_end() { t_capture = nullptr; }

// after a launch of a graph whose body recorded `list` has completed
void profile_account(const ProfList &list)
{
    if (!profiling_enabled()) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (const auto &r : list) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.start, r.stop) == cudaSuccess) {
            g_prof_launches[r.cls] += 1;
            g_prof_ms[r.cls] += ms;
            g_prof_bytes[r.cls] += r.bytes;
        } else {
            cudaGetLastError();   // a failed query must not surface as a later launch's error
        }
    }
}

void profile_release(ProfList &list)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &r : list) { g_pool.push_back(r.start); g_pool.push_back(r.stop); }
    list.clear();
}

void profile_enable(int mode)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    drain_locked();
    if (mode == 1)
        for (int k = 0; k < KC_COUNT; ++k) { g_prof_launches[k] = 0; g_prof_ms[k] = 0.0; g_prof_bytes[k] = 0.0; }
    g_prof_on.store(mode != 0);
}

void profile_read(int cls, long long *launches, double *ms, double *bytes)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    drain_locked();
    *launches = g_prof_launches[cls];
    *ms = g_prof_ms[cls];
    *bytes = g_prof_bytes[cls];
}

int grid_for(int64_t work, int threads, int cap)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

// ------------------------------------------------------------------------------------ scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan of one tile; tile total to sums[blockIdx.x]; the last block also stores the
// running total at out[n] (before the cross-tile offsets are added).
__global__ void scan_tile_kernel(const int *in, int *out, int n, int *sums)
{
    __shared__ int warp_tot[kScanThreads / kWarp];
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems];
    int run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int idx = base + k;
        int x = idx < n ? in[idx] : 0;
        v[k] = run;
        run += x;
    }
    // inclusive scan of per-thread totals across the block
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int t = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
    }
    if (lane == 31) warp_tot[wid] = t;
    __syncthreads();
    if (wid == 0) {
        int w = lane < kScanThreads / kWarp ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / kWarp) warp_tot[lane] = w;
    }
    __syncthreads();
    int excl = t - run + (wid > 0 ? warp_tot[wid - 1] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int idx = base + k;
        if (idx < n) out[idx] = v[k] + excl;
    }
    if (threadIdx.x == kScanThreads - 1) {
        sums[blockIdx.x] = excl + run;
        if (blockIdx.x == gridDim.x - 1) out[n] = excl + run;
    }
}

__global__ void scan_add_kernel(int *out, int n, const int *offs)
{
    const int b = blockIdx.x;
    if (b == 0) return;
    const int add = offs[b];
    const int base = b * kScanTile;
    for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
        int idx = base + k;
        if (idx < n) out[idx] += add;
    }
    if (b == gridDim.x - 1 && threadIdx.x == 0) out[n] += add;
}

cudaError_t scan_exclusive(const int *in, int *out, int n, cudaStream_t s)
{
    if (n <= 0) {
        return cudaMemsetAsync(out, 0, sizeof(int), s);
    }
    int tiles = (n + kScanTile - 1) / kScanTile;
    int *sums = nullptr;
    AMG_CUDA_TRY(cudaMallocAsync(&sums, sizeof(int) * (size_t)(tiles + 1), s));
    scan_tile_kernel<<<tiles, kScanThreads, 0, s>>>(in, out, n, sums); note_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && tiles > 1) {
        e = scan_exclusive(sums, sums, tiles, s);
        if (e == cudaSuccess) {
            scan_add_kernel<<<tiles, kScanThreads, 0, s>>>(out, n, sums); note_launch();
            e = cudaGetLastError();
        }
    }
    cudaError_t e2 = cudaFreeAsync(sums, s);
    return e != cudaSuccess ? e : e2;
}

// Same scan with caller-provided workspace for the tile sums (no allocation); ws must hold
// scan_ws_ints(n) ints.
size_t scan_ws_ints(int n)
{
    size_t total = 0;
    while (n > 1) {
        int tiles = (n + kScanTile - 1) / kScanTile;
        total += (size_t)tiles + 1;
        if (tiles <= 1) break;
        n = tiles;
    }
    return total + 1;
}

cudaError_t scan_exclusive_ws(const int *in, int *out, int n, int *ws, cudaStream_t s)
{
    if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(int), s);
    int tiles = (n + kScanTile - 1) / kScanTile;
    int *sums = ws;
    scan_tile_kernel<<<tiles, kScanThreads, 0, s>>>(in, out, n, sums); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    if (tiles > 1) {
        AMG_CUDA_TRY(scan_exclusive_ws(sums, sums, tiles, ws + tiles + 1, s));
        scan_add_kernel<<<tiles, kScanThreads, 0, s>>>(out, n, sums); note_launch();
        AMG_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

// ------------------------------------------------------------------------------------ fills
__global__ void fill_int_kernel(int *p, int v, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}
__global__ void fill_double_kernel(double *p, double v, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}
cudaError_t fill_int(int *p, int value, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    fill_int_kernel<<<grid_for(n, 256, 4096), 256, 0, s>>>(p, value, n); note_launch();
    return cudaGetLastError();
}
cudaError_t fill_double(double *p, double value, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    fill_double_kernel<<<grid_for(n, 256, 4096), 256, 0, s>>>(p, value, n); note_launch();
    return cudaGetLastError();
}

__global__ void rp_to64_kernel(const int *a, int64_t *b, int n1)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += gridDim.x * blockDim.x) b[i] = a[i];
}
__global__ void rp_to32_kernel(const int64_t *a, int *b, int n1, int *bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += gridDim.x * blockDim.x) {
        int64_t v = a[i];
        if (v < 0 || v > 0x7fffffffLL || (i > 0 && a[i - 1] > v)) atomicAdd(bad, 1);
        b[i] = (int)v;
    }
}
__global__ void d2f_kernel(const double *a, float *b, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}
cudaError_t convert_rowptr_to64(const int *rp32, int64_t *rp64, int n1, cudaStream_t s)
{
    rp_to64_kernel<<<grid_for(n1, 256, 4096), 256, 0, s>>>(rp32, rp64, n1); note_launch();
    return cudaGetLastError();
}
cudaError_t convert_rowptr_to32(const int64_t *rp64, int *rp32, int n1, int *bad, cudaStream_t s)
{
    rp_to32_kernel<<<grid_for(n1, 256, 4096), 256, 0, s>>>(rp64, rp32, n1, bad); note_launch();
    return cudaGetLastError();
}
cudaError_t convert_d2f(const double *in, float *out, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    d2f_kernel<<<grid_for(n, 256, 8192), 256, 0, s>>>(in, out, n); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ reductions
// Fixed grid, fixed per-thread stride order, fixed tree: bitwise reproducible.
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double sh[kReduceThreads / kWarp];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < kReduceThreads / kWarp ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;   // valid in thread 0
}

__global__ void __launch_bounds__(kReduceThreads) dot_kernel(const double *x, const double *y, int n,
                                                            double *partial)
{
    double acc = 0.0;
    for (int i = blockIdx.x * kReduceThreads + threadIdx.x; i < n; i += kReduceBlocks * kReduceThreads)
        acc += x[i] * y[i];
    double t = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kReduceThreads) reduce_partials_kernel(const double *partial, int count,
                                                                        double *out)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < count; i += kReduceThreads) acc += partial[i];
    double t = block_sum(acc);
    if (threadIdx.x == 0) *out = t;
}

cudaError_t dot(const double *x, const double *y, int n, double *partial, double *out, cudaStream_t s)
{
    dot_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(x, y, n, partial); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    reduce_partials_kernel<<<1, kReduceThreads, 0, s>>>(partial, kReduceBlocks, out); note_launch();
    return cudaGetLastError();
}

cudaError_t dot_partial(const double *x, const double *y, int n, double *partial, cudaStream_t s)
{
    dot_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(x, y, n, partial); note_launch();
    return cudaGetLastError();
}

cudaError_t reduce_partials(const double *partial, int count, double *out, cudaStream_t s)
{
    reduce_partials_kernel<<<1, kReduceThreads, 0, s>>>(partial, count, out); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ host copies
// Memory the caller allocated with malloc / numpy (not allocated or registered by CUDA) is
// never handed to the copy engines: it moves through two pinned bounce halves of this
// thread, and the CPU alone reads or writes the caller's pages.  Device, managed and pinned
// memory is copied directly.
namespace {
constexpr size_t kBounceHalf = (size_t)4 << 20;

struct Bounce {
    unsigned char *buf = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    ~Bounce()
    {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (buf) cudaFreeHost(buf);
    }
};
thread_local Bounce t_bounce;

cudaError_t bounce_ready()
{
    Bounce &b = t_bounce;
    if (b.buf) return cudaSuccess;
    AMG_CUDA_TRY(cudaMallocHost((void **)&b.buf, 2 * kBounceHalf));
    for (cudaEvent_t &e : b.ev) AMG_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return cudaSuccess;
}

bool caller_pageable(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeUnregistered;
}
}  // namespace

cudaError_t copy_to_device(void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    if (bytes == 0) return cudaSuccess;
    if (!caller_pageable(src)) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
    AMG_CUDA_TRY(bounce_ready());
    Bounce &b = t_bounce;
    const unsigned char *in = (const unsigned char *)src;
    unsigned char *out = (unsigned char *)dst;
    bool used[2] = {false, false};
    for (size_t off = 0, k = 0; off < bytes; off += kBounceHalf, ++k) {
        const int h = (int)(k & 1);
        const size_t n = std::min(kBounceHalf, bytes - off);
        if (used[h]) AMG_CUDA_TRY(cudaEventSynchronize(b.ev[h]));   // the half's last copy is done
        std::memcpy(b.buf + h * kBounceHalf, in + off, n);
        AMG_CUDA_TRY(cudaMemcpyAsync(out + off, b.buf + h * kBounceHalf, n, cudaMemcpyHostToDevice, s));
        AMG_CUDA_TRY(cudaEventRecord(b.ev[h], s));
        used[h] = true;
    }
    // the halves are reused by this thread's next copy: wait for the last ones
    for (int h = 0; h < 2; ++h)
        if (used[h]) AMG_CUDA_TRY(cudaEventSynchronize(b.ev[h]));
    return cudaSuccess;
}

cudaError_t copy_to_host(void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    if (bytes == 0) return cudaSuccess;
    if (!caller_pageable(dst)) {
        AMG_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
        return cudaStreamSynchronize(s);
    }
    AMG_CUDA_TRY(bounce_ready());
    Bounce &b = t_bounce;
    const unsigned char *in = (const unsigned char *)src;
    unsigned char *out = (unsigned char *)dst;
    const size_t chunks = (bytes + kBounceHalf - 1) / kBounceHalf;
    // chunk k lands in half k & 1; the CPU drains chunk k while chunk k + 1 is in flight
    auto issue = [&](size_t k) -> cudaError_t {
        const size_t off = k * kBounceHalf, n = std::min(kBounceHalf, bytes - off);
        const int h = (int)(k & 1);
        AMG_CUDA_TRY(cudaMemcpyAsync(b.buf + h * kBounceHalf, in + off, n, cudaMemcpyDeviceToHost, s));
        return cudaEventRecord(b.ev[h], s);
    };
    AMG_CUDA_TRY(issue(0));
    for (size_t k = 0; k < chunks; ++k) {
        if (k + 1 < chunks) AMG_CUDA_TRY(issue(k + 1));
        const int h = (int)(k & 1);
        AMG_CUDA_TRY(cudaEventSynchronize(b.ev[h]));
        const size_t off = k * kBounceHalf, n = std::min(kBounceHalf, bytes - off);
        std::memcpy(out + off, b.buf + h * kBounceHalf, n);
    }
    return cudaStreamSynchronize(s);
}

}  // namespace amgk
