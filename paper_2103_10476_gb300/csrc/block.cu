// block.cu -- setup kernels for systems of PDEs: bs unknowns per node (interleaved: unknown
// bs v + c is component c of node v) and k near-null-space vectors.  The paper treats scalar
// PDEs and leaves systems to future work; these extend its steps:
//   * strength between nodes: the Frobenius norm F_IJ of the bs x bs block coupling nodes I and
//     J in Eq. (7) in place of |a_ij| (F_II, F_JJ in place of a_ii, a_jj); for bs = 1 this is
//     Eq. (7) itself;
//   * aggregation: the distance-2 MIS of the strong node graph (the scalar kernels on it);
//   * tentative prolongator: each aggregate's block of B (its nodes' unknowns, nodes and
//     components ascending) factored B_a = Q_a R_a by modified Gram-Schmidt; Pt holds Q_a,
//     the coarse near-null space is R_a (k unknowns per aggregate on the coarse level);
//   * P = Pt - omega Dbar^-1 (Abar Pt) with Abar Pt from the generic SpGEMM (Eq. 3).
// Compiled without FMA contraction: every sum and product is rounded as written.  The block
// norms are summed in the stated order, so the strength decisions match a sequential
// evaluation bit for bit; the QR's inner products are warp sums in a fixed order (values equal
// to a sequential evaluation up to rounding).
#include <climits>

#include "amg_internal.cuh"

namespace amgk {
namespace {

constexpr int kMaxBs = 16;     // unknowns per node at most
constexpr int kMaxK = 8;       // near-null-space vectors at most

// One warp per node I: lane r < bs holds the cursor of row I bs + r; each step the warp takes
// the smallest node id J under the cursors, every lane moves past J's entries in its row, and
// lane 0 emits J (count only when nci is null).  Node ids ascend along a sorted row.
__device__ __forceinline__ int warp_min_int(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__global__ void node_merge_kernel(int nn, const int *rp, const int *ci, int bs, const int *nrp, int *cnt, int *nci)
{
    const int lane = threadIdx.x & 31;
    const int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (I >= nn) return;
    int p = 0, end = 0;
    if (lane < bs) {
        p = rp[I * bs + lane];
        end = rp[I * bs + lane + 1];
    }
    int c = 0;
    int out = nci ? nrp[I] : 0;
    for (;;) {
        const int head = p < end ? ci[p] / bs : INT_MAX;
        const int J = warp_min_int(head);
        if (J == INT_MAX) break;
        while (p < end && ci[p] / bs == J) ++p;
        if (nci && lane == 0) nci[out + c] = J;
        ++c;
    }
    if (!nci && lane == 0) cnt[I] = c;
}

// one thread per node entry t = (I, J): F_IJ = sqrt of the squares of the block's entries,
// summed over its rows in order and each row's entries in order (the columns J bs .. J bs +
// bs - 1 of a sorted row are contiguous: found by binary search); F_II also to fdiag
__global__ void node_norm_kernel(int nn, int64_t nnz_n, const int *rp, const int *ci, const double *v, int bs,
                                 const int *nrp, const int *nci, double *nF, double *fdiag)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nnz_n) return;
    int lo = 0, hi = nn - 1;                     // node I: the last with nrp[I] <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (nrp[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int I = lo, J = nci[t];
    const int c0 = J * bs, c1 = c0 + bs;
    double acc = 0.0;
    for (int r = 0; r < bs; ++r) {
        int a = rp[I * bs + r], b = rp[I * bs + r + 1];
        while (a < b) {                          // first entry with column >= c0
            const int mid = (a + b) >> 1;
            if (ci[mid] < c0) a = mid + 1; else b = mid;
        }
        for (int e = a; e < rp[I * bs + r + 1] && ci[e] < c1; ++e) acc = acc + v[e] * v[e];
    }
    const double f = sqrt(acc);
    nF[t] = f;
    if (J == I) fdiag[I] = f;
}

__global__ void node_strong_kernel(int nn, const int *nrp, const int *nci, const double *nF, const double *fdiag,
                                   double theta, uint8_t *nstrong)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nn) return;
    const double fi = fdiag[I];
    for (int t = nrp[I]; t < nrp[I + 1]; ++t) {
        const int J = nci[t];
        nstrong[t] = (J != I && nF[t] >= theta * sqrt(fi * fdiag[J])) ? 1 : 0;
    }
}

// per stored entry of A: inside a node's block (off the diagonal) strong, else its node
// pair's flag; removed = off the diagonal and not strong; kept[i] = entries of row i kept
__global__ void block_masks_kernel(int n, const int *rp, const int *ci, int bs, const int *nrp, const int *nci,
                                   const uint8_t *nstrong, uint8_t *strong, uint8_t *removed, int *kept)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int I = i / bs;
    const int lo0 = nrp[I], hi0 = nrp[I + 1];
    int k = 0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const int c = ci[e], J = c / bs;
        uint8_t s;
        if (J == I) {
            s = c != i;
        } else {
            int lo = lo0, hi = hi0 - 1;
            s = 0;
            while (lo <= hi) {
                const int mid = (lo + hi) >> 1;
                const int v = nci[mid];
                if (v == J) { s = nstrong[mid]; break; }
                if (v < J) lo = mid + 1; else hi = mid - 1;
            }
        }
        strong[e] = s;
        const uint8_t rm = (c != i && !s) ? 1 : 0;
        removed[e] = rm;
        k += !rm;
    }
    kept[i] = k;
}

// fixed-order warp sum: each lane's partial over its rows t = lane, lane + 32, ... in order,
// then a butterfly over the lanes (every lane receives the same total)
__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// one warp per aggregate: B_a = Q_a R_a by modified Gram-Schmidt in column order, the rows
// spread over the lanes (lane l owns rows l, l + 32, ...); a column left with norm <= 1e-12 of
// its norm before the projections marks *bad (rank-deficient)
__global__ void block_tentative_kernel(int n, int bs, int k, int nagg, const int *mstart, const int *members,
                                       const double *B, double *W, double *Qv, double *Bc, int *bad)
{
    const int lane = threadIdx.x & 31;
    const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (a >= nagg) return;
    const int m0 = mstart[a], m = (mstart[a + 1] - m0) * bs;
    double *w = W + (size_t)m0 * bs * k;
    const size_t nc = (size_t)nagg * k;
    double R[kMaxK * kMaxK];
    for (int j = 0; j < k * k; ++j) R[j] = 0.0;
    for (int j = 0; j < k; ++j)
        for (int t = lane; t < m; t += 32) {
            const int i = members[m0 + t / bs] * bs + t % bs;
            w[(size_t)j * m + t] = B[(size_t)j * n + i];
        }
    for (int j = 0; j < k; ++j) {
        double *wj = w + (size_t)j * m;
        double before = 0.0;
        for (int t = lane; t < m; t += 32) before = before + wj[t] * wj[t];
        before = warp_sum_d(before);
        for (int l = 0; l < j; ++l) {
            const double *wl = w + (size_t)l * m;
            double r = 0.0;
            for (int t = lane; t < m; t += 32) r = r + wl[t] * wj[t];
            r = warp_sum_d(r);
            R[l * k + j] = r;
            for (int t = lane; t < m; t += 32) wj[t] = wj[t] - r * wl[t];
        }
        double s = 0.0;
        for (int t = lane; t < m; t += 32) s = s + wj[t] * wj[t];
        s = warp_sum_d(s);
        const double rjj = sqrt(s);
        if (!(rjj > 1e-12 * sqrt(before))) {
            if (lane == 0) atomicAdd(bad, 1);
            return;                              // uniform over the warp
        }
        for (int t = lane; t < m; t += 32) wj[t] = wj[t] / rjj;
        R[j * k + j] = rjj;
    }
    for (int t = lane; t < m; t += 32) {
        const int i = members[m0 + t / bs] * bs + t % bs;
        for (int j = 0; j < k; ++j) Qv[(size_t)i * k + j] = w[(size_t)j * m + t];
    }
    if (lane < k)
        for (int j = 0; j < k; ++j) Bc[(size_t)lane * nc + (size_t)a * k + j] = R[j * k + lane];
}

// Pt: row i holds k entries, columns agg(i/bs) k + j, values Qv[i k + j]
__global__ void block_pt_kernel(int n, int bs, int k, const int *agg, const double *Qv, int *rp, int *ci, double *v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i == 0) rp[0] = 0;
    rp[i + 1] = (i + 1) * k;
    const int c0 = agg[i / bs] * k;
    for (int j = 0; j < k; ++j) {
        ci[(size_t)i * k + j] = c0 + j;
        v[(size_t)i * k + j] = Qv[(size_t)i * k + j];
    }
}

// P = Pt - (omega / Dbar_i) (Abar Pt), in place over Abar Pt (whose pattern holds Pt's)
__global__ void block_combine_kernel(int n, int bs, int k, const int *agg, const double *Qv, const double *Dsm,
                                     const double *omega, const int *rp, const int *ci, double *v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double scale = *omega / Dsm[i];
    const int c0 = agg[i / bs] * k;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const int c = ci[e];
        const double pt = (c >= c0 && c < c0 + k) ? Qv[(size_t)i * k + (c - c0)] : 0.0;
        v[e] = pt - scale * v[e];
    }
}

}  // namespace

int block_max_bs() { return kMaxBs; }
int block_max_k() { return kMaxK; }

cudaError_t node_counts(const DevCsr &A, int bs, int *cnt, cudaStream_t s)
{
    const int nn = A.n / bs;
    if (nn == 0) return cudaSuccess;
    node_merge_kernel<<<grid_for((int64_t)nn * 32, 256), 256, 0, s>>>(nn, A.rp, A.ci, bs, nullptr, cnt, nullptr); note_launch();
    return cudaGetLastError();
}

cudaError_t node_fill(const DevCsr &A, int bs, const int *nrp, int *nci, double *nF, double *fdiag, cudaStream_t s)
{
    const int nn = A.n / bs;
    if (nn == 0) return cudaSuccess;
    node_merge_kernel<<<grid_for((int64_t)nn * 32, 256), 256, 0, s>>>(nn, A.rp, A.ci, bs, nrp, nullptr, nci); note_launch();
    AMG_CUDA_TRY(cudaGetLastError());
    int64_t nnz_n = 0;
    AMG_CUDA_TRY(cudaMemcpyAsync(&nnz_n, nrp + nn, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (nnz_n == 0) return cudaSuccess;
    node_norm_kernel<<<grid_for(nnz_n, 256), 256, 0, s>>>(nn, nnz_n, A.rp, A.ci, A.v, bs, nrp, nci, nF, fdiag); note_launch();
    return cudaGetLastError();
}

cudaError_t node_strength(int nn, const int *nrp, const int *nci, const double *nF, const double *fdiag, double theta,
                          uint8_t *nstrong, cudaStream_t s)
{
    if (nn == 0) return cudaSuccess;
    node_strong_kernel<<<grid_for(nn, 256), 256, 0, s>>>(nn, nrp, nci, nF, fdiag, theta, nstrong); note_launch();
    return cudaGetLastError();
}

cudaError_t block_masks(const DevCsr &A, int bs, const int *nrp, const int *nci, const uint8_t *nstrong,
                        uint8_t *strong, uint8_t *removed, int *kept, cudaStream_t s)
{
    if (A.n == 0) return cudaSuccess;
    block_masks_kernel<<<grid_for(A.n, 256), 256, 0, s>>>(A.n, A.rp, A.ci, bs, nrp, nci, nstrong, strong, removed,
                                                          kept); note_launch();
    return cudaGetLastError();
}

cudaError_t block_tentative(int n, int bs, int k, int nagg, const int *mstart, const int *members, const double *B,
                            double *W, double *Qv, double *Bc, int *bad, cudaStream_t s)
{
    if (nagg == 0) return cudaSuccess;
    block_tentative_kernel<<<grid_for((int64_t)nagg * 32, 128), 128, 0, s>>>(n, bs, k, nagg, mstart, members, B, W, Qv,
                                                                            Bc, bad); note_launch();
    return cudaGetLastError();
}

cudaError_t block_pt(int n, int bs, int k, const int *agg, const double *Qv, DevCsr &Pt, cudaStream_t s)
{
    if (n == 0) return cudaMemsetAsync(Pt.rp, 0, sizeof(int), s);
    block_pt_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, bs, k, agg, Qv, Pt.rp, Pt.ci, Pt.v); note_launch();
    return cudaGetLastError();
}

cudaError_t block_combine(int n, int bs, int k, const int *agg, const double *Qv, const double *Dsm,
                          const double *omega, DevCsr &AP, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    block_combine_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, bs, k, agg, Qv, Dsm, omega, AP.rp, AP.ci, AP.v); note_launch();
    return cudaGetLastError();
}

}  // namespace amgk
