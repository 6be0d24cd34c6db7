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
// Compiled without FMA contraction: every sum and product is rounded as written, in the
// order stated, so structures and tentative-prolongator values match a sequential evaluation.
#include <climits>

#include "amg_internal.cuh"

namespace amgk {
namespace {

constexpr int kMaxBs = 16;     // unknowns per node at most
constexpr int kMaxK = 8;       // near-null-space vectors at most

// node I's bs rows merged: calls visit(J, p, end) for each coupled node J in ascending order,
// with p[r] at row r's first entry of node J (entries of J are contiguous in a sorted row)
template <typename Visit>
__device__ __forceinline__ void merge_node_rows(const int *rp, const int *ci, int bs, int I, Visit visit)
{
    int p[kMaxBs], end[kMaxBs];
    for (int r = 0; r < bs; ++r) {
        p[r] = rp[I * bs + r];
        end[r] = rp[I * bs + r + 1];
    }
    for (;;) {
        int J = INT_MAX;
        for (int r = 0; r < bs; ++r)
            if (p[r] < end[r]) J = min(J, ci[p[r]] / bs);
        if (J == INT_MAX) break;
        visit(J, p, end);
        for (int r = 0; r < bs; ++r)
            while (p[r] < end[r] && ci[p[r]] / bs == J) ++p[r];
    }
}

__global__ void node_count_kernel(int nn, const int *rp, const int *ci, int bs, int *cnt)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nn) return;
    int c = 0;
    merge_node_rows(rp, ci, bs, I, [&](int, const int *, const int *) { ++c; });
    cnt[I] = c;
}

// nci, F_IJ (squares summed over the block's rows in order, each row's entries in order),
// and F_II per node
__global__ void node_fill_kernel(int nn, const int *rp, const int *ci, const double *v, int bs, const int *nrp,
                                 int *nci, double *nF, double *fdiag)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nn) return;
    int t = nrp[I];
    merge_node_rows(rp, ci, bs, I, [&](int J, const int *p, const int *end) {
        double acc = 0.0;
        for (int r = 0; r < bs; ++r)
            for (int e = p[r]; e < end[r] && ci[e] / bs == J; ++e) acc = acc + v[e] * v[e];
        const double f = sqrt(acc);
        nci[t] = J;
        nF[t] = f;
        if (J == I) fdiag[I] = f;
        ++t;
    });
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

// one thread per aggregate: B_a = Q_a R_a by modified Gram-Schmidt in column order; a column
// left with norm <= 1e-12 of its norm before the projections marks *bad (rank-deficient)
__global__ void block_tentative_kernel(int n, int bs, int k, int nagg, const int *mstart, const int *members,
                                       const double *B, double *W, double *Qv, double *Bc, int *bad)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nagg) return;
    const int m0 = mstart[a], m = (mstart[a + 1] - m0) * bs;
    double *w = W + (size_t)m0 * bs * k;
    const size_t nc = (size_t)nagg * k;
    double R[kMaxK * kMaxK];
    for (int j = 0; j < k * k; ++j) R[j] = 0.0;
    for (int j = 0; j < k; ++j)
        for (int t = 0; t < m; ++t) {
            const int i = members[m0 + t / bs] * bs + t % bs;
            w[(size_t)j * m + t] = B[(size_t)j * n + i];
        }
    for (int j = 0; j < k; ++j) {
        double *wj = w + (size_t)j * m;
        double before = 0.0;
        for (int t = 0; t < m; ++t) before = before + wj[t] * wj[t];
        for (int l = 0; l < j; ++l) {
            const double *wl = w + (size_t)l * m;
            double r = 0.0;
            for (int t = 0; t < m; ++t) r = r + wl[t] * wj[t];
            R[l * k + j] = r;
            for (int t = 0; t < m; ++t) wj[t] = wj[t] - r * wl[t];
        }
        double s = 0.0;
        for (int t = 0; t < m; ++t) s = s + wj[t] * wj[t];
        const double rjj = sqrt(s);
        if (!(rjj > 1e-12 * sqrt(before))) {
            atomicAdd(bad, 1);
            return;
        }
        for (int t = 0; t < m; ++t) wj[t] = wj[t] / rjj;
        R[j * k + j] = rjj;
    }
    for (int t = 0; t < m; ++t) {
        const int i = members[m0 + t / bs] * bs + t % bs;
        for (int j = 0; j < k; ++j) Qv[(size_t)i * k + j] = w[(size_t)j * m + t];
    }
    for (int c = 0; c < k; ++c)
        for (int j = 0; j < k; ++j) Bc[(size_t)c * nc + (size_t)a * k + j] = R[j * k + c];
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
    node_count_kernel<<<grid_for(nn, 128), 128, 0, s>>>(nn, A.rp, A.ci, bs, cnt); note_launch();
    return cudaGetLastError();
}

cudaError_t node_fill(const DevCsr &A, int bs, const int *nrp, int *nci, double *nF, double *fdiag, cudaStream_t s)
{
    const int nn = A.n / bs;
    if (nn == 0) return cudaSuccess;
    node_fill_kernel<<<grid_for(nn, 128), 128, 0, s>>>(nn, A.rp, A.ci, A.v, bs, nrp, nci, nF, fdiag); note_launch();
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
    block_tentative_kernel<<<grid_for(nagg, 64), 64, 0, s>>>(n, bs, k, nagg, mstart, members, B, W, Qv, Bc, bad); note_launch();
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
