// amg_internal.cuh -- internal declarations shared by the library's CUDA translation units.
//
// Layout in device memory: CSR with int32 row pointers (nnz < 2^31 per matrix), int32
// sorted columns and double values (plus float copies of the level operators in mixed
// precision).  Vectors are dense arrays of double or float.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "amg.h"

namespace amgk {

// Kernel-launch counter (every launch site calls note_launch) and per-class kernel timing
// with CUDA events for roofline reports.
void note_launch();
void note_launches(long long k);
long long launch_count();
enum KernelClass { KC_PCG_SPMV = 0, KC_VCYCLE_SPMV = 1, KC_SPGEMM = 2, KC_SETUP_SPMV = 3, KC_COUNT = 4 };
bool profiling_enabled();
void profile_enable(int mode);   // 1 reset and record, 2 record (keep totals), 0 stop
struct ProfRecord {
    int cls;
    cudaEvent_t start, stop;
    double bytes;
};
using ProfList = std::vector<ProfRecord>;
// timing scopes opened while a graph body is captured go to `list` (their events become
// graph nodes); profile_account adds their elapsed times after each launch of the graph
void profile_capture_begin(ProfList *list);
void profile_capture_end();
void profile_account(const ProfList &list);
void profile_release(ProfList &list);
void profile_read(int cls, long long *launches, double *ms, double *bytes);
struct ProfScope {
    ProfScope(int cls, cudaStream_t s, double bytes);
    ~ProfScope();
    int cls;
    cudaStream_t s;
    double bytes;
    cudaEvent_t start = nullptr;
};

constexpr int kWarp = 32;
constexpr int kReduceBlocks = 304;        // fixed grid of the deterministic reductions (2 x 152 SMs)
constexpr int kReduceThreads = 256;

struct DevCsr {
    int n = 0;          // rows
    int ncol = 0;       // columns
    int64_t nnz = 0;
    int *rp = nullptr;  // n + 1
    int *ci = nullptr;  // nnz
    double *v = nullptr;
};

// --------------------------------------------------------------------------------- util.cu
// out[0..n] = exclusive scan of in[0..n-1]; out[n] = total.  in and out may alias.
cudaError_t scan_exclusive(const int *in, int *out, int n, cudaStream_t s);
// the same with caller-provided workspace of scan_ws_ints(n) ints (allocates nothing)
size_t scan_ws_ints(int n);
cudaError_t scan_exclusive_ws(const int *in, int *out, int n, int *ws, cudaStream_t s);
// grid-size helper: enough blocks of `threads` to cover `work` items, capped
int grid_for(int64_t work, int threads, int cap = 1 << 30);
cudaError_t fill_int(int *p, int value, int64_t n, cudaStream_t s);
cudaError_t fill_double(double *p, double value, int64_t n, cudaStream_t s);
cudaError_t convert_rowptr_to64(const int *rp32, int64_t *rp64, int n1, cudaStream_t s);
cudaError_t convert_rowptr_to32(const int64_t *rp64, int *rp32, int n1, int *bad, cudaStream_t s);
cudaError_t convert_d2f(const double *in, float *out, int64_t n, cudaStream_t s);
// Copies between the device and memory the caller owns (host or device).  Host memory that
// CUDA did not allocate or register moves through pinned bounce buffers of the calling
// thread, so the GPU never reads or writes the caller's pageable pages itself.
// copy_to_device returns once `src` may be reused; copy_to_host synchronises `s`.
cudaError_t copy_to_device(void *dst, const void *src, size_t bytes, cudaStream_t s);
cudaError_t copy_to_host(void *dst, const void *src, size_t bytes, cudaStream_t s);

// Deterministic reductions: stage 1 writes kReduceBlocks partial sums, stage 2 sums them in
// a fixed order into *out.
cudaError_t dot(const double *x, const double *y, int n, double *partial, double *out, cudaStream_t s);
cudaError_t reduce_partials(const double *partial, int count, double *out, cudaStream_t s);
cudaError_t dot_partial(const double *x, const double *y, int n, double *partial, cudaStream_t s);

// --------------------------------------------------------------------------------- setup.cu
// Index of each row's diagonal entry (-1 if absent) and its value.
cudaError_t diag_extract(const DevCsr &A, int *diagpos, double *d, cudaStream_t s);
// Eq. (7): strong[e], removed[e] (= weak off-diagonal) and kept-entry counts per row.
// strong_cnt (optional): each row's count of strong entries (the strong graph's row lengths)
cudaError_t strength(const DevCsr &A, const double *d, double theta, uint8_t *strong, uint8_t *removed,
                     int *kept, cudaStream_t s, int *strong_cnt = nullptr);
// nonsymmetric operators: strong[e] = own[e] or own[transpose of e]; removed and kept follow
cudaError_t symmetrize_strength(const DevCsr &A, const uint8_t *own, uint8_t *strong, uint8_t *removed, int *kept,
                                cudaStream_t s);
// §3.1's distance Laplacian on A's pattern (L: one value per stored entry, Ld: its diagonal);
// *bad counts coupled rows at zero distance
cudaError_t distance_laplacian(const DevCsr &A, const double *X, int dim, double *L, double *Ld, int *bad,
                               cudaStream_t s);
// coordinates of the next level: the mean of each aggregate's members (ascending member order)
cudaError_t coarse_coords(int nagg, const int *mstart, const int *members, const double *X, int dim, double *Xc,
                          cudaStream_t s);
// Strong graph (strong off-diagonals only) as CSR: rp from a scan of counts.
cudaError_t strong_graph_counts(const DevCsr &A, const uint8_t *strong, int *cnt, cudaStream_t s);
cudaError_t strong_graph_fill(const DevCsr &A, const uint8_t *strong, const int *grp, int *gci, cudaStream_t s);
// Aggregation on the strong graph; writes agg, root and the aggregate count (device int).
// Returns cudaErrorUnknown-free status; *status_flag set by kernels on internal failure.
struct AggWork {
    unsigned long long *t0, *t1;   // n tuples each
    int *rootof, *join1;           // n each
    int *counter;                  // 2 ints, device
};
cudaError_t aggregate_mis2(int n, const int *grp, const int *gci, uint64_t seed, int level, AggWork w, int *agg,
                           uint8_t *root, int *nagg_host, int *rounds_host, cudaStream_t s);
// Members of each aggregate in ascending order: mstart (nagg+1), members (n).
cudaError_t aggregate_members(int n, int nagg, const int *agg, int *mstart, int *members, int *fill,
                              cudaStream_t s);
// Per aggregate: nrm = sqrt(sum of B^2 over members, ascending); bad > 0 if a norm is 0.
cudaError_t aggregate_norms(int nagg, const int *mstart, const int *members, const double *B, double *nrm,
                            int *bad, cudaStream_t s);
// §2.5: mark pruned strong links (then their transposes) in `removed`, update kept counts.
cudaError_t sprsfy(const DevCsr &A, const uint8_t *strong, const int *agg, const uint8_t *root, int nagg,
                   const int *mstart, const int *members, uint8_t *drop, uint8_t *removed, int *kept,
                   cudaStream_t s);
// Filtered matrix (Eq. 6 or Algorithm 2) into Abar (rp from a scan of kept), plus the
// smoothing diagonal (Dbar, or Dtilde of Eq. 9-11) and the per-row lumping outcome.
cudaError_t filter(const DevCsr &A, const uint8_t *removed, int offlmp, double tau, int onenorm, double sigma,
                   DevCsr &Abar, double *Dsm, uint8_t *lumpflag, int *zero_diag, cudaStream_t s);
// Smoothed prolongator (unit basis), pattern counts then fill.
cudaError_t smooth_counts(const DevCsr &Abar, const int *agg, int *cnt, cudaStream_t s);
cudaError_t smooth_fill(const DevCsr &Abar, const int *agg, const double *B, const double *Dsm,
                        const double *omega_dev, DevCsr &P, cudaStream_t s);
// Algorithm 3 on each row of P (unit basis).
cudaError_t constrain(DevCsr &P, const int *agg, const double *B, uint8_t *cflag, cudaStream_t s);
// Column scaling P_ic /= nrm_c.
cudaError_t scale_columns(DevCsr &P, const double *nrm, cudaStream_t s);
// Transpose (rows of the result sorted).
cudaError_t transpose_counts(const DevCsr &P, int *cnt, cudaStream_t s);
cudaError_t transpose_fill(const DevCsr &P, DevCsr &R, int *fill, cudaStream_t s);
// Power method on D^-1 A (Rayleigh quotient of the last sweep), result on the device.
struct SpmvPlan;
cudaError_t power_lambda(const DevCsr &A, const SpmvPlan &plan, const double *D, int sweeps, uint64_t stream_seed,
                         double *x, double *y, double *partial, double *scal, double *lambda_dev, cudaStream_t s);
uint64_t power_stream_seed(uint64_t seed, int level, int purpose);
cudaError_t omega_from_lambda(const double *lambda_dev, double *omega_dev, cudaStream_t s);
cudaError_t invert_diag(const double *d, double *inv, float *invf, int n, int *zero, cudaStream_t s);

// --------------------------------------------------------------------------------- block.cu
// systems of PDEs (bs unknowns per node, k near-null-space vectors): the node graph of bs x bs
// blocks (counts, then columns, block Frobenius norms and each node's own norm), the block
// strength, the per-entry masks of A, the QR tentative prolongator and P's combination
int block_max_bs();
int block_max_k();
cudaError_t node_counts(const DevCsr &A, int bs, int *cnt, cudaStream_t s);
cudaError_t node_fill(const DevCsr &A, int bs, const int *nrp, int *nci, double *nF, double *fdiag, cudaStream_t s);
cudaError_t node_strength(int nn, const int *nrp, const int *nci, const double *nF, const double *fdiag, double theta,
                          uint8_t *nstrong, cudaStream_t s);
cudaError_t block_masks(const DevCsr &A, int bs, const int *nrp, const int *nci, const uint8_t *nstrong,
                        uint8_t *strong, uint8_t *removed, int *kept, cudaStream_t s);
cudaError_t block_tentative(int n, int bs, int k, int nagg, const int *mstart, const int *members, const double *B,
                            double *W, double *Qv, double *Bc, int *bad, cudaStream_t s);
cudaError_t block_pt(int n, int bs, int k, const int *agg, const double *Qv, DevCsr &Pt, cudaStream_t s);
cudaError_t block_combine(int n, int bs, int k, const int *agg, const double *Qv, const double *Dsm,
                          const double *omega, DevCsr &AP, cudaStream_t s);

// --------------------------------------------------------------------------------- server.cu
// 64-bit content hash of an operator (n, nnz, row pointers, columns, values; device arrays are
// copied to the host first); 0 with *err set when a copy fails.  The server's cache key and the
// router's (router.cu).
uint64_t operator_key(const amg_csr_t *A, std::string *err);

// --------------------------------------------------------------------------------- spgemm.cu
// C = A B, allocating C's arrays with cudaMalloc.  On failure C is left empty.
cudaError_t spgemm(const DevCsr &A, const DevCsr &B, DevCsr &C, int *overflow_host, cudaStream_t s);

// Allocation-free C = A B on device arrays (int64 row pointers in and out), temporaries in a
// fixed file-scope device array; see spgemm.cu.
cudaError_t spgemm_noalloc(int nA, int ncolA, const int64_t *arp64, const int *aci, const double *av, int64_t nnzA,
                           int nB, int ncolB, const int64_t *brp64, const int *bci, const double *bv, int64_t nnzB,
                           int64_t *crp64, int *cci, double *cv, int64_t capacity, int64_t *nnz_out, int *status,
                           std::string *msg, cudaStream_t s);

// --------------------------------------------------------------------------------- coarse.cu
// Dense SPD inverse of the coarsest operator in FP64 (FP32 Cholesky and inverse refined by
// Newton-Schulz in FP64, or the FP64 factorisation when that does not converge).  info = 0
// or the failing pivot row + 1.  work: coarse_work_bytes(n) bytes.
size_t coarse_work_bytes(int n);
// general: the operator may be nonsymmetric (Newton-Schulz from the scaled transpose; info =
// -1 when that does not converge)
cudaError_t coarse_inverse(const DevCsr &A, void *work, double *inv, int *info_dev, cudaStream_t s,
                           bool general = false);

// --------------------------------------------------------------------------------- solve.cu
// SpMV launch plan of one matrix: lanes per row and the shared-memory tile (entries; 0 = none)
// Rows far longer than the rest of their operator (a stalled coarse level can hold rows coupled
// to every other row): each is summed by a whole block of its own (spmv_long_kernel, solve.cu)
// and skipped by the row-tile kernel, whose lanes would otherwise walk it as one serial chain.
// The list travels by value in the kernel's parameters (no device memory of its own).
constexpr int kMaxLongRows = 128;
// Rows split off the row tiles of the solve's products, as the kernels take them (by value).
// rows lists first the rows of more than kSegRowLen entries, summed in segments of kSegRowLen
// entries by a block each (the last block of a row to finish adds the segments' sums in order),
// then the rows of more than kBlockRowLen entries (a block each), then the rest (a warp each).
constexpr int kSegRowLen = 1024;
constexpr int kBlockRowLen = 128;
struct SplitRows {
    const int *rows = nullptr;
    int nseg_rows = 0, nblock = 0, nwarp = 0;
    int nsegb = 0;               // segment blocks of the segmented rows
    const int *seg = nullptr;    // per segment block: row, first entry, end, its row's first segment block, count
    double *part = nullptr;      // per segment block: its sum
    unsigned *tick = nullptr;    // per segmented row (at its first segment block): blocks finished
};
struct LongRows {
    int count = 0;               // rows listed
    int len = 0x7fffffff;        // rows with more entries than this are long
    int rows[kMaxLongRows];
};
struct SpmvPlan {
    int lpr = 2;
    int cap = 0;
    LongRows lr;
    // sliced-ELL copy of the matrix read by the solve's products (solve.cu; ns = 0: none).
    // Columns and the layout are shared by the FP64 and FP32 values.
    int ns = 0;
    const int *sp = nullptr, *sw = nullptr, *sci = nullptr;
    const double *sv64 = nullptr;
    const float *sv32 = nullptr;
    size_t sell_entries = 0;     // stored entries of the copy, padding included
    // rows split off the row tiles for the solve's products (device arrays owned by the
    // hierarchy; sr.rows = nullptr: none): every row with more than split_len entries.  When
    // present it supersedes lr.
    SplitRows sr;
    int split_len = 0x7fffffff;
    int rowk = 0;                // short rows: one thread per row (spmv_rows_kernel)
};
// sliced ELL (slices of 32 rows): slices of an n-row matrix; widths sw[ns], offsets sp[ns+1]
// and the entry count in 64 bits (*total64, device; the offsets hold only when it fits an
// int); then columns and values
int sell_slices(int n);
cudaError_t sell_layout(int n, const int *rp, int *sw, int *sp, unsigned long long *total64, cudaStream_t s);
cudaError_t sell_fill_d(int n, const int *rp, const int *ci, const double *v, int ns, const int *sp, const int *sw,
                        int *sci, double *sv, cudaStream_t s);
cudaError_t sell_fill_f(int n, const int *rp, const float *v, int ns, const int *sp, const int *sw, float *sv,
                        cudaStream_t s);
cudaError_t spmv_plan(const int *rp, int n, int64_t nnz, SpmvPlan *plan, cudaStream_t s);
cudaError_t spmv_plans(int count, SpmvPlan *const *plans, const int *const *rps, const int *ns, const int64_t *nnzs,
                       cudaStream_t s);
// Marks the solve's plans of short rows for the thread-per-row kernel (one synchronisation)
cudaError_t spmv_short_rows(int count, SpmvPlan *const *plans, const int *const *rps, const int *ns,
                            const int64_t *nnzs, cudaStream_t s);
// The split rows of the solve's plans (above): counts with one synchronisation, then a list per
// plan with split rows from alloc(&list, entries) (device memory the caller owns).
cudaError_t spmv_split_rows(int count, SpmvPlan *const *plans, const int *const *rps, const int *ns,
                            const int64_t *nnzs, const std::function<cudaError_t(int **, size_t)> &alloc,
                            cudaStream_t s);
int spmv_partials_needed(int n);
int *spmv_error_flag();
int spmv_take_errors(cudaStream_t s);
struct LevelView {      // what the solve needs of one level, in working precision T
    int n = 0, nc = 0;
    const int *arp = nullptr, *aci = nullptr;
    const void *av = nullptr;               // A values (T)
    const int *prp = nullptr, *pci = nullptr;
    const void *pv = nullptr;               // P values (T)
    const int *rrp = nullptr, *rci = nullptr;
    const void *rv = nullptr;               // R values (T)
    const void *invdiag = nullptr;          // T
    double lambda = 0.0;                    // Chebyshev lambda_max
    int64_t nnz_a = 0;                      // stored entries of A
    SpmvPlan plan_a, plan_p, plan_r;
    void *f = nullptr, *x = nullptr, *x2 = nullptr, *r = nullptr, *d = nullptr;   // T work vectors
};
struct SolveCtx {
    int nlev = 0;
    LevelView lev[32];
    int coarse_n = 0;
    const double *coarse_inv = nullptr;     // dense n x n FP64
    // coarse_degree > 0: the coarsest level is solved by coarse_degree Chebyshev steps on
    // [theta - delta, theta + delta] (its LevelView then holds A, D^-1, x2 and d), not by the inverse
    int coarse_degree = 0;
    double coarse_theta = 0.0, coarse_delta = 0.0;
    double *coarse_tmp_in = nullptr, *coarse_tmp_out = nullptr;
    int cheb_degree = 2;
    double cheb_ratio = 10.0;
    double cheb_boost = 1.1;
    int mixed = 0;
};
// z = V-cycle(r) from z = 0 on the finest level (r, z double on the device).
cudaError_t vcycle(const SolveCtx &c, const double *r, double *z, cudaStream_t s);
// The coarsest level's Chebyshev solve (solve.cu): *degree = 0 when it does not apply (the
// spectrum of D^-1 A too wide for a short polynomial, or the check solve's relative residual
// *check above 1e-12); else the degree and the interval's centre and half-width.
cudaError_t coarse_cheb_setup(const DevCsr &A, const SpmvPlan &pl, const double *invdiag, int *degree,
                              double *theta, double *delta, double *check, cudaStream_t s);

// PCG building blocks (FP64, deterministic reductions; scalars live on the device)
struct PcgScalars {     // device
    double rz, rz_next, rz_new, rz_cross, pq, alpha, beta, rr, bb, tmp;
};
cudaError_t spmv_dot(const DevCsr &A, const SpmvPlan &pl, const double *p, double *q, double *partial,
                     double *result, unsigned *counter, cudaStream_t s);
cudaError_t spmv_scaled_dot(const DevCsr &A, const SpmvPlan &pl, const double *D, const double *x, double *y,
                            double *partial, double *result, unsigned *counter, cudaStream_t s);
cudaError_t spmv_power(const DevCsr &A, const SpmvPlan &pl, const double *invD, const double *x, const double *xx,
                       double *y, double *yy, double *partial, double *lambda, unsigned *counter, cudaStream_t s,
                       bool with_lambda = true);
cudaError_t spmv_d(const DevCsr &A, const SpmvPlan &pl, const double *x, double *y, cudaStream_t s);
cudaError_t residual_d(const DevCsr &A, const SpmvPlan &pl, const double *b, const double *x, double *r,
                       cudaStream_t s);
cudaError_t pcg_update_xr(int n, double *x, double *r, const double *p, const double *q, PcgScalars *sc,
                          const double *pq_partial, int pq_count, double *rr_partial, cudaStream_t s);
int spmv_block_count(int n, const SpmvPlan &pl);
// r . z (and r . z_prev when z_prev is not null: flexible update) then p = z + beta p
cudaError_t pcg_update_p(int n, double *p, const double *r, const double *z, const double *z_prev, PcgScalars *sc,
                         double *pa, double *pb, unsigned *counters, cudaStream_t s);
cudaError_t pcg_store(const double *partial, int count, double *dst, cudaStream_t s);

int pick_lanes(double avg_row);

}  // namespace amgk

// error plumbing shared by the host code
#define AMG_CUDA_TRY(expr)                          \
    do {                                            \
        cudaError_t _e = (expr);                    \
        if (_e != cudaSuccess) return _e;           \
    } while (0)
