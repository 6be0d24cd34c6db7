/*
 * amg.h -- C ABI of the GB300 (sm_103a) smoothed-aggregation AMG library.
 *
 * The library builds a smoothed-aggregation multigrid hierarchy for a sparse symmetric
 * positive definite matrix and solves A x = b with conjugate gradients preconditioned by
 * one V-cycle per iteration.  It follows Hu, Siefert and Tuminaro, "Smooth Aggregation for
 * Difficult Stretched Mesh and Coefficient Variation Problems" (arXiv:2103.10476):
 *   - the problem A_1 u_1 = f_1 and the V-cycle: §1.1, Eq. (1) and Algorithm 1;
 *   - Galerkin coarse operators A_{l+1} = P_l^T A_l P_l: §1.1, Eq. (2);
 *   - smoothed prolongator P = (I - omega D^-1 Abar) Pt, omega = 4 / (3 lambda): Eq. (3);
 *   - aggregates (Eq. 4), tentative prolongator from the near-null space (Eq. 5),
 *     filtered matrix (Eq. 6) and the strength test |a_ij| >= theta sqrt(a_ii a_jj) (Eq. 7);
 *   - the four adaptations, each switchable: 1Norm (§2.1-§2.2, Eq. 9-11), OffLmp (§2.3,
 *     Algorithm 2), Cnstrnt (§2.4, Algorithm 3) and Sprsfy (§2.5);
 *   - Chebyshev smoothing on [b lambda/10, b lambda] with lambda from ten power-method sweeps
 *     (b = 1.1 by default: ten sweeps underestimate lambda_max), and a direct solve on the
 *     coarsest level (§3.1).
 *
 * Every step runs in this library's CUDA kernels on the current device.  All functions
 * return an amg_status_t; no C++ exception crosses the ABI.  A handle is not thread-safe:
 * calls on one handle must not overlap.  Different handles are independent.
 */
#ifndef AMG_GB300_H
#define AMG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AMG_OK = 0,
    AMG_ERR_INVALID_ARG = 1,    /* bad pointer, size, parameter or matrix structure          */
    AMG_ERR_OOM = 2,            /* device allocation failed                                   */
    AMG_ERR_CUDA = 3,           /* a CUDA runtime call failed (see amg_last_error)            */
    AMG_ERR_ZERO_DIAG = 4,      /* a zero diagonal in the filtered or level matrix            */
    AMG_ERR_EIGEN = 5,          /* eigenvalue estimate <= 0 or not finite (§3.1's failure)    */
    AMG_ERR_COARSE_NOT_SPD = 6, /* Cholesky pivot <= 0 on the coarsest level                  */
    AMG_ERR_NOT_CONVERGED = 7,  /* max_iter reached; x holds the last iterate                 */
    AMG_ERR_BUDGET = 8,         /* a memory budget would be exceeded                          */
    AMG_ERR_UNSUPPORTED = 9,    /* size beyond the library's limits, or a mode it lacks       */
    AMG_ERR_INTERNAL = 10,      /* a kernel reported an internal limit (e.g. hash overflow)   */
    AMG_PENDING = 11            /* a served request is not finished yet (amg_server_poll)     */
} amg_status_t;

/* adaptation bits (0 = traditional smoothed aggregation) */
enum { AMG_VAR_1NORM = 1, AMG_VAR_OFFLMP = 2, AMG_VAR_SPRSFY = 4, AMG_VAR_CNSTRNT = 8 };
/* arithmetic of the hierarchy and V-cycle: FP64 throughout, or FP32 levels and V-cycle
 * inside an FP64 conjugate-gradient iteration (outer residual, dot products, eigenvalue
 * estimates and the coarsest factorisation stay FP64) */
enum { AMG_FP64 = 0, AMG_MIXED = 1 };
/* tentative-prolongator columns: divided by the 2-norm of the near-null space on the
 * aggregate (orthonormal), or Eq. (5) as printed (unit) */
enum { AMG_PT_ORTHONORMAL = 0, AMG_PT_UNIT = 1 };
/* eigenvalue used with the 1-norm diagonal: the bound 1 (§2.1) or the power method */
enum { AMG_LAMBDA_ONE = 0, AMG_LAMBDA_POWER = 1 };
/* Strength of connection (Eq. 7) evaluated on A_l itself, or on the distance Laplacian of
 * §3.1: the pattern of A_l with off-diagonal -1 / |x_i - x_j| and a diagonal that makes each
 * row sum to zero, from coordinates given to amg_setup_coords (level 0) and, on coarser
 * levels, the mean coordinates of each aggregate's members. */
enum { AMG_STRENGTH_MATRIX = 0, AMG_STRENGTH_DISTANCE = 1 };
/* Outer Krylov method of amg_solve.  CG for symmetric positive definite operators (§1.1,
 * §3.1); flexible GMRES(restart) with the V-cycle as right preconditioner for nonsymmetric
 * ones (§3's wind pressure system is solved by GMRES preconditioned with smoothed
 * aggregation).  With GMRES the setup treats the operator as nonsymmetric: a connection is
 * strong when Eq. (7) holds for a_ij or for a_ji (the aggregation graph is undirected), and
 * the coarsest inverse makes no use of symmetry. */
enum { AMG_KRYLOV_CG = 0, AMG_KRYLOV_GMRES = 1 };
/* Storage read by the solve's products with the level operators (no counterpart in the paper).
 * A sliced-ELL copy (slices of 32 rows, column-major inside a slice, padded to the slice's
 * longest row; one lane per row with coalesced loads) may be kept beside CSR for a level whose
 * rows average at most 40 entries and whose padding stays within an eighth of its entries.
 * SELL: every such level.  AUTO: those whose FP64 operator (12 bytes per entry) exceeds the L2
 * cache or that have at least 1024 rows per SM (four 256-row sliced blocks per SM); on smaller
 * levels the sliced kernel leaves most SMs idle and the CSR kernel is faster.  CSR: never.  A row is summed in the order of the CSR kernel, so every
 * layout gives identical results; a copy costs 12 bytes per stored entry (16 with AMG_MIXED)
 * plus its padding. */
enum { AMG_LAYOUT_AUTO = 0, AMG_LAYOUT_CSR = 1, AMG_LAYOUT_SELL = 2 };
/* The coarsest-level solve (§3.1: a direct solver on the coarsest level).  INVERSE: a dense
 * FP64 inverse of the coarsest operator, applied by one dense product per V-cycle (the exact
 * solve to rounding).  AUTO (default): the same, except for a coarsest operator of more than 512
 * rows with at most one stored entry in eight whose Jacobi-scaled spectrum is narrow (what
 * stalled aggregation leaves): there the V-cycle applies a fixed Chebyshev polynomial in D^-1 A
 * of the least degree (at most 40) whose error bound on an interval holding that spectrum is
 * below 1e-16.  The interval comes from 16 Lanczos steps (through Jacobi-preconditioned CG),
 * widened by a fifth of its width each way, and is accepted only when a check solve of a
 * pseudo-random right-hand side leaves a relative residual (D^-1 norm) at most 1e-12;
 * otherwise the inverse is formed.  A fixed polynomial is one linear operator, as the inverse
 * is, so PCG keeps its fixed preconditioner; the setup forms no n^2 arrays.  The batch engine
 * and the server form the inverse of such a handle when it joins them.  With AMG_KRYLOV_GMRES
 * the inverse is always used. */
enum { AMG_COARSE_AUTO = 0, AMG_COARSE_INVERSE = 1 };
/* Systems of PDEs (block_size > 1 or nullspace_dim > 1; the paper treats scalar PDEs and leaves
 * systems to future work).  Unknown bs v + c is component c of node v (n a multiple of bs).
 * The near-null space passed to amg_setup is then nullspace_dim vectors of length n, one after
 * another (NULL: the constant of each component, which needs nullspace_dim = block_size).
 * Strength is decided between nodes: the Frobenius norm F_IJ of the bs x bs block coupling
 * nodes I and J stands for |a_ij| in Eq. (7), F_II and F_JJ for a_ii and a_jj; entries inside
 * a node's block are never dropped.  Aggregation is the distance-2 MIS of the strong node graph.
 * Each aggregate's block of B (its nodes' unknowns, nodes and components ascending) is factored
 * by modified Gram-Schmidt, B_a = Q_a R_a: the tentative prolongator holds Q_a and the coarse
 * near-null space is R_a.  P = Pt - omega Dbar^-1 Abar Pt as for scalar problems.  The four
 * adaptations (variants) and the distance strength are not defined for systems: a non-zero
 * variants or AMG_STRENGTH_DISTANCE gives AMG_ERR_UNSUPPORTED, and so does an aggregate too
 * small to carry k independent vectors (a column of its block left with norm <= 1e-12 of its
 * norm before the projections).  amg_export's AMG_EX_AGG and AMG_EX_ROOT are then per node,
 * AMG_EX_NULLSPACE holds the level's k vectors. */

/* Square CSR matrix.  row_ptr has n+1 entries (row_ptr[0] = 0), columns are sorted
 * ascending within each row with no duplicates, and every row stores its diagonal.
 * on_device = 1: the three arrays are device pointers; 0: host pointers.  The library
 * copies the matrix; the caller keeps ownership of these arrays. */
typedef struct {
    int64_t n, nnz;
    const int64_t *row_ptr;
    const int32_t *col;
    const double *val;
    int on_device;
} amg_csr_t;

typedef struct {
    double theta;        /* strength threshold of Eq. (7), in [0, 1]; 0 keeps every entry   */
    unsigned variants;   /* AMG_VAR_* bits                                                   */
    double tau;          /* OffLmp growth factor (1.1)                                       */
    double sigma;        /* 1Norm safeguard minimum root value (1/3)                         */
    int cheb_degree;     /* Chebyshev degree (2)                                             */
    double cheb_ratio;   /* Chebyshev interval [b lambda/ratio, b lambda] (10)               */
    double cheb_boost;   /* b: safety factor on the power-method estimate of lambda_max (1.1) */
    int power_iters;     /* power-method sweeps (10)                                         */
    int max_coarse;      /* stop coarsening at or below this size (500)                      */
    int max_levels;      /* (10)                                                             */
    int precision;       /* AMG_FP64 or AMG_MIXED                                            */
    int pt_scaling;      /* AMG_PT_ORTHONORMAL or AMG_PT_UNIT                                */
    int onenorm_lambda;  /* AMG_LAMBDA_ONE or AMG_LAMBDA_POWER                               */
    int max_iter;        /* PCG iteration limit (1000)                                       */
    uint64_t seed;       /* aggregation priorities and power-method start vectors (0)        */
    double lambda_override; /* > 0: prolongator-smoothing eigenvalue on every level (tests)  */
    void *cuda_stream;   /* cudaStream_t to run on; NULL = the legacy default stream         */
    int strength;        /* AMG_STRENGTH_MATRIX (Eq. 7 on A_l) or AMG_STRENGTH_DISTANCE       */
    int trace;           /* 1: time each setup phase (synchronises the stream at every phase  */
                         /*    boundary; read with amg_setup_trace); 0: no tracing (default)   */
    int krylov;          /* AMG_KRYLOV_CG (symmetric operators) or AMG_KRYLOV_GMRES            */
    int restart;         /* GMRES restart length (30)                                         */
    int spmv_layout;     /* AMG_LAYOUT_AUTO (default), AMG_LAYOUT_CSR or AMG_LAYOUT_SELL       */
    int block_size;      /* systems of PDEs: unknowns per node, interleaved (1: scalar; <= 16)  */
    int nullspace_dim;   /* near-null-space vectors k (1; <= 8); coarse levels have k unknowns  */
                         /*   per aggregate                                                   */
    int coarse_solve;    /* AMG_COARSE_AUTO (default) or AMG_COARSE_INVERSE                     */
} amg_params_t;

typedef struct {
    int iters;           /* PCG iterations (matrix-vector products with A)                   */
    int status;          /* amg_status_t of the call                                         */
    double relres_true;  /* ||b - A x|| / ||b|| recomputed in FP64 at exit                    */
    double setup_ms;     /* wall time of amg_setup                                           */
    double solve_ms;     /* wall time of this amg_solve                                      */
    int levels;
    double op_complexity;/* sum of nnz(A_l) / nnz(A_1)                                       */
} amg_info_t;

typedef struct amg_hierarchy *amg_handle_t;

/* Defaults listed above. */
void amg_params_default(amg_params_t *p);

/* Builds the hierarchy (Eq. 2-7 and §2 per level, then the coarsest factorisation).
 * nullspace: n values on the host or the device, or NULL for the constant vector.
 * On success *out owns all device memory of the hierarchy until amg_free.  On failure *out
 * is NULL and nothing is leaked.  Synchronises the stream before returning. */
amg_status_t amg_setup(const amg_csr_t *A, const double *nullspace, const amg_params_t *p,
                       amg_handle_t *out);

/* amg_setup with coordinates of the rows (for AMG_STRENGTH_DISTANCE, §3.1): coords holds
 * dim (1..3) doubles per row, row-major (x_0, y_0, z_0, x_1, ...), on the same side as A's
 * arrays (host, or device when A->on_device).  The hierarchy keeps a copy of each level's
 * coordinates.  With params->strength = AMG_STRENGTH_DISTANCE, coords NULL or dim outside
 * 1..3 is AMG_ERR_INVALID_ARG, and so are two coupled rows at the same coordinates.
 * amg_setup is this call with coords = NULL. */
amg_status_t amg_setup_coords(const amg_csr_t *A, const double *nullspace, const double *coords, int dim,
                              const amg_params_t *p, amg_handle_t *out);

/* With params.krylov = AMG_KRYLOV_GMRES, amg_solve runs flexible GMRES(restart) instead:
 * per step one V-cycle z_j = M v_j and one product A z_j, classical Gram-Schmidt done twice,
 * Givens rotations; it stops when the minimiser's residual norm is <= tol ||b|| and the
 * recomputed true residual agrees (else it restarts from the current x).  info->iters counts
 * the products with A inside the Arnoldi steps.  Work vectors (2 restart + 2 of them) are
 * allocated with the hierarchy on the first such solve.  amg_solve_multi and the batch engine
 * run PCG only: they return AMG_ERR_UNSUPPORTED for such a handle. */

/* Solves A x = b from x = 0 by PCG with one V-cycle (Algorithm 1) per iteration, until
 * ||r|| / ||b|| <= tol on the recurrence residual and on the recomputed true residual.
 * b and x: n doubles each, host or device (any pointer CUDA can address); they may not
 * alias.  info may be NULL.  Returns AMG_ERR_NOT_CONVERGED (x = last iterate) at max_iter.
 * Synchronises the stream before returning. */
amg_status_t amg_solve(amg_handle_t h, const double *b, double *x, double tol, amg_info_t *info);

/* Several right-hand sides of one system at once (no counterpart in the paper): k (1..8)
 * columns, column j of B and X at B + j n and X + j n (host or device).  Each column is
 * solved as amg_solve would solve it alone (PCG with one V-cycle per iteration from x = 0,
 * its own scalars and stopping test, tolerance tol, the same true-residual check); every
 * sparse product reads the matrix once for all columns.  infos (k entries, may be NULL)
 * receive each column's iterations, status and true residual.  Returns AMG_OK when every
 * column converged, else AMG_ERR_NOT_CONVERGED.  Work vectors for up to 8 columns are
 * allocated with the hierarchy on first use.  Synchronises the stream. */
amg_status_t amg_solve_multi(amg_handle_t h, int k, const double *B, double *X, double tol, amg_info_t *infos);

/* Releases every resource of the handle; NULL is accepted. */
amg_status_t amg_free(amg_handle_t h);

/* Setup phases timed when params.trace = 1 (wall milliseconds on the host, the stream
 * synchronised at each boundary, so each phase includes its device work):
 *   per level l that was coarsened: STRENGTH (Eq. 7 and the strong graph), AGGREGATE (distance-2
 *   MIS and joins), FILTER (aggregate members, Sprsfy, the filtered matrix and its diagonal),
 *   EIGEN (lambda-bar, omega), PROLONG (smoothed P, Cnstrnt, column scaling, R = P^T),
 *   GALERKIN_AP and GALERKIN_RAP (the two products of Eq. 2), SMOOTHER (1/diag and the
 *   Chebyshev eigenvalue);
 *   level 0 only: INPUT (copy and validation of A) and PREPARE (solve vectors, FP32 copies);
 *   the coarsest level only: COARSE (dense Cholesky factor and inverse). */
enum {
    AMG_PH_INPUT = 0, AMG_PH_STRENGTH = 1, AMG_PH_AGGREGATE = 2, AMG_PH_FILTER = 3, AMG_PH_EIGEN = 4,
    AMG_PH_PROLONG = 5, AMG_PH_GALERKIN_AP = 6, AMG_PH_GALERKIN_RAP = 7, AMG_PH_SMOOTHER = 8,
    AMG_PH_COARSE = 9, AMG_PH_PREPARE = 10, AMG_PH_COUNT = 11
};
/* ms[AMG_PH_COUNT] receives level l's phase times (0 where a phase did not run on that level,
 * or without tracing). */
amg_status_t amg_setup_trace(amg_handle_t h, int level, double *ms);

/* Number of levels. */
amg_status_t amg_num_levels(amg_handle_t h, int *levels);

/* The coarsest-level solve the setup chose (params.coarse_solve): *degree = 0 for the dense
 * inverse, else the Chebyshev degree, with the interval [theta - delta, theta + delta] on the
 * spectrum of D^-1 A and the relative residual of the setup's check solve (-1 when no check
 * ran).  Any output pointer may be NULL. */
amg_status_t amg_coarse_solver(amg_handle_t h, int *degree, double *theta, double *delta, double *check);

/* Size of level l: rows, stored entries of A_l, and the number of aggregates formed on it
 * (0 on the coarsest level). */
amg_status_t amg_level_info(amg_handle_t h, int level, int64_t *n, int64_t *nnz, int64_t *nagg);

/* Introspection for parity tests: copies one array of level l to caller-allocated HOST
 * memory.  amg_export_count gives the element count first.  Element types: row pointers
 * int64, columns and aggregate ids int32, values and diagonals double, flags uint8.
 * AMG_EX_SCALARS gives 4 doubles: lambda (smoothing), omega, lambda (Chebyshev), nagg. */
enum {
    AMG_EX_A_ROWPTR = 0, AMG_EX_A_COL = 1, AMG_EX_A_VAL = 2, AMG_EX_STRONG = 3, AMG_EX_REMOVED = 4,
    AMG_EX_LUMPFLAG = 5, AMG_EX_ABAR_ROWPTR = 6, AMG_EX_ABAR_COL = 7, AMG_EX_ABAR_VAL = 8,
    AMG_EX_AGG = 9, AMG_EX_ROOT = 10, AMG_EX_P_ROWPTR = 11, AMG_EX_P_COL = 12, AMG_EX_P_VAL = 13,
    AMG_EX_R_ROWPTR = 14, AMG_EX_R_COL = 15, AMG_EX_R_VAL = 16, AMG_EX_DSMOOTH = 17,
    AMG_EX_SCALARS = 18, AMG_EX_NULLSPACE = 19, AMG_EX_CFLAG = 20, AMG_EX_COORDS = 21
};
amg_status_t amg_export_count(amg_handle_t h, int level, int what, int64_t *count);
amg_status_t amg_export(amg_handle_t h, int level, int what, void *dst_host);

/* One V-cycle z = M^-1 r (Algorithm 1 from z = 0), in the hierarchy's precision.
 * r and z: n doubles, host or device.  Used to test the preconditioner on its own. */
amg_status_t amg_vcycle(amg_handle_t h, const double *r, double *z);

/* Sparse product C = A B on the device (the two-phase hash kernel used for Eq. (2)).
 * A: m x k, B: k x ncolB, both device CSR with sorted columns.  C is allocated by the
 * library (device memory, int64 row pointers); release it with amg_csr_release.
 * Each c_ij is summed over ascending k starting from zero, each term added by one fused
 * multiply-add c = fma(a_ik, b_kj, c) (one rounding per term). */
typedef struct {
    int64_t nrow, ncol, nnz;
    int64_t *row_ptr;
    int32_t *col;
    double *val;
} amg_dcsr_t;
amg_status_t amg_spgemm(const amg_csr_t *A, int64_t ncolA, const amg_csr_t *B, int64_t ncolB,
                        void *cuda_stream, amg_dcsr_t *C);
amg_status_t amg_csr_release(amg_dcsr_t *C);
/* Copies a library-allocated device CSR to caller-allocated host arrays (nrow+1, nnz, nnz). */
amg_status_t amg_dcsr_download(const amg_dcsr_t *C, int64_t *row_ptr, int32_t *col, double *val);

/* Allocation-free sparse product (the paper has no counterpart; it is a deployment aid).
 * Same product and same summation order as amg_spgemm, for callers that must not allocate
 * device memory themselves or through the libraries they call: a process that hands all of
 * the GPU's memory to its own pool, or a serving loop with a fixed memory budget in which a
 * cudaMalloc could fail, and a cudaFree would stall every stream on the device.
 *   A (m x ncolA, ncolA = B's rows) and B (ncolA x ncolB): device CSR arrays (on_device = 1),
 *   int64 row pointers, sorted int32 columns.  The caller provides the result arrays on the
 *   device: C_row_ptr (m + 1 entries), C_col and C_val (capacity entries each).
 *   *nnz_out (host) receives nnz(C).  If it exceeds capacity, nothing is written to C_col or
 *   C_val and AMG_ERR_BUDGET is returned, so the caller can retry with larger arrays.
 *   Checked before any kernel reads a row: row pointers that do not start at 0, decrease or
 *   do not end at nnz, column indices outside the matrix, and NULL col/val arrays of a
 *   matrix with entries give AMG_ERR_INVALID_ARG with nothing written to C.
 * Temporaries live in one 32 MiB array of device memory that is part of the library: every
 * GPU that loads the library holds it until the process exits.  Limits: at most 1,000,000
 * rows in A and in B, at most 2^31 - 16 entries in C, and the hash tables of very long rows
 * must fit in what the row arrays leave of the 32 MiB (their sizes are summed in 64 bits);
 * beyond them the call returns AMG_ERR_UNSUPPORTED (amg_last_error says which).  The first call on a device looks the array up (no allocation); make that first
 * call before any stream capture.  All calls share the array: calls that may overlap on the
 * GPU (different host threads, or streams without ordering between them) race and must be
 * serialised by the caller.  Runs on `cuda_stream` and synchronises it before every return
 * that follows a launch, whatever the status. */
amg_status_t amg_spgemm_noalloc(const amg_csr_t *A, int64_t ncolA, const amg_csr_t *B, int64_t ncolB,
                                void *cuda_stream, int64_t *C_row_ptr, int32_t *C_col, double *C_val,
                                int64_t capacity, int64_t *nnz_out);

/* ---- Many systems at once (no counterpart in the paper, which treats one system; every
 * system is set up and solved with the arithmetic of amg_setup and amg_solve: §1.1, Eq. (2)-(7),
 * §2 and §3.1 per system).
 *
 * amg_setup_batch: count hierarchies, one per A[k] (nullspace may be NULL, or nullspace[k]
 *   NULL, for the constant vector), built concurrently by `threads` host threads (<= 0: up to
 *   16), each on a stream of its own.  out[k] is an ordinary handle (amg_solve, amg_free
 *   work on it) bound to params->cuda_stream.  On failure every out[k] is NULL, nothing is
 *   leaked, and amg_last_error names the first failing system.
 * amg_batch_create: groups the given hierarchies for amg_batch_solve.  All need the same
 *   precision and Chebyshev degree.  The batch refers to the hierarchies' own arrays (the
 *   handles must outlive it) and allocates only vectors and work lists.  The same handle may
 *   appear several times (one system per right-hand side).  tune = 1: lanes per matrix row
 *   of each SpMV are chosen by timing the candidates at the first solve (results can then
 *   differ in the last bits from another batch); 0: from the mean row length
 *   (deterministic).  Runs on cuda_stream.  At most 2^31 rows per level over all systems.
 * amg_batch_solve: PCG with one V-cycle per iteration for every system at once; each system
 *   has its own scalars and stopping test (as amg_solve, tolerance tol) and stops
 *   independently.  b[k], x[k]: system k (the order given to amg_batch_create), n_k doubles,
 *   host or device.  infos (count entries, may be NULL) receive each system's iterations,
 *   status and true residual; solve_ms is the batch's wall time.  Returns AMG_OK when every
 *   system converged, else AMG_ERR_NOT_CONVERGED (or the error that stopped the batch).  One
 *   iteration of the whole batch is replayed as a CUDA graph.  Synchronises the stream.
 * amg_solve_batch: amg_batch_create (tune = 0) + amg_batch_solve + amg_batch_free on h[0]'s
 *   stream.
 * amg_batch_info: systems, levels of the deepest system, fine rows, kernels per replayed
 *   iteration (0 before the first solve). */
typedef struct amg_batch *amg_batch_t;
amg_status_t amg_setup_batch(int count, const amg_csr_t *const *A, const double *const *nullspace,
                             const amg_params_t *params, int threads, amg_handle_t *out);
amg_status_t amg_batch_create(int count, const amg_handle_t *h, void *cuda_stream, int tune, amg_batch_t *out);
amg_status_t amg_batch_solve(amg_batch_t batch, const double *const *b, double *const *x, double tol,
                             amg_info_t *infos);
amg_status_t amg_batch_free(amg_batch_t batch);
amg_status_t amg_solve_batch(int count, const amg_handle_t *h, const double *const *b, double *const *x,
                             double tol, amg_info_t *infos);
amg_status_t amg_batch_info(amg_batch_t batch, int *count, int *levels, int64_t *rows,
                            int64_t *graph_kernels);

/* ---- Serving (no counterpart in the paper): a request loop that admits solves as they
 * arrive and runs them with continuous batching on the batch engine.
 *
 * A request is an operator A (host or device CSR) with nrhs right-hand sides b (nrhs * n
 * doubles, system k at b + k n) and the place for the solutions x (same layout).  The
 * server hashes A's arrays; a request whose operator is resident reuses that hierarchy,
 * otherwise one of the setup threads builds it (amg_setup with the server's parameters).
 * Hierarchies stay resident after their requests finish and are evicted least recently used
 * first when a new one would exceed hbm_budget_bytes (hierarchies plus the engine's vectors
 * and lists).  Every right-hand side becomes one system of the engine as soon as its
 * hierarchy is ready and the engine has room; each PCG iteration of the engine advances every
 * system in flight, and a finished system's x is copied out and its place given to the next.
 * A, b and x belong to the caller and must stay valid until the request is done.
 *
 * amg_server_config_default: hbm_budget_bytes 120 GB, 8 setup threads, 4096 systems and
 *   2^28 fine rows in flight at most, tol 1e-8, tune 1, params = amg_params_default.
 * amg_server_submit: queues a request; *ticket identifies it.  Never blocks on the GPU.
 * amg_server_poll: AMG_PENDING while the request runs; then AMG_OK once, with *info filled
 *   in (info->status holds the request's own outcome); the ticket is released then.
 * amg_server_wait: blocks until the request is done, then as amg_server_poll.
 * amg_server_stats: counters since creation.
 * amg_server_destroy: finishes every request in flight, then releases everything. */
typedef struct amg_server *amg_server_t;
typedef struct {
    size_t hbm_budget_bytes;
    int setup_threads;
    int max_systems;
    int64_t max_rows;
    double tol;
    int tune;
    amg_params_t params;
} amg_server_config_t;
typedef struct {
    int status;          /* AMG_OK, AMG_ERR_NOT_CONVERGED (some right-hand side) or the setup error */
    int nrhs;
    int iters_max;       /* most PCG iterations over the right-hand sides                     */
    int cache_hit;       /* 1: the hierarchy was resident when the request arrived            */
    double relres_max;   /* largest true relative residual over the right-hand sides          */
    double queue_ms;     /* submit -> the first right-hand side enters the engine             */
    double setup_ms;     /* the hierarchy build this request waited for (0 on a hit)          */
    double latency_ms;   /* submit -> every solution copied out                               */
} amg_request_info_t;
typedef struct {
    int64_t submitted, completed, solves, cache_hits, cache_misses, evictions, failed;
    int64_t iterations, commits;
    double engine_busy_ms;
    size_t bytes_hierarchies, bytes_engine;
    int resident_hierarchies;
    char first_error[256];   /* the first failure's message (empty if none)                   */
} amg_server_stats_t;
void amg_server_config_default(amg_server_config_t *cfg);
amg_status_t amg_server_create(const amg_server_config_t *cfg, amg_server_t *out);
amg_status_t amg_server_submit(amg_server_t srv, const amg_csr_t *A, int nrhs, const double *b, double *x,
                               uint64_t *ticket);
amg_status_t amg_server_poll(amg_server_t srv, uint64_t ticket, amg_request_info_t *info);
amg_status_t amg_server_wait(amg_server_t srv, uint64_t ticket, amg_request_info_t *info);
amg_status_t amg_server_stats(amg_server_t srv, amg_server_stats_t *stats);
amg_status_t amg_server_destroy(amg_server_t srv);

/* ---- Requests across several GPUs (no counterpart in the paper, which treats one system).
 * A router gives each operator a home device the first time it sees it and keeps it, so that
 * every repeat of the operator reaches the server that holds its hierarchy.  The operator's
 * key is its content hash (row pointers, columns and values, the server's cache key).  A new
 * operator goes to the device with the least work assigned so far (ties: the lowest index);
 * work counts stored entries, nnz(A) x (nrhs + 20) for an operator new to the device (a setup
 * weighs about twenty solves' matrix passes) and nnz(A) x nrhs for a repeat.  Decisions
 * depend on the request sequence only (never on timing): processes that see the same
 * sequence of requests make the same decisions without any exchange, which lets one process
 * per GPU take its share of a common stream.  Host-side only: no collective, no peer access.
 *
 * amg_router_create: ndev devices (1 ... 4096), numbered 0 ... ndev - 1.
 * amg_router_route: the device of a request for A with nrhs right-hand sides (*device); *key
 *   (may be NULL) receives the content hash and *repeat (may be NULL) 1 when the operator was
 *   seen before.  A on the host or the device (device arrays are copied to the host to be
 *   hashed).  Records the request.  AMG_ERR_CUDA if such a copy fails.
 * amg_router_attach: device's server for amg_router_submit (owned by the caller, who creates
 *   it with that device current and destroys it after the router's last use; NULL detaches).
 * amg_router_submit: routes the request (as amg_router_route) and submits it to the attached
 *   server of its device; *ticket is the router's ticket, *device (may be NULL) the device.
 *   AMG_ERR_INVALID_ARG when that device has no server.  A, b, x as for amg_server_submit.
 * amg_router_poll / amg_router_wait: as amg_server_poll / amg_server_wait for a router ticket;
 *   *device (may be NULL) receives the device that served it.
 * amg_router_stats: for one device, the requests routed to it, the operators whose home it is,
 *   the repeats among those requests and the work assigned (any pointer may be NULL).
 * amg_router_destroy: releases the router (not the attached servers); tickets not yet
 *   collected are dropped. */
typedef struct amg_router *amg_router_t;
amg_status_t amg_router_create(int ndev, amg_router_t *out);
amg_status_t amg_router_route(amg_router_t r, const amg_csr_t *A, int nrhs, int *device, uint64_t *key,
                              int *repeat);
amg_status_t amg_router_attach(amg_router_t r, int device, amg_server_t srv);
amg_status_t amg_router_submit(amg_router_t r, const amg_csr_t *A, int nrhs, const double *b, double *x,
                               uint64_t *ticket, int *device);
amg_status_t amg_router_poll(amg_router_t r, uint64_t ticket, amg_request_info_t *info, int *device);
amg_status_t amg_router_wait(amg_router_t r, uint64_t ticket, amg_request_info_t *info, int *device);
amg_status_t amg_router_stats(amg_router_t r, int device, int64_t *requests, int64_t *operators, int64_t *repeats,
                              double *work);
amg_status_t amg_router_destroy(amg_router_t r);

/* Measurement hooks (no counterpart in the paper).
 * amg_launch_count: kernels launched by this library since it was loaded (all threads).
 * amg_profile_enable(1) resets the totals and starts recording CUDA events around the
 * launches of these kernel classes (on the stream they run on); (2) resumes recording and
 * keeps the totals; (0) stops (the totals stay readable).  A hierarchy whose iteration graph
 * is captured while recording carries the events in that graph.
 *   0: the finest-level FP64 SpMV of the PCG iteration (q = A p with p.q),
 *   1: the finest-level SpMVs of the V-cycle (Chebyshev steps and residual),
 *   2: the sparse products of the Galerkin step (both phases, per product),
 *   3: reserved.
 * amg_profile_read returns, for one class, the number of timed launches, their summed
 * device time in ms and the summed algorithmic bytes (each stored matrix entry, row pointer
 * and vector element counted once per launch). */
int64_t amg_launch_count(void);
amg_status_t amg_profile_enable(int on);
amg_status_t amg_profile_read(int kclass, int64_t *launches, double *total_ms, double *total_bytes);

/* Text of a status code, and of the last CUDA error seen by this thread. */
const char *amg_status_string(amg_status_t s);
const char *amg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
