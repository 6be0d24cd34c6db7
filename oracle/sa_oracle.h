/*
 * sa_oracle.h -- plain, slow, single-threaded FP64 CPU oracle of smoothed-aggregation AMG
 * with the four adaptations of Hu, Siefert and Tuminaro (arXiv:2103.10476).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.  Only the tests,
 * the smoke check and the benchmark's CPU-baseline / reference arm may load it.  It shares
 * no code, header, table or helper with the CUDA library; the two are written separately
 * from the paper.  Every function follows the paper's definitions step by step, in the
 * paper's order, with no blocking, fusion or reordering.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared sa_oracle.c -lm
 * (-ffp-contract=off: no fused multiply-add, so every product and sum is rounded as written.)
 */
#ifndef SA_ORACLE_H
#define SA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes (same numeric meaning as the product library's, by convention) */
enum {
    OC_OK = 0, OC_ERR_INVALID_ARG = 1, OC_ERR_OOM = 2, OC_ERR_ZERO_DIAG = 4, OC_ERR_EIGEN = 5,
    OC_ERR_COARSE_NOT_SPD = 6, OC_ERR_NOT_CONVERGED = 7, OC_ERR_UNSUPPORTED = 9
};
/* adaptation bits (§2.1-§2.5) */
enum { OC_1NORM = 1, OC_OFFLMP = 2, OC_SPRSFY = 4, OC_CNSTRNT = 8 };

/* OffLmp per-row outcome codes (Algorithm 2 branches) */
enum { OC_LUMP_DIAG = 0, OC_LUMP_KPLUS = 1, OC_LUMP_DIAG_KMINUS = 2, OC_LUMP_KPLUS_NEG = 3,
       OC_LUMP_SKIPPED = 4, OC_LUMP_FALLBACK = 5 };

typedef struct {
    int64_t n, nnz;
    int64_t *rp;   /* n+1 */
    int32_t *ci;   /* nnz, ascending within a row */
    double *v;     /* nnz */
} oc_csr;

typedef struct {
    double theta;          /* strength threshold, Eq. (7) */
    unsigned variants;     /* OC_1NORM | OC_OFFLMP | OC_SPRSFY | OC_CNSTRNT */
    double tau;            /* OffLmp growth factor (1.1 in §3.1) */
    double sigma;          /* 1Norm safeguard minimum root value (1/3 in §2.2) */
    int cheb_degree;       /* Chebyshev polynomial degree */
    double cheb_ratio;     /* interval [b lambda/ratio, b lambda] */
    double cheb_boost;     /* b: safety factor on the power-method estimate (1.1) */
    int power_iters;       /* power-method sweeps (10 in §3.1) */
    int max_coarse;        /* coarsest level size */
    int max_levels;
    int pt_unit;           /* 0: orthonormal tentative prolongator columns, 1: Eq. (5) as printed */
    int onenorm_power;     /* 0: lambda := 1 with 1Norm (§2.1), 1: power method */
    uint64_t seed;         /* aggregation priorities and power-method start vectors */
    double lambda_override;/* > 0: use as the prolongator-smoothing eigenvalue on every level */
    int max_iter;          /* PCG iteration limit */
    int strength;          /* 0: Eq. (7) on the matrix; 1: Eq. (7) on the distance Laplacian (§3.1) */
    int krylov;            /* 0: PCG (symmetric operators); 1: flexible GMRES (nonsymmetric operators) */
    int restart;           /* GMRES restart length */
    int block_size;        /* unknowns per node on the finest level (systems of PDEs; 1: scalar) */
    int nullspace_dim;     /* near-null-space vectors k (coarse levels carry k unknowns per node) */
} oc_params;

typedef struct {
    int iters;
    int status;
    double relres_true;
    int levels;
    double op_complexity;
} oc_info;

typedef struct oc_hier oc_hier;

void oc_params_default(oc_params *p);

/* single steps (used by the tests to pin each one) */
void oc_strength(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, double theta,
                 uint8_t *strong);
int oc_distance_laplacian(int64_t n, const int64_t *rp, const int32_t *ci, const double *coords, int dim,
                          double *L);
int oc_coarse_coords(int64_t n, const int32_t *agg, int64_t nagg, const double *coords, int dim, double *out);
int oc_filter(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const uint8_t *removed,
              int offlmp, double tau, oc_csr **out, uint8_t *rowflag);
int64_t oc_mis2_aggregate(int64_t n, const int64_t *rp, const int32_t *ci, const uint8_t *strong,
                          uint64_t seed, int level, int32_t *agg, uint8_t *root);
uint64_t oc_priority(uint64_t seed, int level, int64_t i);
int oc_sprsfy_mark(int64_t n, const int64_t *rp, const int32_t *ci, const uint8_t *strong,
                   const int32_t *agg, const uint8_t *root, int64_t nagg, uint8_t *removed);
int oc_constrain_row(int64_t m, double *p, int64_t ptent_pos, double ptent_val);
int oc_spgemm(const oc_csr *A, const oc_csr *B, int64_t ncolB, oc_csr **out);
int oc_transpose(const oc_csr *A, int64_t ncol, oc_csr **out);
double oc_power_lambda(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *D,
                       int sweeps, uint64_t stream_seed);
uint64_t oc_power_stream_seed(uint64_t seed, int level, int purpose);
int oc_cholesky(int64_t n, const double *a, double *l);
int oc_lu(int64_t n, double *a, int64_t *piv);
void oc_lu_solve(int64_t n, const double *lu, const int64_t *piv, const double *b, double *x);
int oc_gmres_plain(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *b, double *x,
                   double tol, int restart, int max_iter, oc_info *info);
void oc_csr_free(oc_csr *c);
/* systems of PDEs: node graph of bs x bs blocks, block strength, per-aggregate QR */
int64_t oc_node_graph(int64_t n, const int64_t *rp, const int32_t *ci, int bs, int64_t *nrp);
int oc_node_fill(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, int bs, double theta,
                 const int64_t *nrp, int32_t *nci, double *nF, uint8_t *nstrong, uint8_t *strong);
int oc_block_tentative(int64_t n, int bs, int k, const int32_t *node_agg, int64_t nagg, const double *B,
                       double *Qv, double *Bc);

/* the whole method */
int oc_setup(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *nullspace,
             const oc_params *p, oc_hier **out);
int oc_setup_coords(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *nullspace,
                    const double *coords, int dim, const oc_params *p, oc_hier **out);
int oc_prolongator_only(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                        const double *nullspace, const oc_params *p, oc_hier **out);
int oc_solve(oc_hier *h, const double *b, double *x, double tol, oc_info *info);
int oc_pcg_plain(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *b,
                 double *x, double tol, int max_iter, oc_info *info);
int oc_vcycle(oc_hier *h, const double *f, double *u);
/* the Chebyshev smoother of the V-cycle on its own (degree m in D^-1 A on [b lambda/ratio, b lambda]) */
int oc_chebyshev_apply(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *invdiag,
                       double lambda, int degree, double ratio, double boost, const double *f, double *x);
void oc_free(oc_hier *h);

/* introspection */
int oc_nlevels(const oc_hier *h);
int oc_level_get(const oc_hier *h, int level, int what, void *dst, int64_t *len);

#ifdef __cplusplus
}
#endif
#endif
