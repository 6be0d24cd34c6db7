/*
 * sa_oracle.c -- plain FP64 CPU oracle of smoothed-aggregation AMG (SA-AMG) and of the four
 * adaptations 1Norm, OffLmp, Cnstrnt and Sprsfy of Hu, Siefert and Tuminaro,
 * "Smooth Aggregation for Difficult Stretched Mesh and Coefficient Variation Problems"
 * (arXiv:2103.10476).
 *
 * TEST INFRASTRUCTURE ONLY: the reference the CUDA path is checked against.  It is slow on
 * purpose (single thread, dense accumulators, sequential sums in ascending index order, by
 * segments of 256 positions in rows longer than that) and
 * shares nothing with the CUDA library.  The product path never calls it.
 *
 * Where the paper is silent or ambiguous the reading taken is stated at the point of use
 * ("Reading:").  Every floating-point decision (a comparison that selects a branch) is taken
 * on values rounded exactly as written (compiled with -ffp-contract=off).
 */
#include "sa_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OC_MAX_LEVELS 32
#define OC_MAX_DENSE 8192

struct oc_level {
    oc_csr A;             /* level operator A_l                                   */
    uint8_t *strong;      /* per stored entry of A: strong off-diagonal (Eq. 7)   */
    uint8_t *removed;     /* per stored entry of A: dropped from the filtered A    */
    uint8_t *lumpflag;    /* per row: OffLmp outcome (OC_LUMP_*)                   */
    oc_csr Abar;          /* filtered matrix (Eq. 6 / Algorithm 2 / §2.5)          */
    int32_t *agg;         /* aggregate of each vertex                              */
    uint8_t *root;        /* root flag                                             */
    int64_t nagg;
    double *B;            /* near-null space on this level                         */
    double *nrm;          /* per aggregate: 2-norm of B restricted to it           */
    double *Dsm;          /* diagonal used in prolongator smoothing (Dbar or Dtilde) */
    double lambda_bar, omega;
    uint8_t *cflag;       /* Cnstrnt per-row outcome: 0 kept/clipped, 1 zero row, 2 tentative row */
    oc_csr P, R;
    double lambda_cheb;   /* lambda_max(D^-1 A_l) for the Chebyshev smoother       */
    double *invdiag;      /* 1 / diag(A_l)                                         */
    double *coords;       /* dim coordinates per row (distance-Laplacian strength)  */
    int bs, k;            /* unknowns per node; near-null-space vectors (B is n x k) */
    double *Bc;           /* systems: the coarse near-null space (nagg k x k)        */
};

struct oc_hier {
    int nlev;
    int dim;              /* coordinates per row, 0 without coordinates */
    int prolongator_only; /* level 0 holds P but no coarser level was formed */
    struct oc_level lev[OC_MAX_LEVELS];
    double *chol;         /* dense lower Cholesky factor of the coarsest operator */
    double *lu;           /* nonsymmetric operators: dense LU factors (unit lower L) instead */
    int64_t *piv;         /* and the row exchanged with row k at step k */
    oc_params p;
};

/* ---------------------------------------------------------------------------------------- */
/* helpers                                                                                  */
/* ---------------------------------------------------------------------------------------- */

void oc_params_default(oc_params *p)
{
    p->theta = 0.0;
    p->variants = 0;
    p->tau = 1.1;
    p->sigma = 1.0 / 3.0;
    p->cheb_degree = 2;
    p->cheb_ratio = 10.0;
    p->cheb_boost = 1.1;
    p->power_iters = 10;
    p->max_coarse = 500;
    p->max_levels = 10;
    p->pt_unit = 0;
    p->onenorm_power = 0;
    p->seed = 0;
    p->lambda_override = 0.0;
    p->max_iter = 1000;
    p->strength = 0;
    p->krylov = 0;
    p->restart = 30;
    p->block_size = 1;
    p->nullspace_dim = 1;
}

static void csr_release(oc_csr *c)
{
    free(c->rp); free(c->ci); free(c->v);
    c->rp = NULL; c->ci = NULL; c->v = NULL; c->n = 0; c->nnz = 0;
}

void oc_csr_free(oc_csr *c)
{
    if (!c) return;
    csr_release(c);
    free(c);
}

static int csr_alloc(oc_csr *c, int64_t n, int64_t nnz)
{
    c->n = n; c->nnz = nnz;
    c->rp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    c->ci = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    c->v = (double *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
    if (!c->rp || !c->ci || !c->v) { csr_release(c); return OC_ERR_OOM; }
    return OC_OK;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* position of column j in row i, or -1 */
static int64_t find_entry(const int64_t *rp, const int32_t *ci, int64_t i, int32_t j)
{
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
        if (ci[e] == j) return e;
    return -1;
}

/* SplitMix64 finaliser (Steele, Lea and Flood, OOPSLA 2014). */
static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* k-th output (k >= 1) of the SplitMix64 stream started at state s, as a double in [0,1). */
static double stream_u01(uint64_t s, uint64_t k)
{
    uint64_t z = mix64(s + k * 0x9E3779B97F4A7C15ULL);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

/* ---------------------------------------------------------------------------------------- */
/* Strength of connection, Eq. (7)                                                           */
/* ---------------------------------------------------------------------------------------- */

static double diag_of(const int64_t *rp, const int32_t *ci, const double *v, int64_t i)
{
    int64_t e = find_entry(rp, ci, i, (int32_t)i);
    return e < 0 ? 0.0 : v[e];
}

/* strong[e] = 1 iff entry e = (i, j), j != i, satisfies |a_ij| >= theta sqrt(a_ii a_jj).
 * Reading: theta = 0 makes every stored off-diagonal strong (then the filtered matrix equals
 * A, §1.1), including stored zeros; otherwise the inequality is evaluated literally, and a
 * negative a_ii a_jj (sqrt = NaN) makes the entry weak. */
void oc_strength(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, double theta,
                 uint8_t *strong)
{
    double *d = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t i = 0; i < n; ++i) d[i] = diag_of(rp, ci, v, i);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t j = ci[e];
            if (j == i) { strong[e] = 0; continue; }
            if (theta == 0.0) { strong[e] = 1; continue; }
            double prod = d[i] * d[j];
            double thr = theta * sqrt(prod);
            strong[e] = (fabs(v[e]) >= thr) ? 1 : 0;
        }
    }
    free(d);
}

/* Distance Laplacian of §3.1: the pattern of A; off-diagonal L_ij = -1 / |x_i - x_j| (the
 * reciprocal of the negative distance between the coordinates of rows i and j) and L_ii
 * chosen so that the row sums to zero, L_ii = sum over j != i of 1 / |x_i - x_j| in ascending
 * column order.  The distance is sqrt of the squared differences summed in coordinate order.
 * Reading: stored zeros of A are part of the pattern and get a value too.  Returns
 * OC_ERR_INVALID_ARG if two coupled rows have the same coordinates. */
int oc_distance_laplacian(int64_t n, const int64_t *rp, const int32_t *ci, const double *coords, int dim,
                          double *L)
{
    for (int64_t i = 0; i < n; ++i) {
        double diag = 0.0;
        int64_t dpos = -1;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t j = ci[e];
            if (j == i) { dpos = e; continue; }
            double d2 = 0.0;
            for (int c = 0; c < dim; ++c) {
                double dx = coords[i * dim + c] - coords[(int64_t)j * dim + c];
                d2 = d2 + dx * dx;
            }
            double dist = sqrt(d2);
            if (!(dist > 0.0)) return OC_ERR_INVALID_ARG;
            double w = 1.0 / dist;
            L[e] = -w;
            diag = diag + w;
        }
        if (dpos >= 0) L[dpos] = diag;
    }
    return OC_OK;
}

/* Coordinates of the next level (Reading: the paper supplies coordinates for the finest
 * level only; an aggregate's coordinates are the mean of its members', summed in ascending
 * member index and divided by the member count). */
int oc_coarse_coords(int64_t n, const int32_t *agg, int64_t nagg, const double *coords, int dim, double *out)
{
    int64_t *cnt = (int64_t *)calloc((size_t)(nagg > 0 ? nagg : 1), sizeof(int64_t));
    if (!cnt) return OC_ERR_OOM;
    for (int64_t k = 0; k < nagg * dim; ++k) out[k] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t a = agg[i];
        for (int c = 0; c < dim; ++c) out[(int64_t)a * dim + c] = out[(int64_t)a * dim + c] + coords[i * dim + c];
        cnt[a] += 1;
    }
    for (int64_t a = 0; a < nagg; ++a)
        for (int c = 0; c < dim; ++c) out[a * dim + c] = out[a * dim + c] / (double)cnt[a];
    free(cnt);
    return OC_OK;
}

/* ---------------------------------------------------------------------------------------- */
/* Filtered matrix: Eq. (6) (lumping to the diagonal) or Algorithm 2 (OffLmp, §2.3)          */
/* ---------------------------------------------------------------------------------------- */

/* Diagonal-dominance measure of §2.3: sum_{j != i} |a_ij| / |a_ii|. */
/* ---------------------------------------------------------------------------------------- */
/* Systems of PDEs (the paper treats scalar PDEs and leaves systems to future work; the       */
/* readings below extend its steps to bs unknowns per node, interleaved: unknown bs v + c is  */
/* component c of node v, and k near-null-space vectors)                                      */
/* ---------------------------------------------------------------------------------------- */

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* the nodes coupled to node I: node ids of every stored entry of its bs rows, sorted, without
 * repeats; returns how many (written to out) */
static int64_t node_row(const int64_t *rp, const int32_t *ci, int bs, int64_t I, int64_t *out)
{
    int64_t m = 0;
    for (int64_t r = I * bs; r < (I + 1) * bs; ++r)
        for (int64_t e = rp[r]; e < rp[r + 1]; ++e) out[m++] = ci[e] / bs;
    qsort(out, (size_t)m, sizeof(int64_t), cmp_i64);
    int64_t u = 0;
    for (int64_t t = 0; t < m; ++t)
        if (u == 0 || out[t] != out[u - 1]) out[u++] = out[t];
    return u;
}

/* Node graph of the bs x bs blocks: row pointer nrp (n/bs + 1 entries); returns its entry
 * count, -1 when n is not a multiple of bs. */
int64_t oc_node_graph(int64_t n, const int64_t *rp, const int32_t *ci, int bs, int64_t *nrp)
{
    if (bs < 1 || n % bs) return -1;
    int64_t nn = n / bs, maxrow = 0;
    for (int64_t I = 0; I < nn; ++I) {
        int64_t w = rp[(I + 1) * bs] - rp[I * bs];
        if (w > maxrow) maxrow = w;
    }
    int64_t *tmp = (int64_t *)malloc((size_t)(maxrow > 0 ? maxrow : 1) * sizeof(int64_t));
    if (!tmp) return -1;
    nrp[0] = 0;
    for (int64_t I = 0; I < nn; ++I) nrp[I + 1] = nrp[I] + node_row(rp, ci, bs, I, tmp);
    free(tmp);
    return nrp[nn];
}

/* Block strength.  F_IJ = Frobenius norm of the block coupling nodes I and J (squares summed
 * over the block's rows in order, each row's entries in order, then the square root).
 * Reading: Eq. (7) between nodes with F_IJ in place of |a_ij| and F_II, F_JJ in place of
 * a_ii, a_jj: I != J is strong when F_IJ >= theta sqrt(F_II F_JJ) (for bs = 1 this is Eq. (7)
 * itself, sqrt(a^2) being |a| exactly).  Per stored entry of A, strong[e] is the strength of
 * its node pair, and an entry inside a node's own block (off the diagonal) counts as strong:
 * it is never dropped from the filtered matrix. */
int oc_node_fill(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, int bs, double theta,
                 const int64_t *nrp, int32_t *nci, double *nF, uint8_t *nstrong, uint8_t *strong)
{
    if (bs < 1 || n % bs) return OC_ERR_INVALID_ARG;
    int64_t nn = n / bs, maxrow = 0;
    for (int64_t I = 0; I < nn; ++I) {
        int64_t w = rp[(I + 1) * bs] - rp[I * bs];
        if (w > maxrow) maxrow = w;
    }
    int64_t *tmp = (int64_t *)malloc((size_t)(maxrow > 0 ? maxrow : 1) * sizeof(int64_t));
    double *fd = (double *)calloc((size_t)(nn > 0 ? nn : 1), sizeof(double));
    if (!tmp || !fd) { free(tmp); free(fd); return OC_ERR_OOM; }
    for (int64_t I = 0; I < nn; ++I) {
        int64_t m = node_row(rp, ci, bs, I, tmp);
        for (int64_t t = 0; t < m; ++t) {
            int64_t J = tmp[t];
            double acc = 0.0;
            for (int64_t r = I * bs; r < (I + 1) * bs; ++r)
                for (int64_t e = rp[r]; e < rp[r + 1]; ++e)
                    if (ci[e] / bs == J) acc = acc + v[e] * v[e];
            nci[nrp[I] + t] = (int32_t)J;
            nF[nrp[I] + t] = sqrt(acc);
            if (J == I) fd[I] = nF[nrp[I] + t];
        }
    }
    for (int64_t I = 0; I < nn; ++I)
        for (int64_t t = nrp[I]; t < nrp[I + 1]; ++t) {
            int64_t J = nci[t];
            nstrong[t] = (J != I && nF[t] >= theta * sqrt(fd[I] * fd[J])) ? 1 : 0;
        }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int64_t I = i / bs, J = ci[e] / bs;
            if (I == J) { strong[e] = ci[e] != i; continue; }
            uint8_t sflag = 0;
            for (int64_t t = nrp[I]; t < nrp[I + 1]; ++t)
                if (nci[t] == J) sflag = nstrong[t];
            strong[e] = sflag;
        }
    free(tmp);
    free(fd);
    return OC_OK;
}

/* Tentative prolongator for k near-null-space vectors (B: k vectors of length n, one after
 * another).  Aggregate a's rows are the unknowns of its nodes, nodes ascending and components
 * ascending (m rows); its m x k block of B is factored B_a = Q_a R_a by modified Gram-Schmidt
 * in column order (every inner product and norm summed over the rows in order), R_a upper
 * triangular with a positive diagonal.  Row i of Pt holds Q_a's row at columns a k .. a k + k - 1
 * (Qv[i k + j]); the coarse near-null space is R_a (Bc: k vectors of length nagg k, row
 * a k + j of vector c = (R_a)_jc).  So Pt Bc = B and each aggregate's columns are orthonormal.
 * Reading: a column whose norm after the projections falls to 1e-12 of its norm before them
 * (the aggregate is too small to carry k independent vectors) fails with OC_ERR_UNSUPPORTED. */
int oc_block_tentative(int64_t n, int bs, int k, const int32_t *node_agg, int64_t nagg, const double *B,
                       double *Qv, double *Bc)
{
    if (bs < 1 || k < 1 || n % bs) return OC_ERR_INVALID_ARG;
    int64_t nn = n / bs, nc = nagg * k;
    int64_t *start = (int64_t *)calloc((size_t)(nagg + 1), sizeof(int64_t));
    int64_t *members = (int64_t *)malloc((size_t)(nn > 0 ? nn : 1) * sizeof(int64_t));
    int64_t *fillp = (int64_t *)calloc((size_t)(nagg + 1), sizeof(int64_t));
    double *W = (double *)malloc((size_t)(n > 0 ? n : 1) * (size_t)k * sizeof(double));
    double *R = (double *)calloc((size_t)k * (size_t)k, sizeof(double));
    int st = OC_OK;
    if (!start || !members || !fillp || !W || !R) { st = OC_ERR_OOM; goto out; }
    for (int64_t I = 0; I < nn; ++I) start[node_agg[I] + 1]++;
    for (int64_t a = 0; a < nagg; ++a) start[a + 1] += start[a];
    for (int64_t I = 0; I < nn; ++I) members[start[node_agg[I]] + fillp[node_agg[I]]++] = I;
    for (int64_t e = 0; e < nc * k; ++e) Bc[e] = 0.0;
    for (int64_t a = 0; a < nagg && st == OC_OK; ++a) {
        int64_t m = (start[a + 1] - start[a]) * bs;
        /* W[j m + t] = B restricted to the aggregate's rows */
        for (int j = 0; j < k; ++j)
            for (int64_t t = 0; t < m; ++t) {
                int64_t i = members[start[a] + t / bs] * bs + t % bs;
                W[j * m + t] = B[(int64_t)j * n + i];
            }
        for (int j = 0; j < k * k; ++j) R[j] = 0.0;
        for (int j = 0; j < k; ++j) {
            double before = 0.0;
            for (int64_t t = 0; t < m; ++t) before = before + W[j * m + t] * W[j * m + t];
            for (int l = 0; l < j; ++l) {
                double r = 0.0;
                for (int64_t t = 0; t < m; ++t) r = r + W[l * m + t] * W[j * m + t];
                R[l * k + j] = r;
                for (int64_t t = 0; t < m; ++t) W[j * m + t] = W[j * m + t] - r * W[l * m + t];
            }
            double s = 0.0;
            for (int64_t t = 0; t < m; ++t) s = s + W[j * m + t] * W[j * m + t];
            double rjj = sqrt(s);
            if (!(rjj > 1e-12 * sqrt(before))) { st = OC_ERR_UNSUPPORTED; break; }
            for (int64_t t = 0; t < m; ++t) W[j * m + t] = W[j * m + t] / rjj;
            R[j * k + j] = rjj;
        }
        if (st) break;
        for (int64_t t = 0; t < m; ++t) {
            int64_t i = members[start[a] + t / bs] * bs + t % bs;
            for (int j = 0; j < k; ++j) Qv[i * k + j] = W[j * m + t];
        }
        for (int c = 0; c < k; ++c)
            for (int j = 0; j < k; ++j) Bc[(int64_t)c * nc + a * k + j] = R[j * k + c];
    }
out:
    free(start); free(members); free(fillp); free(W); free(R);
    return st;
}

/* Sums along one stored row.  Reading (the paper fixes no summation order): position t of the
 * row (0-based; every stored entry has a position, whether or not it is a term of the sum) lies
 * in segment t / OC_SEG.  A row of at most OC_SEG positions is summed left to right from 0.  In
 * a longer row each segment's terms are summed left to right from 0, then the sums of all the
 * row's segments (0 for one without terms) are added left to right.  Used for the filtered
 * matrix's sums (r_i, kappa+, kappa-, the dominance sum) and the 1Norm sums of Eq. (9)-(10). */
#define OC_SEG 256
typedef struct {
    double tot, seg;
    int64_t cur;          /* the segment being summed */
} rowsum;

static void rs_init(rowsum *s) { s->tot = 0.0; s->seg = 0.0; s->cur = 0; }

/* closes the segments before segment q */
static void rs_to(rowsum *s, int64_t q)
{
    while (s->cur < q) {
        s->tot = s->cur == 0 ? s->seg : s->tot + s->seg;
        s->seg = 0.0;
        ++s->cur;
    }
}

static void rs_add(rowsum *s, int64_t t, double x)
{
    rs_to(s, t / OC_SEG);
    s->seg = s->seg + x;
}

/* the sum over a row of len positions */
static double rs_value(rowsum *s, int64_t len)
{
    rs_to(s, len > 0 ? (len - 1) / OC_SEG : 0);
    return s->cur == 0 ? s->seg : s->tot + s->seg;
}

static double ddom(const double *val, const int32_t *col, int64_t len, int64_t i, double aii)
{
    rowsum s;
    rs_init(&s);
    for (int64_t t = 0; t < len; ++t)
        if (col[t] != i) rs_add(&s, t, fabs(val[t]));
    return rs_value(&s, len) / fabs(aii);
}

/* Algorithm 2 (Lump_AvoidSmallDiag) for one row.  val/col: the stored row of A (length
 * len, ascending columns); rem: 1 for entries in the removal set R_i.  Writes the new row
 * values (same positions; removed entries are ignored by the caller) into out and returns
 * the outcome code.
 *
 * Readings (the paper is ambiguous or garbled at these points):
 *  - r_i = 0 takes the diagonal branch (a no-op) instead of the 0/0 of the K+ branch.
 *  - D(A_i) counts all of A's off-diagonals, including those about to be dropped.
 *  - a row with a_ii <= 0 falls back to lumping onto the diagonal (Eq. 6).
 *  - K- empty: if K+ is not empty all of r_i is spread over K+ (delta = r_i / kappa+, the
 *    entries may turn negative); if no off-diagonal is kept the row is left unlumped (its
 *    row sum is then not preserved).
 *  - the diagonal share r* (and the closed form given after Algorithm 2, whose printed
 *    signs give the signed perturbation -r*): with N = -kappa- - rhat, the growth measure
 *    after lumping r to the diagonal is (N - r) / (a_ii - r) on r in [0, |rhat|].  If
 *    N <= a_ii it does not increase with r and r* = |rhat|.  Otherwise it increases with r:
 *    r* = min(|rhat|, (t a_ii - N) / (t - 1)) when N <= t a_ii (t = tau D(A_i)), and r* = 0
 *    (the smallest growth) when no r meets the bound. */
static int offlmp_row(int64_t i, const int32_t *col, const double *val, const uint8_t *rem, int64_t len,
                      double tau, double *out)
{
    int64_t di = -1;
    for (int64_t t = 0; t < len; ++t) { out[t] = val[t]; if (col[t] == i) di = t; }
    double aii = di >= 0 ? val[di] : 0.0;
    /* r_i: sum of the removed entries */
    rowsum rs;
    rs_init(&rs);
    for (int64_t t = 0; t < len; ++t)
        if (rem[t] && col[t] != i) rs_add(&rs, t, val[t]);
    double r = rs_value(&rs, len);
    if (!(aii > 0.0)) {                    /* reading: fallback to Eq. (6) */
        if (di >= 0) out[di] = aii + r;
        return OC_LUMP_FALLBACK;
    }
    /* r_i >= 0: all of it to the diagonal (lowers the growth measure) */
    if (r >= 0.0) {
        out[di] = aii + r;
        return OC_LUMP_DIAG;
    }
    /* kept positive / negative off-diagonals K+, K- and their sums */
    rowsum sp, sm;
    rs_init(&sp);
    rs_init(&sm);
    int64_t nkp = 0, nkm = 0;
    for (int64_t t = 0; t < len; ++t) {
        if (col[t] == i || rem[t]) continue;
        if (val[t] > 0.0) { rs_add(&sp, t, val[t]); ++nkp; }
        else if (val[t] < 0.0) { rs_add(&sm, t, val[t]); ++nkm; }
    }
    double kp = rs_value(&sp, len), km = rs_value(&sm, len);
    /* |r_i| <= kappa+: K+ absorbs all of it and stays non-negative */
    if (fabs(r) <= kp) {
        double delta = r / kp;
        for (int64_t t = 0; t < len; ++t)
            if (col[t] != i && !rem[t] && val[t] > 0.0) out[t] = val[t] * (1.0 + delta);
        return OC_LUMP_KPLUS;
    }
    /* K- empty */
    if (nkm == 0) {
        if (nkp > 0) {
            double delta = r / kp;
            for (int64_t t = 0; t < len; ++t)
                if (col[t] != i && !rem[t] && val[t] > 0.0) out[t] = val[t] * (1.0 + delta);
            return OC_LUMP_KPLUS_NEG;
        }
        return OC_LUMP_SKIPPED;
    }
    /* K+ takes kappa+ of r_i (its entries become zero); rhat is left */
    for (int64_t t = 0; t < len; ++t)
        if (col[t] != i && !rem[t] && val[t] > 0.0) out[t] = 0.0;
    double rhat = r + kp;
    /* the largest diagonal share r* that keeps the growth bound */
    double t_bound = tau * ddom(val, col, len, i, aii);
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
    /* diagonal takes r*, K- takes the rest in proportion to its entries */
    out[di] = aii - rstar;
    double delta = (rhat + rstar) / km;
    for (int64_t t = 0; t < len; ++t)
        if (col[t] != i && !rem[t] && val[t] < 0.0) out[t] = val[t] * (1.0 + delta);
    return OC_LUMP_DIAG_KMINUS;
}

/* Filtered matrix.  Its pattern is the diagonal plus every stored off-diagonal not in the
 * removal set (removed = weak, plus the §2.5 pruned links); entries that lumping sets to
 * zero stay stored (patterns are symbolic).  offlmp = 0: Eq. (6), the removed entries are
 * summed in ascending column order (by segments in rows of more than OC_SEG entries, rowsum
 * above) and added to a_ii; offlmp = 1: Algorithm 2. */
int oc_filter(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const uint8_t *removed,
              int offlmp, double tau, oc_csr **out, uint8_t *rowflag)
{
    oc_csr *c = (oc_csr *)calloc(1, sizeof(oc_csr));
    if (!c) return OC_ERR_OOM;
    int64_t nnz = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            if (ci[e] == i || !removed[e]) ++nnz;
    if (csr_alloc(c, n, nnz)) { free(c); return OC_ERR_OOM; }
    int64_t maxlen = 0;
    for (int64_t i = 0; i < n; ++i) if (rp[i + 1] - rp[i] > maxlen) maxlen = rp[i + 1] - rp[i];
    double *tmp = (double *)malloc((size_t)(maxlen > 0 ? maxlen : 1) * sizeof(double));
    int64_t pos = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t b = rp[i], len = rp[i + 1] - rp[i];
        int flag = OC_LUMP_DIAG;
        if (offlmp) {
            flag = offlmp_row(i, ci + b, v + b, removed + b, len, tau, tmp);
        } else {
            rowsum rs;
            rs_init(&rs);
            int64_t di = -1;
            for (int64_t t = 0; t < len; ++t) {
                tmp[t] = v[b + t];
                if (ci[b + t] == i) di = t;
                else if (removed[b + t]) rs_add(&rs, t, v[b + t]);
            }
            if (di >= 0) tmp[di] = v[b + di] + rs_value(&rs, len);
        }
        if (rowflag) rowflag[i] = (uint8_t)flag;
        for (int64_t t = 0; t < len; ++t) {
            if (ci[b + t] == i || !removed[b + t]) {
                c->ci[pos] = ci[b + t];
                c->v[pos] = tmp[t];
                ++pos;
            }
        }
        c->rp[i + 1] = pos;
    }
    free(tmp);
    *out = c;
    return OC_OK;
}

/* ---------------------------------------------------------------------------------------- */
/* Aggregation (§1.1 Eq. (4) and the root-plus-neighbours construction of §2.5)              */
/* ---------------------------------------------------------------------------------------- */

/* Vertex priority: the top 30 bits of SplitMix64-mix(seed ^ (level << 40) ^ i), then the
 * index i, compared as one unsigned 64-bit key (all keys distinct). */
uint64_t oc_priority(uint64_t seed, int level, int64_t i)
{
    uint64_t h = mix64(seed ^ ((uint64_t)level << 40) ^ (uint64_t)i);
    return ((h >> 34) << 32) | (uint64_t)(uint32_t)i;
}

typedef struct { uint64_t key; int64_t v; } keyed;
static int cmp_keyed_desc(const void *a, const void *b)
{
    uint64_t x = ((const keyed *)a)->key, y = ((const keyed *)b)->key;
    return (x < y) - (x > y);
}

/* Reading of the paper's aggregation (a root is chosen among vertices that are neither
 * aggregated nor adjacent to an aggregated vertex; the aggregate is the root and its
 * strong neighbours; leftovers join by heuristics):
 *  1. roots = the greedy maximal independent set of the square of the strong graph,
 *     visiting vertices in decreasing priority (a vertex becomes a root when no root lies
 *     within distance 2 of it);
 *  2. a non-root adjacent to one or more roots joins the adjacent root of largest priority;
 *  3. every other vertex (at distance exactly 2 from a root) joins the aggregate of the
 *     neighbour from step 2 whose root has the largest priority;
 *  4. a vertex with no strong neighbour is its own root (a singleton aggregate);
 *  5. aggregates are numbered by increasing root index.
 * The strong graph is the pattern of strong off-diagonals, assumed symmetric. */
int64_t oc_mis2_aggregate(int64_t n, const int64_t *rp, const int32_t *ci, const uint8_t *strong,
                          uint64_t seed, int level, int32_t *agg, uint8_t *root)
{
    if (n <= 0) return 0;
    keyed *ord = (keyed *)malloc((size_t)n * sizeof(keyed));
    uint8_t *covered = (uint8_t *)calloc((size_t)n, 1);
    int64_t *rootof = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!ord || !covered || !rootof) { free(ord); free(covered); free(rootof); return -1; }
    for (int64_t i = 0; i < n; ++i) { ord[i].key = oc_priority(seed, level, i); ord[i].v = i; }
    qsort(ord, (size_t)n, sizeof(keyed), cmp_keyed_desc);
    memset(root, 0, (size_t)n);
    /* step 1: greedy MIS of the distance-2 graph */
    for (int64_t t = 0; t < n; ++t) {
        int64_t v = ord[t].v;
        if (covered[v]) continue;
        root[v] = 1;
        covered[v] = 1;
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
            if (!strong[e]) continue;
            int64_t u = ci[e];
            covered[u] = 1;
            for (int64_t f = rp[u]; f < rp[u + 1]; ++f)
                if (strong[f]) covered[ci[f]] = 1;
        }
    }
    /* step 2 */
    for (int64_t i = 0; i < n; ++i) rootof[i] = root[i] ? i : -1;
    for (int64_t i = 0; i < n; ++i) {
        if (root[i]) continue;
        int64_t best = -1;
        uint64_t bk = 0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            if (!strong[e]) continue;
            int64_t u = ci[e];
            if (root[u]) {
                uint64_t k = oc_priority(seed, level, u);
                if (best < 0 || k > bk) { best = u; bk = k; }
            }
        }
        rootof[i] = best;
    }
    /* step 3 (reads only step-2 assignments) */
    int64_t *join2 = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        join2[i] = rootof[i];
        if (rootof[i] >= 0) continue;
        int64_t best = -1;
        uint64_t bk = 0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            if (!strong[e]) continue;
            int64_t u = ci[e];
            if (!root[u] && rootof[u] >= 0) {
                uint64_t k = oc_priority(seed, level, rootof[u]);
                if (best < 0 || k > bk) { best = rootof[u]; bk = k; }
            }
        }
        join2[i] = best;
    }
    /* step 5: number roots by increasing index */
    int64_t *id = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t nagg = 0;
    for (int64_t i = 0; i < n; ++i) id[i] = root[i] ? nagg++ : -1;
    int64_t bad = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (join2[i] < 0) { agg[i] = -1; ++bad; }
        else agg[i] = (int32_t)id[join2[i]];
    }
    free(ord); free(covered); free(rootof); free(join2); free(id);
    return bad ? -1 : nagg;
}

/* ---------------------------------------------------------------------------------------- */
/* Further sparsification, §2.5                                                              */
/* ---------------------------------------------------------------------------------------- */

/* Marks in `removed` (already holding the weak entries) the strong links that §2.5 prunes,
 * then their transposes.  For each aggregate with root rho:
 *   candidates = aggregates (other than its own) of rho's weak neighbours, minus every
 *                aggregate that holds a strong neighbour of rho;
 *   for each candidate, count the strong links from the non-root members of the aggregate
 *   (all members together -- reading) into it; a count of exactly one prunes that link.
 * Returns the number of pruned links (before symmetrisation). */
int oc_sprsfy_mark(int64_t n, const int64_t *rp, const int32_t *ci, const uint8_t *strong,
                   const int32_t *agg, const uint8_t *root, int64_t nagg, uint8_t *removed)
{
    /* members of each aggregate, ascending */
    int64_t *start = (int64_t *)calloc((size_t)nagg + 1, sizeof(int64_t));
    int64_t *mem = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *rootv = (int64_t *)malloc((size_t)(nagg > 0 ? nagg : 1) * sizeof(int64_t));
    int64_t *fill = (int64_t *)malloc((size_t)(nagg > 0 ? nagg : 1) * sizeof(int64_t));
    int64_t *cnt = (int64_t *)calloc((size_t)(nagg > 0 ? nagg : 1), sizeof(int64_t));
    int64_t *link = (int64_t *)malloc((size_t)(nagg > 0 ? nagg : 1) * sizeof(int64_t));
    uint8_t *cand = (uint8_t *)calloc((size_t)(nagg > 0 ? nagg : 1), 1);
    uint8_t *drop = (uint8_t *)calloc((size_t)(rp[n] > 0 ? rp[n] : 1), 1);
    int64_t *candlist = (int64_t *)malloc((size_t)(nagg > 0 ? nagg : 1) * sizeof(int64_t));
    if (!start || !mem || !rootv || !fill || !cnt || !link || !cand || !drop || !candlist) return -1;
    for (int64_t i = 0; i < n; ++i) start[agg[i] + 1]++;
    for (int64_t a = 0; a < nagg; ++a) start[a + 1] += start[a];
    for (int64_t a = 0; a < nagg; ++a) fill[a] = start[a];
    for (int64_t i = 0; i < n; ++i) {
        mem[fill[agg[i]]++] = i;
        if (root[i]) rootv[agg[i]] = i;
    }
    int npruned = 0;
    for (int64_t a = 0; a < nagg; ++a) {
        int64_t rho = rootv[a];
        int64_t nc = 0;
        /* weak-neighbour aggregates of the root */
        for (int64_t e = rp[rho]; e < rp[rho + 1]; ++e) {
            int64_t j = ci[e];
            if (j == rho || strong[e]) continue;
            int64_t c = agg[j];
            if (c != a && !cand[c]) { cand[c] = 1; candlist[nc++] = c; }
        }
        /* minus aggregates holding a strong neighbour of the root */
        for (int64_t e = rp[rho]; e < rp[rho + 1]; ++e) {
            int64_t j = ci[e];
            if (j == rho || !strong[e]) continue;
            cand[agg[j]] = 0;
        }
        /* count strong links from non-root members into each candidate */
        for (int64_t m = start[a]; m < start[a + 1]; ++m) {
            int64_t vtx = mem[m];
            if (vtx == rho) continue;
            for (int64_t e = rp[vtx]; e < rp[vtx + 1]; ++e) {
                int64_t w = ci[e];
                if (w == vtx || !strong[e]) continue;
                int64_t c = agg[w];
                if (c != a && cand[c]) { if (cnt[c] == 0) link[c] = e; cnt[c]++; }
            }
        }
        for (int64_t t = 0; t < nc; ++t) {
            int64_t c = candlist[t];
            if (cand[c] && cnt[c] == 1) { drop[link[c]] = 1; ++npruned; }
            cand[c] = 0; cnt[c] = 0;
        }
    }
    /* symmetrise: drop (w, v) whenever (v, w) was dropped */
    for (int64_t v = 0; v < n; ++v) {
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
            if (!drop[e]) continue;
            removed[e] = 1;
            int64_t f = find_entry(rp, ci, ci[e], (int32_t)v);
            if (f >= 0) removed[f] = 1;
        }
    }
    free(start); free(mem); free(rootv); free(fill); free(cnt); free(link); free(cand); free(drop);
    free(candlist);
    return npruned;
}

/* ---------------------------------------------------------------------------------------- */
/* Prolongator constraints, §2.4, Algorithm 3                                                */
/* ---------------------------------------------------------------------------------------- */

/* One row p[0..m) of the (unit-basis) smoothed prolongator.  ptent_pos is the position of
 * the tentative prolongator's entry in this row and ptent_val its value.
 * Returns 0 (feasible, clipped in place), 1 (zero row), 2 (infeasible: tentative row).
 * Readings: the loop runs while min < 0 OR max > 1 (the loop's purpose is to remove every
 * violator); ties in argmin / argmax go to the lowest position; the loop stops after at most
 * m passes; if the working set empties while a nonzero remainder is left the row is
 * infeasible.  w starts as the entries that are nonzero. */
int oc_constrain_row(int64_t m, double *p, int64_t ptent_pos, double ptent_val)
{
    double s = 0.0;
    int64_t nw = 0;
    for (int64_t k = 0; k < m; ++k) { s += p[k]; if (p[k] != 0.0) ++nw; }
    int outcome = 0;
    if (s < 0.0 || s > (double)nw) {
        outcome = 2;
    } else if (s == 0.0) {
        for (int64_t k = 0; k < m; ++k) p[k] = 0.0;
        return 1;
    } else {
        uint8_t *inw = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
        for (int64_t k = 0; k < m; ++k) inw[k] = p[k] != 0.0;
        for (int64_t pass = 0; pass <= m; ++pass) {
            int64_t kmin = 0, kmax = 0;
            for (int64_t k = 1; k < m; ++k) {
                if (p[k] < p[kmin]) kmin = k;
                if (p[k] > p[kmax]) kmax = k;
            }
            if (!(p[kmin] < 0.0 || p[kmax] > 1.0)) break;
            double delta = 0.0;
            if (p[kmin] < 0.0) { delta += p[kmin]; p[kmin] = 0.0; if (inw[kmin]) { inw[kmin] = 0; --nw; } }
            if (p[kmax] > 1.0) { delta += p[kmax] - 1.0; p[kmax] = 1.0; if (inw[kmax]) { inw[kmax] = 0; --nw; } }
            if (nw == 0) {
                if (delta != 0.0) outcome = 2;
                break;
            }
            double share = delta / (double)nw;
            for (int64_t k = 0; k < m; ++k) if (inw[k]) p[k] = p[k] + share;
        }
        free(inw);
    }
    if (outcome == 2) {
        for (int64_t k = 0; k < m; ++k) p[k] = 0.0;
        if (ptent_pos >= 0) p[ptent_pos] = ptent_val;
    }
    return outcome;
}

/* ---------------------------------------------------------------------------------------- */
/* Sparse products and transpose                                                             */
/* ---------------------------------------------------------------------------------------- */

/* C = A B by rows (Gustavson): for each i, for k ascending in row i of A, for j in row k of B,
 * acc[j] = fma(a_ik, b_kj, acc[j]) (one rounding per term).  Every reachable (i, j) is stored,
 * whatever its value; columns are sorted.  Each c_ij is therefore accumulated in ascending k
 * starting from 0.
 * Reading for a row of A of more than OC_SEG stored entries (the same segments as rowsum
 * above): the row's positions fall in segments of OC_SEG; each c_ij is accumulated as above
 * over the terms of each segment separately (ascending k from 0), and the segment sums of
 * every segment of the row (0 for a segment without a term for j) are added in segment order. */
int oc_spgemm(const oc_csr *A, const oc_csr *B, int64_t ncolB, oc_csr **out)
{
    int64_t n = A->n;
    double *acc = (double *)calloc((size_t)(ncolB > 0 ? ncolB : 1), sizeof(double));
    int64_t *mark = (int64_t *)malloc((size_t)(ncolB > 0 ? ncolB : 1) * sizeof(int64_t));
    int32_t *cols = (int32_t *)malloc((size_t)(ncolB > 0 ? ncolB : 1) * sizeof(int32_t));
    int64_t *rp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!acc || !mark || !cols || !rp) return OC_ERR_OOM;
    for (int64_t j = 0; j < ncolB; ++j) mark[j] = -1;
    /* symbolic */
    for (int64_t i = 0; i < n; ++i) {
        int64_t cnt = 0;
        for (int64_t e = A->rp[i]; e < A->rp[i + 1]; ++e) {
            int64_t k = A->ci[e];
            for (int64_t f = B->rp[k]; f < B->rp[k + 1]; ++f) {
                int64_t j = B->ci[f];
                if (mark[j] != i) { mark[j] = i; ++cnt; }
            }
        }
        rp[i + 1] = rp[i] + cnt;
    }
    oc_csr *c = (oc_csr *)calloc(1, sizeof(oc_csr));
    c->n = n; c->nnz = rp[n]; c->rp = rp;
    c->ci = (int32_t *)malloc((size_t)(c->nnz > 0 ? c->nnz : 1) * sizeof(int32_t));
    c->v = (double *)malloc((size_t)(c->nnz > 0 ? c->nnz : 1) * sizeof(double));
    for (int64_t j = 0; j < ncolB; ++j) mark[j] = -1;
    /* numeric */
    double *tot = (double *)malloc((size_t)(ncolB > 0 ? ncolB : 1) * sizeof(double));
    if (!tot) return OC_ERR_OOM;
    for (int64_t i = 0; i < n; ++i) {
        int64_t cnt = 0;
        const int64_t len = A->rp[i + 1] - A->rp[i];
        if (len <= OC_SEG) {
            for (int64_t e = A->rp[i]; e < A->rp[i + 1]; ++e) {
                int64_t k = A->ci[e];
                double a = A->v[e];
                for (int64_t f = B->rp[k]; f < B->rp[k + 1]; ++f) {
                    int64_t j = B->ci[f];
                    if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; cols[cnt++] = (int32_t)j; }
                    acc[j] = fma(a, B->v[f], acc[j]);
                }
            }
        } else {
            /* the row's columns first, then one segment at a time */
            for (int64_t e = A->rp[i]; e < A->rp[i + 1]; ++e)
                for (int64_t f = B->rp[A->ci[e]]; f < B->rp[A->ci[e] + 1]; ++f) {
                    int64_t j = B->ci[f];
                    if (mark[j] != i) { mark[j] = i; cols[cnt++] = (int32_t)j; }
                }
            for (int64_t q = 0; q * OC_SEG < len; ++q) {
                for (int64_t t = 0; t < cnt; ++t) acc[cols[t]] = 0.0;
                const int64_t e0 = A->rp[i] + q * OC_SEG;
                const int64_t e1 = e0 + OC_SEG < A->rp[i + 1] ? e0 + OC_SEG : A->rp[i + 1];
                for (int64_t e = e0; e < e1; ++e) {
                    int64_t k = A->ci[e];
                    double a = A->v[e];
                    for (int64_t f = B->rp[k]; f < B->rp[k + 1]; ++f)
                        acc[B->ci[f]] = fma(a, B->v[f], acc[B->ci[f]]);
                }
                for (int64_t t = 0; t < cnt; ++t)
                    tot[cols[t]] = q == 0 ? acc[cols[t]] : tot[cols[t]] + acc[cols[t]];
            }
            for (int64_t t = 0; t < cnt; ++t) acc[cols[t]] = tot[cols[t]];
        }
        qsort(cols, (size_t)cnt, sizeof(int32_t), cmp_i32);
        for (int64_t t = 0; t < cnt; ++t) {
            c->ci[rp[i] + t] = cols[t];
            c->v[rp[i] + t] = acc[cols[t]];
        }
    }
    free(acc); free(mark); free(cols); free(tot);
    *out = c;
    return OC_OK;
}

/* Transpose by a stable counting sort on the column index. */
int oc_transpose(const oc_csr *A, int64_t ncol, oc_csr **out)
{
    oc_csr *t = (oc_csr *)calloc(1, sizeof(oc_csr));
    if (!t || csr_alloc(t, ncol, A->nnz)) return OC_ERR_OOM;
    for (int64_t e = 0; e < A->nnz; ++e) t->rp[A->ci[e] + 1]++;
    for (int64_t j = 0; j < ncol; ++j) t->rp[j + 1] += t->rp[j];
    int64_t *fill = (int64_t *)malloc((size_t)(ncol > 0 ? ncol : 1) * sizeof(int64_t));
    for (int64_t j = 0; j < ncol; ++j) fill[j] = t->rp[j];
    for (int64_t i = 0; i < A->n; ++i)
        for (int64_t e = A->rp[i]; e < A->rp[i + 1]; ++e) {
            int64_t p = fill[A->ci[e]]++;
            t->ci[p] = (int32_t)i;
            t->v[p] = A->v[e];
        }
    free(fill);
    *out = t;
    return OC_OK;
}

/* ---------------------------------------------------------------------------------------- */
/* Eigenvalue estimate: power method (§3.1: ten sweeps)                                      */
/* ---------------------------------------------------------------------------------------- */

/* Start-vector stream of the power method on `level`; purpose 1 = prolongator smoothing,
 * 2 = Chebyshev smoother. */
uint64_t oc_power_stream_seed(uint64_t seed, int level, int purpose)
{
    return seed ^ ((uint64_t)(level + 1) << 48) ^ ((uint64_t)purpose << 56);
}

static void spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s = s + v[e] * x[ci[e]];
        y[i] = s;
    }
}

static double dot(int64_t n, const double *x, const double *y)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s = s + x[i] * y[i];
    return s;
}

/* Power method on M = D^-1 A.  x0_i = 2u_i - 1 with u_i the i-th output of the SplitMix64
 * stream `stream_seed`, then x = x0 / ||x0||; each sweep forms y = M x and the Rayleigh
 * quotient lambda = x . y (x has unit length); between sweeps x = y / ||y||.  The estimate
 * is the quotient of the last sweep (it can be negative, the failure of §3.1). */
double oc_power_lambda(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *D,
                       int sweeps, uint64_t stream_seed)
{
    if (n == 0) return 0.0;
    double *x = (double *)malloc((size_t)n * sizeof(double));
    double *y = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t i = 0; i < n; ++i) x[i] = 2.0 * stream_u01(stream_seed, (uint64_t)i + 1) - 1.0;
    double nx = sqrt(dot(n, x, x));
    for (int64_t i = 0; i < n; ++i) x[i] = x[i] / nx;
    double lambda = 0.0;
    for (int s = 0; s < sweeps; ++s) {
        spmv(n, rp, ci, v, x, y);
        for (int64_t i = 0; i < n; ++i) y[i] = y[i] / D[i];
        lambda = dot(n, x, y);
        if (s + 1 < sweeps) {
            double ny = sqrt(dot(n, y, y));
            for (int64_t i = 0; i < n; ++i) x[i] = y[i] / ny;
        }
    }
    free(x); free(y);
    return lambda;
}

/* ---------------------------------------------------------------------------------------- */
/* Dense Cholesky for the coarsest level (a direct solve, §3.1)                              */
/* ---------------------------------------------------------------------------------------- */

int oc_cholesky(int64_t n, const double *a, double *l)
{
    memset(l, 0, (size_t)(n * n) * sizeof(double));
    for (int64_t j = 0; j < n; ++j) {
        double d = a[j * n + j];
        for (int64_t k = 0; k < j; ++k) d = d - l[j * n + k] * l[j * n + k];
        if (!(d > 0.0)) return OC_ERR_COARSE_NOT_SPD;
        double ljj = sqrt(d);
        l[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            double s = a[i * n + j];
            for (int64_t k = 0; k < j; ++k) s = s - l[i * n + k] * l[j * n + k];
            l[i * n + j] = s / ljj;
        }
    }
    return OC_OK;
}

/* Dense LU with partial pivoting, in place (row-major): at step k the row with the largest
 * |a_ik|, i >= k (the lowest such index on ties), is exchanged with row k; then the
 * multipliers a_ik / a_kk and the update of the trailing rows.  A zero pivot: singular. */
int oc_lu(int64_t n, double *a, int64_t *piv)
{
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = k;
        for (int64_t i = k + 1; i < n; ++i)
            if (fabs(a[i * n + k]) > fabs(a[p * n + k])) p = i;
        piv[k] = p;
        if (p != k)
            for (int64_t j = 0; j < n; ++j) {
                double t = a[k * n + j];
                a[k * n + j] = a[p * n + j];
                a[p * n + j] = t;
            }
        double d = a[k * n + k];
        if (d == 0.0) return OC_ERR_COARSE_NOT_SPD;
        for (int64_t i = k + 1; i < n; ++i) {
            double m = a[i * n + k] / d;
            a[i * n + k] = m;
            for (int64_t j = k + 1; j < n; ++j) a[i * n + j] = a[i * n + j] - m * a[k * n + j];
        }
    }
    return OC_OK;
}

void oc_lu_solve(int64_t n, const double *lu, const int64_t *piv, const double *b, double *x)
{
    for (int64_t i = 0; i < n; ++i) x[i] = b[i];
    for (int64_t k = 0; k < n; ++k)
        if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
    for (int64_t i = 0; i < n; ++i) {
        double s = x[i];
        for (int64_t k = 0; k < i; ++k) s = s - lu[i * n + k] * x[k];
        x[i] = s;
    }
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int64_t k = i + 1; k < n; ++k) s = s - lu[i * n + k] * x[k];
        x[i] = s / lu[i * n + i];
    }
}

static void chol_solve(int64_t n, const double *l, const double *b, double *x)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = b[i];
        for (int64_t k = 0; k < i; ++k) s = s - l[i * n + k] * x[k];
        x[i] = s / l[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int64_t k = i + 1; k < n; ++k) s = s - l[k * n + i] * x[k];
        x[i] = s / l[i * n + i];
    }
}

/* ---------------------------------------------------------------------------------------- */
/* Hierarchy setup                                                                           */
/* ---------------------------------------------------------------------------------------- */

static int csr_copy(oc_csr *dst, int64_t n, const int64_t *rp, const int32_t *ci, const double *v)
{
    if (csr_alloc(dst, n, rp[n])) return OC_ERR_OOM;
    memcpy(dst->rp, rp, (size_t)(n + 1) * sizeof(int64_t));
    memcpy(dst->ci, ci, (size_t)rp[n] * sizeof(int32_t));
    memcpy(dst->v, v, (size_t)rp[n] * sizeof(double));
    return OC_OK;
}

/* Builds P for level L (steps in the order of §1.1 and §2):
 *  strength (Eq. 7) -> aggregates (Eq. 4) -> tentative prolongator (Eq. 5) -> [§2.5 pruning]
 *  -> filtered matrix (Eq. 6 or Algorithm 2) -> diagonal (Dbar, or Dtilde of Eq. 9 with the
 *  safeguard of Eq. 10-11) -> lambda (power method, or 1 with 1Norm) -> omega = 4/(3 lambda)
 *  -> P = (I - omega D^-1 Abar) Pt (Eq. 3) -> [Algorithm 3 per row] -> column scaling. */
static int build_prolongator_block(oc_hier *h, int L, int stop_if_not_coarsened);

static int build_prolongator(oc_hier *h, int L, int stop_if_not_coarsened)
{
    if (h->p.block_size > 1 || h->p.nullspace_dim > 1) return build_prolongator_block(h, L, stop_if_not_coarsened);
    struct oc_level *lv = &h->lev[L];
    const oc_params *p = &h->p;
    oc_csr *A = &lv->A;
    int64_t n = A->n, nnz = A->nnz;
    int st;

    lv->strong = (uint8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
    lv->removed = (uint8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
    lv->lumpflag = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    lv->agg = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    lv->root = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!lv->strong || !lv->removed || !lv->lumpflag || !lv->agg || !lv->root) return OC_ERR_OOM;

    if (p->strength == 1) {
        /* §3.1: Eq. (7) evaluated on the distance Laplacian instead of A */
        if (!lv->coords || h->dim < 1) return OC_ERR_INVALID_ARG;
        double *Ld = (double *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
        if (!Ld) return OC_ERR_OOM;
        st = oc_distance_laplacian(n, A->rp, A->ci, lv->coords, h->dim, Ld);
        if (!st) oc_strength(n, A->rp, A->ci, Ld, p->theta, lv->strong);
        free(Ld);
        if (st) return st;
    } else {
        oc_strength(n, A->rp, A->ci, A->v, p->theta, lv->strong);
    }
    if (p->krylov == 1) {
        /* Reading: for a nonsymmetric operator the connection i-j is strong when Eq. (7) holds
         * for a_ij or for a_ji, so that the aggregation graph is undirected (symmetric
         * operators give the same mask either way). */
        uint8_t *own = (uint8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
        if (!own) return OC_ERR_OOM;
        memcpy(own, lv->strong, (size_t)nnz);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = A->rp[i]; e < A->rp[i + 1]; ++e) {
                int32_t j = A->ci[e];
                if (j == i || own[e]) continue;
                int64_t t = find_entry(A->rp, A->ci, j, (int32_t)i);
                if (t >= 0 && own[t]) lv->strong[e] = 1;
            }
        free(own);
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = A->rp[i]; e < A->rp[i + 1]; ++e)
            lv->removed[e] = (A->ci[e] != i && !lv->strong[e]) ? 1 : 0;

    int64_t nagg = oc_mis2_aggregate(n, A->rp, A->ci, lv->strong, p->seed, L, lv->agg, lv->root);
    if (nagg < 0) return OC_ERR_INVALID_ARG;
    lv->nagg = nagg;
    /* a level whose aggregation does not reduce its size is the coarsest: no prolongator */
    if (stop_if_not_coarsened && (nagg == n || nagg == 0)) return OC_OK;

    /* tentative prolongator, Eq. (5) with B in place of the constant; the orthonormal form
     * divides each column by the 2-norm of B on its aggregate (summed in ascending index) */
    lv->nrm = (double *)calloc((size_t)(nagg > 0 ? nagg : 1), sizeof(double));
    double *ss = (double *)calloc((size_t)(nagg > 0 ? nagg : 1), sizeof(double));
    for (int64_t i = 0; i < n; ++i) ss[lv->agg[i]] = ss[lv->agg[i]] + lv->B[i] * lv->B[i];
    for (int64_t a = 0; a < nagg; ++a) {
        if (!(ss[a] > 0.0)) { free(ss); return OC_ERR_INVALID_ARG; }
        lv->nrm[a] = sqrt(ss[a]);
    }
    free(ss);

    if (p->variants & OC_SPRSFY)
        oc_sprsfy_mark(n, A->rp, A->ci, lv->strong, lv->agg, lv->root, nagg, lv->removed);

    oc_csr *Ab = NULL;
    st = oc_filter(n, A->rp, A->ci, A->v, lv->removed, (p->variants & OC_OFFLMP) ? 1 : 0, p->tau, &Ab,
                   lv->lumpflag);
    if (st) return st;
    lv->Abar = *Ab;
    free(Ab);

    /* diagonal for the smoothing step */
    lv->Dsm = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (p->variants & OC_1NORM) {
        /* Eq. (9): row 1-norm of Abar; Eq. (10)/(11): at least 4 s_i / (3(1 - sigma)),
         * which is 2 s_i for sigma = 1/3; an all-zero row gets 1 */
        double f = (p->sigma == 1.0 / 3.0) ? 2.0 : 4.0 / (3.0 * (1.0 - p->sigma));
        for (int64_t i = 0; i < n; ++i) {
            const int64_t b = lv->Abar.rp[i], len = lv->Abar.rp[i + 1] - b;
            rowsum rd, rsum;
            rs_init(&rd);
            rs_init(&rsum);
            for (int64_t e = b; e < b + len; ++e) {
                rs_add(&rd, e - b, fabs(lv->Abar.v[e]));
                rs_add(&rsum, e - b, lv->Abar.v[e]);
            }
            double d = rs_value(&rd, len), s = rs_value(&rsum, len);
            if (d == 0.0) d = 1.0;
            if (d < f * s) d = f * s;
            lv->Dsm[i] = d;
        }
    } else {
        for (int64_t i = 0; i < n; ++i) {
            double d = diag_of(lv->Abar.rp, lv->Abar.ci, lv->Abar.v, i);
            if (d == 0.0) return OC_ERR_ZERO_DIAG;
            lv->Dsm[i] = d;
        }
    }

    /* eigenvalue estimate of Dsm^-1 Abar and the damping factor of Eq. (3) */
    if (p->lambda_override > 0.0) {
        lv->lambda_bar = p->lambda_override;
    } else if ((p->variants & OC_1NORM) && !p->onenorm_power) {
        lv->lambda_bar = 1.0;              /* §2.1: the Gershgorin bound, used as the estimate */
    } else {
        lv->lambda_bar = oc_power_lambda(n, lv->Abar.rp, lv->Abar.ci, lv->Abar.v, lv->Dsm, p->power_iters,
                                         oc_power_stream_seed(p->seed, L, 1));
    }
    if (!(lv->lambda_bar > 0.0) || !isfinite(lv->lambda_bar)) return OC_ERR_EIGEN;
    lv->omega = 4.0 / (3.0 * lv->lambda_bar);

    /* P = Pt - omega Dsm^-1 (Abar Pt), unit basis (Pt_i = B_i at column agg(i)).
     * Row i's columns are the aggregates of the columns of Abar's row i; (Abar Pt)_ic sums
     * Abar_ik B_k over those k (ascending) with agg(k) = c. */
    {
        oc_csr Pt;
        if (csr_alloc(&Pt, n, n)) return OC_ERR_OOM;
        for (int64_t i = 0; i < n; ++i) { Pt.rp[i + 1] = i + 1; Pt.ci[i] = lv->agg[i]; Pt.v[i] = lv->B[i]; }
        oc_csr *AP = NULL;
        st = oc_spgemm(&lv->Abar, &Pt, nagg, &AP);
        csr_release(&Pt);
        if (st) return st;
        for (int64_t i = 0; i < n; ++i) {
            double scale = lv->omega / lv->Dsm[i];
            for (int64_t e = AP->rp[i]; e < AP->rp[i + 1]; ++e) {
                double pt = (AP->ci[e] == lv->agg[i]) ? lv->B[i] : 0.0;
                AP->v[e] = pt - scale * AP->v[e];
            }
        }
        lv->P = *AP;
        free(AP);
    }

    /* Algorithm 3 on each row (unit basis), then the orthonormal column scaling */
    lv->cflag = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (p->variants & OC_CNSTRNT) {
        for (int64_t i = 0; i < n; ++i) {
            int64_t b = lv->P.rp[i], m = lv->P.rp[i + 1] - b;
            int64_t pos = -1;
            for (int64_t t = 0; t < m; ++t) if (lv->P.ci[b + t] == lv->agg[i]) pos = t;
            lv->cflag[i] = (uint8_t)oc_constrain_row(m, lv->P.v + b, pos, lv->B[i]);
        }
    }
    if (!p->pt_unit)
        for (int64_t e = 0; e < lv->P.nnz; ++e) lv->P.v[e] = lv->P.v[e] / lv->nrm[lv->P.ci[e]];

    oc_csr *R = NULL;
    st = oc_transpose(&lv->P, nagg, &R);
    if (st) return st;
    lv->R = *R;
    free(R);
    return OC_OK;
}

/* The same steps for a system of PDEs (variants off): block strength between nodes
 * (oc_node_fill), MIS-2 aggregation of the node graph, the QR tentative prolongator
 * (oc_block_tentative), the filtered matrix with the dropped entries lumped into the diagonal
 * (Eq. 6), lambda of Dbar^-1 Abar, and P = Pt - omega Dbar^-1 (Abar Pt) (Eq. 3).  agg and root
 * are per node; the coarse level has k unknowns per aggregate. */
static int build_prolongator_block(oc_hier *h, int L, int stop_if_not_coarsened)
{
    struct oc_level *lv = &h->lev[L];
    const oc_params *p = &h->p;
    oc_csr *A = &lv->A;
    int64_t n = A->n, nnz = A->nnz;
    int bs = lv->bs, k = lv->k;
    if (bs < 1 || k < 1 || n % bs) return OC_ERR_INVALID_ARG;
    int64_t nn = n / bs;
    int st;
    lv->strong = (uint8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
    lv->removed = (uint8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
    lv->lumpflag = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    lv->agg = (int32_t *)malloc((size_t)(nn > 0 ? nn : 1) * sizeof(int32_t));
    lv->root = (uint8_t *)malloc((size_t)(nn > 0 ? nn : 1));
    int64_t *nrp = (int64_t *)malloc((size_t)(nn + 1) * sizeof(int64_t));
    if (!lv->strong || !lv->removed || !lv->lumpflag || !lv->agg || !lv->root || !nrp) { free(nrp); return OC_ERR_OOM; }
    int64_t nnzn = oc_node_graph(n, A->rp, A->ci, bs, nrp);
    if (nnzn < 0) { free(nrp); return OC_ERR_INVALID_ARG; }
    int32_t *nci = (int32_t *)malloc((size_t)(nnzn > 0 ? nnzn : 1) * sizeof(int32_t));
    double *nF = (double *)malloc((size_t)(nnzn > 0 ? nnzn : 1) * sizeof(double));
    uint8_t *nstrong = (uint8_t *)malloc((size_t)(nnzn > 0 ? nnzn : 1));
    if (!nci || !nF || !nstrong) { free(nrp); free(nci); free(nF); free(nstrong); return OC_ERR_OOM; }
    st = oc_node_fill(n, A->rp, A->ci, A->v, bs, p->theta, nrp, nci, nF, nstrong, lv->strong);
    int64_t nagg = -1;
    if (!st) nagg = oc_mis2_aggregate(nn, nrp, nci, nstrong, p->seed, L, lv->agg, lv->root);
    free(nrp); free(nci); free(nF); free(nstrong);
    if (st) return st;
    if (nagg < 0) return OC_ERR_INVALID_ARG;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = A->rp[i]; e < A->rp[i + 1]; ++e)
            lv->removed[e] = (A->ci[e] != i && !lv->strong[e]) ? 1 : 0;
    lv->nagg = nagg;
    if (stop_if_not_coarsened && (nagg == 0 || nagg * k >= n)) return OC_OK;
    int64_t nc = nagg * k;

    double *Qv = (double *)malloc((size_t)(n > 0 ? n : 1) * (size_t)k * sizeof(double));
    lv->Bc = (double *)malloc((size_t)(nc > 0 ? nc : 1) * (size_t)k * sizeof(double));
    if (!Qv || !lv->Bc) { free(Qv); return OC_ERR_OOM; }
    st = oc_block_tentative(n, bs, k, lv->agg, nagg, lv->B, Qv, lv->Bc);
    if (st) { free(Qv); return st; }

    oc_csr *Ab = NULL;
    st = oc_filter(n, A->rp, A->ci, A->v, lv->removed, 0, p->tau, &Ab, lv->lumpflag);
    if (st) { free(Qv); return st; }
    lv->Abar = *Ab;
    free(Ab);
    lv->Dsm = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        double d = diag_of(lv->Abar.rp, lv->Abar.ci, lv->Abar.v, i);
        if (d == 0.0) { free(Qv); return OC_ERR_ZERO_DIAG; }
        lv->Dsm[i] = d;
    }
    if (p->lambda_override > 0.0)
        lv->lambda_bar = p->lambda_override;
    else
        lv->lambda_bar = oc_power_lambda(n, lv->Abar.rp, lv->Abar.ci, lv->Abar.v, lv->Dsm, p->power_iters,
                                         oc_power_stream_seed(p->seed, L, 1));
    if (!(lv->lambda_bar > 0.0) || !isfinite(lv->lambda_bar)) { free(Qv); return OC_ERR_EIGEN; }
    lv->omega = 4.0 / (3.0 * lv->lambda_bar);

    /* P = Pt - omega Dbar^-1 (Abar Pt); Pt row i: columns agg(i) k .. agg(i) k + k - 1 */
    oc_csr Pt;
    if (csr_alloc(&Pt, n, n * k)) { free(Qv); return OC_ERR_OOM; }
    for (int64_t i = 0; i < n; ++i) {
        Pt.rp[i + 1] = (i + 1) * k;
        for (int j = 0; j < k; ++j) {
            Pt.ci[i * k + j] = (int32_t)(lv->agg[i / bs] * k + j);
            Pt.v[i * k + j] = Qv[i * k + j];
        }
    }
    oc_csr *AP = NULL;
    st = oc_spgemm(&lv->Abar, &Pt, nc, &AP);
    csr_release(&Pt);
    if (st) { free(Qv); return st; }
    for (int64_t i = 0; i < n; ++i) {
        double scale = lv->omega / lv->Dsm[i];
        int64_t c0 = (int64_t)lv->agg[i / bs] * k;
        for (int64_t e = AP->rp[i]; e < AP->rp[i + 1]; ++e) {
            int64_t c = AP->ci[e];
            double pt = (c >= c0 && c < c0 + k) ? Qv[i * k + (c - c0)] : 0.0;
            AP->v[e] = pt - scale * AP->v[e];
        }
    }
    free(Qv);
    lv->P = *AP;
    free(AP);
    lv->cflag = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    oc_csr *R = NULL;
    st = oc_transpose(&lv->P, nc, &R);
    if (st) return st;
    lv->R = *R;
    free(R);
    return OC_OK;
}

/* Chebyshev eigenvalue and inverse diagonal of A_L */
static int smoother_setup(oc_hier *h, int L)
{
    struct oc_level *lv = &h->lev[L];
    int64_t n = lv->A.n;
    double *d = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    lv->invdiag = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        d[i] = diag_of(lv->A.rp, lv->A.ci, lv->A.v, i);
        if (d[i] == 0.0) { free(d); return OC_ERR_ZERO_DIAG; }
        lv->invdiag[i] = 1.0 / d[i];
    }
    lv->lambda_cheb = oc_power_lambda(n, lv->A.rp, lv->A.ci, lv->A.v, d, h->p.power_iters,
                                      oc_power_stream_seed(h->p.seed, L, 2));
    free(d);
    if (!(lv->lambda_cheb > 0.0) || !isfinite(lv->lambda_cheb)) return OC_ERR_EIGEN;
    return OC_OK;
}

int oc_setup(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *nullspace,
             const oc_params *p, oc_hier **out)
{
    return oc_setup_coords(n, rp, ci, v, nullspace, NULL, 0, p, out);
}

int oc_setup_coords(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *nullspace,
                    const double *coords, int dim, const oc_params *p, oc_hier **out)
{
    *out = NULL;
    if (n < 0 || !rp) return OC_ERR_INVALID_ARG;
    if (p->strength == 1 && (!coords || dim < 1 || dim > 3)) return OC_ERR_INVALID_ARG;
    const int block = p->block_size > 1 || p->nullspace_dim > 1;
    if (p->block_size < 1 || p->nullspace_dim < 1 || n % p->block_size) return OC_ERR_INVALID_ARG;
    if (block && (p->variants || p->strength || (!nullspace && p->nullspace_dim != p->block_size)))
        return p->variants || p->strength ? OC_ERR_UNSUPPORTED : OC_ERR_INVALID_ARG;
    oc_hier *h = (oc_hier *)calloc(1, sizeof(oc_hier));
    if (!h) return OC_ERR_OOM;
    h->p = *p;
    int st = csr_copy(&h->lev[0].A, n, rp, ci, v);
    if (st) { oc_free(h); return st; }
    if (coords && dim >= 1) {
        h->dim = dim;
        h->lev[0].coords = (double *)malloc((size_t)(n > 0 ? n * dim : 1) * sizeof(double));
        if (!h->lev[0].coords) { oc_free(h); return OC_ERR_OOM; }
        memcpy(h->lev[0].coords, coords, (size_t)(n * dim) * sizeof(double));
    }
    {
        /* B: k vectors of length n one after another; without one given, the constant (scalar)
         * or the constant of each component (k = bs) */
        const int k = p->nullspace_dim, bs = p->block_size;
        h->lev[0].bs = bs;
        h->lev[0].k = k;
        h->lev[0].B = (double *)malloc((size_t)(n > 0 ? n : 1) * (size_t)k * sizeof(double));
        if (!h->lev[0].B) { oc_free(h); return OC_ERR_OOM; }
        for (int j = 0; j < k; ++j)
            for (int64_t i = 0; i < n; ++i)
                h->lev[0].B[(int64_t)j * n + i] = nullspace ? nullspace[(int64_t)j * n + i] : (i % bs == j ? 1.0 : 0.0);
    }
    int L = 0;
    for (;;) {
        struct oc_level *lv = &h->lev[L];
        if (lv->A.n <= p->max_coarse || L + 1 >= p->max_levels || L + 1 >= OC_MAX_LEVELS) break;
        st = build_prolongator(h, L, 1);
        if (st) { oc_free(h); return st; }
        if (lv->nagg * lv->k >= lv->A.n || lv->nagg == 0) break;   /* no coarsening: this is the coarsest */
        /* Galerkin product, Eq. (2), with the original A */
        oc_csr *AP = NULL, *Ac = NULL;
        st = oc_spgemm(&lv->A, &lv->P, lv->nagg * lv->k, &AP);
        if (!st) st = oc_spgemm(&lv->R, AP, lv->nagg * lv->k, &Ac);
        oc_csr_free(AP);
        if (st) { oc_free(h); return st; }
        st = smoother_setup(h, L);
        if (st) { oc_csr_free(Ac); oc_free(h); return st; }
        struct oc_level *nx = &h->lev[L + 1];
        nx->A = *Ac;
        free(Ac);
        nx->bs = lv->k;
        nx->k = lv->k;
        if (block) {
            nx->B = lv->Bc;
            lv->Bc = NULL;
        } else {
            nx->B = (double *)malloc((size_t)(lv->nagg > 0 ? lv->nagg : 1) * sizeof(double));
            for (int64_t a = 0; a < lv->nagg; ++a) nx->B[a] = p->pt_unit ? 1.0 : lv->nrm[a];
        }
        if (h->dim > 0) {
            nx->coords = (double *)malloc((size_t)(lv->nagg > 0 ? lv->nagg * h->dim : 1) * sizeof(double));
            if (!nx->coords) { oc_free(h); return OC_ERR_OOM; }
            st = oc_coarse_coords(lv->A.n, lv->agg, lv->nagg, lv->coords, h->dim, nx->coords);
            if (st) { oc_free(h); return st; }
        }
        ++L;
    }
    h->nlev = L + 1;
    /* coarsest level: dense Cholesky */
    struct oc_level *cl = &h->lev[L];
    int64_t nc = cl->A.n;
    if (nc > OC_MAX_DENSE) { oc_free(h); return OC_ERR_UNSUPPORTED; }
    double *dense = (double *)calloc((size_t)(nc * nc > 0 ? nc * nc : 1), sizeof(double));
    for (int64_t i = 0; i < nc; ++i)
        for (int64_t e = cl->A.rp[i]; e < cl->A.rp[i + 1]; ++e) dense[i * nc + cl->A.ci[e]] = cl->A.v[e];
    if (p->krylov == 1) {
        /* nonsymmetric: LU with partial pivoting */
        h->lu = dense;
        h->piv = (int64_t *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(int64_t));
        st = h->piv ? oc_lu(nc, h->lu, h->piv) : OC_ERR_OOM;
    } else {
        h->chol = (double *)calloc((size_t)(nc * nc > 0 ? nc * nc : 1), sizeof(double));
        st = oc_cholesky(nc, dense, h->chol);
        free(dense);
    }
    if (st) { oc_free(h); return st; }
    *out = h;
    return OC_OK;
}

/* ---------------------------------------------------------------------------------------- */
/* Solve: Chebyshev smoother, V-cycle (Algorithm 1) and preconditioned CG                    */
/* ---------------------------------------------------------------------------------------- */

/* Chebyshev polynomial of degree m in D^-1 A on [b lambda/ratio, b lambda], applied to
 * A x = f from the current x (three-term recurrence of Chebyshev acceleration as in
 * Saad, Iterative Methods for Sparse Linear Systems, 2nd ed., Algorithm 12.1):
 *   theta = (a+b)/2, delta = (b-a)/2, sigma1 = theta/delta, rho = 1/sigma1,
 *   d = D^-1 (f - A x) / theta, x += d;
 *   repeat m-1 times: rho' = 1/(2 sigma1 - rho), d = rho' rho d + (2 rho'/delta) D^-1 (f - A x),
 *                     x += d, rho = rho'. */
static void chebyshev(const struct oc_level *lv, int degree, double ratio, double boost, const double *f, double *x,
                      double *r, double *d)
{
    int64_t n = lv->A.n;
    /* Reading: ten power sweeps give a lower estimate of lambda_max(D^-1 A); the interval's
     * upper end is the estimate times a safety factor b (1.1), so that the polynomial does not
     * amplify the top of the spectrum (b = 1 is the estimate itself). */
    double lmax = boost * lv->lambda_cheb, lmin = lmax / ratio;
    double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
    double sigma1 = theta / delta, rho = 1.0 / sigma1;
    spmv(n, lv->A.rp, lv->A.ci, lv->A.v, x, r);
    for (int64_t i = 0; i < n; ++i) {
        d[i] = (lv->invdiag[i] * (f[i] - r[i])) / theta;
        x[i] = x[i] + d[i];
    }
    for (int k = 1; k < degree; ++k) {
        double rho_new = 1.0 / (2.0 * sigma1 - rho);
        double c1 = rho_new * rho, c2 = 2.0 * rho_new / delta;
        spmv(n, lv->A.rp, lv->A.ci, lv->A.v, x, r);
        for (int64_t i = 0; i < n; ++i) {
            d[i] = c1 * d[i] + c2 * (lv->invdiag[i] * (f[i] - r[i]));
            x[i] = x[i] + d[i];
        }
        rho = rho_new;
    }
}

/* The smoother alone, for its pins: the same routine on an operator given as CSR with
 * 1/diag(A) and lambda supplied by the caller. */
int oc_chebyshev_apply(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *invdiag,
                       double lambda, int degree, double ratio, double boost, const double *f, double *x)
{
    if (n < 0 || degree < 1 || !(ratio > 1.0) || !(lambda > 0.0) || !(boost > 0.0)) return OC_ERR_INVALID_ARG;
    struct oc_level lv;
    memset(&lv, 0, sizeof(lv));
    lv.A.n = n; lv.A.nnz = rp[n];
    lv.A.rp = (int64_t *)rp; lv.A.ci = (int32_t *)ci; lv.A.v = (double *)v;
    lv.invdiag = (double *)invdiag;
    lv.lambda_cheb = lambda;
    double *r = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *d = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!r || !d) { free(r); free(d); return OC_ERR_OOM; }
    chebyshev(&lv, degree, ratio, boost, f, x, r, d);
    free(r); free(d);
    return OC_OK;
}

/* Algorithm 1 from level L with u holding the initial guess. */
static void vcycle_level(oc_hier *h, int L, const double *f, double *u)
{
    struct oc_level *lv = &h->lev[L];
    int64_t n = lv->A.n;
    if (L == h->nlev - 1) {
        if (h->lu) oc_lu_solve(n, h->lu, h->piv, f, u);
        else chol_solve(n, h->chol, f, u);
        return;
    }
    double *r = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *d = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    int64_t nc = lv->nagg * lv->k;     /* rows of the next level */
    double *fc = (double *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(double));
    double *uc = (double *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(double));
    chebyshev(lv, h->p.cheb_degree, h->p.cheb_ratio, h->p.cheb_boost, f, u, r, d);
    spmv(n, lv->A.rp, lv->A.ci, lv->A.v, u, r);
    for (int64_t i = 0; i < n; ++i) r[i] = f[i] - r[i];
    spmv(nc, lv->R.rp, lv->R.ci, lv->R.v, r, fc);
    vcycle_level(h, L + 1, fc, uc);
    spmv(n, lv->P.rp, lv->P.ci, lv->P.v, uc, r);
    for (int64_t i = 0; i < n; ++i) u[i] = u[i] + r[i];
    chebyshev(lv, h->p.cheb_degree, h->p.cheb_ratio, h->p.cheb_boost, f, u, r, d);
    free(r); free(d); free(fc); free(uc);
}

int oc_vcycle(oc_hier *h, const double *f, double *u)
{
    memset(u, 0, (size_t)(h->lev[0].A.n > 0 ? h->lev[0].A.n : 1) * sizeof(double));
    vcycle_level(h, 0, f, u);
    return OC_OK;
}

/* Preconditioned CG from x = 0.  Stops when ||r_k|| / ||b|| <= tol on the recurrence
 * residual and the true residual b - A x also meets it; otherwise r is replaced by the true
 * residual and the iteration continues.  apply(M) = one V-cycle, or the identity. */
static int pcg(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, oc_hier *h, const double *b,
               double *x, double tol, int max_iter, oc_info *info)
{
    double *r = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *z = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *pv = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *q = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    memset(x, 0, (size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t i = 0; i < n; ++i) r[i] = b[i];
    double nb = sqrt(dot(n, b, b));
    int it = 0, status = OC_OK;
    double relres = 0.0;
    if (nb == 0.0) goto done;
    if (h) oc_vcycle(h, r, z); else memcpy(z, r, (size_t)n * sizeof(double));
    memcpy(pv, z, (size_t)n * sizeof(double));
    double rz = dot(n, r, z);
    status = OC_ERR_NOT_CONVERGED;
    while (it < max_iter) {
        spmv(n, rp, ci, v, pv, q);
        double pq = dot(n, pv, q);
        double alpha = rz / pq;
        for (int64_t i = 0; i < n; ++i) { x[i] = x[i] + alpha * pv[i]; r[i] = r[i] - alpha * q[i]; }
        ++it;
        double rn = sqrt(dot(n, r, r));
        if (rn / nb <= tol) {
            spmv(n, rp, ci, v, x, q);
            for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
            double tn = sqrt(dot(n, q, q));
            if (tn / nb <= tol) { status = OC_OK; break; }
            memcpy(r, q, (size_t)n * sizeof(double));
        }
        if (h) oc_vcycle(h, r, z); else memcpy(z, r, (size_t)n * sizeof(double));
        double rz_new = dot(n, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (int64_t i = 0; i < n; ++i) pv[i] = z[i] + beta * pv[i];
    }
done:
    spmv(n, rp, ci, v, x, q);
    for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
    relres = nb == 0.0 ? 0.0 : sqrt(dot(n, q, q)) / nb;
    if (info) { info->iters = it; info->status = status; info->relres_true = relres; }
    free(r); free(z); free(pv); free(q);
    return status;
}

/* Flexible GMRES(m) with right preconditioning (Saad, SIAM J. Sci. Comput. 14, 1993), from
 * x = 0: per cycle r = b - A x, v_0 = r / |r|; per step z_j = M v_j (one V-cycle), w = A z_j,
 * classical Gram-Schmidt against v_0..v_j done twice (h = V^T w, w -= V h, each product and
 * sum in ascending index), v_{j+1} = w / |w|; Givens rotations keep the Hessenberg matrix
 * triangular and |g_{j+1}| is the residual norm of the minimiser.  When |g_{j+1}| <= tol |b|,
 * at the cycle's end or at the iteration limit: y from the triangular system, x += Z y, and
 * the true residual decides (stop, or restart from x).  The iteration count is the number of
 * products with A inside the Arnoldi steps.  h NULL: no preconditioner (z_j = v_j). */
static int fgmres(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, oc_hier *h, const double *b,
                  double *x, double tol, int m, int max_iter, oc_info *info)
{
    if (m < 1) m = 1;
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *V = (double *)calloc(nn * (size_t)(m + 1), sizeof(double));
    double *Z = (double *)calloc(nn * (size_t)m, sizeof(double));
    double *w = (double *)malloc(nn * sizeof(double));
    double *H = (double *)calloc((size_t)(m + 1) * (size_t)m, sizeof(double));   /* H[i * m + j] */
    double *g = (double *)calloc((size_t)(m + 1), sizeof(double));
    double *cs = (double *)calloc((size_t)m, sizeof(double)), *sn = (double *)calloc((size_t)m, sizeof(double));
    double *hv = (double *)calloc((size_t)(m + 1), sizeof(double)), *y = (double *)calloc((size_t)m, sizeof(double));
    memset(x, 0, nn * sizeof(double));
    double nb = sqrt(dot(n, b, b));
    int it = 0, status = OC_OK;
    double relres = 0.0;
    if (nb == 0.0) goto done;
    status = OC_ERR_NOT_CONVERGED;
    while (it < max_iter) {
        spmv(n, rp, ci, v, x, w);
        for (int64_t i = 0; i < n; ++i) w[i] = b[i] - w[i];
        double beta = sqrt(dot(n, w, w));
        if (beta / nb <= tol) { status = OC_OK; break; }
        for (int64_t i = 0; i < n; ++i) V[i] = w[i] / beta;
        memset(g, 0, (size_t)(m + 1) * sizeof(double));
        g[0] = beta;
        int j = 0, stop = 0;
        for (; j < m && it < max_iter; ++j) {
            double *vj = V + (size_t)j * nn, *zj = Z + (size_t)j * nn;
            if (h) oc_vcycle(h, vj, zj); else memcpy(zj, vj, nn * sizeof(double));
            spmv(n, rp, ci, v, zj, w);
            ++it;
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = 0.0;
            for (int pass = 0; pass < 2; ++pass) {
                for (int i = 0; i <= j; ++i) hv[i] = dot(n, V + (size_t)i * nn, w);
                for (int64_t e = 0; e < n; ++e) {
                    double t = w[e];
                    for (int i = 0; i <= j; ++i) t = t - hv[i] * V[(size_t)i * nn + e];
                    w[e] = t;
                }
                for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = H[(size_t)i * m + j] + hv[i];
            }
            double hn = sqrt(dot(n, w, w));
            H[(size_t)(j + 1) * m + j] = hn;
            if (hn > 0.0)
                for (int64_t e = 0; e < n; ++e) V[(size_t)(j + 1) * nn + e] = w[e] / hn;
            for (int i = 0; i < j; ++i) {
                double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
            double r = sqrt(a * a + c * c);
            cs[j] = a / r;
            sn[j] = c / r;
            H[(size_t)j * m + j] = r;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            if (fabs(g[j + 1]) / nb <= tol || hn == 0.0) { stop = 1; ++j; break; }
        }
        /* y = H(0:j, 0:j)^-1 g(0:j); x += Z y */
        for (int i = j - 1; i >= 0; --i) {
            double s = g[i];
            for (int k = i + 1; k < j; ++k) s = s - H[(size_t)i * m + k] * y[k];
            y[i] = s / H[(size_t)i * m + i];
        }
        for (int64_t e = 0; e < n; ++e) {
            double t = x[e];
            for (int k = 0; k < j; ++k) t = t + y[k] * Z[(size_t)k * nn + e];
            x[e] = t;
        }
        if (stop || it >= max_iter) {
            spmv(n, rp, ci, v, x, w);
            for (int64_t i = 0; i < n; ++i) w[i] = b[i] - w[i];
            if (sqrt(dot(n, w, w)) / nb <= tol) { status = OC_OK; break; }
        }
    }
done:
    spmv(n, rp, ci, v, x, w);
    for (int64_t i = 0; i < n; ++i) w[i] = b[i] - w[i];
    relres = nb == 0.0 ? 0.0 : sqrt(dot(n, w, w)) / nb;
    if (info) { info->iters = it; info->status = status; info->relres_true = relres; }
    free(V); free(Z); free(w); free(H); free(g); free(cs); free(sn); free(hv); free(y);
    return status;
}

int oc_gmres_plain(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *b, double *x,
                   double tol, int restart, int max_iter, oc_info *info)
{
    return fgmres(n, rp, ci, v, NULL, b, x, tol, restart, max_iter, info);
}

int oc_solve(oc_hier *h, const double *b, double *x, double tol, oc_info *info)
{
    oc_csr *A = &h->lev[0].A;
    int st = h->p.krylov == 1
                 ? fgmres(A->n, A->rp, A->ci, A->v, h, b, x, tol, h->p.restart, h->p.max_iter, info)
                 : pcg(A->n, A->rp, A->ci, A->v, h, b, x, tol, h->p.max_iter, info);
    if (info) {
        info->levels = h->nlev;
        double tot = 0.0;
        for (int L = 0; L < h->nlev; ++L) tot += (double)h->lev[L].A.nnz;
        info->op_complexity = A->nnz > 0 ? tot / (double)A->nnz : 0.0;
    }
    return st;
}

/* Level 0 only: strength, aggregates, filtered matrix and smoothed prolongator, without the
 * Galerkin product or a coarse factorisation (used to check the prolongator on operators
 * whose coarse matrix is singular). */
int oc_prolongator_only(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                        const double *nullspace, const oc_params *p, oc_hier **out)
{
    *out = NULL;
    oc_hier *h = (oc_hier *)calloc(1, sizeof(oc_hier));
    if (!h) return OC_ERR_OOM;
    h->p = *p;
    h->nlev = 1;
    h->prolongator_only = 1;
    int st = csr_copy(&h->lev[0].A, n, rp, ci, v);
    if (st) { oc_free(h); return st; }
    {
        /* B: k vectors of length n one after another; without one given, the constant (scalar)
         * or the constant of each component (k = bs) */
        const int k = p->nullspace_dim, bs = p->block_size;
        h->lev[0].bs = bs;
        h->lev[0].k = k;
        h->lev[0].B = (double *)malloc((size_t)(n > 0 ? n : 1) * (size_t)k * sizeof(double));
        if (!h->lev[0].B) { oc_free(h); return OC_ERR_OOM; }
        for (int j = 0; j < k; ++j)
            for (int64_t i = 0; i < n; ++i)
                h->lev[0].B[(int64_t)j * n + i] = nullspace ? nullspace[(int64_t)j * n + i] : (i % bs == j ? 1.0 : 0.0);
    }
    st = build_prolongator(h, 0, 0);
    if (st) { oc_free(h); return st; }
    *out = h;
    return OC_OK;
}

int oc_pcg_plain(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *b,
                 double *x, double tol, int max_iter, oc_info *info)
{
    return pcg(n, rp, ci, v, NULL, b, x, tol, max_iter, info);
}

void oc_free(oc_hier *h)
{
    if (!h) return;
    for (int L = 0; L < OC_MAX_LEVELS; ++L) {
        struct oc_level *lv = &h->lev[L];
        csr_release(&lv->A); csr_release(&lv->Abar); csr_release(&lv->P); csr_release(&lv->R);
        free(lv->strong); free(lv->removed); free(lv->lumpflag); free(lv->agg); free(lv->root);
        free(lv->B); free(lv->nrm); free(lv->Dsm); free(lv->cflag); free(lv->invdiag); free(lv->coords);
        free(lv->Bc);
    }
    free(h->chol);
    free(h->lu);
    free(h->piv);
    free(h);
}

/* ---------------------------------------------------------------------------------------- */
/* Introspection                                                                             */
/* ---------------------------------------------------------------------------------------- */

int oc_nlevels(const oc_hier *h) { return h ? h->nlev : 0; }

/* what: 0 A.rp, 1 A.ci, 2 A.v, 3 strong, 4 removed, 5 lumpflag, 6 Abar.rp, 7 Abar.ci,
 * 8 Abar.v, 9 agg, 10 root, 11 P.rp, 12 P.ci, 13 P.v, 14 R.rp, 15 R.ci, 16 R.v, 17 Dsm,
 * 18 scalars [lambda_bar, omega, lambda_cheb, nagg], 19 B, 20 cflag, 21 Cholesky factor,
 * 22 coordinates (n * dim), 23 [unknowns per node, near-null-space vectors].
 * Copies into dst when it is not NULL; *len receives the element count. */
int oc_level_get(const oc_hier *h, int L, int what, void *dst, int64_t *len)
{
    if (!h || L < 0 || L >= h->nlev) return OC_ERR_INVALID_ARG;
    const struct oc_level *lv = &h->lev[L];
    int last = (L == h->nlev - 1) && !h->prolongator_only;
    const void *src = NULL;
    size_t es = 0;
    int64_t cnt = 0;
    double sc[4];
    switch (what) {
    case 0: src = lv->A.rp; es = 8; cnt = lv->A.n + 1; break;
    case 1: src = lv->A.ci; es = 4; cnt = lv->A.nnz; break;
    case 2: src = lv->A.v; es = 8; cnt = lv->A.nnz; break;
    case 3: src = lv->strong; es = 1; cnt = last ? 0 : lv->A.nnz; break;
    case 4: src = lv->removed; es = 1; cnt = last ? 0 : lv->A.nnz; break;
    case 5: src = lv->lumpflag; es = 1; cnt = last ? 0 : lv->A.n; break;
    case 6: src = lv->Abar.rp; es = 8; cnt = last ? 0 : lv->Abar.n + 1; break;
    case 7: src = lv->Abar.ci; es = 4; cnt = last ? 0 : lv->Abar.nnz; break;
    case 8: src = lv->Abar.v; es = 8; cnt = last ? 0 : lv->Abar.nnz; break;
    case 9: src = lv->agg; es = 4; cnt = last ? 0 : lv->A.n / (lv->bs > 0 ? lv->bs : 1); break;
    case 10: src = lv->root; es = 1; cnt = last ? 0 : lv->A.n / (lv->bs > 0 ? lv->bs : 1); break;
    case 11: src = lv->P.rp; es = 8; cnt = last ? 0 : lv->P.n + 1; break;
    case 12: src = lv->P.ci; es = 4; cnt = last ? 0 : lv->P.nnz; break;
    case 13: src = lv->P.v; es = 8; cnt = last ? 0 : lv->P.nnz; break;
    case 14: src = lv->R.rp; es = 8; cnt = last ? 0 : lv->R.n + 1; break;
    case 15: src = lv->R.ci; es = 4; cnt = last ? 0 : lv->R.nnz; break;
    case 16: src = lv->R.v; es = 8; cnt = last ? 0 : lv->R.nnz; break;
    case 17: src = lv->Dsm; es = 8; cnt = last ? 0 : lv->A.n; break;
    case 18:
        sc[0] = lv->lambda_bar; sc[1] = lv->omega; sc[2] = lv->lambda_cheb; sc[3] = (double)lv->nagg;
        src = sc; es = 8; cnt = 4; break;
    case 19: src = lv->B; es = 8; cnt = lv->A.n * (lv->k > 0 ? lv->k : 1); break;
    case 20: src = lv->cflag; es = 1; cnt = last ? 0 : lv->A.n; break;
    case 21: src = h->chol; es = 8; cnt = last ? lv->A.n * lv->A.n : 0; break;
    case 22: src = lv->coords; es = 8; cnt = lv->coords ? lv->A.n * h->dim : 0; break;
    case 23: sc[0] = lv->bs; sc[1] = lv->k; src = sc; es = 8; cnt = 2; break;
    default: return OC_ERR_INVALID_ARG;
    }
    if (len) *len = cnt;
    if (dst && cnt > 0 && src) memcpy(dst, src, (size_t)cnt * es);
    return OC_OK;
}
