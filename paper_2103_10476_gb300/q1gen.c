/*
 * q1gen.c -- input generation: the Q1 (trilinear) finite-element diffusion matrix on a
 * tensor-product mesh, the same assembly and the same floating-point operations, in the
 * same order, as problems.q1_matrix (numpy), written in C so that large operators for the
 * serving workload are produced quickly.  It holds none of the multigrid method.  Compiled
 * with -ffp-contract=off so that every product and sum rounds as numpy's does.
 *
 * Stencil of the unknown node (i, j, k) with its neighbour (i+dx, j+dy, k+dz): the sum,
 * over the elements the two nodes share (z outermost, then y, then x, each in ascending
 * element order), of c_e * (Kx My Mz + Mx Ky Mz + Mx My Kz), with the 1-D stiffness
 * K = +-1/h and mass M = 2h/6 (same node) or h/6 (neighbours) of each axis.
 */
#include <stdint.h>
#include <stdlib.h>

typedef struct {
    int valid;
    int e;
    double K, M;
} slot_t;

/* per unknown node index i and offset d in {-1, 0, 1}: up to two shared elements */
static int axis_options(const double *h, int ne, int dirichlet, slot_t *opt, int *nslots)
{
    const int nn = dirichlet ? ne - 1 : ne + 1;
    for (int i = 0; i < nn; ++i) {
        const int full = dirichlet ? i + 1 : i;
        for (int d = -1; d <= 1; ++d) {
            int cand[2], nc;
            if (d == 0) { cand[0] = full - 1; cand[1] = full; nc = 2; }
            else if (d == -1) { cand[0] = full - 1; nc = 1; }
            else { cand[0] = full; nc = 1; }
            nslots[i * 3 + d + 1] = nc;
            for (int s = 0; s < nc; ++s) {
                const int e = cand[s], nb = full + d;
                int valid = e >= 0 && e < ne;
                if (dirichlet) valid = valid && nb >= 1 && nb <= ne - 1;
                else valid = valid && nb >= 0 && nb <= ne;
                const int ec = e < 0 ? 0 : (e > ne - 1 ? ne - 1 : e);
                const double he = h[ec];
                slot_t sl;
                sl.valid = valid;
                sl.e = ec;
                if (d == 0) { sl.K = 1.0 / he; sl.M = 2.0 * he / 6.0; }
                else { sl.K = -1.0 / he; sl.M = he / 6.0; }
                opt[(i * 3 + d + 1) * 2 + s] = sl;
            }
        }
    }
    return nn;
}

/* Fills row_ptr (n + 1), col and val (room for 27 n entries); returns nnz, or -1 if an
 * allocation failed.  coef: nez * ney * nex element coefficients (ez slowest) or NULL. */
int64_t q1_assemble(int nex, int ney, int nez, const double *hx, const double *hy, const double *hz,
                    const double *coef, int dirichlet, int64_t *row_ptr, int32_t *col, double *val)
{
    const int nnx = dirichlet ? nex - 1 : nex + 1, nny = dirichlet ? ney - 1 : ney + 1,
              nnz_ = dirichlet ? nez - 1 : nez + 1;
    slot_t *ox = malloc(sizeof(slot_t) * 6 * (size_t)(nnx > 0 ? nnx : 1));
    slot_t *oy = malloc(sizeof(slot_t) * 6 * (size_t)(nny > 0 ? nny : 1));
    slot_t *oz = malloc(sizeof(slot_t) * 6 * (size_t)(nnz_ > 0 ? nnz_ : 1));
    int *cx = malloc(sizeof(int) * 3 * (size_t)(nnx > 0 ? nnx : 1));
    int *cy = malloc(sizeof(int) * 3 * (size_t)(nny > 0 ? nny : 1));
    int *cz = malloc(sizeof(int) * 3 * (size_t)(nnz_ > 0 ? nnz_ : 1));
    if (!ox || !oy || !oz || !cx || !cy || !cz) {
        free(ox); free(oy); free(oz); free(cx); free(cy); free(cz);
        return -1;
    }
    axis_options(hx, nex, dirichlet, ox, cx);
    axis_options(hy, ney, dirichlet, oy, cy);
    axis_options(hz, nez, dirichlet, oz, cz);
    int64_t nnz = 0;
    int64_t row = 0;
    row_ptr[0] = 0;
    for (int k = 0; k < nnz_; ++k) {
        for (int j = 0; j < nny; ++j) {
            for (int i = 0; i < nnx; ++i, ++row) {
                for (int dz = -1; dz <= 1; ++dz) {
                    for (int dy = -1; dy <= 1; ++dy) {
                        for (int dx = -1; dx <= 1; ++dx) {
                            double acc = 0.0;
                            int any = 0;
                            const int nsz = cz[k * 3 + dz + 1], nsy = cy[j * 3 + dy + 1], nsx = cx[i * 3 + dx + 1];
                            for (int sz = 0; sz < nsz; ++sz) {
                                const slot_t Z = oz[(k * 3 + dz + 1) * 2 + sz];
                                for (int sy = 0; sy < nsy; ++sy) {
                                    const slot_t Y = oy[(j * 3 + dy + 1) * 2 + sy];
                                    for (int sx = 0; sx < nsx; ++sx) {
                                        const slot_t X = ox[(i * 3 + dx + 1) * 2 + sx];
                                        if (!(Z.valid && Y.valid && X.valid)) continue;
                                        const double c =
                                            coef ? coef[((size_t)Z.e * ney + Y.e) * nex + X.e] : 1.0;
                                        const double term = (X.K * Y.M) * Z.M + (X.M * Y.K) * Z.M + (X.M * Y.M) * Z.K;
                                        acc = acc + c * term;
                                        any = 1;
                                    }
                                }
                            }
                            if (any) {
                                col[nnz] = (int32_t)(row + dx + (int64_t)nnx * (dy + (int64_t)nny * dz));
                                val[nnz] = acc;
                                ++nnz;
                            }
                        }
                    }
                }
                row_ptr[row + 1] = nnz;
            }
        }
    }
    free(ox); free(oy); free(oz); free(cx); free(cy); free(cz);
    return nnz;
}
