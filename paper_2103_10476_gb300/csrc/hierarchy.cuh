// hierarchy.cuh -- the hierarchy handle (one system) shared by the C-ABI implementation
// files (api.cu: setup and solve; batch.cu: many systems solved together).
#pragma once

#include <string>
#include <vector>

#include "amg_internal.cuh"

namespace amgk {

struct MultiWork;           // work vectors of amg_solve_multi (multi.cu)
struct GmresWork;           // Krylov basis and work vectors of flexible GMRES (gmres.cu)

struct Level {
    DevCsr A;                 // level operator
    double *diag = nullptr;   // diag(A)
    uint8_t *strong = nullptr, *removed = nullptr, *lumpflag = nullptr, *cflag = nullptr;
    DevCsr Abar;
    int *agg = nullptr;
    uint8_t *root = nullptr;
    int nagg = 0;
    double *B = nullptr, *nrm = nullptr, *Dsm = nullptr;
    double lambda_bar = 0.0, omega = 0.0, lambda_cheb = 0.0;
    DevCsr P, R;
    double *invdiag = nullptr;
    double *coords = nullptr; // dim coordinates per row (distance-Laplacian strength)
    float *invdiag_f = nullptr, *Af = nullptr, *Pf = nullptr, *Rf = nullptr;
    void *vf = nullptr, *vx = nullptr, *vx2 = nullptr, *vr = nullptr, *vd = nullptr;   // solve vectors
    SpmvPlan plan_a, plan_p, plan_r;
    int bs = 1, k = 1;        // unknowns per node; near-null-space vectors (B is n x k)
    double *Bc = nullptr;     // systems: the coarse near-null space formed with P
};

}  // namespace amgk

struct amg_hierarchy {
    using Level = amgk::Level;
    using SpmvPlan = amgk::SpmvPlan;
    using ProfList = amgk::ProfList;
    using PcgScalars = amgk::PcgScalars;
    using SolveCtx = amgk::SolveCtx;
    amg_params_t p;
    cudaStream_t s = nullptr;
    int nlev = 0;
    int dim = 0;                // coordinates per row (0: none given)
    bool block = false;         // a system of PDEs (block_size > 1 or nullspace_dim > 1)
    Level lev[32];
    std::vector<void *> allocs;
    double *coarse_inv = nullptr;
    // the coarsest level's Chebyshev solve (coarse_degree > 0; coarse_inv stays null until the
    // batch engine or the server needs it): degree, interval centre and half-width, and the
    // relative residual of the setup's check solve
    int coarse_degree = 0;
    double coarse_theta = 0.0, coarse_delta = 0.0, coarse_check = -1.0;
    // solve workspace (FP64, finest level)
    double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *pv = nullptr, *q = nullptr, *t = nullptr;
    double *z_prev = nullptr;   // previous preconditioned residual (flexible update, mixed precision)
    double *zb[2] = {nullptr, nullptr};   // the two z buffers (their roles alternate in mixed mode)
    // one PCG iteration (V-cycle, p update, q = A p, x and r update, copy of the r.r partial
    // sums to the host) as a CUDA graph; two graphs in mixed mode (z buffers alternate)
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    ProfList gprof[2];
    int gprof_on[2] = {-1, -1};
    long long gkernels[2] = {0, 0};   // kernels in each graph (added to the launch count per replay)
    bool graph_failed = false;
    double *partial = nullptr, *partial2 = nullptr, *partial3 = nullptr;
    double *rr_host = nullptr;   // pinned copy of the r . r partial sums
    PcgScalars *sc = nullptr;
    unsigned *counters = nullptr;   // ticket counters of the fixed-order reductions (zero between uses)
    SpmvPlan plan0;   // finest-level FP64 operator (PCG)
    SolveCtx ctx;
    double setup_ms = 0.0;
    double phase_ms[32][AMG_PH_COUNT] = {};   // setup phases per level (params.trace)
    double phase_t = 0.0;                     // end of the last traced phase
    int64_t fine_nnz = 0;
    size_t bytes = 0;   // device memory held by the handle
    amgk::MultiWork *multi = nullptr;   // several right-hand sides at once (allocated on first use)
    amgk::GmresWork *gmres = nullptr;   // flexible GMRES basis (allocated on the first GMRES solve)
};


namespace amgk {
// status plumbing shared by the ABI files
amg_status_t fail_cuda(cudaError_t e, const char *where);
void set_last_error(const std::string &msg);
// structural check of the operators a solve reads (A of every level, P and R of every level
// but the coarsest): row pointers start at 0, do not decrease and end at nnz, columns lie in
// range.  Returns the number of faults found (0: intact; -1: the check itself failed) and
// names the first in *detail.  Synchronises s.
int hierarchy_check(const amg_hierarchy *h, cudaStream_t s, std::string *detail);
// with params.trace: synchronise the handle's stream and book the time since the last mark to
// (level, phase)
void trace_mark(amg_hierarchy *h, int level, int phase);
// forms the dense inverse of the coarsest operator of a handle whose V-cycle uses the
// Chebyshev solve (the batch engine and the server apply inverses); synchronises the handle's
// stream.  Does nothing when the inverse exists.
amg_status_t ensure_coarse_inverse(amg_hierarchy *h);
// releases the host side of amg_solve_multi's work vectors (their device memory is in allocs)
void multi_release(amg_hierarchy *h);
// flexible GMRES(params.restart) preconditioned by one V-cycle per step (amg_solve of a handle
// set up with AMG_KRYLOV_GMRES); same arguments, results and info fields as amg_solve
amg_status_t fgmres_solve(amg_hierarchy *h, const double *b, double *x, double tol, amg_info_t *info);
// releases the host side of the GMRES work vectors (their device memory is in allocs)
void gmres_release(amg_hierarchy *h);
}  // namespace amgk
