// engine.cuh -- the segment-indexed multi-system solver behind the batch ABI (batch.cu) and
// the request server (server.cu).
//
// Every member system keeps its own hierarchy (the arrays amg_setup built); the engine
// refers to them through per-slot tables and never copies a matrix.  Work is cut into
// tiles (at most 256/LPR consecutive rows of one system's matrix); a persistent kernel per
// V-cycle step walks a device-side tile list, so one launch covers every system and a
// tile never spans two systems.  Vectors live in two arenas: level 0 (the PCG vectors and
// the finest V-cycle vectors share each system's offset) and all coarser levels.  The
// lists of tiles of systems still iterating are compacted on the device whenever a system
// stops, so a stopped system costs nothing; one PCG iteration of all members is one CUDA
// graph, replayed while members come and go (only its tile lists and counts change).
#pragma once

#include <string>
#include <vector>

#include "hierarchy.cuh"

namespace amgk {

constexpr int kEngLevels = 16;     // deepest hierarchy an engine accepts

struct SegTile {        // rows [row0, row0 + rows) of one slot's matrix
    int slot, row0, rows, pad;
};
struct SegOp {          // one slot's matrix on one level, with where its vectors live
    const int *rp;
    const int *ci;
    const void *v;      // values in the working type
    const void *invd;   // 1 / diag (A only), working type
    const double *coef; // Chebyshev coefficients of this slot and level (A only)
    int xoff, yoff;     // offsets of the column-indexed and row-indexed vectors
    int n, ncol;        // rows and columns (checked against each tile and the vectors)
    int nnz, pad;
};
// Guard of the engine's kernels: a work item that would reach outside its matrix or vector
// arena is skipped and recorded here (count, then the first item's kind, slot, position).
struct EngGuard {
    int count, kind, slot, where;
    int info[12];       // the first item's tile, matrix and vector figures
    int waits;          // blocks whose bounded wait for a bulk copy ran out
};
struct SegCoarse {      // rows [row0, row0 + kCoarseRows) of the dense solve of a slot whose
    const double *inv;  // coarsest level this is (inverse: n x n, row-major)
    int n, off, slot, row0;
};
constexpr int kCoarseRows = 32;    // rows of the coarse solve per work item
struct SegChunk {       // at most kEngChunk fine rows of one slot (PCG vector kernels)
    int slot, begin, end, first, count, id;
};
struct EngScal {        // per-slot PCG scalars (device)
    double rz, rz_new, cross, alpha, pq, rr, tt, bb;
};

// what a launch needs for the guard checks: the slot count, the lengths of the arenas its
// column-indexed and row-indexed vectors live in, and the guard record
struct SegCtx {
    int nslots, xcap, ycap;
    EngGuard *guard;
};

// a list of work items: host copy, the full device list, and the lists compacted by the
// active and flagged masks (counts on the device: [0] active, [1] flagged)
template <typename E>
struct EngList {
    std::vector<E> host;
    E *full = nullptr, *act = nullptr, *flg = nullptr;
    int *count = nullptr;
    int nfull = 0;
    size_t capacity = 0;
    int lpr = 2;        // lanes per row (tile lists)
    int cap = 0;        // shared-memory tile entries (tile lists)
};

class Engine {
public:
    struct Config {
        int mixed = 0;          // FP32 V-cycle inside FP64 PCG
        int degree = 2;         // Chebyshev degree (all members)
        int slots = 0;          // members at most
        int64_t cap0 = 0;       // fine rows of all members at most
        int64_t capc = 0;       // rows of all coarser levels of all members at most
        bool tune = true;       // time the lanes-per-row candidates of each list at the first commit
    };
    struct Slot {
        amg_hierarchy *h = nullptr;
        bool used = false, pending = false;
        int nlev = 0, n0 = 0, csize = 0;
        int64_t o0 = -1, oc = -1;
        int64_t off[kEngLevels] = {};   // arena offsets of each level's rows
        const double *b = nullptr;      // right-hand side of the pending solve (host or device)
        int max_iter = 0;
        double tol = 0.0;
        int active = 0, iters = 0;
        double nb = 0.0, relres = 0.0;
        amg_status_t result = AMG_OK;
    };

    ~Engine();
    amg_status_t init(const Config &c, cudaStream_t s);
    // membership and solves take effect at the next commit
    int add(amg_hierarchy *h);                                  // slot, or -1 (no room)
    void remove(int slot);
    void load(int slot, const double *b, double tol, int max_iter);
    amg_status_t commit();
    // one PCG iteration of every active member; *finished receives the slots that stopped
    amg_status_t step(std::vector<int> *finished);
    amg_status_t download(int slot, double *x);                 // x of a member (host or device)
    int live() const { return live_; }
    const Slot &slot(int k) const { return slots_[k]; }
    int slot_count() const { return (int)slots_.size(); }
    int levels() const { return nlev_; }
    long long kernels_per_iteration() const { return gkernels_[0]; }
    size_t bytes() const { return bytes_; }
    std::string describe() const;   // lanes per row chosen for each list
    // a guard violation recorded since the last call (message), or empty; *slot = its slot
    std::string take_guard(int *slot = nullptr);

private:
    template <typename T>
    cudaError_t alloc(T **p, size_t count);
    void build_lists();
    cudaError_t upload_lists();
    cudaError_t compute_caps();
    cudaError_t compact(bool active);
    cudaError_t push_flags(const std::vector<int> &v, int *dst);
    cudaError_t autotune();
    void heuristic_lanes();
    cudaError_t tail(int parity, cudaStream_t s);
    cudaError_t head(cudaStream_t s);
    template <typename T>
    cudaError_t vcycle(int L, const T *f, T *final_out, T **out, cudaStream_t s);
    cudaError_t true_residual(cudaStream_t s);   // t = b - A x, |t|^2 for the flagged slots
    cudaGraphExec_t graph(int parity);
    void drop_graphs();
    // guard context of a launch whose vectors are in arena xl / yl (0 fine, 1 coarse levels)
    SegCtx ctx(int xl, int yl) const;
    int64_t arena_take(std::vector<std::pair<int64_t, int64_t>> &free_list, int64_t n);
    void arena_give(std::vector<std::pair<int64_t, int64_t>> &free_list, int64_t off, int64_t n);

    Config cfg_;
    cudaStream_t s_ = nullptr, cap_ = nullptr;
    int cstride_ = 5;
    std::vector<void *> allocs_;
    size_t bytes_ = 0;
    std::vector<Slot> slots_;
    std::vector<std::pair<int64_t, int64_t>> free0_, freec_;   // (offset, rows) holes of the arenas
    bool members_changed_ = true, tuned_ = false;
    int nlev_ = 0;                  // levels the V-cycle graph covers
    int live_ = 0;
    int it_ = 0;                    // iterations launched (z-buffer parity in mixed precision)
    // device tables: [level][slot]
    SegOp *opA_ = nullptr, *opP_ = nullptr, *opR_ = nullptr, *op0_ = nullptr;
    SegCoarse *opC_ = nullptr;
    double *coef_ = nullptr;        // [slot][level][cstride]
    std::vector<SegOp> hA_, hP_, hR_, h0_;
    std::vector<SegCoarse> hC_;
    std::vector<double> hcoef_;
    // lists
    EngList<SegTile> lA_[kEngLevels], lP_[kEngLevels], lR_[kEngLevels], l0_;
    EngList<SegCoarse> lC_[kEngLevels];
    EngList<SegChunk> lch_;
    // masks and scalars
    int *active_ = nullptr, *flag_ = nullptr;
    int *hflags_ = nullptr;         // pinned: [0, slots) active, [slots, 2 slots) flag
    cudaEvent_t flag_ev_[2] = {nullptr, nullptr};   // the last upload from each half of hflags_
    EngScal *sc_ = nullptr;
    double *partial_ = nullptr, *partial2_ = nullptr, *rr_dev_ = nullptr, *rr_host_ = nullptr;
    unsigned *ticket_ = nullptr, *ticket2_ = nullptr;
    int *caps_dev_ = nullptr;
    EngGuard *guard_ = nullptr;     // device
    // arenas: level 0 (FP64 PCG vectors; working-type V-cycle vectors) and coarser levels
    double *b_ = nullptr, *x_ = nullptr, *r_ = nullptr, *p_ = nullptr, *q_ = nullptr, *t_ = nullptr;
    double *zb_[2] = {nullptr, nullptr};
    void *f0_ = nullptr, *x0_ = nullptr, *x20_ = nullptr, *r0_ = nullptr, *d0_ = nullptr;
    void *fc_ = nullptr, *xc_ = nullptr, *x2c_ = nullptr, *rc_ = nullptr, *dc_ = nullptr;
    // graphs
    cudaGraphExec_t gexec_[2] = {nullptr, nullptr};
    long long gkernels_[2] = {0, 0};
    bool graph_failed_ = false;
    unsigned coarse_mask_ = 0;      // levels with coarsest-level solves in the captured graphs
    int grid_tiles_ = 0, grid_chunks_ = 0;
};

}  // namespace amgk
