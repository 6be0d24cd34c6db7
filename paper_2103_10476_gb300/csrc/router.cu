// router.cu -- requests across several GPUs (no counterpart in the paper, which solves one
// system at a time): each operator gets a home device the first time it is seen and keeps it,
// so that every repeat reaches the device whose server holds its hierarchy.
//
// The key is the operator's content hash (the server's cache key).  A new operator goes to
// the device with the least work assigned so far (ties: the lowest index), work being a
// count of stored entries: nnz(A) x (right-hand sides + kSetupWeight for a device that has
// not seen the operator), i.e. a setup costs about as much as kSetupWeight solves' worth of
// matrix passes.  The decisions depend only on the sequence of requests, never on timing, so
// processes that see the same request sequence make the same decisions without exchanging
// anything: one process per GPU can each take the requests routed to it from a shared
// stream.  Within one process, servers attached to the router receive their requests
// directly (amg_router_submit).  Host-side only: no collective, no peer access.
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "hierarchy.cuh"

namespace amgk {
namespace {

constexpr double kSetupWeight = 20.0;

struct RouterTicket {
    int device = -1;
    uint64_t server_ticket = 0;
};

}  // namespace
}  // namespace amgk

struct amg_router {
    int ndev = 0;
    std::mutex mu;
    std::unordered_map<uint64_t, int> home;
    std::vector<double> work;
    std::vector<int64_t> requests, operators, repeats;
    std::vector<amg_server_t> servers;
    std::unordered_map<uint64_t, amgk::RouterTicket> tickets;
    uint64_t next_ticket = 1;
};

using namespace amgk;

namespace {

// assigns A's request to a device under the router's lock
amg_status_t route_locked(amg_router *R, const amg_csr_t *A, int nrhs, int *device, uint64_t *key, int *repeat)
{
    std::string err;
    const uint64_t k = operator_key(A, &err);
    if (!err.empty()) {
        set_last_error("amg_router_route: " + err);
        return AMG_ERR_CUDA;
    }
    const double nnz = (double)(A->nnz > 0 ? A->nnz : 1);
    auto it = R->home.find(k);
    int d;
    int rep = 0;
    if (it != R->home.end()) {
        d = it->second;
        rep = 1;
        R->work[(size_t)d] += nnz * (double)nrhs;
        R->repeats[(size_t)d]++;
    } else {
        d = 0;
        for (int t = 1; t < R->ndev; ++t)
            if (R->work[(size_t)t] < R->work[(size_t)d]) d = t;
        R->home.emplace(k, d);
        R->work[(size_t)d] += nnz * ((double)nrhs + kSetupWeight);
        R->operators[(size_t)d]++;
    }
    R->requests[(size_t)d]++;
    *device = d;
    if (key) *key = k;
    if (repeat) *repeat = rep;
    return AMG_OK;
}

bool valid_csr(const amg_csr_t *A)
{
    return A && A->n >= 0 && A->nnz >= 0 && (A->n == 0 || A->row_ptr) && (A->nnz == 0 || (A->col && A->val));
}

}  // namespace

extern "C" {

amg_status_t amg_router_create(int ndev, amg_router_t *out)
{
    if (!out) return AMG_ERR_INVALID_ARG;
    *out = nullptr;
    if (ndev < 1 || ndev > 4096) return AMG_ERR_INVALID_ARG;
    amg_router *R = new (std::nothrow) amg_router();
    if (!R) return AMG_ERR_OOM;
    R->ndev = ndev;
    R->work.assign((size_t)ndev, 0.0);
    R->requests.assign((size_t)ndev, 0);
    R->operators.assign((size_t)ndev, 0);
    R->repeats.assign((size_t)ndev, 0);
    R->servers.assign((size_t)ndev, nullptr);
    *out = R;
    return AMG_OK;
}

amg_status_t amg_router_route(amg_router_t R, const amg_csr_t *A, int nrhs, int *device, uint64_t *key, int *repeat)
{
    if (!R || !valid_csr(A) || nrhs < 0 || !device) return AMG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(R->mu);
    return route_locked(R, A, nrhs, device, key, repeat);
}

amg_status_t amg_router_attach(amg_router_t R, int device, amg_server_t srv)
{
    if (!R || device < 0 || device >= R->ndev) return AMG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(R->mu);
    R->servers[(size_t)device] = srv;
    return AMG_OK;
}

amg_status_t amg_router_submit(amg_router_t R, const amg_csr_t *A, int nrhs, const double *b, double *x,
                               uint64_t *ticket, int *device)
{
    if (!R || !valid_csr(A) || nrhs < 0 || !ticket) return AMG_ERR_INVALID_ARG;
    int d = -1;
    amg_server_t srv = nullptr;
    {
        std::lock_guard<std::mutex> lk(R->mu);
        amg_status_t st = route_locked(R, A, nrhs, &d, nullptr, nullptr);
        if (st != AMG_OK) return st;
        srv = R->servers[(size_t)d];
    }
    if (!srv) {
        set_last_error("amg_router_submit: no server attached to the request's device");
        return AMG_ERR_INVALID_ARG;
    }
    uint64_t st_ticket = 0;
    amg_status_t st = amg_server_submit(srv, A, nrhs, b, x, &st_ticket);
    if (st != AMG_OK) return st;
    std::lock_guard<std::mutex> lk(R->mu);
    const uint64_t t = R->next_ticket++;
    R->tickets[t] = RouterTicket{d, st_ticket};
    *ticket = t;
    if (device) *device = d;
    return AMG_OK;
}

static amg_status_t router_finish(amg_router_t R, uint64_t ticket, amg_request_info_t *info, int *device, bool wait)
{
    if (!R || !info) return AMG_ERR_INVALID_ARG;
    RouterTicket rt;
    amg_server_t srv = nullptr;
    {
        std::lock_guard<std::mutex> lk(R->mu);
        auto it = R->tickets.find(ticket);
        if (it == R->tickets.end()) return AMG_ERR_INVALID_ARG;
        rt = it->second;
        srv = R->servers[(size_t)rt.device];
    }
    if (!srv) return AMG_ERR_INVALID_ARG;
    amg_status_t st = wait ? amg_server_wait(srv, rt.server_ticket, info) : amg_server_poll(srv, rt.server_ticket, info);
    if (st == AMG_PENDING) return st;
    if (device) *device = rt.device;
    std::lock_guard<std::mutex> lk(R->mu);
    R->tickets.erase(ticket);
    return st;
}

amg_status_t amg_router_poll(amg_router_t R, uint64_t ticket, amg_request_info_t *info, int *device)
{
    return router_finish(R, ticket, info, device, false);
}

amg_status_t amg_router_wait(amg_router_t R, uint64_t ticket, amg_request_info_t *info, int *device)
{
    return router_finish(R, ticket, info, device, true);
}

amg_status_t amg_router_stats(amg_router_t R, int device, int64_t *requests, int64_t *operators, int64_t *repeats,
                              double *work)
{
    if (!R || device < 0 || device >= R->ndev) return AMG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(R->mu);
    if (requests) *requests = R->requests[(size_t)device];
    if (operators) *operators = R->operators[(size_t)device];
    if (repeats) *repeats = R->repeats[(size_t)device];
    if (work) *work = R->work[(size_t)device];
    return AMG_OK;
}

amg_status_t amg_router_destroy(amg_router_t R)
{
    delete R;
    return AMG_OK;
}

}  // extern "C"
