// server.cu -- the request loop (no counterpart in the paper): admission by HBM budget,
// hierarchy reuse by operator content, concurrent setups, and continuous batching of every
// right-hand side in flight on one segment-indexed engine (engine.cuh).
//
// Threads.  Setup workers take submitted requests in order, hash the operator and either
// attach the request to a resident (or in-progress) hierarchy or build one with amg_setup on
// their own stream, after evicting unused hierarchies (least recently used first) until the
// new one fits the budget.  The engine thread admits the right-hand sides of ready requests
// into free engine slots, commits, runs one PCG iteration of everything in flight, copies out
// the solutions that finished and frees their slots; so requests that arrive while others are
// on the GPU join at the next iteration and their work shares every launch.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.cuh"

namespace amgk {

// 64-bit content hash of a byte range: four independent multiply-xorshift lanes over 8-byte
// words (the tail zero-padded), folded at the end
static void hash_bytes(const void *p, size_t bytes, uint64_t h[4])
{
    const unsigned char *c = (const unsigned char *)p;
    const uint64_t K = 0x9E3779B97F4A7C15ull;
    size_t i = 0;
    for (; i + 32 <= bytes; i += 32) {
        uint64_t w[4];
        std::memcpy(w, c + i, 32);
        for (int l = 0; l < 4; ++l) {
            h[l] = (h[l] ^ w[l]) * K;
            h[l] ^= h[l] >> 29;
        }
    }
    for (int l = 0; i < bytes; ++l, i += 8) {
        uint64_t w = 0;
        std::memcpy(&w, c + i, std::min<size_t>(8, bytes - i));
        h[l & 3] = (h[l & 3] ^ w) * K;
        h[l & 3] ^= h[l & 3] >> 29;
    }
}

uint64_t operator_key(const amg_csr_t *A, std::string *err)
{
    uint64_t h[4] = {0x243F6A8885A308D3ull, 0x13198A2E03707344ull, 0xA4093822299F31D0ull, 0x082EFA98EC4E6C89ull};
    const int64_t head[2] = {A->n, A->nnz};
    hash_bytes(head, sizeof head, h);
    const size_t brp = sizeof(int64_t) * (size_t)(A->n + 1), bci = sizeof(int32_t) * (size_t)A->nnz,
                 bv = sizeof(double) * (size_t)A->nnz;
    if (A->n == 0) return h[0] ^ h[1];
    if (!A->on_device) {
        hash_bytes(A->row_ptr, brp, h);
        hash_bytes(A->col, bci, h);
        hash_bytes(A->val, bv, h);
    } else {
        std::vector<unsigned char> tmp(std::max(brp, std::max(bci, bv)));
        const void *src[3] = {A->row_ptr, A->col, A->val};
        const size_t len[3] = {brp, bci, bv};
        for (int k = 0; k < 3; ++k) {
            cudaError_t e = cudaMemcpy(tmp.data(), src[k], len[k], cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                *err = cudaGetErrorString(e);
                return 0;
            }
            hash_bytes(tmp.data(), len[k], h);
        }
    }
    uint64_t k = h[0] ^ (h[1] * 0xC2B2AE3D27D4EB4Full) ^ (h[2] * 0x165667B19E3779F9ull) ^ (h[3] * 0x27D4EB2F165667C5ull);
    k ^= k >> 31;
    return k;
}

namespace {

double now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request;

struct Entry {
    uint64_t key = 0;
    amg_hierarchy *h = nullptr;
    int state = 0;              // 0 being built, 1 ready
    size_t bytes = 0;           // the estimate while being built
    int refs = 0;               // requests holding it
    double last_use = 0.0;
    double setup_ms = 0.0;
    std::vector<Request *> waiters;
};

struct Request {
    uint64_t ticket = 0;
    amg_csr_t A{};
    int nrhs = 0;
    const double *b = nullptr;
    double *x = nullptr;
    Entry *e = nullptr;
    double t_submit = 0.0, t_engine = -1.0, t_done = 0.0, setup_ms = 0.0;
    int cache_hit = 0;
    int next_rhs = 0;           // right-hand sides not yet given to the engine
    int remaining = 0;          // right-hand sides not finished
    int iters_max = 0;
    double relres_max = 0.0;
    amg_status_t status = AMG_OK;
    bool done = false;
};

// device bytes a hierarchy of A is expected to hold: bytes per stored entry of A, 64 until a
// hierarchy has been built, then 1.1 x the largest ratio seen (replaced by the real figure
// once this one is built)
size_t estimate_bytes(const amg_csr_t *A, double per_nnz)
{
    return (size_t)(per_nnz * (double)A->nnz) + 160 * (size_t)A->n + (1u << 20);
}

}  // namespace
}  // namespace amgk

struct amg_server {
    amg_server_config_t cfg{};
    int dev = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_engine, cv_done;
    std::deque<amgk::Request *> incoming, ready;
    std::unordered_map<uint64_t, amgk::Entry *> cache;
    std::unordered_map<uint64_t, amgk::Request *> requests;
    uint64_t next_ticket = 1;
    size_t cache_bytes = 0;
    size_t eng_bytes = 0;           // the engine's device bytes (updated by the engine thread)
    double per_nnz = 64.0;          // admission estimate of hierarchy bytes per stored entry
    std::string first_error;        // the first failure's message
    double per_nnz_seen = 0.0;
    bool stop = false, workers_done = false;
    amg_server_stats_t stats{};
    cudaStream_t es = nullptr;
    amgk::Engine eng;
    std::vector<std::thread> workers;
    std::thread engine;
};

namespace amgk {
namespace {

// under the lock: the first failure's message is kept for amg_server_stats
void note_error(amg_server *S, const std::string &msg)
{
    if (S->first_error.empty()) S->first_error = msg.empty() ? std::string("unknown") : msg;
}

// under the lock: a finished request is visible to poll/wait; its hierarchy becomes evictable
void finish_request(amg_server *S, Request *r, amg_status_t status)
{
    if (status != AMG_OK && r->status == AMG_OK) r->status = status;
    r->done = true;
    r->t_done = now_ms();
    if (r->e) {
        r->e->refs--;
        r->e->last_use = r->t_done;
    }
    S->stats.completed++;
    S->stats.solves += r->nrhs;
    S->cv_done.notify_all();
    S->cv_work.notify_all();
}

// under the lock: the least recently used hierarchy no request holds, out of the cache
Entry *take_victim(amg_server *S)
{
    Entry *best = nullptr;
    for (auto &kv : S->cache) {
        Entry *e = kv.second;
        if (e->state == 1 && e->refs == 0 && (!best || e->last_use < best->last_use)) best = e;
    }
    if (best) {
        S->cache.erase(best->key);
        S->cache_bytes -= best->bytes;
        S->stats.evictions++;
    }
    return best;
}

void worker_loop(amg_server *S)
{
    cudaSetDevice(S->dev);
    cudaStream_t ws = nullptr;
    cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_work.wait(lk, [&] { return S->stop || !S->incoming.empty(); });
        if (S->incoming.empty()) break;     // stop, and nothing left to take
        Request *r = S->incoming.front();
        S->incoming.pop_front();
        lk.unlock();
        std::string err;
        const uint64_t key = operator_key(&r->A, &err);
        lk.lock();
        if (!err.empty()) {
            set_last_error("operator hash: " + err);
            note_error(S, "operator hash: " + err);
            finish_request(S, r, AMG_ERR_CUDA);
            S->stats.failed++;
            continue;
        }
        auto it = S->cache.find(key);
        if (it != S->cache.end()) {
            Entry *e = it->second;
            e->refs++;
            r->e = e;
            r->cache_hit = 1;
            S->stats.cache_hits++;
            if (e->state == 1) {
                S->ready.push_back(r);
                S->cv_engine.notify_one();
            } else {
                e->waiters.push_back(r);
            }
            continue;
        }
        // a miss: make room within the budget, then build
        const size_t est = estimate_bytes(&r->A, S->per_nnz);
        bool fits = false;
        for (;;) {
            const size_t used = S->cache_bytes + S->eng_bytes;
            if (used + est <= S->cfg.hbm_budget_bytes) { fits = true; break; }
            Entry *v = take_victim(S);
            if (v) {
                lk.unlock();
                amg_free(v->h);
                delete v;
                lk.lock();
                continue;
            }
            // nothing evictable: wait for requests to finish, unless nothing could ever free
            bool held = false;
            for (auto &kv : S->cache) held |= kv.second->refs > 0 || kv.second->state == 0;
            if (!held) break;
            S->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        }
        S->stats.cache_misses++;
        if (!fits) {
            note_error(S, "a hierarchy larger than the HBM budget");
            finish_request(S, r, AMG_ERR_BUDGET);
            S->stats.failed++;
            continue;
        }
        Entry *e = new Entry();
        e->key = key;
        e->bytes = est;
        e->refs = 1;
        r->e = e;
        S->cache[key] = e;
        S->cache_bytes += est;
        lk.unlock();
        amg_params_t p = S->cfg.params;
        p.cuda_stream = ws;
        p.coarse_solve = AMG_COARSE_INVERSE;           // the engine applies the dense inverse
        amg_handle_t h = nullptr;
        const double t0 = now_ms();
        const amg_status_t st = amg_setup(&r->A, nullptr, &p, &h);
        const double t1 = now_ms();
        const std::string msg = st == AMG_OK ? std::string() : std::string(amg_last_error());
        // the new hierarchy's structure is checked before anything solves with it
        amg_status_t st2 = st;
        std::string chk;
        if (st == AMG_OK) {
            const int f = hierarchy_check(h, ws, &chk);
            if (f != 0) {
                st2 = AMG_ERR_INTERNAL;
                chk = "setup produced an inconsistent hierarchy: " + (f < 0 ? std::string("check failed") : chk);
                amg_free(h);
                h = nullptr;
            }
        }
        lk.lock();
        if (st2 != AMG_OK && st == AMG_OK) {
            S->cache.erase(key);
            S->cache_bytes -= e->bytes;
            std::vector<Request *> all(e->waiters);
            all.push_back(r);
            for (Request *w : all) {
                w->e = nullptr;
                finish_request(S, w, st2);
                S->stats.failed++;
            }
            note_error(S, chk);
            delete e;
            continue;
        }
        if (st == AMG_OK) {
            // the engine's stream orders the eventual release after the engine's last use
            h->s = S->es;
            h->p.cuda_stream = S->es;
            e->h = h;
            e->state = 1;
            S->cache_bytes += h->bytes;
            S->cache_bytes -= e->bytes;
            e->bytes = h->bytes;
            e->setup_ms = t1 - t0;
            if (r->A.nnz > 0) {
                const double ratio = (double)h->bytes / (double)r->A.nnz;
                S->per_nnz_seen = std::max(S->per_nnz_seen, ratio);
                S->per_nnz = 1.1 * S->per_nnz_seen;
            }
            r->setup_ms = e->setup_ms;
            S->ready.push_back(r);
            for (Request *w : e->waiters) {
                w->setup_ms = e->setup_ms;
                S->ready.push_back(w);
            }
            e->waiters.clear();
            S->cv_engine.notify_one();
        } else {
            S->cache.erase(key);
            S->cache_bytes -= e->bytes;
            std::vector<Request *> all(e->waiters);
            all.push_back(r);
            for (Request *w : all) {
                w->e = nullptr;
                finish_request(S, w, st);
                S->stats.failed++;
            }
            note_error(S, std::string("setup: ") + amg_status_string(st) + ": " + msg);
            set_last_error(msg);
            delete e;
        }
    }
    lk.unlock();
    if (ws) cudaStreamDestroy(ws);
}

void engine_loop(amg_server *S)
{
    cudaSetDevice(S->dev);
    Engine &E = S->eng;
    std::deque<Request *> admit;        // requests with right-hand sides not yet in the engine
    std::unordered_map<int, std::pair<Request *, int>> owner;   // slot -> (request, rhs)
    bool removed = false;
    const int64_t max_rows = S->cfg.max_rows;
    const int max_sys = S->cfg.max_systems;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (E.live() == 0 && admit.empty() && S->ready.empty()) {
                if (S->workers_done) break;
                S->cv_engine.wait_for(lk, std::chrono::milliseconds(2));
            }
            while (!S->ready.empty()) {
                Request *r = S->ready.front();
                S->ready.pop_front();
                // a request that can never fit the engine fails at once
                if (r->A.n > max_rows || r->nrhs > max_sys) {
                    set_last_error("request larger than the engine's capacity");
                    note_error(S, "request larger than the engine's capacity");
                    finish_request(S, r, AMG_ERR_BUDGET);
                    S->stats.failed++;
                    continue;
                }
                admit.push_back(r);
            }
        }
        // right-hand sides into free slots, in arrival order
        std::vector<int> loaded;
        while (!admit.empty()) {
            Request *r = admit.front();
            while (r->next_rhs < r->nrhs) {
                const int slot = E.add(r->e->h);
                if (slot < 0) break;
                E.load(slot, r->b + (size_t)r->next_rhs * (size_t)r->A.n, S->cfg.tol, S->cfg.params.max_iter);
                owner[slot] = {r, r->next_rhs};
                loaded.push_back(slot);
                if (r->t_engine < 0) r->t_engine = now_ms();
                r->next_rhs++;
            }
            if (r->next_rhs < r->nrhs) break;
            admit.pop_front();
        }
        std::vector<int> fin;
        amg_status_t st = AMG_OK;
        if (!loaded.empty() || (removed && E.live() == 0)) {
            st = E.commit();
            removed = false;
            std::lock_guard<std::mutex> g(S->mu);
            S->stats.commits++;
            S->eng_bytes = E.bytes();
            // systems that are done at the start (b = 0, or no iterations allowed)
            for (int slot : loaded)
                if (!E.slot(slot).active) fin.push_back(slot);
        }
        if (st == AMG_OK && E.live() > 0) {
            const double t0 = now_ms();
            std::vector<int> f2;
            st = E.step(&f2);
            fin.insert(fin.end(), f2.begin(), f2.end());
            std::lock_guard<std::mutex> g(S->mu);
            S->stats.iterations++;
            S->stats.engine_busy_ms += now_ms() - t0;
        }
        if (st != AMG_OK) {
            // the engine failed: every request in it fails; the engine starts over empty
            const std::string msg = std::string("engine: ") + amg_status_string(st) + ": " + amg_last_error();
            std::lock_guard<std::mutex> g(S->mu);
            note_error(S, msg);
            for (auto &kv : owner) {
                Request *r = kv.second.first;
                E.remove(kv.first);
                if (!r->done && --r->remaining == 0) finish_request(S, r, st);
                else r->status = st;
            }
            owner.clear();
            removed = true;
            continue;
        }
        for (int slot : fin) {
            auto it = owner.find(slot);
            if (it == owner.end()) continue;
            Request *r = it->second.first;
            const int k = it->second.second;
            const Engine::Slot &sl = E.slot(slot);
            const amg_status_t ds = E.download(slot, r->x + (size_t)k * (size_t)r->A.n);
            std::lock_guard<std::mutex> g(S->mu);
            r->iters_max = std::max(r->iters_max, sl.iters);
            r->relres_max = std::max(r->relres_max, sl.relres);
            if (sl.result != AMG_OK && r->status == AMG_OK) r->status = sl.result;
            if (ds != AMG_OK) r->status = ds;
            E.remove(slot);
            owner.erase(it);
            removed = true;
            if (--r->remaining == 0) finish_request(S, r, AMG_OK);
        }
    }
}

}  // namespace
}  // namespace amgk

using namespace amgk;

extern "C" {

void amg_server_config_default(amg_server_config_t *c)
{
    if (!c) return;
    c->hbm_budget_bytes = (size_t)120 << 30;
    c->setup_threads = 8;
    c->max_systems = 4096;
    c->max_rows = (int64_t)1 << 28;
    c->tol = 1e-8;
    c->tune = 1;
    amg_params_default(&c->params);
}

amg_status_t amg_server_create(const amg_server_config_t *cfg, amg_server_t *out)
{
    if (!cfg || !out) return AMG_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->setup_threads < 1 || cfg->max_systems < 1 || cfg->max_rows < 1 || cfg->max_rows > 0x7ffffff0LL ||
        !(cfg->tol >= 0.0) || cfg->params.cheb_degree < 1)
        return AMG_ERR_INVALID_ARG;
    amg_server *S = new amg_server();
    S->cfg = *cfg;
    cudaError_t e = cudaGetDevice(&S->dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->es, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete S;
        return fail_cuda(e, "amg_server_create");
    }
    Engine::Config ec;
    ec.mixed = cfg->params.precision == AMG_MIXED;
    ec.degree = cfg->params.cheb_degree;
    ec.slots = cfg->max_systems;
    ec.cap0 = cfg->max_rows;
    ec.capc = cfg->max_rows;
    ec.tune = cfg->tune != 0;
    amg_status_t st = S->eng.init(ec, S->es);
    if (st == AMG_OK && S->eng.bytes() > cfg->hbm_budget_bytes) {
        set_last_error("the engine's vectors alone exceed the budget");
        st = AMG_ERR_BUDGET;
    }
    if (st != AMG_OK) {
        cudaStream_t es = S->es;
        delete S;
        cudaStreamDestroy(es);
        return st;
    }
    S->eng_bytes = S->eng.bytes();
    for (int t = 0; t < cfg->setup_threads; ++t) S->workers.emplace_back(worker_loop, S);
    S->engine = std::thread(engine_loop, S);
    *out = S;
    return AMG_OK;
}

amg_status_t amg_server_submit(amg_server_t S, const amg_csr_t *A, int nrhs, const double *b, double *x,
                               uint64_t *ticket)
{
    if (!S || !A || !ticket || nrhs < 0 || A->n < 0 || A->nnz < 0) return AMG_ERR_INVALID_ARG;
    if (nrhs > 0 && A->n > 0 && (!b || !x)) return AMG_ERR_INVALID_ARG;
    if (A->n > 0 && (!A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))) return AMG_ERR_INVALID_ARG;
    Request *r = new Request();
    r->A = *A;
    r->nrhs = nrhs;
    r->b = b;
    r->x = x;
    r->remaining = nrhs;
    r->t_submit = now_ms();
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop) {
        delete r;
        return AMG_ERR_INVALID_ARG;
    }
    r->ticket = S->next_ticket++;
    S->requests[r->ticket] = r;
    S->stats.submitted++;
    *ticket = r->ticket;
    if (nrhs == 0) {
        finish_request(S, r, AMG_OK);
        return AMG_OK;
    }
    S->incoming.push_back(r);
    S->cv_work.notify_one();
    return AMG_OK;
}

static void fill_info(const Request *r, amg_request_info_t *info)
{
    if (!info) return;
    info->status = r->status;
    info->nrhs = r->nrhs;
    info->iters_max = r->iters_max;
    info->cache_hit = r->cache_hit;
    info->relres_max = r->relres_max;
    info->queue_ms = r->t_engine >= 0 ? r->t_engine - r->t_submit : r->t_done - r->t_submit;
    info->setup_ms = r->cache_hit ? 0.0 : r->setup_ms;
    info->latency_ms = r->t_done - r->t_submit;
}

amg_status_t amg_server_poll(amg_server_t S, uint64_t ticket, amg_request_info_t *info)
{
    if (!S) return AMG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->requests.find(ticket);
    if (it == S->requests.end()) return AMG_ERR_INVALID_ARG;
    Request *r = it->second;
    if (!r->done) return AMG_PENDING;
    fill_info(r, info);
    S->requests.erase(it);
    delete r;
    return AMG_OK;
}

amg_status_t amg_server_wait(amg_server_t S, uint64_t ticket, amg_request_info_t *info)
{
    if (!S) return AMG_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->requests.find(ticket);
    if (it == S->requests.end()) return AMG_ERR_INVALID_ARG;
    Request *r = it->second;
    S->cv_done.wait(lk, [&] { return r->done; });
    fill_info(r, info);
    S->requests.erase(ticket);
    delete r;
    return AMG_OK;
}

amg_status_t amg_server_stats(amg_server_t S, amg_server_stats_t *out)
{
    if (!S || !out) return AMG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    *out = S->stats;
    out->bytes_hierarchies = S->cache_bytes;
    out->bytes_engine = S->eng_bytes;
    std::memset(out->first_error, 0, sizeof out->first_error);
    std::strncpy(out->first_error, S->first_error.c_str(), sizeof out->first_error - 1);
    int n = 0;
    for (auto &kv : S->cache) n += kv.second->state == 1;
    out->resident_hierarchies = n;
    return AMG_OK;
}

amg_status_t amg_server_destroy(amg_server_t S)
{
    if (!S) return AMG_OK;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (std::thread &t : S->workers) t.join();
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->workers_done = true;
    }
    S->cv_engine.notify_all();
    S->engine.join();
    for (auto &kv : S->cache) {
        amg_free(kv.second->h);
        delete kv.second;
    }
    for (auto &kv : S->requests) delete kv.second;
    cudaStream_t es = S->es;
    delete S;   // the engine releases its memory on es
    cudaStreamDestroy(es);
    return AMG_OK;
}

}  // extern "C"
