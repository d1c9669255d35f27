// Serving loop: runs of different grids, bunches and precisions arrive as requests, are admitted
// by their device-memory footprint into one pool, and are advanced together - each admitted
// request is a run on its own CUDA stream, stepped in chunks, so the kernels of different
// requests overlap on the GPU.  A request that finishes hands its memory back to the pool, and
// the next queued requests are admitted as soon as they fit (continuous batching).
//
// Threads: submit/poll/release run on the caller's threads and only touch the request table
// under a mutex; one scheduler thread owns every CUDA call of the served runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/mithra.h"
#include "kernels.h"
#include "run.h"

namespace {

using mithra::set_last_error;

// First-fit sub-allocator over one device block (256-byte granules, neighbours merged on free).
struct Pool {
    char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;            // offset -> bytes
    std::unordered_map<size_t, size_t> used_;  // offset -> bytes
    size_t in_use = 0, peak = 0;
    std::mutex mu;

    void init(void* b, size_t n)
    {
        base = (char*)b;
        size = n;
        free_.clear();
        used_.clear();
        free_[0] = n;
        in_use = peak = 0;
    }
    void* alloc(size_t bytes)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        std::lock_guard<std::mutex> lk(mu);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[off + bytes] = rest;
            used_[off] = bytes;
            in_use += bytes;
            peak = std::max(peak, in_use);
            return base + off;
        }
        return nullptr;
    }
    void release(void* p)
    {
        std::lock_guard<std::mutex> lk(mu);
        const size_t off = (size_t)((char*)p - base);
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t o = off, n = u->second;
        used_.erase(u);
        in_use -= n;
        auto nx = free_.lower_bound(o);
        if (nx != free_.end() && nx->first == o + n) {
            n += nx->second;
            free_.erase(nx);
        }
        auto pv = free_.lower_bound(o);
        if (pv != free_.begin()) {
            --pv;
            if (pv->first + pv->second == o) {
                o = pv->first;
                n += pv->second;
                free_.erase(pv);
            }
        }
        free_[o] = n;
    }
};

void* pool_alloc(void* ctx, size_t bytes) { return ((Pool*)ctx)->alloc(bytes); }
void pool_free(void* ctx, void* p) { ((Pool*)ctx)->release(p); }

enum State { QUEUED, RUNNING, DONE };

struct Request {
    uint64_t ticket = 0;
    mithra_grid g{};
    mithra_undulator u{};
    mithra_bunch b{};
    std::vector<double> lab;
    int64_t nsteps = 0;
    int64_t reserve = 0;        // footprint reserved at admission
    bool admitted = false;      // holds its reservation
    State state = QUEUED;
    mithra_t run = nullptr;
    cudaStream_t stream = nullptr;
    int64_t enqueued = 0;
    std::deque<cudaEvent_t> inflight;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int status = MITHRA_OK;
    std::string error;
    std::vector<double> p, t;
    double fe = 0, bunch = 0;
    int64_t hbm = 0;
};

struct Server {
    int device = 0;
    Pool pool;
    void* block = nullptr;
    mithra_free_fn block_free = nullptr;
    void* block_ctx = nullptr;
    int max_active = 8, queue_cap = 256, chunk = 16;
    bool grouped = false;                 // one graph launch advances every ready request by its period
    cudaStream_t gstream = nullptr;       // the group launches
    cudaGraphExec_t gexec = nullptr;      // the group of the last launch (rebuilt when it changes)
    std::vector<uintptr_t> gkey;          // its members: ticket and period graph of each
    std::atomic<int64_t> group_launches{0}, group_periods{0};
    int64_t reserved = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> queue;
    std::vector<std::shared_ptr<Request>> active;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> table;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread th;
    int64_t completed = 0;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    void loop();
    void finish(const std::shared_ptr<Request>& r, int status, const char* msg);
    bool launch_group(const std::vector<std::shared_ptr<Request>>& ready, const std::vector<cudaGraph_t>& graphs);
};

// One launch of the ready requests' periods: a graph whose child graphs are the periods (each
// request's own captured steps, on its own buffers), rebuilt only when the members or their
// periods change.  The group stream first waits for every member's stream, and every member's
// stream then waits for the group, so the order of each request's steps is kept.
bool Server::launch_group(const std::vector<std::shared_ptr<Request>>& ready, const std::vector<cudaGraph_t>& graphs)
{
    if (!gstream && cudaStreamCreateWithFlags(&gstream, cudaStreamNonBlocking) != cudaSuccess) {
        gstream = nullptr;
        cudaGetLastError();
        return false;
    }
    std::vector<uintptr_t> key;
    for (size_t i = 0; i < ready.size(); ++i) {
        key.push_back((uintptr_t)ready[i]->ticket);
        key.push_back((uintptr_t)graphs[i]);
    }
    if (key != gkey || !gexec) {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        gkey.clear();
        cudaGraph_t G = nullptr;
        if (cudaGraphCreate(&G, 0) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        bool ok = true;
        for (cudaGraph_t c : graphs) {
            cudaGraphNode_t node;
            if (cudaGraphAddChildGraphNode(&node, G, nullptr, 0, c) != cudaSuccess) {
                ok = false;
                break;
            }
        }
        if (ok && cudaGraphInstantiate(&gexec, G, 0) != cudaSuccess) {
            gexec = nullptr;
            ok = false;
        }
        cudaGraphDestroy(G);
        if (!ok) {
            cudaGetLastError();
            return false;
        }
        gkey = key;
    }
    for (auto& r : ready) {
        cudaEvent_t e;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        cudaEventRecord(e, r->stream);
        cudaStreamWaitEvent(gstream, e, 0);
        cudaEventDestroy(e);
    }
    if (cudaGraphLaunch(gexec, gstream) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaEvent_t g_done;
    cudaEventCreateWithFlags(&g_done, cudaEventDisableTiming);
    cudaEventRecord(g_done, gstream);
    for (auto& r : ready) {
        cudaStreamWaitEvent(r->stream, g_done, 0);
        cudaEvent_t e;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        cudaEventRecord(e, r->stream);
        r->inflight.push_back(e);
        int64_t at = 0;
        const int64_t L = mithra::graph_steps(r->run, &at);
        mithra::period_replayed(r->run);
        r->enqueued += L;
    }
    cudaEventDestroy(g_done);
    ++group_launches;
    group_periods += (int64_t)ready.size();
    return true;
}

std::mutex g_srv_mu;
Server* g_srv = nullptr;

void Server::finish(const std::shared_ptr<Request>& r, int status, const char* msg)
{
    if (r->run && status == MITHRA_OK) {
        size_t n = 0;
        r->p.resize((size_t)r->nsteps);
        r->t.resize((size_t)r->nsteps);
        int rc = mithra_radiated_power(r->run, r->p.data(), r->t.data(), r->p.size(), &n);
        double b3[3] = {0, 0, 0};
        if (rc == MITHRA_OK) rc = mithra_diag(r->run, &r->fe, b3);
        r->bunch = b3[0];
        double info[19];
        if (rc == MITHRA_OK || rc == MITHRA_EDIVERGED) mithra_info(r->run, info, &r->hbm);
        if (rc != MITHRA_OK) {
            status = rc;
            msg = mithra_last_error();
        }
    }
    if (r->run) {
        mithra_destroy(r->run);
        r->run = nullptr;
    }
    for (auto e : r->inflight) cudaEventDestroy(e);
    r->inflight.clear();
    if (r->stream) {
        cudaStreamDestroy(r->stream);
        r->stream = nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (r->admitted) reserved -= r->reserve;
    r->admitted = false;
    r->status = status;
    if (msg) r->error = msg;
    r->t_done = now();
    r->state = DONE;
    r->lab.clear();
    r->lab.shrink_to_fit();
    ++completed;
}

void Server::loop()
{
    cudaSetDevice(device);
    while (true) {
        // admission: first come, first served, as long as the footprint fits
        std::vector<std::shared_ptr<Request>> admit;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (stop) break;
            while (!queue.empty() && (int)(active.size() + admit.size()) < max_active) {
                auto r = queue.front();
                if (r->reserve > (int64_t)pool.size) {
                    queue.pop_front();
                    lk.unlock();
                    finish(r, MITHRA_ENOMEM, "request footprint exceeds the serving pool");
                    lk.lock();
                    continue;
                }
                if (reserved + r->reserve > (int64_t)pool.size) break;
                queue.pop_front();
                reserved += r->reserve;
                r->admitted = true;
                admit.push_back(r);
            }
            if (admit.empty() && active.empty()) {
                cv.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
        }
        for (auto& r : admit) {
            mithra_t run = nullptr;
            r->b.lab_particles = r->lab.empty() ? nullptr : r->lab.data();
            int rc = mithra::create_with(&r->g, 0.0, &r->u, &r->b, pool_alloc, pool_free, &pool, &run);
            if (rc == MITHRA_OK) {
                cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking);
                rc = mithra_set_stream(run, r->stream);
            }
            if (rc != MITHRA_OK) {
                r->run = run;
                finish(r, rc, mithra_last_error());
                continue;
            }
            r->run = run;
            std::lock_guard<std::mutex> lk(mu);
            r->state = RUNNING;
            r->t_admit = now();
            active.push_back(r);
        }
        // advance every active request by a chunk, keeping two chunks in flight per request
        bool progress = !admit.empty();
        std::vector<std::shared_ptr<Request>> done;
        for (auto& r : active) {
            while (!r->inflight.empty() && cudaEventQuery(r->inflight.front()) == cudaSuccess) {
                cudaEventDestroy(r->inflight.front());
                r->inflight.pop_front();
                progress = true;
            }
        }
        // grouped: the requests whose next steps are one replay of their captured period advance
        // together, their periods being the child graphs of one graph and one launch.  A ready
        // request that still has a period in flight waits for partners; one with nothing in
        // flight goes at once (with whoever is ready, or alone on its own stream).
        std::vector<Request*> in_group;
        if (grouped) {
            std::vector<std::shared_ptr<Request>> ready;
            std::vector<cudaGraph_t> graphs;
            bool must_go = false;
            for (auto& r : active) {
                if (r->status != MITHRA_OK || r->enqueued >= r->nsteps || r->inflight.size() >= 2) continue;
                cudaGraph_t gr = mithra::period_graph(r->run, r->nsteps - r->enqueued);
                if (gr) {
                    ready.push_back(r);
                    graphs.push_back(gr);
                    must_go = must_go || r->inflight.empty();
                }
            }
            if (ready.size() >= 2 && launch_group(ready, graphs)) {
                for (auto& r : ready) in_group.push_back(r.get());
                progress = true;
            } else if (ready.size() == 1 && !must_go) {
                in_group.push_back(ready[0].get());   // waits this round
            }
        }
        for (auto& r : active) {
            if (std::find(in_group.begin(), in_group.end(), r.get()) != in_group.end()) continue;
            if (r->enqueued < r->nsteps && r->inflight.size() < 2) {
                // chunks end on the run's graph boundaries, and a whole graph period from a
                // boundary goes as one replay
                int64_t n = std::min<int64_t>(chunk, r->nsteps - r->enqueued);
                int64_t at = 0;
                const int64_t L = mithra::graph_steps(r->run, &at);
                if (L > 0) {
                    if (at >= L && at % L == 0 && r->nsteps - r->enqueued >= L) n = L;
                    else n = std::min<int64_t>(n, L - at % L);
                }
                int rc = mithra_step(r->run, n);
                if (rc != MITHRA_OK) {
                    r->enqueued = r->nsteps;
                    r->status = rc;
                    r->error = mithra_last_error();
                } else {
                    cudaEvent_t e;
                    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
                    cudaEventRecord(e, r->stream);
                    r->inflight.push_back(e);
                    r->enqueued += n;
                }
                progress = true;
            }
            if (r->enqueued >= r->nsteps && r->inflight.empty()) done.push_back(r);
        }
        for (auto& r : done) {
            finish(r, r->status, r->status == MITHRA_OK ? nullptr : r->error.c_str());
            std::lock_guard<std::mutex> lk(mu);
            active.erase(std::find(active.begin(), active.end(), r));
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    // stopping: drop what is still on the device
    if (gstream) cudaStreamSynchronize(gstream);
    for (auto& r : active) finish(r, MITHRA_ETIMEDOUT, "server stopped before the request finished");
    active.clear();
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    if (gstream) cudaStreamDestroy(gstream);
    gstream = nullptr;
    std::lock_guard<std::mutex> lk(mu);
    for (auto& r : queue) {
        r->state = DONE;
        r->status = MITHRA_ETIMEDOUT;
        r->error = "server stopped before the request was admitted";
    }
    queue.clear();
}

}  // namespace

extern "C" int mithra_serve_start(size_t hbm_budget_bytes, int max_active, int queue_capacity, int steps_per_chunk)
{
    return mithra_serve_start_grouped(hbm_budget_bytes, max_active, queue_capacity, steps_per_chunk, 0);
}

extern "C" int mithra_serve_start_grouped(size_t hbm_budget_bytes, int max_active, int queue_capacity,
                                          int steps_per_chunk, int grouped)
{
    std::lock_guard<std::mutex> lk(g_srv_mu);
    if (g_srv) return set_last_error(MITHRA_EINVAL, "serve_start: already running");
    if (hbm_budget_bytes < (1u << 20)) return set_last_error(MITHRA_EINVAL, "serve_start: budget below 1 MiB");
    if (max_active < 1 || queue_capacity < 1 || steps_per_chunk < 1)
        return set_last_error(MITHRA_EINVAL, "serve_start: counts must be >= 1");
    Server* s = new Server();
    cudaGetDevice(&s->device);
    s->max_active = max_active;
    s->queue_cap = queue_capacity;
    s->chunk = steps_per_chunk;
    s->grouped = grouped != 0;
    // the pool comes from the installed allocator (cudaMalloc when none), on the caller's thread
    mithra_alloc_fn a = nullptr;
    mithra_free_fn f = nullptr;
    void* ctx = nullptr;
    mithra::get_allocator(&a, &f, &ctx);
    void* block = nullptr;
    if (a) {
        block = a(ctx, hbm_budget_bytes);
    } else if (cudaMalloc(&block, hbm_budget_bytes) != cudaSuccess) {
        cudaGetLastError();
        block = nullptr;
    }
    if (!block) {
        delete s;
        return set_last_error(MITHRA_ENOMEM, "serve_start: could not allocate the serving pool");
    }
    s->block = block;
    s->block_free = f;
    s->block_ctx = ctx;
    s->pool.init(block, hbm_budget_bytes);
    s->th = std::thread([s] { s->loop(); });
    g_srv = s;
    return MITHRA_OK;
}

extern "C" int mithra_submit(const mithra_grid* g, const mithra_undulator* u, const mithra_bunch* b, int64_t nsteps,
                             uint64_t* ticket)
{
    if (!ticket) return set_last_error(MITHRA_EINVAL, "submit: null ticket");
    int rc = mithra::validate_request(g, 0.0, u, b);
    if (rc) return rc;
    if (nsteps < 1) return set_last_error(MITHRA_EINVAL, "submit: nsteps must be >= 1");
    std::lock_guard<std::mutex> lk(g_srv_mu);
    Server* s = g_srv;
    if (!s) return set_last_error(MITHRA_EINVAL, "submit: the server is not running");
    auto r = std::make_shared<Request>();
    r->g = *g;
    r->u = *u;
    r->b = *b;
    if (b->n > 0 && b->lab_particles) r->lab.assign(b->lab_particles, b->lab_particles + 6 * b->n);
    r->b.lab_particles = nullptr;
    r->nsteps = nsteps;
    r->reserve = mithra::footprint(g, u, b, nsteps);
    {
        std::lock_guard<std::mutex> lq(s->mu);
        if ((int)s->queue.size() >= s->queue_cap) return set_last_error(MITHRA_EAGAIN, "submit: queue full");
        r->ticket = s->next_ticket++;
        r->t_submit = s->now();
        s->queue.push_back(r);
        s->table[r->ticket] = r;
    }
    s->cv.notify_one();
    *ticket = r->ticket;
    return MITHRA_OK;
}

static std::shared_ptr<Request> find_req(uint64_t ticket, Server** out)
{
    std::lock_guard<std::mutex> lk(g_srv_mu);
    *out = g_srv;
    if (!g_srv) return nullptr;
    std::lock_guard<std::mutex> lq(g_srv->mu);
    auto it = g_srv->table.find(ticket);
    return it == g_srv->table.end() ? nullptr : it->second;
}

extern "C" int mithra_poll(uint64_t ticket, int* done, mithra_result* out)
{
    Server* s = nullptr;
    auto r = find_req(ticket, &s);
    if (!s) return set_last_error(MITHRA_EINVAL, "poll: the server is not running");
    if (!r) return set_last_error(MITHRA_ENOTFOUND, "poll: unknown ticket");
    std::lock_guard<std::mutex> lk(s->mu);
    const bool d = r->state == DONE;
    if (done) *done = d ? 1 : 0;
    if (out) {
        std::memset(out, 0, sizeof *out);
        out->status = d ? r->status : MITHRA_OK;
        out->state = (int32_t)r->state;
        out->steps = d ? (r->status == MITHRA_OK ? r->nsteps : 0) : r->enqueued;
        out->t_submit = r->t_submit;
        out->t_admit = r->t_admit;
        out->t_done = r->t_done;
        out->field_energy = r->fe;
        out->bunching = r->bunch;
        double last = 0, peak = 0;
        for (double v : r->p) peak = std::max(peak, v);
        if (!r->p.empty()) last = r->p.back();
        out->power_last = last;
        out->power_peak = peak;
        out->hbm_bytes = r->hbm;
        out->reserved_bytes = r->reserve;
    }
    return MITHRA_OK;
}

extern "C" int mithra_result_series(uint64_t ticket, double* p_lab, double* t_lab, size_t cap, size_t* n_out)
{
    Server* s = nullptr;
    auto r = find_req(ticket, &s);
    if (!s) return set_last_error(MITHRA_EINVAL, "result_series: the server is not running");
    if (!r) return set_last_error(MITHRA_ENOTFOUND, "result_series: unknown ticket");
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->state != DONE) return set_last_error(MITHRA_EAGAIN, "result_series: request not finished");
    if (n_out) *n_out = r->p.size();
    if (!p_lab && !t_lab) return MITHRA_OK;
    if (cap < r->p.size()) return set_last_error(MITHRA_ERANGE, "result_series: buffer too small");
    if (p_lab) std::memcpy(p_lab, r->p.data(), r->p.size() * sizeof(double));
    if (t_lab) std::memcpy(t_lab, r->t.data(), r->t.size() * sizeof(double));
    return MITHRA_OK;
}

extern "C" int mithra_release(uint64_t ticket)
{
    Server* s = nullptr;
    auto r = find_req(ticket, &s);
    if (!s) return set_last_error(MITHRA_EINVAL, "release: the server is not running");
    if (!r) return set_last_error(MITHRA_ENOTFOUND, "release: unknown ticket");
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->state != DONE) return set_last_error(MITHRA_EAGAIN, "release: request not finished");
    s->table.erase(ticket);
    return MITHRA_OK;
}

extern "C" int mithra_serve_stats(int64_t stats[6])
{
    std::lock_guard<std::mutex> lk(g_srv_mu);
    if (!g_srv) return set_last_error(MITHRA_EINVAL, "serve_stats: the server is not running");
    std::lock_guard<std::mutex> lq(g_srv->mu);
    stats[0] = g_srv->completed;
    stats[1] = (int64_t)g_srv->active.size();
    stats[2] = (int64_t)g_srv->queue.size();
    stats[3] = g_srv->reserved;
    {
        std::lock_guard<std::mutex> lp(g_srv->pool.mu);
        stats[4] = (int64_t)g_srv->pool.in_use;
        stats[5] = (int64_t)g_srv->pool.peak;
    }
    return MITHRA_OK;
}

extern "C" int mithra_serve_group_stats(int64_t out[2])
{
    std::lock_guard<std::mutex> lk(g_srv_mu);
    if (!g_srv) return set_last_error(MITHRA_EINVAL, "serve_group_stats: the server is not running");
    out[0] = g_srv->group_launches.load();
    out[1] = g_srv->group_periods.load();
    return MITHRA_OK;
}

extern "C" int mithra_serve_stop(void)
{
    Server* s = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_srv_mu);
        s = g_srv;
        g_srv = nullptr;
    }
    if (!s) return set_last_error(MITHRA_EINVAL, "serve_stop: the server is not running");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    s->th.join();
    if (s->block_free) s->block_free(s->block_ctx, s->block);
    else cudaFree(s->block);
    delete s;
    return MITHRA_OK;
}
