// Re-planning server: continuous batching of DPSO solves (the "online
// re-planning" requirement of Sec. 1 served many requests at a time).
//
// An engine thread owns one CUDA stream.  Each tick it
//   1. admits queued requests in arrival order while slots and the device
//      memory budget allow (cost matrix, swarm initialisation);
//   2. rebuilds the batch when the set of active requests changed;
//   3. advances every active request by the smallest remaining generation
//      budget (capped per tick), so no request runs past its own budget and
//      each result equals a solo dpso_plan of the same request;
//   4. retires finished requests (best tour copied out, memory released).
// Requests arriving while others run join at the next tick and their
// generations share the same launches.
#include <math.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace dpso;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    std::vector<double> xyz, boxes;
    std::vector<int32_t> tags;
    bool has_tags = false;
    int32_t n = 0, m = 0;
    dpso_cost_params cp{};
    dpso_params prm{};
    uint64_t seed = 0;
    int32_t iterations = 0;
    size_t footprint = 0;
    double work = 0.0;  // admission estimate: swarm x budget x n^3
    Clock::time_point submitted;
    // results
    int status = 0;  // 0 queued/running, 1 done, < 0 DPSO_ERR_*
    std::vector<int32_t> tour;
    int64_t cost = 0;
    double latency_s = 0.0;
};

struct Active {
    std::shared_ptr<Request> req;
    dpso_swarm* swarm = nullptr;
    int remaining = 0;  // generations still to run
    int fail = 0;       // status the request failed with while running
};

// Device bytes one request holds while active (the arrays dpso_init
// allocates, each rounded to the 512-byte allocation granule) plus the
// transient buffers of its admission (viewpoints, boxes, the unpadded cost
// matrix).  Only the planning estimate for admission, not an allocator.
size_t request_footprint(int n, int m, int S, int T, int flags) {
    auto a = [](size_t b) { return (b + 511) / 512 * 512; };
    const size_t ldc = (n + 31) / 32 * 32, ldn = (n + 7) / 8 * 8, s = S;
    size_t hist = 1024;
    while (hist < static_cast<size_t>(T)) hist *= 2;
    size_t b = a(n * ldc * 4);                                       // C
    if ((flags & DPSO_FLAG_TWO_OPT) && dpso::two_opt_tiled_rows(n) > 0)
        b += a(static_cast<size_t>(4) * n * dpso::shifted_ld(n) * 4);  // shifted copies
    b += 3 * a(s * ldn * 2) + a(ldn * 2);                             // X, V, P, G
    b += 3 * a(s * 8) + 2 * a(s) + a(s * 4);                          // F, PF, hash, dup, kept, order
    b += a(hist * 8) + 2 * a(sizeof(SwarmDesc) + 1024);               // history, control, meta
    b += a(static_cast<size_t>(n) * 24) + a(static_cast<size_t>(std::max(m, 1)) * 48) +
         a(static_cast<size_t>(n) * n * 4) + a(ldn * 16) + a(static_cast<size_t>(n) * 12);
    return b;
}

}  // namespace

struct dpso_server {
    dpso_server_params prm{};
    int device = 0;
    cudaStream_t stream = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<int64_t, std::shared_ptr<Request>> all;
    int64_t next_id = 1;
    bool stop = false;
    std::thread engine;
    // engine-side state
    std::vector<Active> active;
    dpso_batch* batch = nullptr;
    bool dirty = false;
    size_t used = 0;
    // statistics
    dpso_server_stats st{};
    Clock::time_point start;
};

namespace {

// Cost matrix and swarm for one request on the engine stream.
int admit(dpso_server* sv, Request& r, dpso_swarm** out) {
    cudaStream_t st = sv->stream;
    double *xyz = nullptr, *boxes = nullptr;
    int32_t* C = nullptr;
    int rc = DPSO_OK;
    if (cudaMalloc(&xyz, sizeof(double) * 3 * r.n) != cudaSuccess ||
        cudaMalloc(&boxes, sizeof(double) * 6 * std::max(r.m, 1)) != cudaSuccess ||
        cudaMalloc(&C, sizeof(int32_t) * static_cast<size_t>(r.n) * r.n) != cudaSuccess) {
        cudaGetLastError();
        rc = DPSO_ERR_NO_MEMORY;
    }
    if (!rc && (cudaMemcpyAsync(xyz, r.xyz.data(), sizeof(double) * 3 * r.n,
                                cudaMemcpyHostToDevice, st) != cudaSuccess ||
                (r.m > 0 && cudaMemcpyAsync(boxes, r.boxes.data(), sizeof(double) * 6 * r.m,
                                            cudaMemcpyHostToDevice, st) != cudaSuccess)))
        rc = DPSO_ERR_CUDA;
    if (!rc) rc = dpso_cost_matrix(xyz, r.n, boxes, r.m, &r.cp, C, st);
    if (!rc)
        rc = dpso_init(out, C, r.n, r.has_tags ? r.tags.data() : nullptr, &r.prm, r.seed, st);
    cudaFree(xyz);
    cudaFree(boxes);
    cudaFree(C);
    return rc;
}

// Publishes a request's outcome and releases its share of the budget (the
// caller has already freed its device memory).
void finish(dpso_server* sv, Request& r, int status, bool release) {
    std::lock_guard<std::mutex> lock(sv->mu);
    if (release) sv->used -= r.footprint;
    r.status = status;
    r.latency_s = std::chrono::duration<double>(Clock::now() - r.submitted).count();
    if (status == 1) {
        sv->st.completed += 1;
        sv->st.particle_iterations += static_cast<int64_t>(r.prm.swarm) * r.iterations;
    } else {
        sv->st.failed += 1;
    }
    sv->cv.notify_all();
}

void engine_loop(dpso_server* sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        // 1. admission
        {
            std::unique_lock<std::mutex> lock(sv->mu);
            if (sv->active.empty() && sv->queue.empty() && !sv->stop)
                sv->cv.wait_for(lock, std::chrono::milliseconds(20));
            if (sv->stop) break;
        }
        for (;;) {
            std::shared_ptr<Request> r;
            bool never_fits = false;
            {
                std::lock_guard<std::mutex> lock(sv->mu);
                if (sv->queue.empty() ||
                    static_cast<int>(sv->active.size()) >= sv->prm.max_active)
                    break;
                // the next request: the oldest, or the one with the least
                // estimated work (earliest submitted among equals)
                auto pick = sv->queue.begin();
                if (sv->prm.policy == DPSO_SERVE_SHORTEST_FIRST)
                    for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it)
                        if ((*it)->work < (*pick)->work) pick = it;
                r = *pick;
                never_fits = r->footprint > sv->prm.memory_budget_bytes;
                if (!never_fits && sv->used + r->footprint > sv->prm.memory_budget_bytes) break;
                sv->queue.erase(pick);
                if (!never_fits) sv->used += r->footprint;
            }
            if (never_fits) {
                finish(sv, *r, DPSO_ERR_NO_MEMORY, false);
                continue;
            }
            dpso_swarm* sw = nullptr;
            const int rc = admit(sv, *r, &sw);
            if (rc) {
                finish(sv, *r, rc, true);
                continue;
            }
            sv->active.push_back(Active{r, sw, r->iterations, 0});
            if (r->iterations > 0) sv->dirty = true;
        }
        std::vector<Active> running;
        for (const Active& a : sv->active)
            if (a.remaining > 0) running.push_back(a);
        // 2-3. advance every running request together
        if (!running.empty()) {
            if (sv->dirty || !sv->batch) {
                if (sv->batch) dpso_batch_destroy(sv->batch);
                sv->batch = nullptr;
                std::vector<dpso_swarm*> members;
                for (const Active& a : running) members.push_back(a.swarm);
                int rc = dpso_batch_create(&sv->batch, members.data(),
                                           static_cast<int32_t>(members.size()), sv->stream);
                if (rc) {  // the running requests fail with the batch
                    for (Active& a : sv->active)
                        if (a.remaining > 0) {
                            a.fail = rc;
                            a.remaining = -1;
                        }
                }
                sv->dirty = false;
            }
            if (sv->batch) {
                int g = sv->prm.generations_per_tick;
                for (const Active& a : running) g = std::min(g, a.remaining);
                const int rc = dpso_batch_step(sv->batch, g, sv->stream);
                if (rc == DPSO_OK && cudaStreamSynchronize(sv->stream) == cudaSuccess) {
                    for (Active& a : sv->active)
                        if (a.remaining > 0) a.remaining -= g;
                    std::lock_guard<std::mutex> lock(sv->mu);
                    sv->st.ticks += 1;
                    sv->st.peak_active =
                        std::max<int32_t>(sv->st.peak_active, static_cast<int32_t>(running.size()));
                } else {
                    for (Active& a : sv->active)
                        if (a.remaining > 0) {
                            a.fail = rc ? rc : DPSO_ERR_CUDA;
                            a.remaining = -1;
                        }
                }
            }
        }
        // 4. retirement: the batch goes first (it refers to its members)
        bool any_done = false;
        for (const Active& a : sv->active) any_done = any_done || a.remaining <= 0;
        if (any_done) {
            if (sv->batch) {
                dpso_batch_destroy(sv->batch);
                sv->batch = nullptr;
            }
            std::vector<Active> keep;
            for (Active& a : sv->active) {
                if (a.remaining > 0) {
                    keep.push_back(a);
                    continue;
                }
                Request& r = *a.req;
                int status = a.fail;
                if (!status) {
                    r.tour.assign(r.n, 0);
                    int64_t cost = 0;
                    const int rc = dpso_get_best(a.swarm, r.tour.data(), &cost);
                    r.cost = cost;
                    status = rc ? rc : 1;
                }
                dpso_destroy(a.swarm);
                finish(sv, r, status, true);
            }
            sv->active.swap(keep);
            sv->dirty = true;
        }
    }
    if (sv->batch) dpso_batch_destroy(sv->batch);
    for (Active& a : sv->active) dpso_destroy(a.swarm);
    sv->active.clear();
}

}  // namespace

extern "C" {

void dpso_default_server_params(dpso_server_params* p) {
    if (!p) return;
    p->memory_budget_bytes = 0;
    p->max_active = 64;
    p->generations_per_tick = 8;
    p->policy = DPSO_SERVE_ARRIVAL_ORDER;
    p->reserved = 0;
}

int dpso_server_create(dpso_server** out, const dpso_server_params* p) {
    if (!out || !p || p->max_active < 1 || p->generations_per_tick < 1 ||
        (p->policy != DPSO_SERVE_ARRIVAL_ORDER && p->policy != DPSO_SERVE_SHORTEST_FIRST) ||
        p->reserved != 0)
        return DPSO_ERR_ARG;
    *out = nullptr;
    dpso_server* sv = new dpso_server();
    sv->prm = *p;
    if (cudaGetDevice(&sv->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete sv;
        return DPSO_ERR_CUDA;
    }
    if (sv->prm.memory_budget_bytes == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaStreamDestroy(sv->stream);
            delete sv;
            return DPSO_ERR_CUDA;
        }
        sv->prm.memory_budget_bytes = free_b / 2;
    }
    sv->start = Clock::now();
    sv->engine = std::thread(engine_loop, sv);
    *out = sv;
    return DPSO_OK;
}

int dpso_server_footprint(const dpso_request* r, uint64_t* bytes) {
    if (!r || !bytes || r->n < 3 || r->m < 0 || r->iterations < 0 || r->params.swarm < 1)
        return DPSO_ERR_ARG;
    if (r->n > DPSO_MAX_N || r->params.swarm > DPSO_MAX_SWARM) return DPSO_ERR_RANGE;
    *bytes = request_footprint(r->n, r->m, r->params.swarm, r->iterations, r->params.flags);
    return DPSO_OK;
}

int dpso_server_submit(dpso_server* sv, const dpso_request* r, int64_t* id) {
    if (!sv || !r || !id || !r->xyz_host || r->n < 3 || r->m < 0 || (r->m > 0 && !r->boxes_host) ||
        r->iterations < 0 || r->reserved != 0)
        return DPSO_ERR_ARG;
    if (r->n > DPSO_MAX_N) return DPSO_ERR_RANGE;
    const int pv = validate_params(&r->params);
    if (pv) return pv;
    if (!isfinite(r->cost.uav_radius_m) || r->cost.uav_radius_m < 0.0 ||
        r->cost.blocked_penalty_mm < 0 || r->cost.reserved != 0)
        return DPSO_ERR_ARG;
    auto q = std::make_shared<Request>();
    q->n = r->n;
    q->m = r->m;
    q->xyz.assign(r->xyz_host, r->xyz_host + 3 * static_cast<size_t>(r->n));
    if (r->m > 0) q->boxes.assign(r->boxes_host, r->boxes_host + 6 * static_cast<size_t>(r->m));
    if (r->tags_host) {
        q->tags.assign(r->tags_host, r->tags_host + 3 * static_cast<size_t>(r->n));
        q->has_tags = true;
    }
    q->cp = r->cost;
    q->prm = r->params;
    q->seed = r->seed;
    q->iterations = r->iterations;
    q->footprint = request_footprint(r->n, r->m, r->params.swarm, r->iterations, r->params.flags);
    q->work = static_cast<double>(r->params.swarm) * r->iterations * r->n * r->n * r->n;
    q->submitted = Clock::now();
    std::lock_guard<std::mutex> lock(sv->mu);
    q->id = sv->next_id++;
    sv->all[q->id] = q;
    sv->queue.push_back(q);
    sv->st.submitted += 1;
    sv->cv.notify_all();
    *id = q->id;
    return DPSO_OK;
}

int dpso_server_poll(dpso_server* sv, int64_t id, int32_t* state, int32_t* tour_host,
                     int32_t tour_cap, int64_t* cost, double* latency_s) {
    if (!sv || !state) return DPSO_ERR_ARG;
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->all.find(id);
    if (it == sv->all.end()) return DPSO_ERR_ARG;
    const Request& r = *it->second;
    *state = r.status;
    if (r.status == 1) {
        if (tour_host) {
            if (tour_cap < r.n) return DPSO_ERR_ARG;
            memcpy(tour_host, r.tour.data(), sizeof(int32_t) * r.n);
        }
        if (cost) *cost = r.cost;
    }
    if (latency_s) *latency_s = r.status != 0 ? r.latency_s : 0.0;
    return DPSO_OK;
}

int dpso_server_wait(dpso_server* sv, int64_t id, double timeout_s, int32_t* state) {
    if (!sv || !state) return DPSO_ERR_ARG;
    std::unique_lock<std::mutex> lock(sv->mu);
    auto it = sv->all.find(id);
    if (it == sv->all.end()) return DPSO_ERR_ARG;
    std::shared_ptr<Request> r = it->second;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout_s));
    while (r->status == 0 && Clock::now() < deadline)
        sv->cv.wait_until(lock, deadline);
    *state = r->status;
    return r->status == 0 ? DPSO_ERR_TIMEOUT : DPSO_OK;
}

int dpso_server_stats_get(dpso_server* sv, dpso_server_stats* out) {
    if (!sv || !out) return DPSO_ERR_ARG;
    std::lock_guard<std::mutex> lock(sv->mu);
    *out = sv->st;
    out->queued = static_cast<int32_t>(sv->queue.size());
    out->memory_used_bytes = sv->used;
    out->elapsed_s = std::chrono::duration<double>(Clock::now() - sv->start).count();
    return DPSO_OK;
}

void dpso_server_destroy(dpso_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        sv->cv.notify_all();
    }
    if (sv->engine.joinable()) sv->engine.join();
    cudaStreamSynchronize(sv->stream);
    cudaStreamDestroy(sv->stream);
    delete sv;
}

}  // extern "C"
