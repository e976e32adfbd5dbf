// Re-planning server: continuous batching of DPSO solves (the "online
// re-planning" requirement of Sec. 1 served many requests at a time).
//
// Requests are served in size-class lanes (by viewpoint count: below 100,
// 100-199, 200-399, ..., the last lane taking the rest).  Each lane has an
// engine thread and a CUDA stream of its own, so the lanes' launches overlap
// on the device and a small request's generations do not wait for a large
// one's.  Each tick a lane
//   1. admits queued requests of its class (in arrival order, or least
//      estimated work first) while the server's slots and device memory
//      budget allow (cost matrix, swarm initialisation);
//   2. rebuilds its batch when its set of active requests changed;
//   3. advances every active request of the lane by the smallest remaining
//      generation budget (capped per tick), so no request runs past its own
//      budget and each result equals a solo dpso_plan of the same request;
//   4. retires finished requests (best tour copied out, memory released).
// Requests arriving while others run join their lane at its next tick and
// their generations share the lane's launches.
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
    int lane = 0;
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

// One size-class lane: engine thread, stream, running requests and batch
// (the last three touched only by the lane's thread).
struct Lane {
    int index = 0;
    int admitted = 0;  // requests of this lane admitted and not yet retired (under mu)
    cudaStream_t stream = nullptr;
    std::thread engine;
    std::vector<Active> active;
    dpso_batch* batch = nullptr;
    bool dirty = false;
};

struct dpso_server {
    dpso_server_params prm{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<int64_t, std::shared_ptr<Request>> all;
    int64_t next_id = 1;
    bool stop = false;
    std::vector<std::unique_ptr<Lane>> lanes;
    // The lanes' library calls (admission, batch building, enqueueing,
    // retirement) take turns under lib_mu, so that no lane frees device
    // memory or captures a graph while another captures; only the waits for
    // their streams run concurrently (and the launches on the device).
    std::mutex lib_mu;
    // shared by the lanes, under mu
    size_t used = 0;
    int n_active = 0;  // requests admitted and not yet retired, all lanes
    // statistics
    dpso_server_stats st{};
    Clock::time_point start;
};

namespace {

// The lane of a request of n viewpoints: 0 below 100, then one lane per
// doubling (100-199, 200-399, ...), the last lane taking the rest.
int lane_of(int n, int lanes) {
    int k = 0;
    while (k + 1 < lanes && n >= (100 << k)) ++k;
    return k;
}

// Cost matrix and swarm for one request on its lane's stream.
int admit(cudaStream_t st, Request& r, dpso_swarm** out) {
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
void finish(dpso_server* sv, Lane* ln, Request& r, int status, bool release) {
    std::lock_guard<std::mutex> lock(sv->mu);
    if (release) {
        sv->used -= r.footprint;
        sv->n_active -= 1;
        ln->admitted -= 1;
    }
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

void engine_loop(dpso_server* sv, Lane* ln) {
    cudaSetDevice(sv->device);
    for (;;) {
        // 1. admission
        {
            std::unique_lock<std::mutex> lock(sv->mu);
            if (ln->active.empty() && !sv->stop) {
                bool mine = false;
                for (const auto& q : sv->queue) mine = mine || q->lane == ln->index;
                if (!mine) sv->cv.wait_for(lock, std::chrono::milliseconds(20));
            }
            if (sv->stop) break;
        }
        for (;;) {
            std::shared_ptr<Request> r;
            bool never_fits = false;
            {
                std::lock_guard<std::mutex> lock(sv->mu);
                if (sv->n_active >= sv->prm.max_active) break;
                // a lane holds at most its share of the slots while another
                // lane has requests waiting
                const int share = std::max(1, sv->prm.max_active / sv->prm.lanes);
                if (ln->admitted >= share) {
                    bool others = false;
                    for (const auto& q : sv->queue) others = others || q->lane != ln->index;
                    if (others) break;
                }
                // the lane's next request: the oldest, or the one with the
                // least estimated work (earliest submitted among equals)
                auto pick = sv->queue.end();
                for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
                    if ((*it)->lane != ln->index) continue;
                    if (pick == sv->queue.end()) {
                        pick = it;
                        if (sv->prm.policy != DPSO_SERVE_SHORTEST_FIRST) break;
                    } else if ((*it)->work < (*pick)->work) {
                        pick = it;
                    }
                }
                if (pick == sv->queue.end()) break;
                r = *pick;
                never_fits = r->footprint > sv->prm.memory_budget_bytes;
                if (!never_fits && sv->used + r->footprint > sv->prm.memory_budget_bytes) break;
                sv->queue.erase(pick);
                if (!never_fits) {
                    sv->used += r->footprint;
                    sv->n_active += 1;
                    ln->admitted += 1;
                }
            }
            if (never_fits) {
                finish(sv, ln, *r, DPSO_ERR_NO_MEMORY, false);
                continue;
            }
            dpso_swarm* sw = nullptr;
            int rc;
            {
                std::lock_guard<std::mutex> lib(sv->lib_mu);
                rc = admit(ln->stream, *r, &sw);
            }
            if (rc) {
                finish(sv, ln, *r, rc, true);
                continue;
            }
            ln->active.push_back(Active{r, sw, r->iterations, 0});
            if (r->iterations > 0) ln->dirty = true;
        }
        std::vector<Active> running;
        for (const Active& a : ln->active)
            if (a.remaining > 0) running.push_back(a);
        // 2-3. advance every running request of the lane together
        if (!running.empty()) {
            std::unique_lock<std::mutex> lib(sv->lib_mu);
            if (ln->dirty || !ln->batch) {
                if (ln->batch) dpso_batch_destroy(ln->batch);
                ln->batch = nullptr;
                std::vector<dpso_swarm*> members;
                for (const Active& a : running) members.push_back(a.swarm);
                int rc = dpso_batch_create(&ln->batch, members.data(),
                                           static_cast<int32_t>(members.size()), ln->stream);
                if (rc) {  // the running requests fail with the batch
                    for (Active& a : ln->active)
                        if (a.remaining > 0) {
                            a.fail = rc;
                            a.remaining = -1;
                        }
                }
                ln->dirty = false;
            }
            if (ln->batch) {
                int g = sv->prm.generations_per_tick;
                for (const Active& a : running) g = std::min(g, a.remaining);
                const int rc = dpso_batch_step(ln->batch, g, ln->stream);
                lib.unlock();
                if (rc == DPSO_OK && cudaStreamSynchronize(ln->stream) == cudaSuccess) {
                    for (Active& a : ln->active)
                        if (a.remaining > 0) a.remaining -= g;
                    std::lock_guard<std::mutex> lock(sv->mu);
                    sv->st.ticks += 1;
                    sv->st.peak_active = std::max<int32_t>(sv->st.peak_active, sv->n_active);
                } else {
                    for (Active& a : ln->active)
                        if (a.remaining > 0) {
                            a.fail = rc ? rc : DPSO_ERR_CUDA;
                            a.remaining = -1;
                        }
                }
            }
        } else if (!ln->active.empty()) {
            std::lock_guard<std::mutex> lock(sv->mu);
            sv->st.peak_active = std::max<int32_t>(sv->st.peak_active, sv->n_active);
        }
        // 4. retirement: the batch goes first (it refers to its members)
        bool any_done = false;
        for (const Active& a : ln->active) any_done = any_done || a.remaining <= 0;
        if (any_done) {
            std::lock_guard<std::mutex> lib(sv->lib_mu);
            if (ln->batch) {
                dpso_batch_destroy(ln->batch);
                ln->batch = nullptr;
            }
            std::vector<Active> keep;
            for (Active& a : ln->active) {
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
                finish(sv, ln, r, status, true);
            }
            ln->active.swap(keep);
            ln->dirty = true;
        }
    }
    std::lock_guard<std::mutex> lib(sv->lib_mu);
    if (ln->batch) dpso_batch_destroy(ln->batch);
    ln->batch = nullptr;
    for (Active& a : ln->active) dpso_destroy(a.swarm);
    ln->active.clear();
}

}  // namespace

extern "C" {

void dpso_default_server_params(dpso_server_params* p) {
    if (!p) return;
    p->memory_budget_bytes = 0;
    p->max_active = 64;
    p->generations_per_tick = 8;
    p->policy = DPSO_SERVE_ARRIVAL_ORDER;
    p->lanes = 4;
}

int dpso_server_create(dpso_server** out, const dpso_server_params* p) {
    if (!out || !p || p->max_active < 1 || p->generations_per_tick < 1 ||
        (p->policy != DPSO_SERVE_ARRIVAL_ORDER && p->policy != DPSO_SERVE_SHORTEST_FIRST) ||
        p->lanes < 0 || p->lanes > DPSO_SERVE_MAX_LANES)
        return DPSO_ERR_ARG;
    *out = nullptr;
    dpso_server* sv = new dpso_server();
    sv->prm = *p;
    if (sv->prm.lanes == 0) sv->prm.lanes = 4;
    auto fail = [&](int code) {
        for (auto& ln : sv->lanes)
            if (ln->stream) cudaStreamDestroy(ln->stream);
        delete sv;
        return code;
    };
    if (cudaGetDevice(&sv->device) != cudaSuccess) return fail(DPSO_ERR_CUDA);
    // lanes of smaller requests get higher stream priorities: when a large
    // lane's generation frees the SMs, a small lane's waiting kernels go first
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess)
        return fail(DPSO_ERR_CUDA);
    for (int k = 0; k < sv->prm.lanes; ++k) {
        auto ln = std::make_unique<Lane>();
        ln->index = k;
        const int prio = std::min(least, greatest + k);  // greatest is numerically lowest
        if (cudaStreamCreateWithPriority(&ln->stream, cudaStreamNonBlocking, prio) != cudaSuccess)
            return fail(DPSO_ERR_CUDA);
        sv->lanes.push_back(std::move(ln));
    }
    if (sv->prm.memory_budget_bytes == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(DPSO_ERR_CUDA);
        sv->prm.memory_budget_bytes = free_b / 2;
    }
    sv->start = Clock::now();
    for (auto& ln : sv->lanes) ln->engine = std::thread(engine_loop, sv, ln.get());
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
    q->lane = lane_of(q->n, sv->prm.lanes);
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
    for (auto& ln : sv->lanes) {
        if (ln->engine.joinable()) ln->engine.join();
        cudaStreamSynchronize(ln->stream);
        cudaStreamDestroy(ln->stream);
    }
    delete sv;
}

}  // extern "C"
