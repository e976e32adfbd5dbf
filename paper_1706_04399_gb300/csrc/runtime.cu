// Host runtime and C ABI of the DPSO library: swarm lifecycle, the generation
// loop of Fig. "pseudocode" replayed from CUDA graphs, checkpoints, and the
// standalone entry points (fitness, 2-opt, Philox draws, synchronous plan).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <vector>

#include "common.cuh"

namespace dpso {

// Parameter ranges every entry point that takes dpso_params accepts.
int validate_params(const dpso_params* p) {
    if (!p) return DPSO_ERR_ARG;
    auto unit = [](double v) { return isfinite(v) && v >= 0.0 && v <= 1.0; };
    if (!unit(p->w) || !unit(p->phi1) || !unit(p->phi2)) return DPSO_ERR_ARG;
    if (p->swarm < 1 || p->mut_period < 1 || p->mut_swaps < 0 || p->det_frac_pct < 0 ||
        p->det_frac_pct > 100 || p->stall_limit < 0 || p->max_moves < 0 ||
        p->two_opt_trigger < 0 || p->two_opt_trigger > 1 || (p->flags & ~15) != 0)
        return DPSO_ERR_ARG;
    if (p->swarm > DPSO_MAX_SWARM) return DPSO_ERR_RANGE;
    return DPSO_OK;
}

}  // namespace dpso

using namespace dpso;

namespace {

#define CK(expr)                                   \
    do {                                           \
        if ((expr) != cudaSuccess) return DPSO_ERR_CUDA; \
    } while (0)

// Makes `dev` current for the scope of a call and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

unsigned long long q32(double c) { return static_cast<unsigned long long>(llround(ldexp(c, 32))); }

constexpr uint32_t kStateMagic = 0x4f535044u;  // "DPSO"
constexpr uint32_t kStateVersion = 1;

// Events recorded per generation: before the update, then after the update,
// the mutation, the first gbest pass, the edge exchange and the second gbest
// pass.
constexpr int kPhaseEvents = 6;

struct StateHeader {
    uint32_t magic, version;
    int32_t n, S, t, stall, done, n_det;
    int64_t gf;
    uint64_t pairs, moves, runs;
    uint64_t seed;
    dpso_params prm;
};

// A swarm's descriptors as the batched launches read them (device memory).
struct SwarmMeta {
    SwarmDesc desc;
    TwoOptTask task;
    int off[2];   // particle offsets of a batch of one: {0, S}
    int toff[2];  // tour offsets of the one 2-opt problem: {0, S}
    unsigned int queue;
    unsigned int pad;
};

}  // namespace

struct dpso_swarm {
    int device = 0, num_sms = 0;
    dpso_params prm{};
    Consts k{};
    SwarmDev d{};
    int* C = nullptr;
    int* Cs = nullptr;  // row-shifted copies of C for the TMA 2-opt (or null)
    uint16_t *X = nullptr, *V = nullptr, *P = nullptr, *G = nullptr;
    long long *F = nullptr, *PF = nullptr;
    unsigned long long* hash = nullptr;
    unsigned char *dup = nullptr, *kept = nullptr;
    int* order = nullptr;  // exchange order, recomputed every generation
    Ctl* ctl = nullptr;
    SwarmMeta* meta = nullptr;  // device: descriptors of this swarm as a batch of one
    long long* hist = nullptr;
    int hist_cap = 0;
    int n_det = 0;
    int t_host = 0;
    cudaStream_t last = nullptr;
    cudaStream_t cap = nullptr;
    // the two generation graphs (index 0: without mutation, 1: with it); each
    // holds kPhaseEvents event-record nodes at the phase boundaries, which
    // record into ev_cap unless timing mode rebinds them to pool events
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaGraphNode_t ev_node[2][kPhaseEvents] = {};
    cudaEvent_t ev_cap[kPhaseEvents] = {};
    // timing mode
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;       // kPhaseEvents events per timed generation
    std::vector<std::array<int, 2>> pending; // (first event, mutation generation)
    dpso_timing acc{};
};

namespace {

void free_swarm(dpso_swarm* s) {
    if (!s) return;
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k) {
        if (s->exec[k]) cudaGraphExecDestroy(s->exec[k]);
        if (s->graph[k]) cudaGraphDestroy(s->graph[k]);
    }
    for (cudaEvent_t e : s->ev_cap)
        if (e) cudaEventDestroy(e);
    void* bufs[] = {s->C,    s->Cs,   s->X,   s->V,     s->P,   s->G,    s->F,    s->PF,
                    s->hash, s->dup,  s->kept, s->order, s->ctl, s->meta, s->hist};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (s->cap) cudaStreamDestroy(s->cap);
    delete s;
}

// Allocates and zero-fills on `st`, so the fill is ordered before later work
// on that stream (a plain cudaMemset runs on the legacy stream, which
// non-blocking streams do not wait for).
template <typename T>
int dalloc(T** p, size_t count, cudaStream_t st) {
    if (cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return DPSO_ERR_NO_MEMORY;
    }
    if (cudaMemsetAsync(*p, 0, count * sizeof(T), st) != cudaSuccess) return DPSO_ERR_CUDA;
    return DPSO_OK;
}

// Host-side copies of the descriptors the batched launches take.
TwoOptTask swarm_task(const dpso_swarm* s) {
    TwoOptTask a{};
    a.C = s->C;
    a.Cs = s->Cs;
    a.ldc = s->k.ldc;
    a.n = s->k.n;
    a.tours = s->X;
    a.ldt = s->k.ldn;
    a.count = s->k.S;
    a.cost = s->F;
    a.pbest = s->P;
    a.pcost = s->PF;
    a.max_moves = s->k.max_moves;
    a.gate = &s->ctl->run_two_opt;
    a.pairs = &s->ctl->pairs;
    a.moves = &s->ctl->moves;
    a.status = &s->ctl->status;
    a.evals = &s->ctl->evals;
    a.order = s->order;
    a.kind = (s->k.flags & DPSO_FLAG_NODE_SWAP) ? 1 : 0;
    return a;
}

int swarm_arrays(const Consts& k) { return k.w_q >= (1ull << 32) ? 5 : 7; }

BatchView swarm_view(const dpso_swarm* s) {
    return BatchView{&s->meta->desc, s->meta->off, 1, s->k.S, s->k.ldn, swarm_arrays(s->k), s->k.S};
}

TwoOptBatch swarm_two_opt(const dpso_swarm* s) {
    TwoOptBatch tb{&s->meta->task, s->meta->toff, 1, s->k.S, s->k.n, s->Cs != nullptr, 0,
                   &s->meta->queue};
    tb.kind = (s->k.flags & DPSO_FLAG_NODE_SWAP) ? 1 : 0;
    return tb;
}

// One generation of Fig. "pseudocode" for one swarm: particle update,
// mutation (when due), gbest, then the edge exchange and a second gbest pass
// (both no-ops unless the first gbest pass scheduled the exchange).  With
// `ev`, an external event-record node is captured at each phase boundary
// (move | mutation | gbest | 2-opt | gbest).
cudaError_t enqueue_generation(dpso_swarm* s, bool mut_iter, cudaStream_t st,
                               const cudaEvent_t* ev = nullptr) {
    const bool two = (s->k.flags & DPSO_FLAG_TWO_OPT) != 0;
    const BatchView bv = swarm_view(s);
    const TwoOptBatch tb = swarm_two_opt(s);
    auto mark = [&](int q) {
        return ev ? cudaEventRecordWithFlags(ev[q], st, cudaEventRecordExternal) : cudaSuccess;
    };
    cudaError_t e = mark(0);
    if (e == cudaSuccess) e = launch_move(bv, st);
    if (e == cudaSuccess) e = mark(1);
    if (e == cudaSuccess && mut_iter) e = launch_mutation(bv, st);
    if (e == cudaSuccess) e = mark(2);
    if (e == cudaSuccess) e = launch_gbest(bv, 0, st);
    if (e == cudaSuccess) e = mark(3);
    if (e == cudaSuccess && two) e = launch_rank_cost(bv, st);
    if (e == cudaSuccess && two) e = cudaMemsetAsync(tb.queue, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess && two) e = launch_two_opt(tb, s->num_sms, st);
    if (e == cudaSuccess) e = mark(4);
    if (e == cudaSuccess && two) e = launch_gbest(bv, 1, st);
    if (e == cudaSuccess) e = mark(5);
    return e;
}

// Timing mode: rebinds the graph's event-record nodes to kPhaseEvents fresh
// pool events and replays it (an update of a graph exec affects only later
// launches, so generations already enqueued keep their own events).
cudaError_t launch_generation_timed(dpso_swarm* s, bool mut_iter, cudaStream_t st) {
    const size_t base = s->pending.size() * kPhaseEvents;
    while (s->ev_pool.size() < base + kPhaseEvents) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        s->ev_pool.push_back(e);
    }
    const int g = mut_iter ? 1 : 0;
    for (int q = 0; q < kPhaseEvents; ++q) {
        cudaError_t r =
            cudaGraphExecEventRecordNodeSetEvent(s->exec[g], s->ev_node[g][q], s->ev_pool[base + q]);
        if (r != cudaSuccess) return r;
    }
    cudaError_t e = cudaGraphLaunch(s->exec[g], st);
    if (e == cudaSuccess) s->pending.push_back({static_cast<int>(base), g});
    return e;
}

int collect_timing(dpso_swarm* s) {
    for (const auto& pr : s->pending) {
        cudaEvent_t* ev = s->ev_pool.data() + pr[0];  // kPhaseEvents events
        float t[5];
        for (int q = 0; q < 5; ++q) CK(cudaEventElapsedTime(&t[q], ev[q], ev[q + 1]));
        const bool two = (s->k.flags & DPSO_FLAG_TWO_OPT) != 0;
        s->acc.ms[DPSO_PHASE_MOVE] += t[0];
        s->acc.ms[DPSO_PHASE_MUTATION] += t[1];
        s->acc.ms[DPSO_PHASE_GBEST] += t[2] + t[4];
        s->acc.ms[DPSO_PHASE_TWO_OPT] += t[3];
        s->acc.launches[DPSO_PHASE_MOVE] += 1;
        s->acc.launches[DPSO_PHASE_MUTATION] += pr[1] ? 4 : 0;
        s->acc.launches[DPSO_PHASE_GBEST] += two ? 2 : 1;
        s->acc.launches[DPSO_PHASE_TWO_OPT] += two ? 1 : 0;
        s->acc.generations += 1;
    }
    s->pending.clear();
    return DPSO_OK;
}

// Captures the generation graph with (g = 1) or without (g = 0) mutation,
// keeps it (its event-record nodes are rebound in timing mode) and
// instantiates it.
int capture(dpso_swarm* s, int g) {
    for (cudaEvent_t& e : s->ev_cap)
        if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeRelaxed));
    const cudaError_t e = enqueue_generation(s, g == 1, s->cap, s->ev_cap);
    const cudaError_t e2 = cudaStreamEndCapture(s->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return DPSO_ERR_CUDA;
    }
    s->graph[g] = graph;
    size_t count = 0;
    CK(cudaGraphGetNodes(graph, nullptr, &count));
    std::vector<cudaGraphNode_t> nodes(count);
    CK(cudaGraphGetNodes(graph, nodes.data(), &count));
    int found = 0;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType type;
        CK(cudaGraphNodeGetType(nd, &type));
        if (type != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev = nullptr;
        CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
        for (int q = 0; q < kPhaseEvents; ++q)
            if (ev == s->ev_cap[q] && !s->ev_node[g][q]) {
                s->ev_node[g][q] = nd;
                ++found;
            }
    }
    if (found != kPhaseEvents) return DPSO_ERR_INTERNAL;
    CK(cudaGraphInstantiate(&s->exec[g], graph, 0));
    return DPSO_OK;
}

// Makes room for `need` history entries (the device reads the pointer from
// its control block, so the captured graphs stay valid).
int ensure_history(dpso_swarm* s, int need) {
    if (need <= s->hist_cap) return DPSO_OK;
    int cap = std::max(1024, s->hist_cap);
    while (cap < need) cap *= 2;
    long long* nh = nullptr;
    int st = dalloc(&nh, static_cast<size_t>(cap), s->last);
    if (st) return st;
    // after the generations already enqueued on the swarm's stream, before
    // the ones the caller enqueues next
    if (s->hist_cap > 0)
        CK(cudaMemcpyAsync(nh, s->hist, sizeof(long long) * s->hist_cap, cudaMemcpyDeviceToDevice,
                           s->last));
    CK(cudaMemcpyAsync(&s->ctl->hist, &nh, sizeof(nh), cudaMemcpyHostToDevice, s->last));
    CK(cudaMemcpyAsync(&s->ctl->hist_cap, &cap, sizeof(cap), cudaMemcpyHostToDevice, s->last));
    CK(cudaStreamSynchronize(s->last));
    cudaFree(s->hist);
    s->hist = nh;
    s->hist_cap = cap;
    return DPSO_OK;
}

int read_ctl(dpso_swarm* s, Ctl* c) {
    CK(cudaStreamSynchronize(s->last));
    CK(cudaMemcpy(c, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    return DPSO_OK;
}

}  // namespace

namespace dpso {
// Flags (bit 0 of *err) any of the count x n tours that is not a permutation.
__global__ void tours_valid_kernel(const uint16_t* tours, int n, int* err) {
    extern __shared__ unsigned char seen[];
    const uint16_t* x = tours + static_cast<size_t>(blockIdx.x) * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) seen[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int v = x[i];
        if (v >= n) atomicOr(err, 1);
        else seen[v] = 1;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (!seen[i]) atomicOr(err, 1);
}
}  // namespace dpso

extern "C" {

void dpso_default_params(dpso_params* p) {
    if (!p) return;
    p->w = 1.0;
    p->phi1 = 0.4;
    p->phi2 = 0.4;
    p->swarm = 100;
    p->mut_period = 3;
    p->mut_swaps = 2;
    p->det_frac_pct = 10;
    p->stall_limit = 0;
    p->flags = DPSO_FLAG_DET_INIT | DPSO_FLAG_MUTATION | DPSO_FLAG_TWO_OPT;
    p->two_opt_trigger = 0;
    p->max_moves = 0;
}

void dpso_default_cost_params(dpso_cost_params* p) {
    if (!p) return;
    p->uav_radius_m = 0.0;
    p->blocked_penalty_mm = 1000000;
    p->reserved = 0;
}

const char* dpso_status_string(int status) {
    switch (status) {
        case DPSO_OK: return "ok";
        case DPSO_ERR_ARG: return "invalid argument";
        case DPSO_ERR_RANGE: return "value out of range";
        case DPSO_ERR_NO_MEMORY: return "out of device memory";
        case DPSO_ERR_CUDA: return "CUDA runtime error";
        case DPSO_ERR_TIMEOUT: return "device wait timed out";
        case DPSO_ERR_INTERNAL: return "internal error";
        default: return "unknown status";
    }
}

int dpso_fitness(const int32_t* C_dev, int32_t n, const uint16_t* tours_dev, int32_t count,
                 int64_t* cost_dev, void* stream) {
    if (!C_dev || !tours_dev || !cost_dev || n < 1 || count < 0) return DPSO_ERR_ARG;
    if (n > DPSO_MAX_N) return DPSO_ERR_RANGE;
    CK(launch_fitness(C_dev, n, n, tours_dev, n, count, reinterpret_cast<long long*>(cost_dev),
                      static_cast<cudaStream_t>(stream)));
    return DPSO_OK;
}

}  // extern "C"

namespace {

// dpso_two_opt and dpso_node_swap: validate, fitness, one persistent exchange
// launch over `count` tours (kind 0: 2-opt, 1: node swap), counters back.
int exchange_tours(int kind, const int32_t* C_dev, int32_t n, uint16_t* tours_dev,
                   int32_t count, int64_t* cost_dev, int32_t max_moves, int64_t* pairs_host,
                   int64_t* moves_host, void* stream) {
    if (!C_dev || !tours_dev || !cost_dev || n < 3 || count < 0 || max_moves < 0)
        return DPSO_ERR_ARG;
    if (n > DPSO_MAX_N || (kind == 1 && node_swap_tiled_rows(n) == 0)) return DPSO_ERR_RANGE;
    if (pairs_host) *pairs_host = 0;
    if (moves_host) *moves_host = 0;
    if (count == 0) return DPSO_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // scratch: error word, work queue, counters, and the one-problem task list
    struct Scratch {
        int err;
        unsigned int queue;
        unsigned long long pairs, moves;
        TwoOptTask task;
        int toff[2];
    };
    Scratch* scratch = nullptr;
    if (cudaMallocAsync(&scratch, sizeof(Scratch), st) != cudaSuccess) {
        cudaGetLastError();
        return DPSO_ERR_NO_MEMORY;
    }
    int* err = &scratch->err;
    int herr = 0;
    unsigned long long counters[2] = {0, 0};
    Scratch host{};
    host.toff[1] = count;
    cudaError_t e = cudaMemcpyAsync(scratch, &host, sizeof(Scratch), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_check_cost_limit(C_dev, n, n, kind ? DPSO_NODE_SWAP_COST_MAX : DPSO_COST_MAX, err, st);
    if (e == cudaSuccess) {
        tours_valid_kernel<<<count, 256, n, st>>>(tours_dev, n, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    int* Cs = nullptr;
    if (e == cudaSuccess && herr == 0 && two_opt_tiled_rows(n) > 0) {
        if (cudaMallocAsync(&Cs, sizeof(int) * 4 * static_cast<size_t>(n) * shifted_ld(n), st) !=
            cudaSuccess) {
            cudaGetLastError();
            Cs = nullptr;  // 2-opt falls back to the kernel that stages rows itself
            if (kind == 1) e = cudaErrorMemoryAllocation;
        } else {
            e = build_shifted_copies(C_dev, n, n, Cs, st);
        }
    }
    if (e == cudaSuccess && herr == 0) {
        e = launch_fitness(C_dev, n, n, tours_dev, n, count, reinterpret_cast<long long*>(cost_dev),
                           st);
        TwoOptTask& a = host.task;
        a.C = C_dev;
        a.Cs = Cs;
        a.ldc = n;
        a.n = n;
        a.tours = tours_dev;
        a.ldt = n;
        a.count = count;
        a.cost = reinterpret_cast<long long*>(cost_dev);
        a.max_moves = max_moves;
        a.pairs = &scratch->pairs;
        a.moves = &scratch->moves;
        a.status = err;
        a.kind = kind;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&scratch->task, &host.task, sizeof(TwoOptTask),
                                cudaMemcpyHostToDevice, st);
        TwoOptBatch tb{&scratch->task, scratch->toff, 1, count, n, Cs != nullptr, 0,
                       &scratch->queue};
        tb.kind = kind;
        if (e == cudaSuccess) e = launch_two_opt(tb, sms, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(counters, &scratch->pairs, sizeof(counters), cudaMemcpyDeviceToHost,
                                st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host.task is read by the copy
    }
    cudaFreeAsync(scratch, st);
    if (Cs) cudaFreeAsync(Cs, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaErrorMemoryAllocation) return DPSO_ERR_NO_MEMORY;
    if (e != cudaSuccess) return DPSO_ERR_CUDA;
    if (herr == DPSO_ERR_INTERNAL || herr == DPSO_ERR_TIMEOUT) return herr;
    if (herr & 1) return DPSO_ERR_ARG;
    if (herr & 2) return DPSO_ERR_RANGE;
    if (pairs_host) *pairs_host = static_cast<int64_t>(counters[0]);
    if (moves_host) *moves_host = static_cast<int64_t>(counters[1]);
    return DPSO_OK;
}

}  // namespace

extern "C" {

int dpso_two_opt(const int32_t* C_dev, int32_t n, uint16_t* tours_dev, int32_t count,
                 int64_t* cost_dev, int32_t max_moves, int64_t* pairs_host, int64_t* moves_host,
                 void* stream) {
    return exchange_tours(0, C_dev, n, tours_dev, count, cost_dev, max_moves, pairs_host,
                          moves_host, stream);
}

int dpso_node_swap(const int32_t* C_dev, int32_t n, uint16_t* tours_dev, int32_t count,
                   int64_t* cost_dev, int32_t max_moves, int64_t* pairs_host,
                   int64_t* moves_host, void* stream) {
    return exchange_tours(1, C_dev, n, tours_dev, count, cost_dev, max_moves, pairs_host,
                          moves_host, stream);
}

int dpso_philox_draws(uint64_t seed, uint32_t phase, uint32_t iteration, uint32_t particle,
                      int32_t count, uint32_t* out_dev, void* stream) {
    if (count < 0 || (count > 0 && !out_dev)) return DPSO_ERR_ARG;
    CK(launch_philox_draws(seed, phase, iteration, particle, count, out_dev,
                           static_cast<cudaStream_t>(stream)));
    return DPSO_OK;
}

int dpso_init(dpso_swarm** out, const int32_t* C_dev, int32_t n, const int32_t* tags_host,
              const dpso_params* p, uint64_t seed, void* stream) {
    if (!out || !C_dev) return DPSO_ERR_ARG;
    *out = nullptr;
    int st = validate_params(p);
    if (st) return st;
    if (n < 3) return DPSO_ERR_ARG;
    if (n > DPSO_MAX_N) return DPSO_ERR_RANGE;
    const bool det = (p->flags & DPSO_FLAG_DET_INIT) && tags_host;
    if (det) {
        std::vector<std::array<int, 3>> tg(n);
        for (int i = 0; i < n; ++i) {
            for (int a = 0; a < 3; ++a) {
                tg[i][a] = tags_host[3 * i + a];
                if (tg[i][a] < 0) return DPSO_ERR_ARG;
            }
        }
        std::sort(tg.begin(), tg.end());
        for (int i = 1; i < n; ++i)
            if (tg[i] == tg[i - 1]) return DPSO_ERR_ARG;
    }

    dpso_swarm* s = new dpso_swarm();
    cudaStream_t ust = static_cast<cudaStream_t>(stream);
    s->last = ust;
    s->prm = *p;
    auto fail = [&](int code) {
        free_swarm(s);
        return code;
    };
    if (cudaGetDevice(&s->device) != cudaSuccess) return fail(DPSO_ERR_CUDA);
    if (cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) !=
        cudaSuccess)
        return fail(DPSO_ERR_CUDA);
    if (two_opt_rows(n) == 0) return fail(DPSO_ERR_RANGE);
    const bool node_swap = (p->flags & DPSO_FLAG_TWO_OPT) && (p->flags & DPSO_FLAG_NODE_SWAP);
    if (node_swap && node_swap_tiled_rows(n) == 0) return fail(DPSO_ERR_RANGE);

    Consts& k = s->k;
    k.n = n;
    k.S = p->swarm;
    k.ldc = round_up(n, 32);
    k.ldn = round_up(n, 8);
    k.flags = p->flags;
    k.mut_period = p->mut_period;
    k.mut_swaps = p->mut_swaps;
    k.trigger = p->two_opt_trigger;
    k.max_moves = p->max_moves;
    k.stall_limit = p->stall_limit;
    k.w_q = q32(p->w);
    k.phi1_q = q32(p->phi1);
    k.phi2_q = q32(p->phi2);
    k.seed = seed;
    const size_t S = static_cast<size_t>(k.S), ldn = static_cast<size_t>(k.ldn);

    if ((st = dalloc(&s->C, static_cast<size_t>(n) * k.ldc, ust)) ||
        (st = dalloc(&s->X, S * ldn, ust)) || (st = dalloc(&s->V, S * ldn, ust)) ||
        (st = dalloc(&s->P, S * ldn, ust)) || (st = dalloc(&s->G, ldn, ust)) ||
        (st = dalloc(&s->F, S, ust)) || (st = dalloc(&s->PF, S, ust)) ||
        (st = dalloc(&s->hash, S, ust)) || (st = dalloc(&s->dup, S, ust)) ||
        (st = dalloc(&s->kept, S, ust)) || (st = dalloc(&s->order, S, ust)) ||
        (st = dalloc(&s->ctl, 1, ust)) ||
        (st = dalloc(&s->meta, 1, ust)))
        return fail(st);
    if ((st = ensure_history(s, 1024))) return fail(st);
    s->d = SwarmDev{s->C,    s->X,   s->V,    s->P,   s->G,    s->F,
                    s->PF,   s->hash, s->dup, s->kept, s->ctl, s->order};
    {
        // identity until the first generation ranks the particles
        std::vector<int> ident(S);
        for (size_t i = 0; i < S; ++i) ident[i] = static_cast<int>(i);
        if (cudaMemcpyAsync(s->order, ident.data(), sizeof(int) * S, cudaMemcpyHostToDevice,
                            ust) != cudaSuccess ||
            cudaStreamSynchronize(ust) != cudaSuccess)
            return fail(DPSO_ERR_CUDA);
    }

    int* err = nullptr;
    uint16_t* orders = nullptr;
    int* tags_dev = nullptr;
    if ((st = dalloc(&err, 1, ust))) return fail(st);
    auto fail2 = [&](int code) {
        cudaFree(err);
        cudaFree(orders);
        cudaFree(tags_dev);
        return fail(code);
    };
    if (cudaMemcpy2DAsync(s->C, sizeof(int) * k.ldc, C_dev, sizeof(int) * n, sizeof(int) * n, n,
                          cudaMemcpyDeviceToDevice, ust) != cudaSuccess ||
        launch_check_cost_limit(s->C, n, k.ldc,
                                node_swap ? DPSO_NODE_SWAP_COST_MAX : DPSO_COST_MAX, err,
                                ust) != cudaSuccess)
        return fail2(DPSO_ERR_CUDA);
    if (det) {
        s->n_det = static_cast<int>((static_cast<long long>(k.S) * p->det_frac_pct) / 100);
        s->n_det = std::min(k.S, std::max(1, s->n_det));
        if ((st = dalloc(&orders, 8 * ldn, ust)) ||
            (st = dalloc(&tags_dev, 3 * static_cast<size_t>(n), ust)))
            return fail2(st);
        if (cudaMemcpyAsync(tags_dev, tags_host, sizeof(int) * 3 * n, cudaMemcpyHostToDevice, ust) !=
                cudaSuccess ||
            launch_det_orders(tags_dev, n, orders, k.ldn, err, ust) != cudaSuccess)
            return fail2(DPSO_ERR_CUDA);
    }
    int herr = 0;
    if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ust) != cudaSuccess ||
        cudaStreamSynchronize(ust) != cudaSuccess)
        return fail2(DPSO_ERR_CUDA);
    if (herr & 1) return fail2(DPSO_ERR_ARG);
    if (herr & 2) return fail2(DPSO_ERR_RANGE);
    if ((p->flags & DPSO_FLAG_TWO_OPT) && two_opt_tiled_rows(n) > 0) {
        if ((st = dalloc(&s->Cs, static_cast<size_t>(4) * n * shifted_ld(n), ust)))
            return fail2(st);
        if (build_shifted_copies(s->C, k.ldc, n, s->Cs, ust) != cudaSuccess)
            return fail2(DPSO_ERR_CUDA);
    }
    {
        SwarmMeta m{};
        m.desc.k = k;
        m.desc.d = s->d;
        m.task = swarm_task(s);
        m.off[1] = k.S;
        m.toff[1] = k.S;
        if (cudaMemcpyAsync(s->meta, &m, sizeof(m), cudaMemcpyHostToDevice, ust) != cudaSuccess ||
            cudaStreamSynchronize(ust) != cudaSuccess)
            return fail2(DPSO_ERR_CUDA);
    }

    if (launch_init_particles(k, s->d, orders, s->n_det, ust) != cudaSuccess ||
        launch_fitness(s->C, k.ldc, n, s->X, k.ldn, k.S, s->F, ust) != cudaSuccess ||
        cudaMemcpyAsync(s->PF, s->F, sizeof(long long) * S, cudaMemcpyDeviceToDevice, ust) !=
            cudaSuccess ||
        launch_gbest_init(k, s->d, ust) != cudaSuccess ||
        cudaMemcpyAsync(&s->ctl->n_det, &s->n_det, sizeof(int), cudaMemcpyHostToDevice, ust) !=
            cudaSuccess ||
        cudaStreamSynchronize(ust) != cudaSuccess)
        return fail2(DPSO_ERR_CUDA);
    cudaFree(err);
    cudaFree(orders);
    cudaFree(tags_dev);

    if (cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) != cudaSuccess)
        return fail(DPSO_ERR_CUDA);
    if ((st = capture(s, 0)) || (st = capture(s, 1))) return fail(st);
    *out = s;
    return DPSO_OK;
}

int dpso_step(dpso_swarm* s, int32_t iterations, void* stream) {
    if (!s || iterations < 0) return DPSO_ERR_ARG;
    if (iterations == 0) return DPSO_OK;
    DeviceGuard g(s->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (st != s->last) {
        // order this call after everything already enqueued on the previous stream
        CK(cudaStreamSynchronize(s->last));
        s->last = st;
    }
    const int st2 = ensure_history(s, s->t_host + iterations);
    if (st2) return st2;
    for (int it = 0; it < iterations; ++it) {
        const int t = s->t_host + 1 + it;
        const bool mut = (s->k.flags & DPSO_FLAG_MUTATION) && (t % s->k.mut_period == 0);
        if (s->timing) CK(launch_generation_timed(s, mut, st));
        else CK(cudaGraphLaunch(s->exec[mut ? 1 : 0], st));
    }
    s->t_host += iterations;
    return DPSO_OK;
}

int dpso_get_best(dpso_swarm* s, int32_t* tour_host, int64_t* cost) {
    if (!s || !tour_host || !cost) return DPSO_ERR_ARG;
    DeviceGuard g(s->device);
    Ctl c;
    const int st = read_ctl(s, &c);
    if (st) return st;
    std::vector<uint16_t> tmp(s->k.n);
    CK(cudaMemcpy(tmp.data(), s->G, sizeof(uint16_t) * s->k.n, cudaMemcpyDeviceToHost));
    for (int i = 0; i < s->k.n; ++i) tour_host[i] = tmp[i];
    *cost = c.gf;
    return c.status ? c.status : DPSO_OK;
}

int dpso_get_history(dpso_swarm* s, int64_t* gbest_host, int32_t cap, int32_t* len) {
    if (!s || !len || cap < 0 || (cap > 0 && !gbest_host)) return DPSO_ERR_ARG;
    DeviceGuard g(s->device);
    Ctl c;
    const int st = read_ctl(s, &c);
    if (st) return st;
    *len = c.t;
    const int k = std::min(cap, c.t);
    if (k > 0) CK(cudaMemcpy(gbest_host, s->hist, sizeof(int64_t) * k, cudaMemcpyDeviceToHost));
    return DPSO_OK;
}

int dpso_get_stats(dpso_swarm* s, dpso_stats* out) {
    if (!s || !out) return DPSO_ERR_ARG;
    DeviceGuard g(s->device);
    Ctl c;
    const int st = read_ctl(s, &c);
    if (st) return st;
    memset(out, 0, sizeof(*out));
    out->iterations = c.t;
    out->stalled = c.done;
    out->gbest_cost = c.gf;
    out->two_opt_pairs = static_cast<int64_t>(c.pairs);
    out->two_opt_moves = static_cast<int64_t>(c.moves);
    out->two_opt_runs = static_cast<int64_t>(c.runs);
    out->two_opt_evaluated = static_cast<int64_t>(c.evals);
    out->device_status = c.status;
    return DPSO_OK;
}

int dpso_get_state(dpso_swarm* s, void* buf, size_t* bytes) {
    if (!s || !bytes) return DPSO_ERR_ARG;
    DeviceGuard g(s->device);
    Ctl c;
    int st = read_ctl(s, &c);
    if (st) return st;
    const size_t n = s->k.n, S = s->k.S;
    const size_t need = sizeof(StateHeader) + 3 * S * n * sizeof(uint16_t) + n * sizeof(uint16_t) +
                        2 * S * sizeof(int64_t) + static_cast<size_t>(c.t) * sizeof(int64_t);
    if (!buf) {
        *bytes = need;
        return DPSO_OK;
    }
    if (*bytes < need) return DPSO_ERR_ARG;
    unsigned char* o = static_cast<unsigned char*>(buf);
    StateHeader h{};
    h.magic = kStateMagic;
    h.version = kStateVersion;
    h.n = s->k.n;
    h.S = s->k.S;
    h.t = c.t;
    h.stall = c.stall;
    h.done = c.done;
    h.n_det = c.n_det;
    h.gf = c.gf;
    h.pairs = c.pairs;
    h.moves = c.moves;
    h.runs = c.runs;
    h.seed = s->k.seed;
    h.prm = s->prm;
    memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    const size_t row = n * sizeof(uint16_t), pitch = s->k.ldn * sizeof(uint16_t);
    for (uint16_t* A : {s->X, s->V, s->P}) {
        CK(cudaMemcpy2D(o, row, A, pitch, row, S, cudaMemcpyDeviceToHost));
        o += row * S;
    }
    CK(cudaMemcpy(o, s->G, row, cudaMemcpyDeviceToHost));
    o += row;
    CK(cudaMemcpy(o, s->F, S * sizeof(int64_t), cudaMemcpyDeviceToHost));
    o += S * sizeof(int64_t);
    CK(cudaMemcpy(o, s->PF, S * sizeof(int64_t), cudaMemcpyDeviceToHost));
    o += S * sizeof(int64_t);
    if (c.t > 0) CK(cudaMemcpy(o, s->hist, sizeof(int64_t) * c.t, cudaMemcpyDeviceToHost));
    *bytes = need;
    return DPSO_OK;
}

int dpso_set_state(dpso_swarm* s, const void* buf, size_t bytes) {
    if (!s || !buf || bytes < sizeof(StateHeader)) return DPSO_ERR_ARG;
    DeviceGuard g(s->device);
    StateHeader h;
    memcpy(&h, buf, sizeof(h));
    if (h.magic != kStateMagic || h.version != kStateVersion || h.n != s->k.n || h.S != s->k.S ||
        h.seed != s->k.seed || memcmp(&h.prm, &s->prm, sizeof(dpso_params)) != 0 || h.t < 0)
        return DPSO_ERR_ARG;
    const size_t n = s->k.n, S = s->k.S;
    const size_t need = sizeof(StateHeader) + 3 * S * n * sizeof(uint16_t) + n * sizeof(uint16_t) +
                        2 * S * sizeof(int64_t) + static_cast<size_t>(h.t) * sizeof(int64_t);
    if (bytes < need) return DPSO_ERR_ARG;
    CK(cudaStreamSynchronize(s->last));
    int st = ensure_history(s, std::max(h.t, 1));
    if (st) return st;
    // every copy is ordered on the swarm's own stream, which is then waited
    // for: a copy from pageable memory may return before its transfer lands,
    // and the caller's next launch may be on a non-blocking stream
    cudaStream_t st0 = s->last;
    const unsigned char* o = static_cast<const unsigned char*>(buf) + sizeof(h);
    const size_t row = n * sizeof(uint16_t), pitch = s->k.ldn * sizeof(uint16_t);
    for (uint16_t* A : {s->X, s->V, s->P}) {
        CK(cudaMemcpy2DAsync(A, pitch, o, row, row, S, cudaMemcpyHostToDevice, st0));
        o += row * S;
    }
    CK(cudaMemcpyAsync(s->G, o, row, cudaMemcpyHostToDevice, st0));
    o += row;
    CK(cudaMemcpyAsync(s->F, o, S * sizeof(int64_t), cudaMemcpyHostToDevice, st0));
    o += S * sizeof(int64_t);
    CK(cudaMemcpyAsync(s->PF, o, S * sizeof(int64_t), cudaMemcpyHostToDevice, st0));
    o += S * sizeof(int64_t);
    if (h.t > 0)
        CK(cudaMemcpyAsync(s->hist, o, sizeof(int64_t) * h.t, cudaMemcpyHostToDevice, st0));
    Ctl c;
    CK(cudaMemcpyAsync(&c, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st0));
    CK(cudaStreamSynchronize(st0));
    c.gf = h.gf;
    c.gf_start = h.gf;
    c.t = h.t;
    c.stall = h.stall;
    c.done = h.done;
    c.run_two_opt = 0;
    c.status = DPSO_OK;
    c.n_det = h.n_det;
    c.queue = 0;
    c.pairs = h.pairs;
    c.moves = h.moves;
    c.runs = h.runs;
    CK(cudaMemcpyAsync(s->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, st0));
    CK(cudaStreamSynchronize(st0));
    s->t_host = h.t;
    return DPSO_OK;
}

int dpso_set_timing(dpso_swarm* s, int on) {
    if (!s) return DPSO_ERR_ARG;
    DeviceGuard g(s->device);
    CK(cudaStreamSynchronize(s->last));
    s->pending.clear();
    s->acc = dpso_timing{};
    s->timing = on != 0;
    return DPSO_OK;
}

int dpso_get_timing(dpso_swarm* s, dpso_timing* out) {
    if (!s || !out) return DPSO_ERR_ARG;
    DeviceGuard g(s->device);
    CK(cudaStreamSynchronize(s->last));
    const int st = collect_timing(s);
    if (st) return st;
    *out = s->acc;
    return DPSO_OK;
}

void dpso_destroy(dpso_swarm* s) {
    if (!s) return;
    DeviceGuard g(s->device);
    cudaStreamSynchronize(s->last);
    free_swarm(s);
}

// ------------------------------------------------------------------ batches

}  // extern "C"

struct dpso_batch {
    // One persistent 2-opt launch per class of members sharing a launch shape.
    struct TwoOptClass {
        TwoOptTask* tasks = nullptr;  // device, the class's members by descending n
        int* toff = nullptr;          // device, tour offsets (nprob + 1)
        unsigned int* queue = nullptr;
        TwoOptBatch tb{};
    };
    int device = 0, num_sms = 0;
    std::vector<dpso_swarm*> members;
    SwarmDesc* desc = nullptr;  // device, members in creation order
    int* off = nullptr;         // device, ninst + 1
    BatchView bv{};
    bool any_two_opt = false;
    bool shifted = true;                 // every exchanging member has the shifted copies
    std::vector<TwoOptTask> tasks;       // host: every exchanging member, by descending n
    std::vector<TwoOptClass> cls;
    std::vector<cudaStream_t> side;      // capture streams of the classes after the first
    std::vector<cudaEvent_t> ev;         // fork, then one join per side stream
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t last = nullptr;
};

namespace {

void free_classes(dpso_batch* b) {
    for (auto& c : b->cls) {
        void* bufs[] = {c.tasks, c.toff, c.queue};
        for (void* p : bufs)
            if (p) cudaFree(p);
    }
    b->cls.clear();
}

void free_batch(dpso_batch* b) {
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    free_classes(b);
    void* bufs[] = {b->desc, b->off};
    for (void* p : bufs)
        if (p) cudaFree(p);
    for (cudaStream_t s : b->side) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

// Default launch shape of the tiled kernel for tours of n viewpoints and the
// resident CTAs per SM it gets (all zero: the general kernel).
struct ShapeKey {
    int kind = 0, rows = 0, tpc = 0, tg = 0, ctas = 0;
    bool operator==(const ShapeKey& o) const {
        return kind == o.kind && rows == o.rows && tpc == o.tpc && tg == o.tg && ctas == o.ctas;
    }
};

ShapeKey default_shape(int n, bool shifted, int kind) {
    ShapeKey k;
    k.kind = kind;
    if (kind == 1) {  // node swap: one kernel shape per tile height
        k.rows = node_swap_tiled_rows(n);
        return k;
    }
    if (!shifted || two_opt_tiled_rows(n) == 0) return k;
    k.rows = two_opt_tiled_rows(n);
    k.tpc = two_opt_tiled_tpc(n, k.rows);
    k.tg = two_opt_tiled_tg(n, k.rows, k.tpc);
    k.ctas = two_opt_tiled_ctas(n, k.rows, k.tpc, k.tg);
    return k;
}

// Splits the exchanging members into launch classes: runs of members (by
// descending n) whose default shape and resident CTAs per SM agree, each
// launched with that shape; or one class with a pinned shape for all.
int build_classes(dpso_batch* b, const dpso_two_opt_shape* pinned) {
    free_classes(b);
    const int nt = static_cast<int>(b->tasks.size());
    std::vector<std::pair<int, int>> runs;  // [first, last) task ranges
    std::vector<ShapeKey> keys;
    for (int i = 0; i < nt; ++i) {
        ShapeKey k;
        if (pinned)
            k.kind = b->tasks[i].kind;  // one class per exchange kind
        else
            k = default_shape(b->tasks[i].n, b->tasks[i].Cs != nullptr, b->tasks[i].kind);
        if (i == 0 || !(k == keys.back())) {
            runs.push_back({i, i + 1});
            keys.push_back(k);
        } else {
            runs.back().second = i + 1;
        }
    }
    for (size_t c = 0; c < runs.size(); ++c) {
        dpso_batch::TwoOptClass cl;
        const int first = runs[c].first, cnt = runs[c].second - runs[c].first;
        std::vector<int> toff(1, 0);
        int max_n = 0;
        bool shifted = true;  // the tiled kernel needs every member's shifted copies
        for (int i = first; i < first + cnt; ++i) {
            toff.push_back(toff.back() + b->tasks[i].count);
            max_n = std::max(max_n, b->tasks[i].n);
            shifted = shifted && b->tasks[i].Cs != nullptr;
        }
        int st = DPSO_OK;
        if ((st = dalloc(&cl.tasks, cnt, b->last)) || (st = dalloc(&cl.toff, cnt + 1, b->last)) ||
            (st = dalloc(&cl.queue, 1, b->last))) {
            b->cls.push_back(cl);
            return st;
        }
        b->cls.push_back(cl);
        CK(cudaMemcpyAsync(cl.tasks, b->tasks.data() + first, sizeof(TwoOptTask) * cnt,
                           cudaMemcpyHostToDevice, b->last));
        CK(cudaMemcpyAsync(cl.toff, toff.data(), sizeof(int) * (cnt + 1), cudaMemcpyHostToDevice,
                           b->last));
        CK(cudaStreamSynchronize(b->last));  // the host vectors go out of scope
        TwoOptBatch& tb = b->cls.back().tb;
        tb = TwoOptBatch{cl.tasks, cl.toff, cnt, toff.back(), max_n, shifted, 0, cl.queue};
        tb.kind = keys[c].kind;
        if (keys[c].kind == 1) {
            // node swap: the tile height follows max_n
        } else if (pinned) {
            tb.rows = pinned->rows;
            tb.tpc = pinned->tours_per_cta;
            tb.tg = pinned->tiles_in_flight;
        } else if (keys[c].rows > 0) {
            tb.rows = keys[c].rows;
            tb.tpc = keys[c].tpc;
            tb.tg = keys[c].tg;
        }
    }
    // one capture stream and one join event per class after the first
    while (b->side.size() + 1 < b->cls.size()) {
        cudaStream_t s = nullptr;
        CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        b->side.push_back(s);
    }
    while (b->ev.size() < b->cls.size()) {
        cudaEvent_t e = nullptr;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->ev.push_back(e);
    }
    return DPSO_OK;
}

// One generation of every member: the particle update, mutation, gbest, the
// exchange order, then the classes' 2-opt launches side by side (forked from
// and joined back into `st`), then the second gbest pass.
cudaError_t enqueue_batch_classes(dpso_batch* b, cudaStream_t st) {
    cudaError_t e = launch_move(b->bv, st);
    if (e == cudaSuccess) e = launch_mutation(b->bv, st);
    if (e == cudaSuccess) e = launch_gbest(b->bv, 0, st);
    if (e != cudaSuccess || !b->any_two_opt) return e;
    e = launch_rank_cost(b->bv, st);
    if (e == cudaSuccess && b->cls.size() > 1) e = cudaEventRecord(b->ev[0], st);
    for (size_t c = 1; c < b->cls.size() && e == cudaSuccess; ++c) {
        cudaStream_t s = b->side[c - 1];
        e = cudaStreamWaitEvent(s, b->ev[0], 0);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->cls[c].queue, 0, sizeof(unsigned int), s);
        if (e == cudaSuccess) e = launch_two_opt(b->cls[c].tb, b->num_sms, s);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev[c], s);
    }
    if (e == cudaSuccess && !b->cls.empty()) {
        e = cudaMemsetAsync(b->cls[0].queue, 0, sizeof(unsigned int), st);
        if (e == cudaSuccess) e = launch_two_opt(b->cls[0].tb, b->num_sms, st);
    }
    for (size_t c = 1; c < b->cls.size() && e == cudaSuccess; ++c)
        e = cudaStreamWaitEvent(st, b->ev[c], 0);
    if (e == cudaSuccess) e = launch_gbest(b->bv, 1, st);
    return e;
}

int capture_batch(dpso_batch* b) {
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
    const cudaError_t e = enqueue_batch_classes(b, b->cap);
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return DPSO_ERR_CUDA;
    }
    const cudaError_t e3 = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    return e3 == cudaSuccess ? DPSO_OK : DPSO_ERR_CUDA;
}

// Times every shape that fits a class on scratch copies of its tours (gates
// ignored, at most kProbeMoves moves per tour) and keeps the fastest.
int autotune_class(dpso_batch* b, dpso_batch::TwoOptClass& cl, cudaStream_t st) {
    constexpr int kProbeMoves = 8;
    if (cl.tb.kind != 0 || cl.tb.nprob <= 0 || !cl.tb.shifted ||
        two_opt_tiled_rows(cl.tb.max_n) == 0)
        return DPSO_OK;
    std::vector<TwoOptTask> tasks(cl.tb.nprob);
    CK(cudaMemcpy(tasks.data(), cl.tasks, sizeof(TwoOptTask) * cl.tb.nprob,
                  cudaMemcpyDeviceToHost));
    const std::vector<TwoOptTask> orig = tasks;
    std::vector<void*> scratch;
    TwoOptTask* dtasks = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&](int code) {
        cudaStreamSynchronize(st);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (dtasks) cudaFree(dtasks);
        for (void* p : scratch) cudaFree(p);
        return code;
    };
    int st2 = DPSO_OK;
    for (TwoOptTask& t : tasks) {
        uint16_t* tours = nullptr;
        long long* cost = nullptr;
        unsigned long long* cnt = nullptr;
        int* status = nullptr;
        if ((st2 = dalloc(&tours, static_cast<size_t>(t.count) * t.ldt, st)) ||
            (st2 = dalloc(&cost, t.count, st)) || (st2 = dalloc(&cnt, 2, st)) ||
            (st2 = dalloc(&status, 1, st)))
            return cleanup(st2);
        scratch.insert(scratch.end(), {tours, cost, cnt, status});
        t.tours = tours;
        t.cost = cost;
        t.pbest = nullptr;
        t.pcost = nullptr;
        t.gate = nullptr;
        t.pairs = cnt;
        t.moves = cnt + 1;
        t.status = status;
        t.max_moves = kProbeMoves;
        t.order = nullptr;
        t.evals = nullptr;
    }
    if ((st2 = dalloc(&dtasks, tasks.size(), st))) return cleanup(st2);
    if (cudaMemcpyAsync(dtasks, tasks.data(), sizeof(TwoOptTask) * tasks.size(),
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        return cleanup(DPSO_ERR_CUDA);
    float best = 1e30f;
    int rows_b = 0, tpc_b = 0, tg_b = 0;
    constexpr int kShapes[4][2] = {{1, 1}, {2, 1}, {4, 1}, {1, 2}};  // (tours per CTA, tiles)
    for (int rows : {32, 30, 24, 16, 8}) {
        for (const auto& sh : kShapes) {
            const int tpc = sh[0], tg = sh[1];
            if (!two_opt_tiled_fits(cl.tb.max_n, rows, tpc, tg)) continue;
            for (size_t i = 0; i < tasks.size(); ++i) {  // restore the tours
                if (cudaMemcpy2DAsync(tasks[i].tours, sizeof(uint16_t) * tasks[i].ldt,
                                      orig[i].tours, sizeof(uint16_t) * orig[i].ldt,
                                      sizeof(uint16_t) * tasks[i].n, tasks[i].count,
                                      cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                    cudaMemcpyAsync(tasks[i].cost, orig[i].cost,
                                    sizeof(long long) * tasks[i].count, cudaMemcpyDeviceToDevice,
                                    st) != cudaSuccess)
                    return cleanup(DPSO_ERR_CUDA);
            }
            TwoOptBatch tb = cl.tb;
            tb.tasks = dtasks;
            if (cudaMemsetAsync(tb.queue, 0, sizeof(unsigned int), st) != cudaSuccess ||
                cudaEventRecord(e0, st) != cudaSuccess)
                return cleanup(DPSO_ERR_CUDA);
            const cudaError_t le = launch_two_opt_tiled(tb, rows, tpc, tg, b->num_sms, st);
            if (le == cudaErrorInvalidValue || le == cudaErrorInvalidConfiguration) {
                cudaGetLastError();  // this shape does not fit: skip it
                continue;
            }
            float ms = 0.f;
            if (le != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
                cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                return cleanup(DPSO_ERR_CUDA);
            if (ms < best) {
                best = ms;
                rows_b = rows;
                tpc_b = tpc;
                tg_b = tg;
            }
        }
    }
    if (rows_b > 0) {
        cl.tb.rows = rows_b;
        cl.tb.tpc = tpc_b;
        cl.tb.tg = tg_b;
    }
    return cleanup(DPSO_OK);
}

}  // namespace

extern "C" {

int dpso_batch_create(dpso_batch** out, dpso_swarm* const* swarms, int32_t count, void* stream) {
    if (!out || !swarms || count < 1) return DPSO_ERR_ARG;
    *out = nullptr;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    for (int i = 0; i < count; ++i) {
        if (!swarms[i] || swarms[i]->device != dev) return DPSO_ERR_ARG;
        for (int j = 0; j < i; ++j)
            if (swarms[j] == swarms[i]) return DPSO_ERR_ARG;
    }
    dpso_batch* b = new dpso_batch();
    b->device = dev;
    b->last = static_cast<cudaStream_t>(stream);
    b->members.assign(swarms, swarms + count);
    auto fail = [&](int code) {
        free_batch(b);
        return code;
    };
    if (cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(DPSO_ERR_CUDA);
    std::vector<SwarmDesc> desc(count);
    std::vector<int> off(count + 1, 0);
    int max_ldn = 0, max_S = 0, arrays = 5;
    for (int i = 0; i < count; ++i) {
        const dpso_swarm* s = swarms[i];
        desc[i].k = s->k;
        desc[i].d = s->d;
        off[i + 1] = off[i] + s->k.S;
        max_ldn = std::max(max_ldn, s->k.ldn);
        max_S = std::max(max_S, s->k.S);
        arrays = std::max(arrays, swarm_arrays(s->k));
    }
    // exchanging members by decreasing tour length: long tours start first
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return swarms[x]->k.n > swarms[y]->k.n; });
    for (int i : order) {
        if (!(swarms[i]->k.flags & DPSO_FLAG_TWO_OPT)) continue;
        b->tasks.push_back(swarm_task(swarms[i]));
        b->shifted = b->shifted && swarms[i]->Cs != nullptr;
    }
    b->any_two_opt = !b->tasks.empty();
    int st = DPSO_OK;
    if ((st = dalloc(&b->desc, count, b->last)) || (st = dalloc(&b->off, count + 1, b->last)))
        return fail(st);
    if (cudaMemcpyAsync(b->desc, desc.data(), sizeof(SwarmDesc) * count, cudaMemcpyHostToDevice,
                        b->last) != cudaSuccess ||
        cudaMemcpyAsync(b->off, off.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice,
                        b->last) != cudaSuccess ||
        cudaStreamSynchronize(b->last) != cudaSuccess)
        return fail(DPSO_ERR_CUDA);
    b->bv = BatchView{b->desc, b->off, count, off[count], max_ldn, arrays, max_S};
    if ((st = build_classes(b, nullptr))) return fail(st);
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
        return fail(DPSO_ERR_CUDA);
    if ((st = capture_batch(b))) return fail(st);
    *out = b;
    return DPSO_OK;
}

int dpso_batch_step(dpso_batch* b, int32_t iterations, void* stream) {
    if (!b || iterations < 0) return DPSO_ERR_ARG;
    if (iterations == 0) return DPSO_OK;
    DeviceGuard g(b->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (dpso_swarm* s : b->members) {
        if (s->last != st) {
            CK(cudaStreamSynchronize(s->last));
            s->last = st;
        }
        const int r = ensure_history(s, s->t_host + iterations);
        if (r) return r;
    }
    if (b->last != st) {
        CK(cudaStreamSynchronize(b->last));
        b->last = st;
    }
    for (int it = 0; it < iterations; ++it) CK(cudaGraphLaunch(b->graph, st));
    for (dpso_swarm* s : b->members) s->t_host += iterations;
    return DPSO_OK;
}

int dpso_batch_autotune(dpso_batch* b, dpso_two_opt_shape* chosen, void* stream) {
    if (!b) return DPSO_ERR_ARG;
    DeviceGuard g(b->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaStreamSynchronize(b->last));
    b->last = st;
    for (auto& cl : b->cls) {
        const int r = autotune_class(b, cl, st);
        if (r) return r;
    }
    const int r = capture_batch(b);
    if (r) return r;
    if (chosen) {  // the shape of the class holding the longest tours
        *chosen = dpso_two_opt_shape{0, 0, 0};
        if (!b->cls.empty()) {
            const TwoOptBatch& tb = b->cls[0].tb;
            int rows = tb.rows, tpc = tb.tpc, tg = tb.tg;
            if (rows <= 0) {  // the class runs the default shape for its tours
                int sms = 0;
                CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
                two_opt_default_shape(tb.max_n, tb.total, sms, &rows, &tpc, &tg);
            } else {
                if (tpc <= 0) tpc = two_opt_tiled_tpc(tb.max_n, rows);
                if (tg <= 0) tg = two_opt_tiled_tg(tb.max_n, rows, tpc);
            }
            *chosen = dpso_two_opt_shape{rows, tpc, tg};
        }
    }
    return DPSO_OK;
}

int dpso_two_opt_default_shape(int32_t n, int32_t count, int32_t num_sms,
                               dpso_two_opt_shape* out) {
    if (!out || n < 3 || count < 0 || num_sms < 1) return DPSO_ERR_ARG;
    *out = dpso_two_opt_shape{0, 0, 0};
    if (n > DPSO_MAX_N) return DPSO_OK;
    int rows = 0, tpc = 0, tg = 0;
    two_opt_default_shape(n, count, num_sms, &rows, &tpc, &tg);
    if (rows > 0) *out = dpso_two_opt_shape{rows, tpc, tg};
    return DPSO_OK;
}

int dpso_batch_set_two_opt_shape(dpso_batch* b, const dpso_two_opt_shape* shape) {
    if (!b) return DPSO_ERR_ARG;
    DeviceGuard g(b->device);
    const bool defaults =
        !shape || (shape->rows == 0 && shape->tours_per_cta == 0 && shape->tiles_in_flight == 0);
    if (!defaults) {
        int max_n = 0;  // the shape applies to the edge-exchange (2-opt) members
        for (const TwoOptTask& t : b->tasks)
            if (t.kind == 0) max_n = std::max(max_n, t.n);
        if (!b->shifted || max_n == 0 ||
            !two_opt_tiled_fits(max_n, shape->rows, shape->tours_per_cta, shape->tiles_in_flight))
            return DPSO_ERR_ARG;
    }
    CK(cudaStreamSynchronize(b->last));
    const int st = build_classes(b, defaults ? nullptr : shape);
    if (st) return st;
    return capture_batch(b);
}

void dpso_batch_destroy(dpso_batch* b) {
    if (!b) return;
    DeviceGuard g(b->device);
    cudaStreamSynchronize(b->last);
    free_batch(b);
}

int dpso_plan(const double* xyz_host, int32_t n, const double* boxes_host, int32_t m,
              const int32_t* tags_host, const dpso_cost_params* cp, const dpso_params* p,
              uint64_t seed, int32_t iterations, int32_t* tour_host, int64_t* cost) {
    if (!xyz_host || !cp || !p || !tour_host || !cost || n < 3 || m < 0 || iterations < 0 ||
        (m > 0 && !boxes_host))
        return DPSO_ERR_ARG;
    if (n > DPSO_MAX_N) return DPSO_ERR_RANGE;
    int st = validate_params(p);
    if (st) return st;
    cudaStream_t s = nullptr;
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    double *xyz = nullptr, *boxes = nullptr;
    int* C = nullptr;
    dpso_swarm* sw = nullptr;
    st = DPSO_OK;
    if (cudaMalloc(&xyz, sizeof(double) * 3 * n) != cudaSuccess ||
        cudaMalloc(&boxes, sizeof(double) * 6 * std::max(m, 1)) != cudaSuccess ||
        cudaMalloc(&C, sizeof(int) * static_cast<size_t>(n) * n) != cudaSuccess) {
        cudaGetLastError();
        st = DPSO_ERR_NO_MEMORY;
    }
    if (!st && (cudaMemcpyAsync(xyz, xyz_host, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s) !=
                    cudaSuccess ||
                (m > 0 && cudaMemcpyAsync(boxes, boxes_host, sizeof(double) * 6 * m,
                                          cudaMemcpyHostToDevice, s) != cudaSuccess)))
        st = DPSO_ERR_CUDA;
    if (!st) st = dpso_cost_matrix(xyz, n, boxes, m, cp, C, s);
    if (!st) st = dpso_init(&sw, C, n, tags_host, p, seed, s);
    if (!st) st = dpso_step(sw, iterations, s);
    if (!st) st = dpso_get_best(sw, tour_host, cost);
    if (sw) dpso_destroy(sw);
    cudaFree(xyz);
    cudaFree(boxes);
    cudaFree(C);
    cudaStreamDestroy(s);
    return st;
}

}  // extern "C"
