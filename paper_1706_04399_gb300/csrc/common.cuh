// Internal declarations shared by the CUDA translation units of the DPSO
// library (enhanced discrete PSO, Phung et al., arXiv:1706.04399).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dpso.h"

namespace dpso {

// Random-stream phases: the fourth counter word of every Philox draw.
constexpr uint32_t kPhaseInit = 1;      // initial random permutations
constexpr uint32_t kPhaseVelocity = 2;  // r1, r2 of Eq. (velocity)
constexpr uint32_t kPhaseMutation = 3;  // Sec. 3.2.2 disturbance swaps

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit products (counter words 0 and 2 by 0xD2511F53 and 0xCD9E8D57),
// high halves xor-ed with the other counter words and the key, the key bumped
// by the Weyl constants 0x9E3779B9 / 0xBB67AE85 before every round but the
// first.
// ---------------------------------------------------------------------------
struct Block4 {
    uint32_t v[4];
};

__device__ __forceinline__ Block4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                         uint64_t seed) {
    uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return Block4{{c0, c1, c2, c3}};
}

// Draw `d` of (seed, phase, iteration, particle): word d%4 of the block at
// counter (d/4, particle, iteration, phase).
__device__ __forceinline__ uint32_t draw(uint64_t seed, uint32_t phase, uint32_t iter,
                                         uint32_t particle, uint32_t d) {
    const Block4 b = philox(d >> 2, particle, iter, phase, seed);
    return b.v[d & 3u];
}

// Integer in [0, m): multiply-shift of a 32-bit draw (no rejection).
__device__ __forceinline__ uint32_t bounded(uint32_t u, uint32_t m) { return __umulhi(u, m); }

// ---------------------------------------------------------------------------
// Device control block of one swarm (one per swarm, in device memory).
// ---------------------------------------------------------------------------
struct Ctl {
    long long gf;        // gbest cost
    long long gf_start;  // gbest cost when the running generation began
    int t;               // generations completed
    int stall;           // consecutive generations without strict improvement
    int done;            // stall limit reached
    int run_two_opt;     // edge exchange scheduled in the running generation
    int status;          // sticky device error (DPSO_OK or DPSO_ERR_*)
    int n_det;           // particles seeded back-and-forth
    unsigned int queue;  // 2-opt work counter
    unsigned int pad0;
    unsigned long long pairs;  // 2-opt candidate pairs evaluated
    unsigned long long moves;  // 2-opt moves applied
    unsigned long long runs;   // generations with an edge exchange
    unsigned long long evals;  // candidate pairs the exchange kernels evaluated
    long long* hist;           // gbest cost after each generation
    int hist_cap;
    int pad1;
};

// Solver constants derived on the host from dpso_params.
struct Consts {
    int n, S;
    int ldc;  // int32 row stride of the cost matrix copy
    int ldn;  // uint16 row stride of tours / velocities
    int flags, mut_period, mut_swaps, trigger, max_moves, stall_limit;
    unsigned long long w_q, phi1_q, phi2_q;  // coefficients in Q32 (1.0 = 2^32)
    unsigned long long seed;
};

// Device arrays of one swarm.
struct SwarmDev {
    const int* C;  // n x ldc
    uint16_t* X;   // positions, S x ldn
    uint16_t* V;   // velocities as label permutations, S x ldn
    uint16_t* P;   // pbest positions, S x ldn
    uint16_t* G;   // gbest, ldn
    long long* F;  // fitness of X
    long long* PF; // fitness of P
    unsigned long long* hash;  // mutation scratch: tour hashes
    unsigned char* dup;        // mutation scratch: duplicate flags
    unsigned char* kept;       // mutation scratch: kept flags
    Ctl* ctl;
    int* order;  // exchange order: particles by decreasing fitness (S ints)
};

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// ---- launchers (cost.cu) ----
cudaError_t launch_cost_matrix(const double* xyz, int n, const double* boxes, int m, double radius,
                               int penalty, int* C, int ldc, int* err, cudaStream_t st);
cudaError_t launch_check_inputs(const double* xyz, int n, const double* boxes, int m, int* err,
                                cudaStream_t st);
cudaError_t launch_check_cost(const int* C, int n, int ldc, int* err, cudaStream_t st);
cudaError_t launch_check_cost_limit(const int* C, int n, int ldc, int limit, int* err,
                                    cudaStream_t st);

// One swarm as the generation kernels see it.
struct SwarmDesc {
    Consts k;
    SwarmDev d;
};

// Swarms advanced together by one set of launches: desc[ninst] and
// off[ninst + 1] (prefix sums of the swarm sizes) live in device memory.  A
// single swarm is a batch of one.  Every instance's arithmetic depends only on
// its own data, so results do not depend on the company it keeps.
struct BatchView {
    const SwarmDesc* desc;
    const int* off;
    int ninst;
    int total;    // off[ninst]: particles in the batch
    int max_ldn;  // largest ldn: sizes the move kernel's shared memory
    int arrays;   // shared arrays per particle in the move kernel: 7 if any w < 1, else 5
    int max_S;    // largest swarm of the batch
};

// Instance owning global item g: the largest i with off[i] <= g.
__device__ __forceinline__ int find_inst(const int* __restrict__ off, int ninst, int g) {
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// True when instance `k`'s running generation (t + 1) is a mutation generation.
__device__ __forceinline__ bool mutation_due(const Consts& k, const Ctl* c) {
    return !c->done && (k.flags & DPSO_FLAG_MUTATION) && ((c->t + 1) % k.mut_period == 0);
}

// ---- launchers (swarm.cu) ----
cudaError_t launch_fitness(const int* C, int ldc, int n, const uint16_t* tours, int ldt, int count,
                           long long* out, cudaStream_t st);
cudaError_t launch_det_orders(const int* tags, int n, uint16_t* orders, int ldn, int* err,
                              cudaStream_t st);
cudaError_t launch_init_particles(const Consts& k, const SwarmDev& d, const uint16_t* orders,
                                  int n_det, cudaStream_t st);
cudaError_t launch_gbest_init(const Consts& k, const SwarmDev& d, cudaStream_t st);
cudaError_t launch_move(const BatchView& b, cudaStream_t st);
cudaError_t launch_mutation(const BatchView& b, cudaStream_t st);
cudaError_t launch_rank_cost(const BatchView& b, cudaStream_t st);
cudaError_t launch_gbest(const BatchView& b, int second, cudaStream_t st);
cudaError_t launch_philox_draws(unsigned long long seed, uint32_t phase, uint32_t iter,
                                uint32_t particle, int count, uint32_t* out, cudaStream_t st);

// ---- launchers (two_opt.cu, two_opt_tiled.cu) ----
// One 2-opt problem: best-improvement 2-opt on `count` tours of length n (row
// stride ldt), updating tours, costs and (when pbest != nullptr) the pbest
// arrays.  When `gate` is non-null nothing happens unless *gate != 0.
struct TwoOptTask {
    const int* C;
    const int* Cs;  // optional: four row-shifted copies of C (build_shifted_copies)
    int ldc, n;
    uint16_t* tours;
    int ldt, count;
    long long* cost;
    uint16_t* pbest;
    long long* pcost;
    int max_moves;
    int pad;
    const int* gate;
    unsigned long long* pairs;
    unsigned long long* moves;
    int* status;  // receives DPSO_ERR_INTERNAL if the move guard trips
    // Optional per-tour counters: when tour_passes is set, each tour's passes
    // and moves are written there instead of being added to *pairs / *moves.
    unsigned int* tour_passes;
    unsigned int* tour_moves;
    // Optional processing order: work item k of this task is tour order[k]
    // (a permutation of 0..count-1); NULL means tour k.  Results do not depend
    // on it, only the time the last tour finishes does.
    const int* order;
    int kind;  // exchange neighbourhood: 0 edge exchange (2-opt), 1 node swap
    // Optional: receives the candidate pairs the kernel actually evaluated
    // (fewer than *pairs, the pairs a plain best-improvement pass scans, when
    // the kernel reuses the previous pass's row minima).
    unsigned long long* evals;
};

// One persistent launch over every tour of several problems: tasks[nprob] and
// off[nprob + 1] (prefix sums of the counts) in device memory, one work queue
// (zero on entry).
struct TwoOptBatch {
    const TwoOptTask* tasks;
    const int* off;
    int nprob, total;
    int max_n;        // sizes shared memory and the tile height
    bool shifted;     // every task has Cs: the tiled kernel may be used
    int rows;         // tile height of the tiled kernel (0: the default for max_n)
    unsigned int* queue;
    int tpc;          // tours per CTA of the tiled kernel (0: the default for max_n)
    int tg;           // tile subgroups per tour of the tiled kernel (0: the default)
    int kind;         // exchange of every task: 0 edge exchange (2-opt), 1 node swap
};
cudaError_t launch_two_opt(const TwoOptBatch& b, int num_sms, cudaStream_t st);

// ---- two_opt_tiled.cu: pipelined tiled variant (needs the shifted copies) ----
// Row pitch (words) of the shifted copies and of the staged rows: room for a
// shift of up to 3 words, a multiple of 4 words (16-byte rows), ldq/4 odd.
// Raises a kernel's dynamic shared-memory limit to the most the device
// allows beside the kernel's static shared memory, and checks that `smem`
// bytes fit.  Every caller sets the same value, so launches of one kernel
// with different sizes from several host threads never lower the limit
// under one another (the attribute is per kernel, not per launch).
template <typename Kernel>
inline cudaError_t raise_smem_limit(Kernel* kernel, size_t smem) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const int dyn_max = optin - static_cast<int>(fa.sharedSizeBytes);
    if (dyn_max < 0 || smem > static_cast<size_t>(dyn_max)) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
}

__host__ __device__ inline int shifted_ld(int n) {
    int q = (n + 3 + 3) / 4 * 4;
    if (((q / 4) & 1) == 0) q += 4;
    return q;
}
size_t two_opt_tiled_smem(int n, int rows_per_tile, int stages);
int two_opt_tiled_rows(int n);  // default tile height, 0 when no height fits
// Shape of a launch over `count` tours with no pinned shape (rows 0: none fits).
void two_opt_default_shape(int n, int count, int num_sms, int* rows, int* tpc, int* tg);
int two_opt_tiled_tpc(int n, int rows);  // default tours per CTA
int two_opt_tiled_tg(int n, int rows, int tpc);  // default tiles in flight per tour
int two_opt_tiled_ctas(int n, int rows, int tpc, int tg);  // resident CTAs per SM
bool two_opt_tiled_fits(int n, int rows, int tpc, int tg);  // a valid shape that fits
cudaError_t build_shifted_copies(const int* C, int ldc, int n, int* Cs, cudaStream_t st);
cudaError_t launch_two_opt_tiled(const TwoOptBatch& b, int rows, int tpc, int tg, int num_sms,
                                 cudaStream_t st);
cudaError_t launch_two_opt_general(const TwoOptBatch& b, int num_sms, cudaStream_t st);

// ---- node_swap_tiled.cu: node-swap exchange (needs the shifted copies and
// entries of C at most DPSO_NODE_SWAP_COST_MAX) ----
size_t node_swap_tiled_smem(int n, int rows);
int node_swap_tiled_rows(int n);  // 0 when no tile height fits
cudaError_t launch_node_swap_tiled(const TwoOptBatch& b, int num_sms, cudaStream_t st);

// ---- runtime.cu ----
__global__ void tours_valid_kernel(const uint16_t* tours, int n, int* err);
int two_opt_rows(int n);
int validate_params(const dpso_params* p);

}  // namespace dpso
