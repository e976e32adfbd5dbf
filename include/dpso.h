/*
 * dpso.h -- C ABI of the GB300 library for the enhanced discrete particle swarm
 * optimisation (DPSO) of Phung, Quach, Dinh, Ha, "Enhanced Discrete Particle
 * Swarm Optimization Path Planning for UAV Vision-based Surface Inspection"
 * (arXiv:1706.04399).
 *
 * The inspection path is the extended travelling-salesman tour of Sec. 2.3
 * over camera viewpoints: Eq. (min) under the degree and no-subtour
 * constraints.  The solver is the DPSO of Sec. 3 and Fig. "pseudocode":
 * swap-sequence velocities (Sec. 3.1), deterministic initialisation
 * (Sec. 3.2.1), random mutation (Sec. 3.2.2) and edge exchange (Sec. 3.2.3),
 * with the particles evolved in parallel on the GPU (Sec. 3.2.4).
 *
 * Conventions for every call:
 *   - Return value: DPSO_OK (0) on success, else a negative DPSO_ERR_* code.
 *     No C++ exception crosses this boundary.
 *   - A pointer named *_dev is a CUDA device pointer on the current device (for
 *     example a torch tensor's data_ptr()); *_host is ordinary host memory.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Asynchronous calls only enqueue work on it; the caller
 *     keeps their input buffers alive until the stream has passed the call.
 *   - Tours are permutations of 0..n-1 without the closing copy of the first
 *     node (Sec. 3.1 stores n_{N+1} = n_1; here it is implied).
 *   - Costs are integer millimetres (int32 per edge, int64 per tour).
 *   - Limits: 3 <= n <= DPSO_MAX_N viewpoints, 1 <= swarm <= DPSO_MAX_SWARM,
 *     every edge cost in [0, DPSO_COST_MAX].
 */
#ifndef DPSO_H
#define DPSO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DPSO_OK 0
#define DPSO_ERR_ARG (-1)       /* invalid argument (sizes, NaN, duplicate tags, asymmetric C) */
#define DPSO_ERR_RANGE (-2)     /* n or swarm above the limits, or an edge cost > DPSO_COST_MAX */
#define DPSO_ERR_NO_MEMORY (-3) /* device allocation failed or over the memory budget */
#define DPSO_ERR_CUDA (-4)      /* a CUDA runtime call failed */
#define DPSO_ERR_TIMEOUT (-5)   /* a bounded device-side wait ran out */
#define DPSO_ERR_INTERNAL (-6)  /* an internal consistency check failed */

#define DPSO_MAX_N 8192
#define DPSO_MAX_SWARM 65535
#define DPSO_COST_MAX (1 << 29)

/* dpso_params.flags */
#define DPSO_FLAG_DET_INIT 1 /* Sec. 3.2.1 back-and-forth seeding (needs grid tags) */
#define DPSO_FLAG_MUTATION 2 /* Sec. 3.2.2 random mutation */
#define DPSO_FLAG_TWO_OPT 4  /* Sec. 3.2.3 edge exchange */
/* With DPSO_FLAG_TWO_OPT: the exchange swaps two nodes (every pair of
 * positions, the node-swap reading of the paper's GPU listing) instead of
 * exchanging two edges.  Needs edge costs <= DPSO_NODE_SWAP_COST_MAX. */
#define DPSO_FLAG_NODE_SWAP 8
#define DPSO_NODE_SWAP_COST_MAX (1 << 28)

/*
 * Swarm parameters (Fig. "pseudocode"; Sec. 4 uses w = 1, phi1 = phi2 = 0.4,
 * mutation every 3 generations).
 *   w, phi1, phi2     inertial, cognitive and social coefficients of
 *                     Eq. (velocity), each in [0, 1]
 *   swarm             number of particles
 *   mut_period        mutate every mut_period-th generation (>= 1)
 *   mut_swaps         position swaps applied to each disturbed particle (>= 0)
 *   det_frac_pct      percent of particles seeded back-and-forth (0..100);
 *                     at least one when DPSO_FLAG_DET_INIT is set and tags given
 *   stall_limit       stop after this many generations without a strict gbest
 *                     improvement (0 = never)
 *   flags             DPSO_FLAG_* bits
 *   two_opt_trigger   0: edge exchange in every generation whose gbest did not
 *                     strictly improve; 1: only in such mutation generations
 *   max_moves         cap on 2-opt moves per particle per exchange (0 = none)
 */
typedef struct dpso_params {
    double w, phi1, phi2;
    int32_t swarm, mut_period, mut_swaps, det_frac_pct, stall_limit, flags,
        two_opt_trigger, max_moves;
} dpso_params;

/*
 * Edge-cost model (Sec. 2.3): straight-segment Euclidean length in mm, rounded
 * to nearest in FP64, plus blocked_penalty_mm when the closed segment meets an
 * obstacle box grown by uav_radius_m on every side (the "very large cost" of a
 * blocked pair; Sec. 2.2's inflation by the UAV size).
 */
typedef struct dpso_cost_params {
    double uav_radius_m;
    int32_t blocked_penalty_mm;
    int32_t reserved; /* must be 0 */
} dpso_cost_params;

/* Counters of a swarm. */
typedef struct dpso_stats {
    int32_t iterations;     /* generations completed */
    int32_t stalled;        /* 1 once stall_limit stopped the loop */
    int64_t gbest_cost;     /* current gbest tour cost */
    int64_t two_opt_pairs;  /* candidate pairs a plain best-improvement scan
                               evaluates: passes x n(n-3)/2 per tour */
    int64_t two_opt_moves;  /* 2-opt moves applied */
    int64_t two_opt_runs;   /* generations in which the edge exchange ran */
    int32_t device_status;  /* sticky device-side error code (DPSO_OK if none) */
    int32_t reserved;
    int64_t two_opt_evaluated; /* candidate pairs the kernels evaluated: at most
                                  two_opt_pairs, fewer when a pass reuses the
                                  previous pass's row minima (rows a move left
                                  unchanged are not evaluated again); a count
                                  of this process's work, not saved in a state */
} dpso_stats;

/* Per-phase device time of a swarm's generations while timing is on
 * (dpso_set_timing), accumulated from CUDA events recorded on the stream the
 * kernels run on.  Index: DPSO_PHASE_*. */
#define DPSO_PHASE_MOVE 0     /* Eqs. (velocity), (position), fitness, pbest */
#define DPSO_PHASE_MUTATION 1 /* Sec. 3.2.2 */
#define DPSO_PHASE_GBEST 2    /* both gbest passes */
#define DPSO_PHASE_TWO_OPT 3  /* Sec. 3.2.3 */
#define DPSO_NUM_PHASES 4
typedef struct dpso_timing {
    double ms[DPSO_NUM_PHASES];       /* summed device milliseconds */
    int64_t launches[DPSO_NUM_PHASES]; /* kernels launched */
    int32_t generations;               /* generations timed */
    int32_t reserved;
} dpso_timing;

typedef struct dpso_swarm dpso_swarm;

/* Fills the defaults: w=1, phi1=phi2=0.4 (Sec. 4), swarm=100, mut_period=3,
 * mut_swaps=2, det_frac_pct=10 (Fig. "pseudocode"), stall_limit=0, all
 * flags, trigger 0, max_moves 0. */
void dpso_default_params(dpso_params *p);
/* uav_radius_m = 0, blocked_penalty_mm = 1 000 000. */
void dpso_default_cost_params(dpso_cost_params *p);
/* Static string for a status code. */
const char *dpso_status_string(int status);

/*
 * Edge-cost matrix (Sec. 2.3).  xyz_dev: n x 3 float64 viewpoints (metres,
 * row-major).  boxes_dev: m x 6 float64 boxes (lo_x, lo_y, lo_z, hi_x, hi_y,
 * hi_z); may be NULL when m == 0.  C_dev: caller-owned n x n int32, row-major,
 * written with C[i][j] = C[j][i] (computed for i < j) and a zero diagonal.
 * 1 <= n <= DPSO_MAX_N.  Synchronises `stream` to report DPSO_ERR_ARG (a
 * non-finite coordinate or lo > hi) or DPSO_ERR_RANGE (an entry above
 * DPSO_COST_MAX; such entries are clamped to DPSO_COST_MAX).
 */
int dpso_cost_matrix(const double *xyz_dev, int32_t n, const double *boxes_dev, int32_t m,
                     const dpso_cost_params *cp, int32_t *C_dev, void *stream);

/*
 * Tour cost, Eq. (min): cost_dev[t] = sum_k C[x_k][x_(k+1) mod n] for each of
 * `count` tours.  tours_dev: count x n uint16, row-major.  C_dev: n x n int32.
 * Asynchronous.  Tours are not validated; a label outside [0, n) adds nothing
 * and is never used to index C.
 */
int dpso_fitness(const int32_t *C_dev, int32_t n, const uint16_t *tours_dev, int32_t count,
                 int64_t *cost_dev, void *stream);

/*
 * Edge exchange, Sec. 3.2.3: best-improvement 2-opt applied to each of `count`
 * tours until no exchange of two non-adjacent edges shortens it (or max_moves
 * moves, 0 = no cap).  Ties take the smallest (i, j).  tours_dev (count x n
 * uint16) is rewritten in place; cost_dev (count int64) receives the final
 * costs.  C_dev must be symmetric with a zero diagonal and entries in
 * [0, DPSO_COST_MAX].  Library-allocated scratch holds the work queue and the
 * counters.  Synchronises `stream`; pairs_host / moves_host (may be NULL)
 * receive the candidate pairs evaluated and moves applied.
 */
int dpso_two_opt(const int32_t *C_dev, int32_t n, uint16_t *tours_dev, int32_t count,
                 int64_t *cost_dev, int32_t max_moves, int64_t *pairs_host,
                 int64_t *moves_host, void *stream);

/*
 * dpso_two_opt without any device allocation (the paper has no counterpart;
 * this is a deployment variant).  Same arguments, the same tours, costs,
 * pair and move counts, and the same synchronisation as dpso_two_opt, but it
 * always runs the general (untiled) 2-opt kernel, which is slower for tours
 * the tiled kernel takes (n <= 4145): the tiled kernel reads four row-shifted
 * copies of the cost matrix that would have to be allocated.  Its scratch --
 * error word, work queue, totals, the task descriptor and per-tour pass /
 * move counts -- lives in one fixed 128 KiB device array inside the library
 * (held by every GPU that loads it, until exit) instead of being allocated
 * per call; it calls no allocating routine.
 * For callers that must not allocate device memory while running: an on-board
 * re-planning loop whose GPU memory is reserved once at start-up (an
 * allocation can synchronise the device or fail under fragmentation in
 * flight), or a process whose device memory belongs to another allocator.
 * Every call looks up the array's address on the current device (no
 * allocation); the first call on a device loads the library's kernels there:
 * make it before any stream capture.  All calls share the array, so calls
 * that overlap on the GPU (other streams, other host threads) race; the
 * caller must serialise them.
 * Returns DPSO_OK; DPSO_ERR_ARG (null pointer, n < 3, count or max_moves < 0,
 * an asymmetric cost matrix or a non-zero diagonal, a tour that is not a
 * permutation); DPSO_ERR_RANGE (n > DPSO_MAX_N, a cost outside [0,
 * DPSO_COST_MAX], or count > DPSO_NOALLOC_MAX_TOURS, the last before any
 * device work); DPSO_ERR_CUDA; DPSO_ERR_INTERNAL.  It never returns
 * DPSO_ERR_NO_MEMORY or DPSO_ERR_TIMEOUT.
 */
#define DPSO_NOALLOC_MAX_TOURS 16350
int dpso_two_opt_noalloc(const int32_t *C_dev, int32_t n, uint16_t *tours_dev, int32_t count,
                         int64_t *cost_dev, int32_t max_moves, int64_t *pairs_host,
                         int64_t *moves_host, void *stream);

/*
 * Edge costs by A* over a voxel grid (Sec. 2.2, Eqs. (L) and (cost)), the
 * paper's alternative to straight segments.  The grid is given: `origin`
 * (m), `voxel_m` (edge, m), `dims` (nx, ny, nz; each <= 4096); voxel (x, y, z)
 * has index (z ny + y) nx + x and centre origin + (i + 0.5) voxel_m per axis.
 * A voxel is occupied when its centre lies in a closed box or within the
 * UAV's sphere of such a voxel's centre: dx^2 + dy^2 + dz^2 <= inflate_r2
 * (voxels^2, <= 1024).  A* runs between the voxels of viewpoints i < j
 * (floor((p - origin) / voxel_m) per axis) over free voxels: 26 neighbours,
 * step cost weights[0] dx^2 + weights[1] dy^2 + weights[2] dz^2 (<= 1000
 * each), heuristic the squared voxel distance to the goal, closed voxels never
 * reopened, ties to the smallest (f, h, voxel).  C[i][j] = C[j][i] =
 * unit_mm x the path cost; blocked_cost when a viewpoint lies outside the grid
 * or in an occupied voxel, or when max_expansions voxels were closed without
 * reaching the goal.
 */
#define DPSO_ASTAR_MAX_EXPANSIONS 100000
typedef struct {
    double origin[3];
    double voxel_m;
    int32_t dims[3];
    int32_t inflate_r2;
    int32_t weights[3];
    int32_t unit_mm;
    int32_t blocked_cost;
    int32_t max_expansions; /* <= DPSO_ASTAR_MAX_EXPANSIONS */
    int32_t reserved;       /* must be 0 */
} dpso_astar_params;

/* voxel_m 0.5, dims 1 x 1 x 1, weights 1, unit_mm 500, blocked_cost 1e8,
 * max_expansions 20000, no inflation, origin 0. */
void dpso_default_astar_params(dpso_astar_params *p);

/* Occupancy (uint8, nx ny nz, 1 = occupied) of the grid for m boxes (device,
 * m x 6 lo/hi).  Synchronises `stream`.  Errors: DPSO_ERR_ARG, DPSO_ERR_RANGE
 * (grid or inflation above the limits), DPSO_ERR_NO_MEMORY. */
int dpso_voxel_occupancy(const double *boxes_dev, int32_t m, const dpso_astar_params *ap,
                         uint8_t *occ_dev, void *stream);

/* n x n int32 A* cost matrix (device, row-major) for n viewpoints (device,
 * n x 3) over the occupancy `occ_dev`.  One thread per pair; each search
 * first gets room for 256 expansions, and pairs that need more are searched
 * again with room for max_expansions.  Synchronises `stream`.  Errors:
 * DPSO_ERR_ARG, DPSO_ERR_RANGE (also: an entry above DPSO_COST_MAX, clamped),
 * DPSO_ERR_NO_MEMORY. */
int dpso_cost_matrix_astar(const double *xyz_dev, int32_t n, const uint8_t *occ_dev,
                           const dpso_astar_params *ap, int32_t *C_dev, void *stream);

/*
 * Node-swap exchange (the "swap nodes(i,j) and evaluate fitness" reading of
 * the edge exchange in the paper's GPU listing, Sec. 3.2.3): for each of the
 * `count` tours, repeatedly swap the two positions i < j (every pair of the
 * cyclic tour) whose swap shortens the tour most, ties to the smallest
 * (delta, i, j), until no swap improves or `max_moves` (> 0) swaps were made.
 * Arguments, layout and errors as dpso_two_opt, except that entries of C must
 * be at most DPSO_NODE_SWAP_COST_MAX (else DPSO_ERR_RANGE, as for n too large
 * for a shared-memory tile); *pairs_host counts n(n-1)/2 per pass.
 * Synchronises `stream`.
 */
int dpso_node_swap(const int32_t *C_dev, int32_t n, uint16_t *tours_dev, int32_t count,
                   int64_t *cost_dev, int32_t max_moves, int64_t *pairs_host,
                   int64_t *moves_host, void *stream);

/*
 * Creates a swarm over the n x n cost matrix C_dev (copied; the caller may free
 * it after the call) and runs the initialisation block of Fig. "pseudocode":
 * positions (back-and-forth for a fraction, Sec. 3.2.1, else seeded random
 * permutations), fitness, pbest = position, empty velocity, gbest.
 * tags_host: n x 3 int32 (face, row, col) grid tags, non-negative and unique,
 * or NULL (then every particle is random).  The library owns *out.
 * Synchronises `stream`.  Errors: DPSO_ERR_ARG (parameters, tags, C not
 * symmetric or diagonal not zero), DPSO_ERR_RANGE, DPSO_ERR_NO_MEMORY.
 */
int dpso_init(dpso_swarm **out, const int32_t *C_dev, int32_t n, const int32_t *tags_host,
              const dpso_params *p, uint64_t seed, void *stream);

/*
 * Enqueues `iterations` generations of Fig. "pseudocode" on `stream`
 * (asynchronous; replays CUDA graphs).  Generations after a stall stop are
 * no-ops.  Calls on one swarm must be ordered (same stream, or synchronised).
 */
int dpso_step(dpso_swarm *s, int32_t iterations, void *stream);

/* Best tour (n int32) and its cost; synchronises the swarm's last stream. */
int dpso_get_best(dpso_swarm *s, int32_t *tour_host, int64_t *cost);

/* gbest cost after each completed generation; *len receives the number of
 * completed generations, at most `cap` values are written. */
int dpso_get_history(dpso_swarm *s, int64_t *gbest_host, int32_t cap, int32_t *len);

/* Counters; synchronises. */
int dpso_get_stats(dpso_swarm *s, dpso_stats *st);

/*
 * Timing mode (tracing): each generation graph that dpso_step replays holds
 * event-record nodes at its phase boundaries; while timing is on, dpso_step
 * points them at fresh CUDA events before every replay (the same graph, the
 * same kernels), and dpso_get_timing synchronises and returns the
 * accumulated phase times.  Turning it on or off clears the accumulators.
 * Results are identical either way.
 */
int dpso_set_timing(dpso_swarm *s, int on);
int dpso_get_timing(dpso_swarm *s, dpso_timing *out);

/*
 * Checkpoint: serialises the whole swarm (positions, velocities as
 * permutations, pbests, fitness, gbest, generation and stall counters,
 * counters, history) into buf.  With buf == NULL only *bytes is set to the
 * size needed; otherwise *bytes is the buffer size on input and the size
 * written on output.  Synchronises.
 */
int dpso_get_state(dpso_swarm *s, void *buf, size_t *bytes);

/* Restores a checkpoint taken from a swarm with the same n, swarm size and
 * parameters.  The random streams are counter-based, so a resumed run is
 * bit-identical to an uninterrupted one.  Synchronises. */
int dpso_set_state(dpso_swarm *s, const void *buf, size_t bytes);

/* Frees the swarm (synchronises its stream first).  NULL is ignored. */
void dpso_destroy(dpso_swarm *s);

/*
 * Batches (many independent instances advanced together).  A batch groups
 * existing swarms of any sizes (all on the current device, each in at most one
 * batch in use at a time).  dpso_batch_step runs `iterations` generations of
 * every member with one set of launches per generation, replayed from a CUDA
 * graph: one warp per particle of every member for Eqs. (velocity) and
 * (position), one block per member for the gbest, and one persistent 2-opt
 * launch over every member's tours (Sec. 3.2.3), longest tours first.  Each
 * member follows exactly the trajectory it would follow alone (its arithmetic
 * reads only its own data and its own counter-based random stream).  The
 * members remain usable through the dpso_get_* calls; do not step a member
 * alone while its batch is in use.  The batch owns only descriptors; destroy
 * it before its members.  dpso_batch_create synchronises `stream`.
 */
typedef struct dpso_batch dpso_batch;
int dpso_batch_create(dpso_batch **out, dpso_swarm *const *swarms, int32_t count, void *stream);
int dpso_batch_step(dpso_batch *b, int32_t iterations, void *stream);
/* Launch shape of the tiled 2-opt kernel: tile height (rows: 32 / 30 / 24 /
 * 16 / 8), tours per CTA (1 / 2 / 4) and tiles of one tour in flight at once
 * (1, or 2 with one tour per CTA: two 8-warp subgroups of a 16-warp CTA).
 * All zero means the defaults for the longest tour of the batch. */
typedef struct {
    int32_t rows;
    int32_t tours_per_cta;
    int32_t tiles_in_flight;
} dpso_two_opt_shape;

/* Picks the 2-opt launch shape for this batch by timing every shape that fits
 * on scratch copies of the members' current tours (at most 8 moves per tour
 * each, so the probe costs a few passes; best called right after creation).
 * Results do not depend on the choice.  *chosen (may be NULL) receives the
 * shape in use.  Synchronises `stream`. */
int dpso_batch_autotune(dpso_batch *b, dpso_two_opt_shape *chosen, void *stream);
/* Sets the 2-opt launch shape by hand (NULL or all zero: the defaults).
 * DPSO_ERR_ARG when the shape is not one of the above, does not fit in shared
 * memory for the longest member, or the members lack the row-shifted cost
 * copies the tiled kernel reads.  Results do not depend on the shape.
 * Synchronises the batch's stream. */
int dpso_batch_set_two_opt_shape(dpso_batch *b, const dpso_two_opt_shape *shape);
/* The 2-opt launch shape used when none is pinned, for a launch over `count`
 * tours of n viewpoints on a GPU with `num_sms` SMs (a launch implementation
 * choice; the paper has none).  Up to n = 256: 32-row tiles, two tours per
 * CTA; beyond: the shape with the most tile rows in flight per SM, except that
 * tours whose tallest fitting tile has 16 rows or fewer take 8-row tiles with
 * two tours per CTA when those fit and count >= 2 * num_sms.  All zero when
 * no tiled shape fits (the general kernel runs).  Host only, no device call.
 * DPSO_ERR_ARG for a NULL out, n < 3, count < 0 or num_sms < 1. */
int dpso_two_opt_default_shape(int32_t n, int32_t count, int32_t num_sms,
                               dpso_two_opt_shape *out);
void dpso_batch_destroy(dpso_batch *b);

/*
 * Synchronous convenience solve from host buffers: copies the inputs to the
 * device, builds the cost matrix, initialises a swarm, runs `iterations`
 * generations and copies the best tour (n int32) and cost back.  boxes_host
 * may be NULL when m == 0; tags_host may be NULL.
 */
int dpso_plan(const double *xyz_host, int32_t n, const double *boxes_host, int32_t m,
              const int32_t *tags_host, const dpso_cost_params *cp, const dpso_params *p,
              uint64_t seed, int32_t iterations, int32_t *tour_host, int64_t *cost);

/*
 * Re-planning server (the on-line re-planning requirement of Sec. 1 served
 * for many requests at once; the paper has no server of its own).
 *
 * Requests are served in `lanes` size classes by viewpoint count n: lane 0
 * takes n < 100, lane k (k >= 1) 100 * 2^(k-1) <= n < 100 * 2^k, the last
 * lane every larger n.  Each lane has an engine thread and a CUDA stream of
 * its own on the device that is current at creation, so the lanes' launches
 * overlap on the device and a small request's generations do not wait for a
 * large one's.  Requests are copied at submission and queued; each tick of
 * a lane admits queued requests of its class (in the order `policy` sets)
 * while fewer than `max_active` requests are running in the whole server
 * (a lane holding max_active / lanes of them admits more only while no
 * other lane has requests waiting; lanes of smaller requests run on streams
 * of higher priority) and their estimated device footprint fits in
 * `memory_budget_bytes` (cost
 * matrix by dpso_cost_matrix, swarm by dpso_init; the state then stays on
 * the device until the request ends), groups the lane's running requests
 * into one batch (dpso_batch_*) and advances it by their smallest remaining
 * generation budget, at most `generations_per_tick` generations.  No request
 * runs past its own budget, so each result (tour and cost) is bit-identical
 * to dpso_plan of the same request alone, whatever else is in the mix.
 * Finished requests leave the batch at the lane's next tick and release
 * their memory.
 */
typedef struct dpso_server dpso_server;

/* Admission order of queued requests: arrival, or least estimated work first
 * (swarm x generation budget x n^3, the edge exchange's growth; ties by
 * arrival).  The second lowers the latency of small requests in a burst and
 * can delay large ones while smaller ones keep arriving.  Neither changes
 * any result. */
#define DPSO_SERVE_ARRIVAL_ORDER 0
#define DPSO_SERVE_SHORTEST_FIRST 1

#define DPSO_SERVE_MAX_LANES 8

typedef struct {
    uint64_t memory_budget_bytes; /* 0: half of the free device memory at creation */
    int32_t max_active;           /* running requests at most, all lanes (default 64) */
    int32_t generations_per_tick; /* generations per engine tick at most (default 8) */
    int32_t policy;               /* DPSO_SERVE_* (default arrival order) */
    int32_t lanes;                /* size-class lanes, 1..DPSO_SERVE_MAX_LANES; 0: 4
                                     (the default) */
} dpso_server_params;

typedef struct {
    const double *xyz_host;   /* n x 3 viewpoints (m); copied at submission */
    const double *boxes_host; /* m x 6 boxes (lo xyz, hi xyz), or NULL when m == 0 */
    const int32_t *tags_host; /* n x 3 grid tags, or NULL */
    int32_t n, m;
    int32_t iterations; /* generation budget, >= 0 */
    int32_t reserved;   /* must be 0 */
    uint64_t seed;
    dpso_cost_params cost;
    dpso_params params;
} dpso_request;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t ticks;               /* batch launches of the engine */
    int64_t particle_iterations; /* swarm x budget summed over completed requests */
    uint64_t memory_used_bytes;  /* footprint of the admitted requests now */
    int32_t peak_active;         /* most requests advanced in one tick */
    int32_t queued;              /* submitted and not yet admitted */
    double elapsed_s;            /* since creation */
} dpso_server_stats;

void dpso_default_server_params(dpso_server_params *p);
/* Starts the engines (one per lane).  Errors: DPSO_ERR_ARG (max_active or
 * generations_per_tick < 1, an unknown policy, lanes outside 0..8),
 * DPSO_ERR_CUDA. */
int dpso_server_create(dpso_server **out, const dpso_server_params *p);
/* Queues a request (host buffers copied; the caller may free them at once)
 * and returns its id (> 0).  Does not block on the device.  Errors:
 * DPSO_ERR_ARG (bad sizes or parameters), DPSO_ERR_RANGE (n > DPSO_MAX_N). */
int dpso_server_submit(dpso_server *s, const dpso_request *r, int64_t *id);
/* The device bytes admission charges for a request (host only, no device
 * needed): the swarm arrays dpso_init allocates for its n, swarm size,
 * generation budget and flags, plus the transient cost-matrix buffers. */
int dpso_server_footprint(const dpso_request *r, uint64_t *bytes);
/* *state: 0 queued or running, 1 done, or the negative status the request
 * failed with (DPSO_ERR_NO_MEMORY when its footprint exceeds the whole
 * budget).  When done, copies the best tour (tour_cap >= n, tour_host may be
 * NULL) and its cost; *latency_s (may be NULL) is the time from submission
 * to completion.  Errors: DPSO_ERR_ARG (unknown id, tour_cap < n). */
int dpso_server_poll(dpso_server *s, int64_t id, int32_t *state, int32_t *tour_host,
                     int32_t tour_cap, int64_t *cost, double *latency_s);
/* Blocks until the request leaves state 0 or timeout_s passes
 * (DPSO_ERR_TIMEOUT); *state as in dpso_server_poll. */
int dpso_server_wait(dpso_server *s, int64_t id, double timeout_s, int32_t *state);
int dpso_server_stats_get(dpso_server *s, dpso_server_stats *out);
/* Stops the engine after its current tick, frees every request's device
 * memory and the server.  Requests not yet done are dropped.  NULL ignored. */
void dpso_server_destroy(dpso_server *s);

/*
 * Philox4x32-10 draws as the solver takes them (counter = (draw/4, particle,
 * iteration, phase), key = the seed's two 32-bit halves, word draw%4), for
 * `count` consecutive draws starting at draw 0: out_dev[d] for d < count.
 * Exposed so the random stream itself can be checked.  Asynchronous.
 */
int dpso_philox_draws(uint64_t seed, uint32_t phase, uint32_t iteration, uint32_t particle,
                      int32_t count, uint32_t *out_dev, void *stream);

/*
 * Measurement aid (no counterpart in the paper): the device's L2 read
 * bandwidth in GB/s, the bound on staging cost-matrix rows in the 2-opt
 * kernel.  Reads an L2-resident device buffer of `bytes` (allocated and freed
 * by the call) `reps` times with 16-byte loads from every SM; best of five
 * timed runs with CUDA events on `stream`.  Synchronises `stream`.
 */
int dpso_probe_l2_read_gbs(size_t bytes, int32_t reps, double *gbs, void *stream);

/*
 * Measurement aid (no counterpart in the paper): the rate, in GB/s of 4-byte
 * words delivered, of independent random 4-byte gathers from an L2-resident
 * device buffer of `bytes` (4096 .. 2^33; allocated and freed by the call):
 * the access shape of a tour-fitness evaluation, Eq. (min), where each term
 * C[x_k][x_k+1] is one such gather.  Every thread of 8 CTAs per SM issues
 * `reps` rounds of eight gathers; best of five timed runs with CUDA events on
 * `stream`.  Synchronises `stream`.
 */
int dpso_probe_l2_gather_gbs(size_t bytes, int32_t reps, double *gbs, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DPSO_H */
