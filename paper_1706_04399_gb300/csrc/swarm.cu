// Particle kernels of the enhanced DPSO (Phung et al., arXiv:1706.04399):
// tour fitness (Eq. min), initialisation (Sec. 3.2.1 and Fig. "pseudocode"),
// the velocity / position update (Eqs. velocity, position with the Sec. 3.1
// operators), random mutation (Sec. 3.2.2) and the pbest / gbest reduction.
//
// Velocities are stored as the label permutation their transposition list
// induces (x + v only depends on it).  With w = 1 the list is never truncated,
// so this is exact; with w < 1 the list is taken to be the canonical one of
// that permutation, (identity + v) - identity.
#include "common.cuh"

namespace dpso {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Warp-cooperative Eq. (min) for the tour x (closing edge included).
__device__ __forceinline__ long long tour_cost_warp(const int* __restrict__ C, int ldc, int n,
                                                    const uint16_t* x, int lane) {
    long long f = 0;
    // eight positions per lane per round, their gathers issued together
    for (int base = 0; base < n; base += 256) {
        int a[8], b[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = base + lane + 32 * k;
            a[k] = i < n ? x[i] : 0;
            b[k] = i < n ? x[i + 1 == n ? 0 : i + 1] : 0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (base + lane + 32 * k < n) f += C[(size_t)a[k] * ldc + b[k]];
    }
    return warp_sum(f);
}

// ------------------------------------------------------------------ fitness
// Public entry: labels outside [0, n) contribute nothing (never read C).
__global__ void fitness_kernel(const int* __restrict__ C, int ldc, int n,
                               const uint16_t* __restrict__ tours, int ldt, int count,
                               long long* __restrict__ out) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= count) return;
    const uint16_t* x = tours + (size_t)w * ldt;
    long long f = 0;
    // A round covers 256 positions, eight per lane (lane, lane + 32, ...): the
    // labels of all eight edges are read first, then the eight gathers from C
    // are issued together, so every lane keeps eight L2 requests in flight.
    for (int base = 0; base < n; base += 256) {
        int a[8], b[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = base + lane + 32 * k;
            a[k] = i < n ? x[i] : n;
            b[k] = i < n ? x[i + 1 == n ? 0 : i + 1] : n;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (a[k] < n && b[k] < n) f += C[(size_t)a[k] * ldc + b[k]];
    }
    f = warp_sum(f);
    if (lane == 0) out[w] = f;
}

// ----------------------------------------------------- deterministic orders
// Back-and-forth order of variant v (Sec. 3.2.1): bit0 walks lines along
// columns instead of rows, bit1 visits lines in descending order, bit2 flips
// the direction of even lines; line L runs forward iff (L odd) == bit2.  The
// key of a viewpoint is (face, line', pos'); its rank among all keys is its
// place in the order.  Duplicate keys (duplicate tags) set *err.

struct Key {
    int face, line, pos;
};

__device__ __forceinline__ Key det_key(const int* tags, int i, int v) {
    const int face = tags[3 * i], row = tags[3 * i + 1], col = tags[3 * i + 2];
    const int line = (v & 1) ? col : row;
    const int pos = (v & 1) ? row : col;
    const bool backward = ((line & 1) != 0) != ((v & 4) != 0);
    return Key{face, (v & 2) ? -line : line, backward ? -pos : pos};
}

__device__ __forceinline__ bool key_less(const Key& a, const Key& b) {
    if (a.face != b.face) return a.face < b.face;
    if (a.line != b.line) return a.line < b.line;
    return a.pos < b.pos;
}

__global__ void det_orders_kernel(const int* __restrict__ tags, int n, uint16_t* orders, int ldn,
                                  int* err) {
    const int v = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ int st[3 * 512];
    Key mine{0, 0, 0};
    if (i < n) mine = det_key(tags, i, v);
    int rank = 0, same = 0;
    for (int j0 = 0; j0 < n; j0 += 512) {
        const int cnt = min(512, n - j0);
        __syncthreads();
        for (int e = threadIdx.x; e < 3 * cnt; e += blockDim.x) st[e] = tags[3 * j0 + e];
        __syncthreads();
        if (i < n) {
            for (int j = 0; j < cnt; ++j) {
                const Key o = det_key(st, j, v);
                rank += key_less(o, mine);
                same += !key_less(o, mine) && !key_less(mine, o);
            }
        }
    }
    if (i < n) {
        if (same != 1) atomicOr(err, 1);
        else orders[(size_t)v * ldn + rank] = static_cast<uint16_t>(i);
    }
}

// ----------------------------------------------------------- initialisation
// Particle p < n_det takes variant p%8 rotated left by floor(p/8); the others
// are Fisher-Yates shuffles of the identity: for i = n-1 .. 1, j = draw
// (n-1-i) of phase 1 bounded to [0, i], swap x[i], x[j].  v = identity,
// pbest = x.

__global__ void init_particles_kernel(Consts k, SwarmDev d, const uint16_t* __restrict__ orders,
                                      int n_det) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= k.S) return;
    const int n = k.n;
    uint16_t* x = d.X + (size_t)p * k.ldn;
    if (p < n_det) {
        const uint16_t* ord = orders + (size_t)(p % 8) * k.ldn;
        const int rot = (p / 8) % n;
        for (int i = 0; i < n; ++i) x[i] = ord[(i + rot) % n];
    } else {
        for (int i = 0; i < n; ++i) x[i] = static_cast<uint16_t>(i);
        for (int d0 = 0; d0 < n - 1; d0 += 4) {
            const Block4 b = philox(static_cast<uint32_t>(d0 >> 2), p, 0, kPhaseInit, k.seed);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int dd = d0 + q;
                if (dd >= n - 1) break;
                const int i = n - 1 - dd;
                const int j = static_cast<int>(bounded(b.v[q], static_cast<uint32_t>(i + 1)));
                const uint16_t tmp = x[i];
                x[i] = x[j];
                x[j] = tmp;
            }
        }
    }
    uint16_t* pb = d.P + (size_t)p * k.ldn;
    uint16_t* v = d.V + (size_t)p * k.ldn;
    for (int i = 0; i < n; ++i) {
        pb[i] = x[i];
        v[i] = static_cast<uint16_t>(i);
    }
}

// ------------------------------------------------------------ gbest (init)

__device__ __forceinline__ unsigned long long fit_key(long long f, int p) {
    return (static_cast<unsigned long long>(f) << 16) | static_cast<unsigned long long>(p);
}

// Block-wide minimum of (fitness, index) keys; result valid in every thread.
__device__ unsigned long long block_min_key(const long long* __restrict__ f, int S) {
    __shared__ unsigned long long red[32];
    unsigned long long best = ~0ull;
    for (int p = threadIdx.x; p < S; p += blockDim.x) best = min(best, fit_key(f[p], p));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(kFull, best, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = best;
    __syncthreads();
    if (w == 0) {
        best = lane < (int)(blockDim.x >> 5) ? red[lane] : ~0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(kFull, best, o));
        if (lane == 0) red[0] = best;
    }
    __syncthreads();
    best = red[0];
    __syncthreads();
    return best;
}

__global__ void gbest_init_kernel(Consts k, SwarmDev d) {
    const unsigned long long key = block_min_key(d.F, k.S);
    const int bp = static_cast<int>(key & 0xffffu);
    for (int i = threadIdx.x; i < k.n; i += blockDim.x) d.G[i] = d.X[(size_t)bp * k.ldn + i];
    if (threadIdx.x == 0) {
        Ctl* c = d.ctl;
        c->gf = d.F[bp];
        c->gf_start = d.F[bp];
        c->t = 0;
        c->stall = 0;
        c->done = 0;
        c->run_two_opt = 0;
        c->queue = 0;
    }
}

// ---------------------------------------------------------------- the move
// Sec. 3.1 subtraction x2 - x1 read as the greedy left-to-right list: scan
// positions, and where the running copy y differs from the target, swap the
// labels y[k] and tgt[k] (found through the inverse map pos).  The swap is
// written branch-free; when y[k] == tgt[k] it stores the same values back.
// Stops after `limit` transpositions; returns how many were applied.  tgt is
// read in 16-byte chunks (rows are padded to multiples of 8 labels).
__device__ int greedy_subtract(uint16_t* y, uint16_t* pos, const uint16_t* __restrict__ tgt,
                               int n, int limit) {
    int cnt = 0;
    if (limit <= 0) return 0;
    uint4 cur = *reinterpret_cast<const uint4*>(tgt);
    for (int k0 = 0; k0 < n; k0 += 8) {
        const uint4 nxt = (k0 + 8 < n) ? *reinterpret_cast<const uint4*>(tgt + k0 + 8) : cur;
        const uint32_t w[4] = {cur.x, cur.y, cur.z, cur.w};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int kk = k0 + q;
            if (kk >= n) break;
            const uint16_t b = static_cast<uint16_t>(w[q >> 1] >> ((q & 1) * 16));
            const uint16_t a = y[kk];
            const uint16_t pb = pos[b];
            y[kk] = b;
            y[pb] = a;
            pos[b] = static_cast<uint16_t>(kk);
            pos[a] = pb;
            cnt += (a != b);
            if (cnt >= limit) return cnt;
        }
        cur = nxt;
    }
    return cnt;
}

// floor(c |v|) with c = phi * u / 2^32 in Q32 fixed point.
__device__ __forceinline__ int scaled_count(unsigned long long phi_q, uint32_t u, int len) {
    const unsigned long long cq = (phi_q * static_cast<unsigned long long>(u)) >> 32;
    return static_cast<int>((cq * static_cast<unsigned long long>(len)) >> 32);
}

// One warp per particle.  Shared memory per warp: ya/pa (copy of x moved
// toward P and its inverse), yb/pb (toward G), ix (inverse of x) and, when
// w < 1, yw/pw (identity moved toward the velocity permutation).
//   1. full greedy passes give |P - x|, |G - x| (and |v|): lanes 0, 1 (2)
//   2. truncated passes apply the first ka / kb (kw) transpositions
//   3. v <- sigma_b o sigma_a o sigma_wv, x <- v o x, fitness, pbest
// One warp per particle of any instance in the batch.  Shared memory per
// warp: ya/pa (copy of x moved toward P and its inverse), yb/pb (toward G),
// ix (inverse of x) and, when the instance has w < 1, yw/pw (identity moved
// toward the velocity permutation).
//   1. full greedy passes give |P - x|, |G - x| (and |v|): lanes 0, 1 (2)
//   2. truncated passes apply the first ka / kb (kw) transpositions
//   3. v <- sigma_b o sigma_a o sigma_wv, x <- v o x, fitness, pbest
__global__ void move_kernel(BatchView b) {
    extern __shared__ __align__(16) uint16_t sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * (blockDim.x >> 5) + warp;
    if (g >= b.total) return;
    const int inst = find_inst(b.off, b.ninst, g);
    const int p = g - b.off[inst];
    const Consts k = b.desc[inst].k;
    const SwarmDev d = b.desc[inst].d;
    const Ctl* ctl = d.ctl;
    if (ctl->done) return;
    const int t = ctl->t + 1;
    const int n = k.n, ldn = k.ldn;
    const bool partial = k.w_q < (1ull << 32);
    uint16_t* ya = sm + static_cast<size_t>(warp) * b.arrays * b.max_ldn;
    uint16_t* pa = ya + ldn;
    uint16_t* yb = pa + ldn;
    uint16_t* pb = yb + ldn;
    uint16_t* ix = pb + ldn;
    uint16_t* yw = ix + ldn;
    uint16_t* pw = yw + ldn;
    uint16_t* x = d.X + static_cast<size_t>(p) * ldn;
    uint16_t* v = d.V + static_cast<size_t>(p) * ldn;
    uint16_t* P = d.P + static_cast<size_t>(p) * ldn;
    const uint16_t* G = d.G;
    const int lanes = partial ? (k.w_q == 0 ? 2 : 3) : 2;

    auto reset = [&]() {
        for (int i = lane; i < n; i += 32) {
            const uint16_t xi = x[i];
            ix[xi] = static_cast<uint16_t>(i);
            ya[i] = xi;
            pa[xi] = static_cast<uint16_t>(i);
            yb[i] = xi;
            pb[xi] = static_cast<uint16_t>(i);
            if (partial) {
                yw[i] = static_cast<uint16_t>(i);
                pw[i] = static_cast<uint16_t>(i);
            }
        }
        __syncwarp();
    };
    auto run = [&](int lim_a, int lim_b, int lim_w) {
        int c = 0;
        if (lane == 0) c = greedy_subtract(ya, pa, P, n, lim_a);
        else if (lane == 1) c = greedy_subtract(yb, pb, G, n, lim_b);
        else if (lane == 2 && lanes == 3) c = greedy_subtract(yw, pw, v, n, lim_w);
        __syncwarp();
        return c;
    };

    reset();
    const int c0 = run(n, n, n);
    const int La = __shfl_sync(kFull, c0, 0), Lb = __shfl_sync(kFull, c0, 1);
    const int Lw = __shfl_sync(kFull, c0, 2);
    const Block4 r = philox(0, p, t, kPhaseVelocity, k.seed);
    const int ka = scaled_count(k.phi1_q, r.v[0], La);
    const int kb = scaled_count(k.phi2_q, r.v[1], Lb);
    const int kw = partial ? static_cast<int>(
                                 (k.w_q * static_cast<unsigned long long>(lanes == 3 ? Lw : 0)) >> 32)
                           : 0;
    reset();
    run(ka, kb, kw);

    // sigma_a(m) = ya[ix[m]], sigma_b(m) = yb[ix[m]]; new velocity into pa.
    for (int l = lane; l < n; l += 32) {
        uint16_t m = partial ? yw[l] : v[l];
        m = ya[ix[m]];
        m = yb[ix[m]];
        pa[l] = m;
    }
    __syncwarp();
    for (int l = lane; l < n; l += 32) v[l] = pa[l];
    for (int i = lane; i < n; i += 32) {
        const uint16_t xn = pa[x[i]];
        pb[i] = xn;
        x[i] = xn;
    }
    __syncwarp();
    const long long f = tour_cost_warp(d.C, k.ldc, n, pb, lane);
    const long long pf = d.PF[p];  // read by every lane before lane 0 may write it
    __syncwarp();
    if (lane == 0) d.F[p] = f;
    if (f < pf) {
        for (int i = lane; i < n; i += 32) P[i] = pb[i];
        if (lane == 0) d.PF[p] = f;
    }
}

// ---------------------------------------------------------------- mutation
// Sec. 3.2.2: order the particles by (fitness, index); a particle equal (as a
// tour array) to an earlier one in that order is a duplicate; the first
// ceil(S/3) non-duplicates are kept; every other particle gets mut_swaps
// swaps of two distinct positions (phase-3 draws 2q, 2q+1), an empty
// velocity, a new fitness and a pbest update.  Equal tours have equal
// fitness, so "earlier" means equal fitness and a smaller index; a 64-bit
// hash screens the candidates and full compares decide.

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Global particle g of the batch -> (instance, particle); false when g is past
// the batch or the instance does not mutate in its running generation.
__device__ __forceinline__ bool mut_item(const BatchView& b, int g, Consts& k, SwarmDev& d,
                                         int& p) {
    if (g >= b.total) return false;
    const int inst = find_inst(b.off, b.ninst, g);
    p = g - b.off[inst];
    k = b.desc[inst].k;
    d = b.desc[inst].d;
    return mutation_due(k, d.ctl);
}

__global__ void mut_hash_kernel(BatchView b) {
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    Consts k;
    SwarmDev d;
    int p;
    if (!mut_item(b, g, k, d, p)) return;
    const uint16_t* x = d.X + static_cast<size_t>(p) * k.ldn;
    unsigned long long h = 0;
    for (int i = lane; i < k.n; i += 32)
        h += mix64((static_cast<unsigned long long>(i) << 16) | x[i]);
    h = warp_sum_u(h);
    if (lane == 0) d.hash[p] = h;
}

__device__ bool tours_equal(const uint16_t* a, const uint16_t* b, int ldn) {
    const uint4* va = reinterpret_cast<const uint4*>(a);
    const uint4* vb = reinterpret_cast<const uint4*>(b);
    for (int i = 0; i < ldn / 8; ++i) {
        const uint4 u = va[i], w = vb[i];
        if (u.x != w.x || u.y != w.y || u.z != w.z || u.w != w.w) return false;
    }
    return true;
}

__global__ void mut_dup_kernel(BatchView b) {
    Consts k;
    SwarmDev d;
    int p;
    if (!mut_item(b, blockIdx.x * blockDim.x + threadIdx.x, k, d, p)) return;
    const long long fp = d.F[p];
    const unsigned long long hp = d.hash[p];
    unsigned char dup = 0;
    for (int q = 0; q < p && !dup; ++q)
        if (d.F[q] == fp && d.hash[q] == hp)
            dup = tours_equal(d.X + static_cast<size_t>(q) * k.ldn,
                              d.X + static_cast<size_t>(p) * k.ldn, k.ldn);
    d.dup[p] = dup;
}

__global__ void mut_kept_kernel(BatchView b) {
    Consts k;
    SwarmDev d;
    int p;
    if (!mut_item(b, blockIdx.x * blockDim.x + threadIdx.x, k, d, p)) return;
    unsigned char kept = 0;
    if (!d.dup[p]) {
        const long long fp = d.F[p];
        int rank = 0;
        for (int q = 0; q < k.S; ++q)
            rank += !d.dup[q] && (d.F[q] < fp || (d.F[q] == fp && q < p));
        kept = rank < (k.S + 2) / 3;
    }
    d.kept[p] = kept;
}

__global__ void mut_apply_kernel(BatchView b) {
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    Consts k;
    SwarmDev d;
    int p;
    if (!mut_item(b, g, k, d, p) || d.kept[p]) return;
    const int t = d.ctl->t + 1, n = k.n;
    uint16_t* x = d.X + static_cast<size_t>(p) * k.ldn;
    if (lane == 0) {
        for (int q = 0; q < k.mut_swaps; ++q) {
            const uint32_t di = 2u * q, dj = 2u * q + 1u;
            const Block4 bi = philox(di >> 2, p, t, kPhaseMutation, k.seed);
            const Block4 bj = philox(dj >> 2, p, t, kPhaseMutation, k.seed);
            const int i = static_cast<int>(bounded(bi.v[di & 3u], static_cast<uint32_t>(n)));
            int j = static_cast<int>(bounded(bj.v[dj & 3u], static_cast<uint32_t>(n - 1)));
            j += (j >= i);
            const uint16_t tmp = x[i];
            x[i] = x[j];
            x[j] = tmp;
        }
    }
    __syncwarp();
    uint16_t* v = d.V + static_cast<size_t>(p) * k.ldn;
    for (int i = lane; i < n; i += 32) v[i] = static_cast<uint16_t>(i);
    const long long f = tour_cost_warp(d.C, k.ldc, n, x, lane);
    const long long pf = d.PF[p];
    __syncwarp();
    if (lane == 0) d.F[p] = f;
    if (f < pf) {
        uint16_t* P = d.P + static_cast<size_t>(p) * k.ldn;
        for (int i = lane; i < n; i += 32) P[i] = x[i];
        if (lane == 0) d.PF[p] = f;
    }
}

// ------------------------------------------------------------------ gbest
// Fig. "pseudocode": the particle with the smallest (pbest fitness, index)
// replaces the gbest only on strict improvement.  Pass 0 runs after the
// particle loop (and mutation) and schedules the edge exchange; pass 1 runs
// after the exchange.  The generation is closed (history, stall counter,
// generation counter, stop flag) by the last pass that runs.  One block per
// instance of the batch.

__global__ void gbest_kernel(BatchView b, int second) {
    const Consts k = b.desc[blockIdx.x].k;
    const SwarmDev d = b.desc[blockIdx.x].d;
    Ctl* c = d.ctl;
    if (c->done) return;
    if (second && !c->run_two_opt) return;
    const bool mut_iter = mutation_due(k, c);
    const unsigned long long key = block_min_key(d.PF, k.S);
    const long long best = static_cast<long long>(key >> 16);
    const int bp = static_cast<int>(key & 0xffffu);
    const long long gf_old = c->gf;
    __syncthreads();
    if (best < gf_old)
        for (int i = threadIdx.x; i < k.n; i += blockDim.x)
            d.G[i] = d.P[static_cast<size_t>(bp) * k.ldn + i];
    if (threadIdx.x != 0) return;
    const int t = c->t + 1;
    if (!second) c->gf_start = gf_old;
    if (best < gf_old) c->gf = best;
    if (t <= c->hist_cap) c->hist[t - 1] = c->gf;
    else c->status = DPSO_ERR_INTERNAL;
    const bool improved = c->gf < c->gf_start;
    if (!second) {
        const bool run = (k.flags & DPSO_FLAG_TWO_OPT) && !improved && (k.trigger == 0 || mut_iter);
        c->run_two_opt = run ? 1 : 0;
        if (run) {
            c->runs += 1;
            return;
        }
    } else {
        c->run_two_opt = 0;
    }
    c->stall = improved ? 0 : c->stall + 1;
    c->t = t;
    if (k.stall_limit > 0 && c->stall >= k.stall_limit) c->done = 1;
}

// ------------------------------------------------------ exchange order
// order[r] = the particle of rank r by (fitness descending, index ascending)
// within each instance, so the edge exchange starts the tours expected to
// need the most passes first (longest-processing-time-first list
// scheduling; the post-move fitness is the estimate).  Block (x, y) ranks
// particles x*256 .. x*256+255 of instance y against all of its particles.
__global__ void rank_cost_kernel(BatchView b) {
    const int inst = blockIdx.y;
    const SwarmDesc& ds = b.desc[inst];
    const int S = ds.k.S;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x * blockDim.x >= S) return;  // whole block past this swarm
    const long long* __restrict__ F = ds.d.F;
    __shared__ long long sf[256];
    const long long mine = p < S ? F[p] : 0;
    int rank = 0;
    for (int q0 = 0; q0 < S; q0 += 256) {
        const int cnt = min(256, S - q0);
        __syncthreads();
        if (threadIdx.x < cnt) sf[threadIdx.x] = F[q0 + threadIdx.x];
        __syncthreads();
        if (p < S) {
            for (int j = 0; j < cnt; ++j) {
                const long long o = sf[j];
                rank += (o > mine) | ((o == mine) & (q0 + j < p));
            }
        }
    }
    if (p < S) ds.d.order[rank] = p;
}

__global__ void philox_draws_kernel(unsigned long long seed, uint32_t phase, uint32_t iter,
                                    uint32_t particle, int count, uint32_t* out) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d < count) out[d] = draw(seed, phase, iter, particle, static_cast<uint32_t>(d));
}

// Warps per block of the move kernel: up to 8, within 200 KB of shared memory.
int move_warps(const BatchView& b) {
    const size_t per = static_cast<size_t>(b.arrays) * b.max_ldn * sizeof(uint16_t);
    int w = 8;
    while (w > 1 && per * w > 200 * 1024) --w;
    return w;
}

}  // namespace

cudaError_t launch_fitness(const int* C, int ldc, int n, const uint16_t* tours, int ldt, int count,
                           long long* out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (count * 32 + threads - 1) / threads;
    fitness_kernel<<<blocks, threads, 0, st>>>(C, ldc, n, tours, ldt, count, out);
    return cudaGetLastError();
}

cudaError_t launch_det_orders(const int* tags, int n, uint16_t* orders, int ldn, int* err,
                              cudaStream_t st) {
    dim3 grid((n + 255) / 256, 8);
    det_orders_kernel<<<grid, 256, 0, st>>>(tags, n, orders, ldn, err);
    return cudaGetLastError();
}

cudaError_t launch_init_particles(const Consts& k, const SwarmDev& d, const uint16_t* orders,
                                  int n_det, cudaStream_t st) {
    init_particles_kernel<<<(k.S + 63) / 64, 64, 0, st>>>(k, d, orders, n_det);
    return cudaGetLastError();
}

cudaError_t launch_gbest_init(const Consts& k, const SwarmDev& d, cudaStream_t st) {
    gbest_init_kernel<<<1, 1024, 0, st>>>(k, d);
    return cudaGetLastError();
}

cudaError_t launch_move(const BatchView& b, cudaStream_t st) {
    if (b.total <= 0) return cudaSuccess;
    const int w = move_warps(b);
    const size_t smem = static_cast<size_t>(b.arrays) * b.max_ldn * sizeof(uint16_t) * w;
    const cudaError_t e = raise_smem_limit(move_kernel, smem);
    if (e != cudaSuccess) return e;
    move_kernel<<<(b.total + w - 1) / w, 32 * w, smem, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_mutation(const BatchView& b, cudaStream_t st) {
    if (b.total <= 0) return cudaSuccess;
    const int wb = (b.total * 32 + 255) / 256, tb = (b.total + 255) / 256;
    mut_hash_kernel<<<wb, 256, 0, st>>>(b);
    mut_dup_kernel<<<tb, 256, 0, st>>>(b);
    mut_kept_kernel<<<tb, 256, 0, st>>>(b);
    mut_apply_kernel<<<wb, 256, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_rank_cost(const BatchView& b, cudaStream_t st) {
    if (b.ninst <= 0 || b.max_S <= 0) return cudaSuccess;
    dim3 grid((b.max_S + 255) / 256, b.ninst);
    rank_cost_kernel<<<grid, 256, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_gbest(const BatchView& b, int second, cudaStream_t st) {
    if (b.ninst <= 0) return cudaSuccess;
    gbest_kernel<<<b.ninst, 1024, 0, st>>>(b, second);
    return cudaGetLastError();
}

cudaError_t launch_philox_draws(unsigned long long seed, uint32_t phase, uint32_t iter,
                                uint32_t particle, int count, uint32_t* out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    philox_draws_kernel<<<(count + 255) / 256, 256, 0, st>>>(seed, phase, iter, particle, count,
                                                             out);
    return cudaGetLastError();
}

}  // namespace dpso
