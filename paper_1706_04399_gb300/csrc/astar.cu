// Edge costs by A* over a voxel grid (Sec. 2.2, Eqs. (L) and (cost)): the
// paper's alternative to straight segments.  The grid (origin, voxel edge,
// dimensions) is an input; voxel (x, y, z) has index (z ny + y) nx + x and
// centre origin + (i + 0.5) voxel per axis (doubles, correctly rounded, no
// contraction, as on the host).
//
//  * Occupancy: a voxel is occupied when its centre lies in a closed box, or
//    when its centre is within the UAV's sphere (r2 voxels^2) of such a
//    voxel's centre.
//  * Search: one thread per viewpoint pair (i < j), A* from the voxel of i to
//    that of j over free voxels with 26 neighbours, step cost
//    a1 dx^2 + a2 dy^2 + a3 dz^2, heuristic the squared voxel distance to the
//    goal, a closed list (no reopening) and lazy open-list entries popped by
//    the smallest (f, h, voxel); with that total order the expansion order,
//    hence the cost, does not depend on how the priority queue is built.
//  * Pairs whose voxels lie in different connected components of the free
//    voxels (union-find over the 26-neighbourhood) are blocked without a
//    search: A* could only exhaust its open list or its cap there.
//  * Pass 1: one warp per search, its map and open list in shared memory
//    (astar_warp_kernel); a search that outgrows them is searched again, from
//    the start, by pass 2: one thread per search with its own binary heap and
//    open-addressing map (voxel -> best g, closed; slots stamped by search,
//    so nothing is cleared) in device scratch, room for the full expansion
//    cap.  Grids or weights too large for the warp pass's packed keys take
//    the thread pass twice instead: room for 256 expansions, then the cap.
//  * C[i][j] = C[j][i] = g * unit_mm; blocked_cost where a viewpoint lies
//    outside the grid or in an occupied voxel, or the cap was exhausted.
#include <climits>
#include <vector>

#include "common.cuh"

namespace dpso {
namespace {

struct AstarGrid {
    double ox, oy, oz, voxel;
    int nx, ny, nz;
};

__device__ __forceinline__ double centre(double o, int i, double voxel) {
    return __dadd_rn(o, __dmul_rn(__dadd_rn(static_cast<double>(i), 0.5), voxel));
}

__global__ void voxel_core_kernel(AstarGrid gr, const double* __restrict__ boxes, int m,
                                  unsigned char* __restrict__ core) {
    const long long nv = static_cast<long long>(gr.nx) * gr.ny * gr.nz;
    for (long long v = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; v < nv;
         v += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(v % gr.nx), y = static_cast<int>((v / gr.nx) % gr.ny),
                  z = static_cast<int>(v / (static_cast<long long>(gr.nx) * gr.ny));
        const double cx = centre(gr.ox, x, gr.voxel), cy = centre(gr.oy, y, gr.voxel),
                     cz = centre(gr.oz, z, gr.voxel);
        unsigned char in = 0;
        for (int b = 0; b < m && !in; ++b) {
            const double* bx = boxes + 6 * static_cast<size_t>(b);
            in = cx >= bx[0] && cx <= bx[3] && cy >= bx[1] && cy <= bx[4] && cz >= bx[2] &&
                 cz <= bx[5];
        }
        core[v] = in;
    }
}

__global__ void voxel_inflate_kernel(AstarGrid gr, int r2, int R,
                                     const unsigned char* __restrict__ core,
                                     unsigned char* __restrict__ occ) {
    const long long nv = static_cast<long long>(gr.nx) * gr.ny * gr.nz;
    for (long long v = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; v < nv;
         v += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(v % gr.nx), y = static_cast<int>((v / gr.nx) % gr.ny),
                  z = static_cast<int>(v / (static_cast<long long>(gr.nx) * gr.ny));
        unsigned char o = 0;
        for (int dz = -R; dz <= R && !o; ++dz)
            for (int dy = -R; dy <= R && !o; ++dy)
                for (int dx = -R; dx <= R && !o; ++dx) {
                    if (dx * dx + dy * dy + dz * dz > r2) continue;
                    const int xx = x + dx, yy = y + dy, zz = z + dz;
                    if (xx < 0 || yy < 0 || zz < 0 || xx >= gr.nx || yy >= gr.ny || zz >= gr.nz)
                        continue;
                    o = core[(static_cast<long long>(zz) * gr.ny + yy) * gr.nx + xx];
                }
        occ[v] = o;
    }
}

// Voxel of each viewpoint, or -1 outside the grid or in an occupied voxel.
__global__ void viewpoint_voxel_kernel(AstarGrid gr, const double* __restrict__ xyz, int n,
                                       const unsigned char* __restrict__ occ, int* __restrict__ vox) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double o[3] = {gr.ox, gr.oy, gr.oz};
    const int d[3] = {gr.nx, gr.ny, gr.nz};
    long long c[3];
    bool inside = true;
    for (int k = 0; k < 3; ++k) {
        c[k] = static_cast<long long>(floor(__ddiv_rn(__dsub_rn(xyz[3 * i + k], o[k]), gr.voxel)));
        inside = inside && c[k] >= 0 && c[k] < d[k];
    }
    int v = -1;
    if (inside) {
        v = static_cast<int>((c[2] * gr.ny + c[1]) * gr.nx + c[0]);
        if (occ[v]) v = -1;
    }
    vox[i] = v;
}

struct OpenEntry {
    long long f;
    long long g;
    int h;
    int v;
};

__device__ __forceinline__ bool open_less(const OpenEntry& a, const OpenEntry& b) {
    if (a.f != b.f) return a.f < b.f;
    if (a.h != b.h) return a.h < b.h;
    return a.v < b.v;
}

// Voxel -> best g and closed flag.  A slot belongs to the search whose stamp
// it carries (tag >> 1; the scratch starts zeroed and stamps start at 1), so
// no search has to clear the map of the previous one.
struct MapSlot {
    int v;
    unsigned tag;  // (stamp << 1) | closed
    long long g;
};

struct AstarArgs {
    AstarGrid gr;
    const unsigned char* occ;
    const int* vox;
    const int* comp;     // connected component (smallest voxel index) of free voxels
    const int2* pairs;   // (i, j), i < j
    int stamp0;          // stamp of pairs[0] (stamps are unique within a pass)
    int npairs;
    int a1, a2, a3;
    long long unit_mm;
    int blocked_cost;
    int max_exp;          // this pass' expansion budget
    bool final_pass;      // exhausting max_exp means blocked (else: retry later)
    int heap_cap;         // entries per search (26 max_exp + 1)
    int map_bits;         // map slots per search = 2^map_bits (>= 2 heap_cap)
    OpenEntry* heap;      // npairs x heap_cap
    MapSlot* map;         // npairs x 2^map_bits
    int* C;
    int n;
    int* retry;           // pass 1: 1 for pairs to search again
    int* err;             // bit 1: an entry above DPSO_COST_MAX (clamped)
};

__device__ __forceinline__ unsigned slot_of(int v, int bits) {
    return (static_cast<unsigned>(v) * 2654435761u) >> (32 - bits);
}

// Finds (insert = false) or inserts the slot of voxel v for this search.
__device__ MapSlot* map_find(MapSlot* map, int bits, unsigned stamp, int v, bool insert) {
    const unsigned mask = (1u << bits) - 1u;
    unsigned s = slot_of(v, bits);
    for (unsigned probe = 0; probe <= mask; ++probe, s = (s + 1) & mask) {
        MapSlot* e = map + s;
        const bool mine = (e->tag >> 1) == stamp;
        if (mine && e->v == v) return e;
        if (!mine) {
            if (!insert) return nullptr;
            e->v = v;
            e->tag = stamp << 1;
            e->g = LLONG_MAX;
            return e;
        }
    }
    return nullptr;  // full (cannot happen at load <= 1/2)
}

__global__ void astar_pairs_kernel(AstarArgs A) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.npairs) return;
    const int2 pr = A.pairs[k];
    const int s = A.vox[pr.x], t = A.vox[pr.y];
    long long result = -1;  // path cost, or -1: blocked
    bool retry = false;
    // different components: no search can reach t (it would exhaust its open
    // list or its cap), so the pair is blocked without one
    if (s >= 0 && t >= 0 && A.comp[s] == A.comp[t]) {
        OpenEntry* heap = A.heap + static_cast<size_t>(k) * A.heap_cap;
        MapSlot* map = A.map + (static_cast<size_t>(k) << A.map_bits);
        const unsigned stamp = static_cast<unsigned>(A.stamp0 + k);
        const int nx = A.gr.nx, ny = A.gr.ny, nz = A.gr.nz;
        const int tx = t % nx, ty = (t / nx) % ny, tz = t / (nx * ny);
        int len = 0;
        auto push = [&](const OpenEntry& e) {
            int i = len++;
            while (i > 0) {
                const int parent = (i - 1) / 2;
                if (!open_less(e, heap[parent])) break;
                heap[i] = heap[parent];
                i = parent;
            }
            heap[i] = e;
        };
        auto pop = [&]() {
            const OpenEntry top = heap[0], last = heap[--len];
            int i = 0;
            for (;;) {
                int c = 2 * i + 1;
                if (c >= len) break;
                if (c + 1 < len && open_less(heap[c + 1], heap[c])) ++c;
                if (!open_less(heap[c], last)) break;
                heap[i] = heap[c];
                i = c;
            }
            if (len > 0) heap[i] = last;
            return top;
        };
        {
            const int sx = s % nx, sy = (s / nx) % ny, sz = s / (nx * ny);
            const int h0 = (sx - tx) * (sx - tx) + (sy - ty) * (sy - ty) + (sz - tz) * (sz - tz);
            MapSlot* e0 = map_find(map, A.map_bits, stamp, s, true);
            e0->g = 0;
            push(OpenEntry{h0, 0, h0, s});
        }
        int expanded = 0;
        while (len > 0) {
            const OpenEntry e = pop();
            MapSlot* me = map_find(map, A.map_bits, stamp, e.v, false);
            if (me->tag & 1u) continue;
            me->tag |= 1u;
            if (e.v == t) {
                result = e.g;
                break;
            }
            if (expanded >= A.max_exp) {
                retry = !A.final_pass;
                break;
            }
            ++expanded;
            const int x = e.v % nx, y = (e.v / nx) % ny, z = e.v / (nx * ny);
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (!dx && !dy && !dz) continue;
                        const int xx = x + dx, yy = y + dy, zz = z + dz;
                        if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) continue;
                        const int v = (zz * ny + yy) * nx + xx;
                        if (A.occ[v]) continue;
                        MapSlot* sl = map_find(map, A.map_bits, stamp, v, true);
                        if (sl->tag & 1u) continue;
                        const long long g = e.g + static_cast<long long>(A.a1) * dx * dx +
                                            static_cast<long long>(A.a2) * dy * dy +
                                            static_cast<long long>(A.a3) * dz * dz;
                        if (g >= sl->g) continue;
                        sl->g = g;
                        const int h = (xx - tx) * (xx - tx) + (yy - ty) * (yy - ty) +
                                      (zz - tz) * (zz - tz);
                        push(OpenEntry{g + h, g, h, v});
                    }
        }
    }
    if (retry) {
        A.retry[k] = 1;
        return;
    }
    long long c = result < 0 ? A.blocked_cost : result * A.unit_mm;
    if (c > DPSO_COST_MAX) {
        atomicOr(A.err, 2);
        c = DPSO_COST_MAX;
    }
    A.C[static_cast<size_t>(pr.x) * A.n + pr.y] = static_cast<int>(c);
    A.C[static_cast<size_t>(pr.y) * A.n + pr.x] = static_cast<int>(c);
}

// The same search with one warp per pair and the whole state in shared
// memory, for searches that stay small (which, with the squared-distance
// heuristic, is nearly all of them).  Per warp:
//   map:  kWarpSlots slots (voxel | closed bit, best g), linear probing with
//         lanes inserting concurrently by 64-bit CAS (nothing is deleted
//         within a search, so a lane that finds an empty slot knows its voxel
//         is not further along);
//   open: an append-only array of keys (f << 42 | h << 24 | voxel), popped
//         entries overwritten with ~0.  Keys of live entries are distinct
//         (a voxel is pushed again only with a smaller g), so the pop is a
//         warp-wide minimum and its owner lane is unique.
// A pop, the closed test, the goal and cap tests are uniform over the warp;
// lanes 0..25 then relax one neighbour each and append their entries in lane
// order.  The pushes of one expansion are the sequential search's (each
// neighbour's test reads only its own slot), and the pop order depends only
// on the set of keys, so the result is the sequential search's.  A search
// that would outgrow the map or the open array is left to the global pass
// (retry flag).  Host-checked bounds keep f < 2^22, h < 2^18 and every grid
// dimension at most 256.
constexpr int kWarpSlots = 2048;         // map slots per warp
constexpr int kWarpOpen = 2048;          // open entries per warp
constexpr int kWarpDistinct = 1900;      // inserts before a search hands over
constexpr int kWarpsPerBlock = 7;        // 7 x 32 KB of shared memory per block
constexpr unsigned long long kEmptySlot = ~0ull;
constexpr unsigned kClosed = 1u << 30;   // closed bit of a slot's voxel word

struct WarpArgs {
    AstarGrid gr;
    const unsigned char* occ;
    const int* vox;
    const int* comp;
    const int2* pairs;
    int npairs;
    unsigned* queue;  // next pair (zero on entry)
    int a1, a2, a3;
    long long unit_mm;
    int blocked_cost;
    int max_exp;
    int* C;
    int n;
    int* retry;  // 1: left to the global pass
    int* err;
};

// Voxels in the warp pass are named by packed coordinates x | y << 8 | z << 16
// (every grid dimension at most 256), which order like the voxel index
// (z ny + y) nx + x, so keys need no division to give back coordinates.
__device__ __forceinline__ int pack_xyz(int x, int y, int z) { return x | (y << 8) | (z << 16); }

// Warp-wide minimum of a 64-bit key: the minimum of the high words, then of
// the low words among the lanes holding it.
__device__ __forceinline__ unsigned long long warp_min_key(unsigned long long v) {
    const unsigned hi = static_cast<unsigned>(v >> 32);
    const unsigned mhi = __reduce_min_sync(0xffffffffu, hi);
    const unsigned lo = hi == mhi ? static_cast<unsigned>(v) : 0xffffffffu;
    const unsigned mlo = __reduce_min_sync(0xffffffffu, lo);
    return (static_cast<unsigned long long>(mhi) << 32) | mlo;
}

__global__ void __launch_bounds__(32 * kWarpsPerBlock) astar_warp_kernel(WarpArgs A) {
    extern __shared__ unsigned long long sm_astar[];
    const int lane = threadIdx.x & 31;
    unsigned long long* const open = sm_astar + (threadIdx.x >> 5) * (kWarpOpen + kWarpSlots);
    unsigned long long* const map = open + kWarpOpen;
    const int nx = A.gr.nx, ny = A.gr.ny, nz = A.gr.nz;
    const int nxy = nx * ny;
    // this lane's neighbour offset (lanes 0..25; the 27 offsets minus the centre)
    const int d = lane < 13 ? lane : lane + 1;
    const int ddx = d % 3 - 1, ddy = (d / 3) % 3 - 1, ddz = d / 9 - 1;
    const int step = A.a1 * ddx * ddx + A.a2 * ddy * ddy + A.a3 * ddz * ddz;
    auto slot0 = [](int c) { return (static_cast<unsigned>(c) * 2654435761u) >> 21; };  // 11 bits
    auto cw = [](unsigned long long e) { return static_cast<int>((e >> 32) & (kClosed - 1)); };
    constexpr unsigned long long kClosedBit = static_cast<unsigned long long>(kClosed) << 32;
    for (;;) {
        int k = 0;
        if (lane == 0) k = static_cast<int>(atomicAdd(A.queue, 1u));
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= A.npairs) break;
        const int2 pr = A.pairs[k];
        const int s = A.vox[pr.x], t = A.vox[pr.y];
        long long result = -1;
        bool handover = false;
        if (s >= 0 && t >= 0 && A.comp[s] == A.comp[t]) {
            for (int i = lane; i < kWarpSlots; i += 32) map[i] = kEmptySlot;
            const int tx = t % nx, ty = (t / nx) % ny, tz = t / nxy;
            const int sx = s % nx, sy = (s / nx) % ny, sz = s / nxy;
            const int tc = pack_xyz(tx, ty, tz), sc = pack_xyz(sx, sy, sz);
            const int h0 = (sx - tx) * (sx - tx) + (sy - ty) * (sy - ty) + (sz - tz) * (sz - tz);
            __syncwarp();
            if (lane == 0) {
                map[slot0(sc)] = static_cast<unsigned long long>(sc) << 32;  // g = 0
                open[0] = (static_cast<unsigned long long>(h0) << 42) |
                          (static_cast<unsigned long long>(h0) << 24) | static_cast<unsigned>(sc);
            }
            int len = 1, distinct = 1, expanded = 0;
            __syncwarp();
            for (;;) {
                // pop the smallest (f, h, voxel); four independent loads per round
                unsigned long long mine = ~0ull;
                int at = -1;
                for (int i = lane; i < len; i += 128) {
                    const unsigned long long k0 = open[i];
                    const unsigned long long k1 = i + 32 < len ? open[i + 32] : ~0ull;
                    const unsigned long long k2 = i + 64 < len ? open[i + 64] : ~0ull;
                    const unsigned long long k3 = i + 96 < len ? open[i + 96] : ~0ull;
                    if (k0 < mine) { mine = k0; at = i; }
                    if (k1 < mine) { mine = k1; at = i + 32; }
                    if (k2 < mine) { mine = k2; at = i + 64; }
                    if (k3 < mine) { mine = k3; at = i + 96; }
                }
                const unsigned long long top = warp_min_key(mine);
                if (top == ~0ull) break;  // the open list is exhausted
                if (mine == top) open[at] = ~0ull;
                const int c = static_cast<int>(top & 0xffffffu);
                const int h = static_cast<int>((top >> 24) & 0x3ffffu);
                const int g = static_cast<int>(top >> 42) - h;
                // its slot exists (inserted when it was pushed); the probe is
                // bounded all the same, and a miss hands the pair over
                unsigned sv = slot0(c);
                unsigned long long e = map[sv];
                for (int probe = 1; probe < kWarpSlots && cw(e) != c; ++probe) {
                    sv = (sv + 1) & (kWarpSlots - 1);
                    e = map[sv];
                }
                __syncwarp();
                if (cw(e) != c) {
                    handover = true;
                    break;
                }
                if (e & kClosedBit) continue;  // stale entry
                if (lane == 0) map[sv] = e | kClosedBit;
                if (c == tc) {
                    result = g;
                    break;
                }
                if (expanded >= A.max_exp) break;  // cap: blocked
                ++expanded;
                if (distinct + 26 > kWarpDistinct || len + 26 > kWarpOpen) {
                    handover = true;
                    break;
                }
                const int xx = (c & 0xff) + ddx, yy = ((c >> 8) & 0xff) + ddy, zz = (c >> 16) + ddz;
                bool push = false, inserted = false, lost = false;
                unsigned long long key = 0;
                if (lane < 26 && xx >= 0 && yy >= 0 && zz >= 0 && xx < nx && yy < ny && zz < nz &&
                    !__ldg(A.occ + (zz * ny + yy) * nx + xx)) {
                    const int u = pack_xyz(xx, yy, zz);
                    const int gu = g + step;
                    const unsigned long long want =
                        (static_cast<unsigned long long>(u) << 32) | static_cast<unsigned>(gu);
                    unsigned su = slot0(u);
                    // fewer than kWarpSlots voxels are ever inserted, so an
                    // empty slot ends the probe within kWarpSlots steps
                    lost = true;
                    for (int probe = 0; probe < kWarpSlots; ++probe) {
                        unsigned long long cur = map[su];
                        if (cur == kEmptySlot) {
                            cur = atomicCAS(map + su, kEmptySlot, want);
                            if (cur == kEmptySlot) {
                                inserted = push = true;
                                lost = false;
                                break;
                            }
                        }
                        if (cw(cur) == u) {
                            if (!(cur & kClosedBit) && gu < static_cast<int>(cur & 0xffffffffu)) {
                                map[su] = want;
                                push = true;
                            }
                            lost = false;
                            break;
                        }
                        su = (su + 1) & (kWarpSlots - 1);
                    }
                    if (push) {
                        const int hu =
                            (xx - tx) * (xx - tx) + (yy - ty) * (yy - ty) + (zz - tz) * (zz - tz);
                        key = (static_cast<unsigned long long>(gu + hu) << 42) |
                              (static_cast<unsigned long long>(hu) << 24) | static_cast<unsigned>(u);
                    }
                }
                if (__any_sync(0xffffffffu, lost)) {  // cannot happen (see above)
                    handover = true;
                    break;
                }
                const unsigned pb = __ballot_sync(0xffffffffu, push);
                if (push) open[len + __popc(pb & ((1u << lane) - 1u))] = key;
                len += __popc(pb);
                distinct += __popc(__ballot_sync(0xffffffffu, inserted));
                __syncwarp();
            }
        }
        if (lane == 0) {
            if (handover) {
                A.retry[k] = 1;
            } else {
                long long cost = result < 0 ? A.blocked_cost : result * A.unit_mm;
                if (cost > DPSO_COST_MAX) {
                    atomicOr(A.err, 2);
                    cost = DPSO_COST_MAX;
                }
                A.C[static_cast<size_t>(pr.x) * A.n + pr.y] = static_cast<int>(cost);
                A.C[static_cast<size_t>(pr.y) * A.n + pr.x] = static_cast<int>(cost);
            }
        }
        __syncwarp();
    }
}

// Connected components of the free voxels (26-neighbourhood) by union-find:
// every root ends at the smallest voxel index of its component whatever the
// order of the unions (hook the larger root under the smaller by CAS).
__device__ int cc_find(int* parent, int v) {
    int p = parent[v];
    while (p != v) {
        const int gp = parent[p];
        if (gp != p) parent[v] = gp;  // halve the path (benign races)
        v = p;
        p = gp;
    }
    return v;
}

__global__ void cc_init_kernel(const unsigned char* __restrict__ occ, long long nv, int* parent) {
    for (long long v = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; v < nv;
         v += static_cast<long long>(gridDim.x) * blockDim.x)
        parent[v] = occ[v] ? -1 : static_cast<int>(v);
}

__global__ void cc_union_kernel(AstarGrid gr, const unsigned char* __restrict__ occ, int* parent) {
    const long long nv = static_cast<long long>(gr.nx) * gr.ny * gr.nz;
    for (long long v = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; v < nv;
         v += static_cast<long long>(gridDim.x) * blockDim.x) {
        if (occ[v]) continue;
        const int x = static_cast<int>(v % gr.nx), y = static_cast<int>((v / gr.nx) % gr.ny),
                  z = static_cast<int>(v / (static_cast<long long>(gr.nx) * gr.ny));
        for (int d = 14; d < 27; ++d) {  // the 13 neighbours after v in index order
            const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
            const int xx = x + dx, yy = y + dy, zz = z + dz;
            if (xx < 0 || yy < 0 || zz < 0 || xx >= gr.nx || yy >= gr.ny || zz >= gr.nz) continue;
            const int u = (zz * gr.ny + yy) * gr.nx + xx;
            if (occ[u]) continue;
            int a = cc_find(parent, static_cast<int>(v)), b = cc_find(parent, u);
            while (a != b) {
                if (a > b) {
                    const int t = a;
                    a = b;
                    b = t;
                }
                const int old = atomicCAS(parent + b, b, a);  // hook root b under a
                if (old == b) break;
                b = cc_find(parent, old);
                a = cc_find(parent, a);
            }
        }
    }
}

__global__ void cc_flatten_kernel(long long nv, int* parent) {
    for (long long v = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; v < nv;
         v += static_cast<long long>(gridDim.x) * blockDim.x)
        if (parent[v] >= 0) parent[v] = cc_find(parent, static_cast<int>(v));
}

__global__ void zero_diagonal_kernel(int* C, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) C[static_cast<size_t>(i) * n + i] = 0;
}

constexpr int kPass1Expansions = 256;

int map_bits_for(long long entries) {
    int b = 4;
    while ((1ll << b) < 2 * entries) ++b;
    return b;
}

int check_params(const dpso_astar_params* ap) {
    if (!ap || !(ap->voxel_m > 0.0) || !isfinite(ap->voxel_m) || ap->inflate_r2 < 0 ||
        ap->unit_mm < 0 || ap->blocked_cost < 0 || ap->max_expansions < 0 || ap->reserved != 0)
        return DPSO_ERR_ARG;
    for (int k = 0; k < 3; ++k) {
        if (!isfinite(ap->origin[k]) || ap->dims[k] < 1 || ap->weights[k] < 0) return DPSO_ERR_ARG;
        if (ap->dims[k] > 4096 || ap->weights[k] > 1000) return DPSO_ERR_RANGE;
    }
    if (static_cast<long long>(ap->dims[0]) * ap->dims[1] * ap->dims[2] > INT_MAX ||
        ap->max_expansions > DPSO_ASTAR_MAX_EXPANSIONS || ap->inflate_r2 > 1024)
        return DPSO_ERR_RANGE;
    return DPSO_OK;
}

// The warp pass packs (f, h, voxel) into 22 + 18 + 24 bits: every grid
// dimension at most 256 (8 bits per packed coordinate), every heuristic
// (squared voxel distance) below 2^18, and every f = g + h below 2^22, where
// g <= (max_expansions + 2) x the largest step.
bool warp_pass_fits(const dpso_astar_params* ap) {
    long long hmax = 0;
    for (int k = 0; k < 3; ++k) hmax += static_cast<long long>(ap->dims[k] - 1) * (ap->dims[k] - 1);
    const long long gmax = (static_cast<long long>(ap->max_expansions) + 2) *
                           (static_cast<long long>(ap->weights[0]) + ap->weights[1] + ap->weights[2]);
    return ap->dims[0] <= 256 && ap->dims[1] <= 256 && ap->dims[2] <= 256 && hmax < (1ll << 18) &&
           gmax + hmax < (1ll << 22);
}

cudaError_t run_warp_pass(const WarpArgs& W, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int smem = kWarpsPerBlock * (kWarpOpen + kWarpSlots) * static_cast<int>(sizeof(unsigned long long));
    if (e == cudaSuccess)
        e = raise_smem_limit(astar_warp_kernel, smem);
    if (e != cudaSuccess) return e;
    const int blocks = std::max(1, std::min(sms, (W.npairs + kWarpsPerBlock - 1) / kWarpsPerBlock));
    astar_warp_kernel<<<blocks, 32 * kWarpsPerBlock, smem, st>>>(W);
    return cudaGetLastError();
}

AstarGrid grid_of(const dpso_astar_params* ap) {
    return AstarGrid{ap->origin[0], ap->origin[1], ap->origin[2], ap->voxel_m,
                     ap->dims[0],   ap->dims[1],   ap->dims[2]};
}

// One pass over `pairs` (device) in chunks that fit `budget` bytes of scratch.
cudaError_t run_pass(AstarArgs A, const int2* pairs, int npairs, size_t budget, cudaStream_t st) {
    const size_t per = static_cast<size_t>(A.heap_cap) * sizeof(OpenEntry) +
                       (size_t(1) << A.map_bits) * sizeof(MapSlot);
    const int chunk = static_cast<int>(std::max<size_t>(1, std::min<size_t>(npairs, budget / per)));
    OpenEntry* heap = nullptr;
    MapSlot* map = nullptr;
    cudaError_t e = cudaMallocAsync(&heap, per * chunk, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(heap, 0, per * chunk, st);  // map tags 0: no search owns a slot
    if (e != cudaSuccess) {
        cudaFreeAsync(heap, st);
        return e;
    }
    map = reinterpret_cast<MapSlot*>(reinterpret_cast<char*>(heap) +
                                     static_cast<size_t>(A.heap_cap) * sizeof(OpenEntry) * chunk);
    A.heap = heap;
    A.map = map;
    int* retry_base = A.retry;
    for (int first = 0; first < npairs && e == cudaSuccess; first += chunk) {
        A.pairs = pairs + first;
        A.npairs = std::min(chunk, npairs - first);
        A.stamp0 = first + 1;
        A.retry = retry_base ? retry_base + first : nullptr;
        astar_pairs_kernel<<<(A.npairs + 127) / 128, 128, 0, st>>>(A);
        e = cudaGetLastError();
    }
    cudaFreeAsync(heap, st);
    return e;
}

}  // namespace
}  // namespace dpso

using namespace dpso;

extern "C" {

void dpso_default_astar_params(dpso_astar_params* p) {
    if (!p) return;
    *p = dpso_astar_params{};
    p->voxel_m = 0.5;
    p->dims[0] = p->dims[1] = p->dims[2] = 1;
    p->weights[0] = p->weights[1] = p->weights[2] = 1;
    p->unit_mm = 500;
    p->blocked_cost = 100000000;
    p->max_expansions = 20000;
}

int dpso_voxel_occupancy(const double* boxes_dev, int32_t m, const dpso_astar_params* ap,
                         uint8_t* occ_dev, void* stream) {
    int st = check_params(ap);
    if (st) return st;
    if (!occ_dev || m < 0 || (m > 0 && !boxes_dev)) return DPSO_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const AstarGrid gr = grid_of(ap);
    const long long nv = static_cast<long long>(gr.nx) * gr.ny * gr.nz;
    unsigned char* core = nullptr;
    if (cudaMallocAsync(&core, nv, s) != cudaSuccess) {
        cudaGetLastError();
        return DPSO_ERR_NO_MEMORY;
    }
    int R = 0;
    while ((R + 1) * (R + 1) <= ap->inflate_r2) ++R;
    const int blocks = static_cast<int>(std::min<long long>((nv + 255) / 256, 65536));
    voxel_core_kernel<<<blocks, 256, 0, s>>>(gr, boxes_dev, m, core);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        voxel_inflate_kernel<<<blocks, 256, 0, s>>>(gr, ap->inflate_r2, R, core, occ_dev);
        e = cudaGetLastError();
    }
    cudaFreeAsync(core, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? DPSO_OK : DPSO_ERR_CUDA;
}

int dpso_cost_matrix_astar(const double* xyz_dev, int32_t n, const uint8_t* occ_dev,
                           const dpso_astar_params* ap, int32_t* C_dev, void* stream) {
    int st = check_params(ap);
    if (st) return st;
    if (!xyz_dev || !occ_dev || !C_dev || n < 1) return DPSO_ERR_ARG;
    if (n > DPSO_MAX_N) return DPSO_ERR_RANGE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long np = static_cast<long long>(n) * (n - 1) / 2;
    std::vector<int2> pairs;
    pairs.reserve(static_cast<size_t>(np));
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) pairs.push_back(make_int2(i, j));
    int *vox = nullptr, *retry = nullptr, *err = nullptr, *comp = nullptr;
    unsigned* queue = nullptr;
    int2* dpairs = nullptr;
    const long long nv = static_cast<long long>(ap->dims[0]) * ap->dims[1] * ap->dims[2];
    auto cleanup = [&](int code) {
        cudaFreeAsync(comp, s);
        cudaFreeAsync(vox, s);
        cudaFreeAsync(retry, s);
        cudaFreeAsync(err, s);
        cudaFreeAsync(dpairs, s);
        cudaFreeAsync(queue, s);
        cudaStreamSynchronize(s);
        return code;
    };
    if (cudaMallocAsync(&vox, sizeof(int) * n, s) != cudaSuccess ||
        cudaMallocAsync(&retry, sizeof(int) * std::max<long long>(np, 1), s) != cudaSuccess ||
        cudaMallocAsync(&err, sizeof(int), s) != cudaSuccess ||
        cudaMallocAsync(&comp, sizeof(int) * nv, s) != cudaSuccess ||
        cudaMallocAsync(&dpairs, sizeof(int2) * std::max<long long>(np, 1), s) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(DPSO_ERR_NO_MEMORY);
    }
    const AstarGrid gr = grid_of(ap);
    cudaError_t e = cudaMemsetAsync(retry, 0, sizeof(int) * std::max<long long>(np, 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess && np > 0)
        e = cudaMemcpyAsync(dpairs, pairs.data(), sizeof(int2) * np, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        viewpoint_voxel_kernel<<<(n + 127) / 128, 128, 0, s>>>(gr, xyz_dev, n, occ_dev, vox);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        zero_diagonal_kernel<<<(n + 127) / 128, 128, 0, s>>>(C_dev, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {  // components of the free voxels
        const int blocks = static_cast<int>(std::min<long long>((nv + 255) / 256, 65536));
        cc_init_kernel<<<blocks, 256, 0, s>>>(occ_dev, nv, comp);
        cc_union_kernel<<<blocks, 256, 0, s>>>(gr, occ_dev, comp);
        cc_flatten_kernel<<<blocks, 256, 0, s>>>(nv, comp);
        e = cudaGetLastError();
    }
    AstarArgs A{};
    A.gr = gr;
    A.occ = occ_dev;
    A.vox = vox;
    A.comp = comp;
    A.a1 = ap->weights[0];
    A.a2 = ap->weights[1];
    A.a3 = ap->weights[2];
    A.unit_mm = ap->unit_mm;
    A.blocked_cost = ap->blocked_cost;
    A.C = C_dev;
    A.n = n;
    A.err = err;
    constexpr size_t kBudget = size_t(4) << 30;  // scratch bytes per pass
    A.retry = retry;
    if (warp_pass_fits(ap)) {
        // pass 1: every pair, one warp per search in shared memory, the full
        // cap; searches that outgrow the warp's map or open array are retried
        WarpArgs W{};
        W.gr = gr;
        W.occ = occ_dev;
        W.vox = vox;
        W.comp = comp;
        W.pairs = dpairs;
        W.npairs = static_cast<int>(np);
        W.a1 = ap->weights[0];
        W.a2 = ap->weights[1];
        W.a3 = ap->weights[2];
        W.unit_mm = ap->unit_mm;
        W.blocked_cost = ap->blocked_cost;
        W.max_exp = ap->max_expansions;
        W.C = C_dev;
        W.n = n;
        W.retry = retry;
        W.err = err;
        A.final_pass = false;
        if (e == cudaSuccess && np > 0) {
            e = cudaMallocAsync(&queue, sizeof(unsigned), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(queue, 0, sizeof(unsigned), s);
            W.queue = queue;
            if (e == cudaSuccess) e = run_warp_pass(W, s);
        }
    } else {
        // pass 1: every pair, room for a short search
        const int e1 = std::min(kPass1Expansions, ap->max_expansions);
        A.max_exp = e1;
        A.final_pass = e1 == ap->max_expansions;
        A.heap_cap = 26 * e1 + 1;
        A.map_bits = map_bits_for(A.heap_cap);
        if (e == cudaSuccess && np > 0) e = run_pass(A, dpairs, static_cast<int>(np), kBudget, s);
    }
    // pass 2: the pairs that need more room, searched again from the start
    std::vector<int> flags(static_cast<size_t>(np));
    if (e == cudaSuccess && np > 0 && !A.final_pass) {
        e = cudaMemcpyAsync(flags.data(), retry, sizeof(int) * np, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        std::vector<int2> again;
        for (long long k = 0; k < np; ++k)
            if (flags[k]) again.push_back(pairs[k]);
        if (e == cudaSuccess && !again.empty()) {
            e = cudaMemcpyAsync(dpairs, again.data(), sizeof(int2) * again.size(),
                                cudaMemcpyHostToDevice, s);
            A.max_exp = ap->max_expansions;
            A.final_pass = true;
            A.heap_cap = 26 * ap->max_expansions + 1;
            A.map_bits = map_bits_for(A.heap_cap);
            A.retry = nullptr;
            if (e == cudaSuccess)
                e = run_pass(A, dpairs, static_cast<int>(again.size()), kBudget, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // `again` is read by the copy
        }
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaErrorMemoryAllocation) return cleanup(DPSO_ERR_NO_MEMORY);
    if (e != cudaSuccess) return cleanup(DPSO_ERR_CUDA);
    return cleanup(herr & 2 ? DPSO_ERR_RANGE : DPSO_OK);
}

}  // extern "C"
