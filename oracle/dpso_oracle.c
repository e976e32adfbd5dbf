/*
 * CPU oracle for the enhanced discrete PSO of Phung et al.,
 * "Enhanced Discrete Particle Swarm Optimization Path Planning for UAV
 * Vision-based Surface Inspection" (arXiv:1706.04399).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * reference that the CUDA library is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * Every step follows the paper's text in the paper's order:
 *   - Sec. 2.3            edge costs l_ij, blocked pairs get a very large cost
 *   - Eq. (min)           tour cost  sum l_ij lambda_ij
 *   - Sec. 3.1            positions, velocities as transposition lists, and the
 *                         operators x+v, x2-x1, v1 (+) v2, c.v
 *   - Eqs. (velocity), (position)   the particle update
 *   - Sec. 3.2.1          deterministic (back-and-forth) initialisation
 *   - Sec. 3.2.2          random mutation
 *   - Sec. 3.2.3          edge exchange (2-opt, best improvement)
 *   - Fig. "pseudocode"   the enhanced DPSO loop
 * Where the paper is silent the reading used is stated at the spot.
 *
 * Velocities are kept as literal transposition lists, as in Sec. 3.1 (the CUDA
 * path stores the permutation a list induces instead; the two agree exactly).
 *
 * Parity is pinned for: Philox (published known-answer vectors), the cost
 * matrix (hand-checkable integer grid values, exact dyadic blocking), the
 * operators (the Sec. 3.1 worked example and the algebraic definitions),
 * fitness (brute force over all tours for n <= 9 and closed-form grid optima),
 * 2-opt (2-optimality and per-move fitness deltas), mutation (kept particles
 * unchanged, disturbed count) and the loop (monotone gbest history, gbest =
 * min pbest, valid permutations).  The full stochastic trajectory has no
 * closed form: beyond those invariants it is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_DET_INIT 1
#define ORC_MUTATION 2
#define ORC_TWO_OPT 4
#define ORC_NODE_SWAP 8 /* the exchange swaps two nodes instead of two edges */

#define ORC_ERR_ARG (-1)
#define ORC_ERR_RANGE (-2)
#define ORC_ERR_MEM (-3)

#define ORC_COST_MAX (1 << 29)

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11.  Round: two 32x32->64 products of counter words */
/* 0 and 2 with the published multipliers, outputs permuted and xor-ed with  */
/* the key; the key is advanced by the published Weyl constants between     */
/* rounds.                                                                   */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One 32-bit draw.  Counter = (draw/4, particle, iteration, phase), key =
 * the 64-bit seed split into halves; the draw takes output word draw%4.
 * Phases: 1 = initial permutation, 2 = velocity coefficients, 3 = mutation. */
uint32_t orc_draw(uint64_t seed, uint32_t phase, uint32_t iter, uint32_t particle,
                  uint32_t draw)
{
    uint32_t ctr[4] = {draw >> 2, particle, iter, phase};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[draw & 3u];
}

/* Draws 0..count-1 of one (seed, phase, iteration, particle) stream. */
void orc_draws(uint64_t seed, uint32_t phase, uint32_t iter, uint32_t particle, int32_t count,
               uint32_t *out)
{
    for (int32_t d = 0; d < count; ++d)
        out[d] = orc_draw(seed, phase, iter, particle, (uint32_t)d);
}

/* Integer in [0, m) from a 32-bit draw: multiply-shift without rejection. */
static uint32_t bounded(uint32_t u, uint32_t m)
{
    return (uint32_t)(((uint64_t)u * (uint64_t)m) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.3: edge length l_ij between viewpoints.  Reading: the straight    */
/* segment's Euclidean length in millimetres, rounded to nearest (ties to    */
/* even) in FP64, plus a fixed penalty when the closed segment meets any     */
/* obstacle box grown by the UAV radius (the "very large cost" of a blocked  */
/* pair; the Sec. 2.2 voxel inflation made axis-aligned).                    */
/* ------------------------------------------------------------------------ */

/* Slab test of the closed segment p + t (q - p), t in [0,1], against the
 * closed box [lo - r, hi + r]. */
int orc_segment_blocked(const double *p, const double *q, const double *box, double r)
{
    double tmin = 0.0, tmax = 1.0;
    for (int k = 0; k < 3; ++k) {
        double lo = box[k] - r;
        double hi = box[3 + k] + r;
        double d = q[k] - p[k];
        if (d == 0.0) {
            if (p[k] < lo || p[k] > hi)
                return 0;
        } else {
            double t1 = (lo - p[k]) / d;
            double t2 = (hi - p[k]) / d;
            if (t1 > t2) {
                double t = t1;
                t1 = t2;
                t2 = t;
            }
            if (t1 > tmin)
                tmin = t1;
            if (t2 < tmax)
                tmax = t2;
        }
    }
    return tmin <= tmax;
}

/* C[i][j] for i<j, mirrored; zero diagonal.  Returns ORC_ERR_RANGE when an
 * entry exceeds 2^29 (the fixed-point range the integer deltas rely on). */
int orc_cost_matrix(const double *xyz, int32_t n, const double *boxes, int32_t m,
                    double radius, int32_t penalty, int32_t *C)
{
    if (n < 1 || m < 0 || penalty < 0)
        return ORC_ERR_ARG;
    int status = 0;
    for (int32_t i = 0; i < n; ++i) {
        C[(int64_t)i * n + i] = 0;
        for (int32_t j = i + 1; j < n; ++j) {
            const double *p = xyz + 3 * (int64_t)i;
            const double *q = xyz + 3 * (int64_t)j;
            double dx = q[0] - p[0];
            double dy = q[1] - p[1];
            double dz = q[2] - p[2];
            double s = dx * dx;
            s = s + dy * dy;
            s = s + dz * dz;
            double dist = sqrt(s);
            long long mm = llrint(1000.0 * dist);
            int blocked = 0;
            for (int32_t b = 0; b < m && !blocked; ++b)
                blocked = orc_segment_blocked(p, q, boxes + 6 * (int64_t)b, radius);
            long long v = mm + (blocked ? (long long)penalty : 0);
            if (v > ORC_COST_MAX) {
                status = ORC_ERR_RANGE;
                v = ORC_COST_MAX;
            }
            C[(int64_t)i * n + j] = (int32_t)v;
            C[(int64_t)j * n + i] = (int32_t)v;
        }
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2 edge costs by A* over a voxel grid (the alternative to the       */
/* straight segments above).  The grid is given: origin (m), voxel edge (m), */
/* dims[3] voxels, voxel (x, y, z) at index (z * ny + y) * nx + x with centre */
/* origin + (i + 0.5) * voxel per axis.                                      */
/* ------------------------------------------------------------------------ */

/* Occupancy: a voxel is occupied when its centre lies in a closed box, or
 * when its centre is within the UAV's sphere of such a voxel's centre:
 * dx^2 + dy^2 + dz^2 <= r2 in voxel units (r2 = the inflation radius
 * squared, in voxels^2, given as an integer). */
int orc_voxel_occupancy(const double *origin, double voxel, const int32_t *dims,
                        const double *boxes, int32_t m, int32_t r2, uint8_t *occ)
{
    int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    if (nx < 1 || ny < 1 || nz < 1 || m < 0 || r2 < 0 || !(voxel > 0.0))
        return ORC_ERR_ARG;
    int64_t nv = nx * ny * nz;
    uint8_t *core = (uint8_t *)calloc((size_t)nv, 1);
    if (!core)
        return ORC_ERR_MEM;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                double c[3] = {origin[0] + ((double)x + 0.5) * voxel,
                               origin[1] + ((double)y + 0.5) * voxel,
                               origin[2] + ((double)z + 0.5) * voxel};
                for (int32_t b = 0; b < m; ++b) {
                    const double *bx = boxes + 6 * (int64_t)b;
                    if (c[0] >= bx[0] && c[0] <= bx[3] && c[1] >= bx[1] && c[1] <= bx[4] &&
                        c[2] >= bx[2] && c[2] <= bx[5]) {
                        core[(z * ny + y) * nx + x] = 1;
                        break;
                    }
                }
            }
    int32_t R = 0;
    while ((int64_t)(R + 1) * (R + 1) <= r2)
        ++R;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                int o = 0;
                for (int32_t dz = -R; dz <= R && !o; ++dz)
                    for (int32_t dy = -R; dy <= R && !o; ++dy)
                        for (int32_t dx = -R; dx <= R && !o; ++dx) {
                            if (dx * dx + dy * dy + dz * dz > r2)
                                continue;
                            int64_t xx = x + dx, yy = y + dy, zz = z + dz;
                            if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz)
                                continue;
                            o = core[(zz * ny + yy) * nx + xx];
                        }
                occ[(z * ny + y) * nx + x] = (uint8_t)o;
            }
    free(core);
    return 0;
}

/* Open-list entry; the list pops the smallest (f, h, voxel).  Equal keys only
 * arise for repeated entries of one voxel, so the expansion order is the
 * same for any correct priority queue. */
typedef struct {
    int64_t f, h;
    int64_t v;
    int64_t g;
} orc_open;

static int open_less(const orc_open *a, const orc_open *b)
{
    if (a->f != b->f)
        return a->f < b->f;
    if (a->h != b->h)
        return a->h < b->h;
    return a->v < b->v;
}

typedef struct {
    orc_open *heap;
    int64_t len, cap;
    int64_t *best; /* best g per voxel, valid where stamp == cur */
    int32_t *stamp, *closed, cur;
} orc_astar_ws;

static void heap_push(orc_astar_ws *w, orc_open e)
{
    if (w->len == w->cap) {
        w->cap = w->cap ? 2 * w->cap : 1024;
        w->heap = (orc_open *)realloc(w->heap, sizeof(orc_open) * (size_t)w->cap);
    }
    int64_t i = w->len++;
    while (i > 0) {
        int64_t parent = (i - 1) / 2;
        if (!open_less(&e, &w->heap[parent]))
            break;
        w->heap[i] = w->heap[parent];
        i = parent;
    }
    w->heap[i] = e;
}

static orc_open heap_pop(orc_astar_ws *w)
{
    orc_open top = w->heap[0], last = w->heap[--w->len];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= w->len)
            break;
        if (c + 1 < w->len && open_less(&w->heap[c + 1], &w->heap[c]))
            ++c;
        if (!open_less(&w->heap[c], &last))
            break;
        w->heap[i] = w->heap[c];
        i = c;
    }
    if (w->len > 0)
        w->heap[i] = last;
    return top;
}

/* A* from voxel s to voxel t over free voxels, 26 neighbours, step cost
 * a[0] dx^2 + a[1] dy^2 + a[2] dz^2, heuristic the squared voxel distance to
 * t, closed voxels never reopened.  Returns the cost g of t, or -1 when t is
 * not reached before max_exp voxels other than t have been closed. */
static int64_t astar_one(const uint8_t *occ, const int32_t *dims, int64_t s, int64_t t,
                         const int32_t *a, int32_t max_exp, orc_astar_ws *w)
{
    int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    int64_t tx = t % nx, ty = (t / nx) % ny, tz = t / (nx * ny);
    ++w->cur;
    w->len = 0;
    int64_t sx = s % nx, sy = (s / nx) % ny, sz = s / (nx * ny);
    int64_t h0 = (sx - tx) * (sx - tx) + (sy - ty) * (sy - ty) + (sz - tz) * (sz - tz);
    w->stamp[s] = w->cur;
    w->best[s] = 0;
    orc_open e0 = {h0, h0, s, 0};
    heap_push(w, e0);
    int64_t expanded = 0;
    while (w->len > 0) {
        orc_open e = heap_pop(w);
        if (w->closed[e.v] == w->cur)
            continue;
        w->closed[e.v] = w->cur;
        if (e.v == t)
            return e.g;
        if (expanded >= max_exp)
            return -1;
        ++expanded;
        int64_t x = e.v % nx, y = (e.v / nx) % ny, z = e.v / (nx * ny);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dx && !dy && !dz)
                        continue;
                    int64_t xx = x + dx, yy = y + dy, zz = z + dz;
                    if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz)
                        continue;
                    int64_t v = (zz * ny + yy) * nx + xx;
                    if (occ[v] || w->closed[v] == w->cur)
                        continue;
                    int64_t g = e.g + (int64_t)a[0] * dx * dx + (int64_t)a[1] * dy * dy +
                                (int64_t)a[2] * dz * dz;
                    if (w->stamp[v] == w->cur && g >= w->best[v])
                        continue;
                    w->stamp[v] = w->cur;
                    w->best[v] = g;
                    int64_t h = (xx - tx) * (xx - tx) + (yy - ty) * (yy - ty) + (zz - tz) * (zz - tz);
                    orc_open ne = {g + h, h, v, g};
                    heap_push(w, ne);
                }
    }
    return -1;
}

/* C[i][j] = unit_mm * (A* cost from the voxel of viewpoint i to that of j),
 * i < j, mirrored, zero diagonal; blocked_cost where a viewpoint lies outside
 * the grid or in an occupied voxel, or no path was found within max_exp
 * expansions.  The voxel of a point is floor((p - origin) / voxel) per axis.
 * Returns ORC_ERR_RANGE (entries clamped) when an entry exceeds 2^29. */
int orc_cost_matrix_astar(const double *xyz, int32_t n, const uint8_t *occ,
                          const double *origin, double voxel, const int32_t *dims,
                          const int32_t *a, int32_t unit_mm, int32_t blocked_cost,
                          int32_t max_exp, int32_t *C)
{
    if (n < 1 || unit_mm < 0 || blocked_cost < 0 || max_exp < 0 || a[0] < 0 || a[1] < 0 ||
        a[2] < 0 || !(voxel > 0.0))
        return ORC_ERR_ARG;
    int64_t nx = dims[0], ny = dims[1], nz = dims[2], nv = nx * ny * nz;
    int64_t *vox = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    orc_astar_ws w = {0};
    w.best = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    w.stamp = (int32_t *)calloc((size_t)nv, sizeof(int32_t));
    w.closed = (int32_t *)calloc((size_t)nv, sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i) {
        int64_t c[3];
        int inside = 1;
        for (int k = 0; k < 3; ++k) {
            c[k] = (int64_t)floor((xyz[3 * (int64_t)i + k] - origin[k]) / voxel);
            inside &= c[k] >= 0 && c[k] < dims[k];
        }
        vox[i] = inside ? (c[2] * ny + c[1]) * nx + c[0] : -1;
        if (vox[i] >= 0 && occ[vox[i]])
            vox[i] = -1;
    }
    int status = 0;
    for (int32_t i = 0; i < n; ++i) {
        C[(int64_t)i * n + i] = 0;
        for (int32_t j = i + 1; j < n; ++j) {
            int64_t g = (vox[i] < 0 || vox[j] < 0) ? -1 : astar_one(occ, dims, vox[i], vox[j], a,
                                                                    max_exp, &w);
            int64_t v = g < 0 ? (int64_t)blocked_cost : g * unit_mm;
            if (v > ORC_COST_MAX) {
                status = ORC_ERR_RANGE;
                v = ORC_COST_MAX;
            }
            C[(int64_t)i * n + j] = (int32_t)v;
            C[(int64_t)j * n + i] = (int32_t)v;
        }
    }
    free(vox);
    free(w.heap);
    free(w.best);
    free(w.stamp);
    free(w.closed);
    return status;
}

/* Eq. (min) for the tour x (closing edge included). */
int64_t orc_fitness(const int32_t *C, int32_t n, const uint16_t *x)
{
    int64_t f = 0;
    for (int32_t k = 0; k < n; ++k)
        f += C[(int64_t)x[k] * n + x[(k + 1) % n]];
    return f;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1 operators.  A velocity is a list of transpositions of node      */
/* LABELS (the worked example (1,4,2,3,5,1)+((1,2),(2,3)) = (3,4,1,2,5,3)    */
/* changes n_1 itself, so a transposition swaps labels wherever they sit).   */
/* Lists are stored as 2*len uint16 values (a0,b0,a1,b1,...).               */
/* ------------------------------------------------------------------------ */

/* x + v: apply the transpositions in order. */
void orc_apply(uint16_t *x, int32_t n, const uint16_t *v, int64_t len)
{
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t k = 0; k < n; ++k)
        pos[x[k]] = k;
    for (int64_t e = 0; e < len; ++e) {
        uint16_t a = v[2 * e], b = v[2 * e + 1];
        int32_t pa = pos[a], pb = pos[b];
        x[pa] = b;
        x[pb] = a;
        pos[a] = pb;
        pos[b] = pa;
    }
    free(pos);
}

/* x2 - x1: the velocity v with x1 + v = x2.  Reading (the paper only states
 * the property): scan positions left to right and, where the running copy of
 * x1 differs from x2, emit the transposition (current label, wanted label).
 * This yields n - cycles(x2 o x1^-1) transpositions, the minimum.  v_out needs
 * room for 2*(n-1) values.  Returns the length. */
int64_t orc_subtract(const uint16_t *x2, const uint16_t *x1, int32_t n, uint16_t *v_out)
{
    uint16_t *y = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n);
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    memcpy(y, x1, sizeof(uint16_t) * (size_t)n);
    for (int32_t k = 0; k < n; ++k)
        pos[y[k]] = k;
    int64_t len = 0;
    for (int32_t k = 0; k < n; ++k) {
        if (y[k] != x2[k]) {
            uint16_t a = y[k], b = x2[k];
            v_out[2 * len] = a;
            v_out[2 * len + 1] = b;
            ++len;
            /* the transposition (a b) applied to y: a sits at k, b at pos[b] */
            int32_t pb = pos[b];
            y[k] = b;
            y[pb] = a;
            pos[b] = k;
            pos[a] = pb;
        }
    }
    free(pos);
    free(y);
    return len;
}

/* c.v keeps the first floor(c |v|) transpositions (Sec. 3.1, 0 < c <= 1).
 * Reading for the rounding: c = phi * r with r = u / 2^32, evaluated in
 * fixed point: cq = (phi_q u) >> 32 with phi_q = round(phi 2^32), then
 * k = (cq |v|) >> 32. */
static uint64_t fixed_q32(double c)
{
    return (uint64_t)llround(ldexp(c, 32));
}

static int64_t scaled_count(uint64_t phi_q, uint32_t u, int64_t len)
{
    uint64_t cq = (phi_q * (uint64_t)u) >> 32;
    return (int64_t)((cq * (uint64_t)len) >> 32);
}

/* Length kept by (phi r).v for a list of length len (exported for tests). */
int64_t orc_scaled_count(double phi, uint32_t u, int64_t len)
{
    return scaled_count(fixed_q32(phi), u, len);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2.1 deterministic initialisation: back-and-forth tours over the    */
/* grid tags.  Reading: variant s in 0..7 -- bit0 walks lines along columns  */
/* instead of rows, bit1 visits lines in descending order, bit2 flips the    */
/* direction of even lines; line L is walked forward iff (L odd) == bit2.    */
/* Faces are concatenated in ascending face id.                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t face, line, pos, node;
} orc_key;

static int key_cmp(const void *pa, const void *pb)
{
    const orc_key *a = (const orc_key *)pa, *b = (const orc_key *)pb;
    if (a->face != b->face)
        return a->face < b->face ? -1 : 1;
    if (a->line != b->line)
        return a->line < b->line ? -1 : 1;
    if (a->pos != b->pos)
        return a->pos < b->pos ? -1 : 1;
    return 0;
}

/* Back-and-forth order of variant s (0..7).  Returns ORC_ERR_ARG when tags
 * are negative or not unique. */
int orc_boustrophedon(const int32_t *tags, int32_t n, int32_t s, uint16_t *order)
{
    orc_key *k = (orc_key *)malloc(sizeof(orc_key) * (size_t)n);
    int bad = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t face = tags[3 * i], row = tags[3 * i + 1], col = tags[3 * i + 2];
        if (face < 0 || row < 0 || col < 0)
            bad = 1;
        int32_t line = (s & 1) ? col : row;
        int32_t pos = (s & 1) ? row : col;
        int backward = ((line & 1) != 0) != ((s & 4) != 0);
        k[i].face = face;
        k[i].line = (s & 2) ? -line : line;
        k[i].pos = backward ? -pos : pos;
        k[i].node = i;
    }
    qsort(k, (size_t)n, sizeof(orc_key), key_cmp);
    for (int32_t i = 0; i + 1 < n; ++i)
        if (key_cmp(&k[i], &k[i + 1]) == 0)
            bad = 1;
    for (int32_t i = 0; i < n; ++i)
        order[i] = (uint16_t)k[i].node;
    free(k);
    return bad ? ORC_ERR_ARG : 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2.3 edge exchange.  Every exchange of two non-adjacent edges      */
/* (x_i,x_i+1), (x_j,x_j+1) is evaluated; the one with the largest gain is  */
/* applied by reversing x[i+1..j]; repeated until no exchange improves.     */
/* Ties go to the smallest (i, j).  Returns moves applied.                  */
/* ------------------------------------------------------------------------ */
int64_t orc_two_opt(const int32_t *C, int32_t n, uint16_t *x, int64_t *f,
                    int32_t max_moves, int64_t *pairs_out)
{
    int64_t moves = 0, pairs = 0;
    for (;;) {
        if (max_moves > 0 && moves >= max_moves)
            break;
        int64_t best = 0;
        int32_t bi = -1, bj = -1;
        for (int32_t i = 0; i < n; ++i) {
            for (int32_t j = i + 2; j < n; ++j) {
                if (i == 0 && j == n - 1)
                    continue;
                int32_t a = x[i], b = x[i + 1], c = x[j], d = x[(j + 1) % n];
                int64_t delta = (int64_t)C[(int64_t)a * n + c] + C[(int64_t)b * n + d]
                                - C[(int64_t)a * n + b] - C[(int64_t)c * n + d];
                ++pairs;
                if (delta < best) {
                    best = delta;
                    bi = i;
                    bj = j;
                }
            }
        }
        if (bi < 0)
            break;
        for (int32_t lo = bi + 1, hi = bj; lo < hi; ++lo, --hi) {
            uint16_t t = x[lo];
            x[lo] = x[hi];
            x[hi] = t;
        }
        *f += best;
        ++moves;
    }
    if (pairs_out)
        *pairs_out += pairs;
    return moves;
}

/* ------------------------------------------------------------------------ */
/* Node-swap exchange (the "swap nodes(i,j) and evaluate fitness" reading of  */
/* the exchange in the paper's GPU listing): every pair of positions i < j of */
/* the cyclic tour is evaluated; the swap of x[i] and x[j] with the most      */
/* improvement is applied; repeated until no swap improves.  Ties go to the   */
/* smallest (i, j).  The change of a swap is the change of the edges that     */
/* touch position i or j, each counted once (adjacent positions share one).   */
/* Returns moves applied; *pairs_out grows by n(n-1)/2 per pass.              */
/* ------------------------------------------------------------------------ */
static int64_t swap_delta(const int32_t *C, int32_t n, const uint16_t *x, int32_t i, int32_t j)
{
    int32_t starts[4] = {(i - 1 + n) % n, i, (j - 1 + n) % n, j}; /* edge (k, k+1 mod n) */
    int32_t uniq[4], nu = 0;
    for (int q = 0; q < 4; ++q) {
        int seen = 0;
        for (int r = 0; r < nu; ++r)
            seen |= uniq[r] == starts[q];
        if (!seen)
            uniq[nu++] = starts[q];
    }
    int64_t before = 0, after = 0;
    for (int r = 0; r < nu; ++r) {
        int32_t u = uniq[r], v = (uniq[r] + 1) % n;
        before += C[(int64_t)x[u] * n + x[v]];
        int32_t xu = u == i ? x[j] : (u == j ? x[i] : x[u]);
        int32_t xv = v == i ? x[j] : (v == j ? x[i] : x[v]);
        after += C[(int64_t)xu * n + xv];
    }
    return after - before;
}

int64_t orc_node_swap(const int32_t *C, int32_t n, uint16_t *x, int64_t *f,
                      int32_t max_moves, int64_t *pairs_out)
{
    int64_t moves = 0, pairs = 0;
    for (;;) {
        if (max_moves > 0 && moves >= max_moves)
            break;
        int64_t best = 0;
        int32_t bi = -1, bj = -1;
        for (int32_t i = 0; i < n; ++i) {
            for (int32_t j = i + 1; j < n; ++j) {
                int64_t delta = swap_delta(C, n, x, i, j);
                ++pairs;
                if (delta < best) {
                    best = delta;
                    bi = i;
                    bj = j;
                }
            }
        }
        if (bi < 0)
            break;
        uint16_t t = x[bi];
        x[bi] = x[bj];
        x[bj] = t;
        *f += best;
        ++moves;
    }
    if (pairs_out)
        *pairs_out += pairs;
    return moves;
}

/* ------------------------------------------------------------------------ */
/* The swarm and the loop of Fig. "pseudocode".                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint16_t *t; /* 2*len labels */
    int64_t len, cap;
} orc_vel;

typedef struct {
    int32_t n, S;
    int32_t *C;
    double w, phi1, phi2;
    int32_t mut_period, mut_swaps, det_frac_pct, stall_limit, flags, trigger, max_moves;
    uint64_t seed;
    uint16_t *X, *P, *G;
    int64_t *F, *PF, gf;
    orc_vel *V;
    int32_t t, stall, done;
    int64_t *hist;
    int32_t hist_len, hist_cap;
    int64_t pairs, moves, two_opt_runs;
    int32_t last_improved, last_two_opt;
    /* a generation between orc_swarm_iterate_begin and _end: its number, the
     * gbest cost it started from, whether the exchange runs */
    int32_t gen_t, gen_open, gen_exchange;
    int64_t gen_gf0;
    uint16_t *scratch; /* 2*(n-1) transpositions */
} orc_swarm;

static int vel_reserve(orc_vel *v, int64_t len)
{
    if (len <= v->cap)
        return 0;
    int64_t cap = v->cap ? v->cap : 16;
    while (cap < len)
        cap *= 2;
    uint16_t *t = (uint16_t *)realloc(v->t, sizeof(uint16_t) * 2 * (size_t)cap);
    if (!t)
        return ORC_ERR_MEM;
    v->t = t;
    v->cap = cap;
    return 0;
}

static int vel_append(orc_vel *v, const uint16_t *t, int64_t len)
{
    if (vel_reserve(v, v->len + len))
        return ORC_ERR_MEM;
    memcpy(v->t + 2 * v->len, t, sizeof(uint16_t) * 2 * (size_t)len);
    v->len += len;
    return 0;
}

void orc_swarm_free(orc_swarm *sw)
{
    if (!sw)
        return;
    if (sw->V)
        for (int32_t p = 0; p < sw->S; ++p)
            free(sw->V[p].t);
    free(sw->V);
    free(sw->C);
    free(sw->X);
    free(sw->P);
    free(sw->G);
    free(sw->F);
    free(sw->PF);
    free(sw->hist);
    free(sw->scratch);
    free(sw);
}

static uint16_t *row_of(uint16_t *A, int32_t n, int32_t p)
{
    return A + (int64_t)p * n;
}

/* gbest = the particle with the smallest (pbest fitness, index); the
 * swarm's best is replaced only on strict improvement (Fig. "pseudocode"). */
void orc_swarm_gbest(orc_swarm *sw)
{
    int32_t bp = 0;
    for (int32_t p = 1; p < sw->S; ++p)
        if (sw->PF[p] < sw->PF[bp])
            bp = p;
    if (sw->PF[bp] < sw->gf) {
        sw->gf = sw->PF[bp];
        memcpy(sw->G, row_of(sw->P, sw->n, bp), sizeof(uint16_t) * (size_t)sw->n);
    }
}

static void pbest(orc_swarm *sw, int32_t p)
{
    if (sw->F[p] < sw->PF[p]) {
        sw->PF[p] = sw->F[p];
        memcpy(row_of(sw->P, sw->n, p), row_of(sw->X, sw->n, p),
               sizeof(uint16_t) * (size_t)sw->n);
    }
}

/* Initialisation block of Fig. "pseudocode": positions (some back-and-forth,
 * the rest random), fitness, pbest = itself, empty velocity, gbest.
 * Reading of "10% specific": n_det = max(1, floor(S * pct / 100)) particles
 * take variant p%8 rotated left by floor(p/8); the others are Fisher-Yates
 * shuffles of the identity driven by phase-1 draws. */
orc_swarm *orc_swarm_new(const int32_t *C, int32_t n, const int32_t *tags, int32_t S,
                         double w, double phi1, double phi2, int32_t mut_period,
                         int32_t mut_swaps, int32_t det_frac_pct, int32_t stall_limit,
                         int32_t flags, int32_t trigger, int32_t max_moves, uint64_t seed,
                         int32_t *status)
{
    *status = 0;
    if (n < 3 || n > 65535 || S < 1 || S > 65535 || !(w >= 0.0 && w <= 1.0) ||
        !(phi1 >= 0.0 && phi1 <= 1.0) || !(phi2 >= 0.0 && phi2 <= 1.0) || mut_period < 1 ||
        mut_swaps < 0 || det_frac_pct < 0 || det_frac_pct > 100 || stall_limit < 0 ||
        max_moves < 0 || trigger < 0 || trigger > 1) {
        *status = ORC_ERR_ARG;
        return NULL;
    }
    orc_swarm *sw = (orc_swarm *)calloc(1, sizeof(orc_swarm));
    sw->n = n;
    sw->S = S;
    sw->w = w;
    sw->phi1 = phi1;
    sw->phi2 = phi2;
    sw->mut_period = mut_period;
    sw->mut_swaps = mut_swaps;
    sw->det_frac_pct = det_frac_pct;
    sw->stall_limit = stall_limit;
    sw->flags = flags;
    sw->trigger = trigger;
    sw->max_moves = max_moves;
    sw->seed = seed;
    size_t nn = (size_t)n * (size_t)n;
    sw->C = (int32_t *)malloc(sizeof(int32_t) * nn);
    memcpy(sw->C, C, sizeof(int32_t) * nn);
    sw->X = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n * (size_t)S);
    sw->P = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n * (size_t)S);
    sw->G = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n);
    sw->F = (int64_t *)malloc(sizeof(int64_t) * (size_t)S);
    sw->PF = (int64_t *)malloc(sizeof(int64_t) * (size_t)S);
    sw->V = (orc_vel *)calloc((size_t)S, sizeof(orc_vel));
    sw->scratch = (uint16_t *)malloc(sizeof(uint16_t) * 2 * (size_t)n);
    sw->hist_cap = 64;
    sw->hist = (int64_t *)malloc(sizeof(int64_t) * (size_t)sw->hist_cap);

    int32_t n_det = 0;
    if ((flags & ORC_DET_INIT) && tags) {
        n_det = (int32_t)(((int64_t)S * det_frac_pct) / 100);
        if (n_det < 1)
            n_det = 1;
        if (n_det > S)
            n_det = S;
    }
    uint16_t *orders = (uint16_t *)malloc(sizeof(uint16_t) * 8 * (size_t)n);
    if (n_det > 0) {
        for (int32_t s = 0; s < 8; ++s) {
            if (orc_boustrophedon(tags, n, s, orders + (int64_t)s * n) != 0) {
                *status = ORC_ERR_ARG;
                free(orders);
                orc_swarm_free(sw);
                return NULL;
            }
        }
    }
    for (int32_t p = 0; p < S; ++p) {
        uint16_t *x = row_of(sw->X, n, p);
        if (p < n_det) {
            const uint16_t *ord = orders + (int64_t)(p % 8) * n;
            int32_t rot = (p / 8) % n;
            for (int32_t k = 0; k < n; ++k)
                x[k] = ord[(k + rot) % n];
        } else {
            for (int32_t k = 0; k < n; ++k)
                x[k] = (uint16_t)k;
            for (int32_t i = n - 1; i >= 1; --i) {
                uint32_t u = orc_draw(seed, 1, 0, (uint32_t)p, (uint32_t)(n - 1 - i));
                int32_t j = (int32_t)bounded(u, (uint32_t)(i + 1));
                uint16_t t = x[i];
                x[i] = x[j];
                x[j] = t;
            }
        }
        sw->F[p] = orc_fitness(sw->C, n, x);
        sw->PF[p] = sw->F[p];
        memcpy(row_of(sw->P, n, p), x, sizeof(uint16_t) * (size_t)n);
        sw->V[p].len = 0;
    }
    free(orders);
    int32_t bp = 0;
    for (int32_t p = 1; p < S; ++p)
        if (sw->F[p] < sw->F[bp])
            bp = p;
    sw->gf = sw->F[bp];
    memcpy(sw->G, row_of(sw->X, n, bp), sizeof(uint16_t) * (size_t)n);
    return sw;
}

/* Eqs. (velocity) and (position) for one particle, against the gbest G0 of
 * the start of the iteration (the gbest is updated after the particle loop,
 * Fig. "pseudocode").  v <- w.v (+) phi1 r1.(P - x) (+) phi2 r2.(G - x);
 * x <- x + v; fitness; pbest on strict improvement.  r1, r2 are one draw
 * each per particle per iteration (phase 2, draws 0 and 1).  With w = 1 the
 * list is kept whole; for w < 1 it is first replaced by the canonical list of
 * the permutation it induces, (identity + v) - identity, and then truncated. */
static int move_particle(orc_swarm *sw, int32_t p, int32_t t, const uint16_t *G0)
{
    int32_t n = sw->n;
    uint16_t *x = row_of(sw->X, n, p);
    orc_vel *v = &sw->V[p];
    uint32_t u1 = orc_draw(sw->seed, 2, (uint32_t)t, (uint32_t)p, 0);
    uint32_t u2 = orc_draw(sw->seed, 2, (uint32_t)t, (uint32_t)p, 1);
    uint64_t w_q = fixed_q32(sw->w);

    if (w_q < ((uint64_t)1 << 32)) {
        uint16_t *id = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n);
        for (int32_t k = 0; k < n; ++k)
            id[k] = (uint16_t)k;
        uint16_t *perm = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n);
        memcpy(perm, id, sizeof(uint16_t) * (size_t)n);
        orc_apply(perm, n, v->t, v->len);
        int64_t len = orc_subtract(perm, id, n, sw->scratch);
        int64_t keep = (int64_t)((w_q * (uint64_t)len) >> 32);
        v->len = 0;
        if (vel_append(v, sw->scratch, keep))
            return ORC_ERR_MEM;
        free(perm);
        free(id);
    }

    int64_t la = orc_subtract(row_of(sw->P, n, p), x, n, sw->scratch);
    int64_t ka = scaled_count(fixed_q32(sw->phi1), u1, la);
    if (vel_append(v, sw->scratch, ka))
        return ORC_ERR_MEM;
    int64_t lb = orc_subtract(G0, x, n, sw->scratch);
    int64_t kb = scaled_count(fixed_q32(sw->phi2), u2, lb);
    if (vel_append(v, sw->scratch, kb))
        return ORC_ERR_MEM;

    orc_apply(x, n, v->t, v->len);
    sw->F[p] = orc_fitness(sw->C, n, x);
    pbest(sw, p);
    return 0;
}

int orc_swarm_move(orc_swarm *sw, int32_t t)
{
    uint16_t *G0 = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)sw->n);
    memcpy(G0, sw->G, sizeof(uint16_t) * (size_t)sw->n);
    int st = 0;
    for (int32_t p = 0; p < sw->S && !st; ++p)
        st = move_particle(sw, p, t, G0);
    free(G0);
    return st;
}

/* Sec. 3.2.2 random mutation.  Readings: particles are ordered by (fitness,
 * index); a particle is identical to an earlier one in that order when the
 * tour arrays are equal; the first ceil(S/3) distinct particles are kept and
 * every other particle is disturbed by mut_swaps swaps of two distinct
 * positions (phase-3 draws 2q, 2q+1), its velocity emptied, then re-scored
 * and its pbest updated.  kept_out (may be NULL) receives 1 for kept. */
typedef struct {
    int64_t f;
    int32_t p;
} orc_fi;

static int fi_cmp(const void *pa, const void *pb)
{
    const orc_fi *a = (const orc_fi *)pa, *b = (const orc_fi *)pb;
    if (a->f != b->f)
        return a->f < b->f ? -1 : 1;
    return a->p < b->p ? -1 : (a->p > b->p);
}

int orc_swarm_mutate(orc_swarm *sw, int32_t t, int32_t *kept_out)
{
    int32_t n = sw->n, S = sw->S;
    orc_fi *ord = (orc_fi *)malloc(sizeof(orc_fi) * (size_t)S);
    for (int32_t p = 0; p < S; ++p) {
        ord[p].f = sw->F[p];
        ord[p].p = p;
    }
    qsort(ord, (size_t)S, sizeof(orc_fi), fi_cmp);
    int32_t *kept = (int32_t *)calloc((size_t)S, sizeof(int32_t));
    int32_t K = (S + 2) / 3, nkept = 0;
    for (int32_t r = 0; r < S; ++r) {
        int32_t p = ord[r].p;
        int dup = 0;
        for (int32_t q = r - 1; q >= 0 && ord[q].f == ord[r].f && !dup; --q)
            dup = memcmp(row_of(sw->X, n, ord[q].p), row_of(sw->X, n, p),
                         sizeof(uint16_t) * (size_t)n) == 0;
        if (!dup && nkept < K) {
            kept[p] = 1;
            ++nkept;
        }
    }
    for (int32_t p = 0; p < S; ++p) {
        if (kept[p])
            continue;
        uint16_t *x = row_of(sw->X, n, p);
        for (int32_t q = 0; q < sw->mut_swaps; ++q) {
            uint32_t ui = orc_draw(sw->seed, 3, (uint32_t)t, (uint32_t)p, (uint32_t)(2 * q));
            uint32_t uj = orc_draw(sw->seed, 3, (uint32_t)t, (uint32_t)p, (uint32_t)(2 * q + 1));
            int32_t i = (int32_t)bounded(ui, (uint32_t)n);
            int32_t j = (int32_t)bounded(uj, (uint32_t)(n - 1));
            if (j >= i)
                ++j;
            uint16_t tmp = x[i];
            x[i] = x[j];
            x[j] = tmp;
        }
        sw->V[p].len = 0;
        sw->F[p] = orc_fitness(sw->C, n, x);
        pbest(sw, p);
    }
    if (kept_out)
        memcpy(kept_out, kept, sizeof(int32_t) * (size_t)S);
    free(kept);
    free(ord);
    return 0;
}

/* Edge exchange on a subset of particles (all when idx == NULL), then pbest. */
void orc_swarm_two_opt(orc_swarm *sw, const int32_t *idx, int32_t count)
{
    int32_t total = idx ? count : sw->S;
    for (int32_t r = 0; r < total; ++r) {
        int32_t p = idx ? idx[r] : r;
        if (sw->flags & ORC_NODE_SWAP)
            sw->moves += orc_node_swap(sw->C, sw->n, row_of(sw->X, sw->n, p), &sw->F[p],
                                       sw->max_moves, &sw->pairs);
        else
            sw->moves += orc_two_opt(sw->C, sw->n, row_of(sw->X, sw->n, p), &sw->F[p],
                                     sw->max_moves, &sw->pairs);
        pbest(sw, p);
    }
}

/* The edge exchange (then pbest) of particles idx[0..count-1], with its
 * pair and move counts written to out[0], out[1] instead of being added to
 * the swarm's counters: it reads and writes only those particles' rows, so
 * calls on disjoint particle sets may run at the same time.  The caller adds
 * the counts with orc_swarm_add_counters. */
void orc_swarm_two_opt_part(orc_swarm *sw, const int32_t *idx, int32_t count, int64_t out[2])
{
    int64_t pairs = 0, moves = 0;
    for (int32_t r = 0; r < count; ++r) {
        int32_t p = idx[r];
        if (sw->flags & ORC_NODE_SWAP)
            moves += orc_node_swap(sw->C, sw->n, row_of(sw->X, sw->n, p), &sw->F[p],
                                   sw->max_moves, &pairs);
        else
            moves += orc_two_opt(sw->C, sw->n, row_of(sw->X, sw->n, p), &sw->F[p],
                                 sw->max_moves, &pairs);
        pbest(sw, p);
    }
    out[0] = pairs;
    out[1] = moves;
}

void orc_swarm_add_counters(orc_swarm *sw, int64_t pairs, int64_t moves)
{
    sw->pairs += pairs;
    sw->moves += moves;
}

static void hist_put(orc_swarm *sw, int32_t t, int64_t v)
{
    if (t > sw->hist_cap) {
        while (sw->hist_cap < t)
            sw->hist_cap *= 2;
        sw->hist = (int64_t *)realloc(sw->hist, sizeof(int64_t) * (size_t)sw->hist_cap);
    }
    sw->hist[t - 1] = v;
    if (t > sw->hist_len)
        sw->hist_len = t;
}

/* One generation of Fig. "pseudocode": move all particles, mutate every
 * mut_period-th generation, update gbest, and run the edge exchange when the
 * gbest did not strictly improve in this generation (trigger 0), or only in
 * mutation generations that did not improve it (trigger 1, the wording of
 * Sec. 4).
 *
 * The generation is split in two around the exchange so that a caller may
 * run the exchange itself (it is independent per particle):
 * orc_swarm_iterate_begin does everything up to the exchange and sets
 * *run_exchange; orc_swarm_iterate_end does what follows it (gbest, history,
 * stall).  orc_swarm_iterate runs begin, the exchange of every particle in
 * index order, and end.  Returns 1 when the loop has stopped (stall limit),
 * a negative code on error, else 0. */
int orc_swarm_iterate_begin(orc_swarm *sw, int32_t *run_exchange)
{
    *run_exchange = 0;
    if (sw->done)
        return 1;
    if (sw->gen_open)
        return ORC_ERR_ARG;
    int32_t t = sw->t + 1;
    sw->gen_gf0 = sw->gf;
    int st = orc_swarm_move(sw, t);
    if (st)
        return st;
    int mut = (sw->flags & ORC_MUTATION) && (t % sw->mut_period == 0);
    if (mut)
        orc_swarm_mutate(sw, t, NULL);
    orc_swarm_gbest(sw);
    int improved = sw->gf < sw->gen_gf0;
    hist_put(sw, t, sw->gf);
    sw->gen_t = t;
    sw->gen_open = 1;
    sw->gen_exchange = (sw->flags & ORC_TWO_OPT) && !improved && (sw->trigger == 0 || mut);
    *run_exchange = sw->gen_exchange;
    return 0;
}

int orc_swarm_iterate_end(orc_swarm *sw)
{
    if (!sw->gen_open)
        return ORC_ERR_ARG;
    int32_t t = sw->gen_t;
    sw->last_two_opt = sw->gen_exchange;
    if (sw->gen_exchange) {
        sw->two_opt_runs += 1;
        orc_swarm_gbest(sw);
        hist_put(sw, t, sw->gf);
    }
    int improved = sw->gf < sw->gen_gf0;
    sw->last_improved = improved;
    sw->stall = improved ? 0 : sw->stall + 1;
    sw->t = t;
    sw->gen_open = 0;
    if (sw->stall_limit > 0 && sw->stall >= sw->stall_limit)
        sw->done = 1;
    return 0;
}

int orc_swarm_iterate(orc_swarm *sw)
{
    int32_t run2 = 0;
    int st = orc_swarm_iterate_begin(sw, &run2);
    if (st)
        return st;
    if (run2)
        orc_swarm_two_opt(sw, NULL, 0);
    return orc_swarm_iterate_end(sw);
}

int orc_swarm_run(orc_swarm *sw, int32_t iterations)
{
    for (int32_t k = 0; k < iterations; ++k) {
        int st = orc_swarm_iterate(sw);
        if (st < 0)
            return st;
        if (sw->done)
            break;
    }
    return 0;
}

/* ---- accessors for the Python wrapper ---- */
int32_t orc_swarm_n(const orc_swarm *sw) { return sw->n; }
int32_t orc_swarm_size(const orc_swarm *sw) { return sw->S; }
int32_t orc_swarm_t(const orc_swarm *sw) { return sw->t; }
int32_t orc_swarm_done(const orc_swarm *sw) { return sw->done; }
int32_t orc_swarm_stall(const orc_swarm *sw) { return sw->stall; }
int64_t orc_swarm_gf(const orc_swarm *sw) { return sw->gf; }
int32_t orc_swarm_last_two_opt(const orc_swarm *sw) { return sw->last_two_opt; }
int32_t orc_swarm_last_improved(const orc_swarm *sw) { return sw->last_improved; }

void orc_swarm_counters(const orc_swarm *sw, int64_t out[3])
{
    out[0] = sw->pairs;
    out[1] = sw->moves;
    out[2] = sw->two_opt_runs;
}

/* Copies out X, P (S*n), G (n), F, PF (S), and V as the permutation each list
 * induces on the identity (S*n).  Any pointer may be NULL. */
void orc_swarm_export(const orc_swarm *sw, uint16_t *X, uint16_t *P, uint16_t *G,
                      int64_t *F, int64_t *PF, uint16_t *Vperm)
{
    size_t sn = (size_t)sw->S * (size_t)sw->n;
    if (X)
        memcpy(X, sw->X, sizeof(uint16_t) * sn);
    if (P)
        memcpy(P, sw->P, sizeof(uint16_t) * sn);
    if (G)
        memcpy(G, sw->G, sizeof(uint16_t) * (size_t)sw->n);
    if (F)
        memcpy(F, sw->F, sizeof(int64_t) * (size_t)sw->S);
    if (PF)
        memcpy(PF, sw->PF, sizeof(int64_t) * (size_t)sw->S);
    if (Vperm) {
        for (int32_t p = 0; p < sw->S; ++p) {
            uint16_t *y = Vperm + (int64_t)p * sw->n;
            for (int32_t k = 0; k < sw->n; ++k)
                y[k] = (uint16_t)k;
            orc_apply(y, sw->n, sw->V[p].t, sw->V[p].len);
        }
    }
}

/* Snapshot replay: replaces the swarm's state with one taken from another
 * run of the same loop (same instance and parameters), so that the next
 * generations of both can be compared.  Arrays as orc_swarm_export writes
 * them: X, P (S*n), G (n), F, PF (S), and Vperm (S*n), each velocity given
 * as the permutation it induces on the identity.  A velocity is stored as the
 * list Sec. 3.1's subtraction gives for it, (identity + v) - identity: x + v
 * depends only on that permutation (every transposition swaps two labels),
 * w.v with w = 1 keeps the list whole, and with w < 1 the list is first
 * replaced by exactly this canonical list, so the loop continues as it would
 * from the original lists.  gf, t, stall, done: the loop state; hist: the
 * t gbest costs so far; counters: the exchange's pairs, moves and runs.
 * Returns ORC_ERR_ARG, leaving the swarm unchanged, when a row of X, P, G or
 * Vperm is not a permutation of 0..n-1 or t < 0; ORC_ERR_MEM when out of
 * memory. */
static int is_perm(const uint16_t *x, int32_t n, uint8_t *seen)
{
    memset(seen, 0, (size_t)n);
    for (int32_t k = 0; k < n; ++k) {
        if (x[k] >= n || seen[x[k]])
            return 0;
        seen[x[k]] = 1;
    }
    return 1;
}

int orc_swarm_import(orc_swarm *sw, const uint16_t *X, const uint16_t *P, const uint16_t *G,
                     const int64_t *F, const int64_t *PF, const uint16_t *Vperm, int64_t gf,
                     int32_t t, int32_t stall, int32_t done, const int64_t *hist,
                     const int64_t counters[3])
{
    int32_t n = sw->n, S = sw->S;
    if (t < 0 || stall < 0)
        return ORC_ERR_ARG;
    uint8_t *seen = (uint8_t *)malloc((size_t)n);
    uint16_t *id = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n);
    if (!seen || !id) {
        free(seen);
        free(id);
        return ORC_ERR_MEM;
    }
    int ok = is_perm(G, n, seen);
    for (int32_t p = 0; p < S && ok; ++p)
        ok = is_perm(X + (int64_t)p * n, n, seen) && is_perm(P + (int64_t)p * n, n, seen) &&
             is_perm(Vperm + (int64_t)p * n, n, seen);
    free(seen);
    if (!ok) {
        free(id);
        return ORC_ERR_ARG;
    }
    for (int32_t k = 0; k < n; ++k)
        id[k] = (uint16_t)k;
    for (int32_t p = 0; p < S; ++p) {
        int64_t len = orc_subtract(Vperm + (int64_t)p * n, id, n, sw->scratch);
        sw->V[p].len = 0;
        if (vel_append(&sw->V[p], sw->scratch, len)) {
            free(id);
            return ORC_ERR_MEM;
        }
    }
    free(id);
    size_t sn = (size_t)S * (size_t)n;
    memcpy(sw->X, X, sizeof(uint16_t) * sn);
    memcpy(sw->P, P, sizeof(uint16_t) * sn);
    memcpy(sw->G, G, sizeof(uint16_t) * (size_t)n);
    memcpy(sw->F, F, sizeof(int64_t) * (size_t)S);
    memcpy(sw->PF, PF, sizeof(int64_t) * (size_t)S);
    sw->gf = gf;
    sw->t = t;
    sw->stall = stall;
    sw->done = done != 0;
    sw->gen_open = 0;
    sw->hist_len = 0;
    for (int32_t k = 1; k <= t; ++k)
        hist_put(sw, k, hist[k - 1]);
    sw->pairs = counters[0];
    sw->moves = counters[1];
    sw->two_opt_runs = counters[2];
    return 0;
}

int64_t orc_swarm_vel_len(const orc_swarm *sw, int32_t p) { return sw->V[p].len; }

int32_t orc_swarm_history(const orc_swarm *sw, int64_t *out, int32_t cap)
{
    int32_t k = sw->hist_len < cap ? sw->hist_len : cap;
    if (out && k > 0)
        memcpy(out, sw->hist, sizeof(int64_t) * (size_t)k);
    return sw->hist_len;
}
