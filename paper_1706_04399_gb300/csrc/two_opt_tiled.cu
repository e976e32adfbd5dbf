// Edge exchange of Sec. 3.2.3 (best-improvement 2-opt to 2-optimality), the
// pipelined tiled variant for tours whose 33-row tiles fit in shared memory.
//
// Same mathematics and tie order as two_opt.cu:
//   delta(i, j) = C[x_i][x_j] + C[x_i+1][x_j+1] - C[x_i][x_i+1] - C[x_j][x_j+1],
//   the applied move is the smallest (delta, i, j) with delta < 0.
//
// Layout and mapping:
//  * A persistent grid takes tours from a work queue; a tour is solved by 8
//    warps (8 / TPC when a CTA holds TPC short tours, 16 when two tile
//    subgroups of 8 warps evaluate two tiles of a pass at once).
//  * A tile is R positions I..I+R-1 (R = 32 or 30; fewer for long tours), one
//    per lane; its R+1 cost rows C[x_I..x_I+R] are staged in shared memory,
//    one bulk copy per row, posted by a few lanes of every warp of the group
//    and counted on an mbarrier (a tile costs a handful of instructions instead
//    of one 16-byte copy per lane-chunk).
//  * 16-byte copies need 16-byte-aligned rows, which alone would put rows a,
//    a+8, a+16, a+24 in the same bank.  The cost matrix is therefore kept in
//    four copies whose rows are shifted right by 0..3 words; row a of a tile is
//    taken from copy (a>>3)&3 into a row pitch ldq with ldq/4 odd, so the 32
//    lanes reading one column hit 32 distinct banks.  Eight-row tiles need no
//    shift (at a pitch with pitch/4 odd, rows 0..7, and rows 1..8, each fall
//    on distinct bank quads; a lane reads rows r and r + 1): their
//    segment-tile kernels stage from copy 0 at a compile-time pitch class, so
//    that a lane's two rows are a constant apart.
//  * Column records rec[c] = {4 x_c+1, -C[x_c][x_c+1]} give the second
//    gather's byte offset and the edge term in one broadcast load; the first
//    gather's offset 4 x_c is the previous record's.
//  * Each lane tracks, over its columns in increasing order (groups of four),
//    the minimum of C[x_i][x_c] + C[x_i+1][x_c+1] - C[x_c][x_c+1] and the
//    first group holding it, with selects only (no divergent branch in the
//    column loop).  Subtracting C[x_i][x_i+1] gives a candidate (delta, i,
//    group) as a packed 64-bit key; the warps of a tile fold theirs per row.
//  * Row cache: each row's smallest improving key (delta < 0; else none)
//    survives from pass to pass.  A move that reverses positions a+1..b
//    changes the deltas of rows a..b, and of rows below a only in columns
//    a..b; rows past b keep theirs.  The next pass stages only the rows
//    C[x_a..x_b+1] of the reversed segment, in segment tiles starting at a:
//    each evaluates its own rows over every column and, since C is
//    symmetric (C[x_i][x_j] = C[x_j][x_i]), every row i < a over its columns
//    j in the tile, with one j per lane reading the staged rows C[x_j],
//    C[x_j+1] at x_i, x_i+1 (the same two gathers per pair, conflict-free;
//    the minimum over j is taken across lanes, only for groups where some
//    lane holds an improving pair).  Rows below a whose cached move lay in a
//    group touching a..b are evaluated afresh in full, in the grid tiles that
//    hold them.  The pass's move is the smallest cached key; its exact column
//    and the two new edge costs are read from C.
//  * Pairs with j = i+1 and (0, n-1) have delta = 0 for a symmetric C and
//    never win, so only the triangle at the start of each tile is masked.
#include <climits>

#include "tiled_common.cuh"

namespace dpso {
namespace {

using namespace tiled;

// Builds copy k (k = 0..3) of C with every row shifted right by k words:
// Cs[(k n + r) ldq + k + l] = C[r][l], zeros elsewhere.
__global__ void shift_copies_kernel(const int* __restrict__ C, int ldc, int n, int ldq,
                                    int* __restrict__ Cs) {
    const int r = blockIdx.x, k = blockIdx.y;
    int* dst = Cs + (static_cast<size_t>(k) * n + r) * ldq;
    for (int w = threadIdx.x; w < ldq; w += blockDim.x) {
        const int l = w - k;
        dst[w] = (l >= 0 && l < n) ? C[static_cast<size_t>(r) * ldc + l] : 0;
    }
}

}  // namespace

// Tours of at least this many viewpoints use segment tiles (see the kernel).
constexpr int kSegmentMinN = 512;

// Compile-time pitches (words) of the staged rows of 8-row segment tiles with
// one tour per CTA: 256 k + 4 for k = 2..16, each 4 times an odd number.
constexpr int kPitchStep = 256, kPitchMin = 2, kPitchMax = 16;

// The staged rows' pitch for tours of up to n viewpoints: the smallest
// compile-time class holding a row for 8-row segment tiles with one tile in
// flight (n >= kSegmentMinN; tours per CTA must be 1 for segment tiles, and a
// larger class only costs shared memory elsewhere), else the row size itself.
__host__ __device__ inline int staged_pitch(int n, int rows, int stages) {
    const int ld = shifted_ld(n);
    if (rows != 8 || stages != 1 || n < kSegmentMinN) return ld;
    const int k = (ld - 4 + kPitchStep - 1) / kPitchStep;
    return k <= kPitchMax ? kPitchStep * max(k, kPitchMin) + 4 : ld;
}

// Tiles of a tour's fixed tile grid (rows 0..n-3 in tiles of `rows`).
__host__ __device__ inline int grid_tiles(int n, int rows) { return (n - 2 + rows - 1) / rows; }

size_t two_opt_tiled_smem(int n, int rows_per_tile, int stages) {
    const size_t rows = static_cast<size_t>(stages) * (rows_per_tile + 1) *
                        staged_pitch(n, rows_per_tile, stages) * sizeof(int);
    const size_t rec = static_cast<size_t>(n + 4) * sizeof(int2);
    const size_t xs = static_cast<size_t>((n + 1 + 7) / 8 * 8) * sizeof(uint16_t);
    // the row cache
    const size_t cache = static_cast<size_t>((n + 1) & ~1) * sizeof(uint64_t);
    // the pass's need-tile bitmask (words) and list (uint16), 8-byte multiples
    const int nt = grid_tiles(n, rows_per_tile);
    const size_t bits = static_cast<size_t>((nt + 63) / 64 * 2) * sizeof(unsigned);
    const size_t list = static_cast<size_t>((nt + 3) / 4 * 4) * sizeof(uint16_t);
    return rows + rec + xs + cache + bits + list;
}

namespace {

// Record term of the padding columns past n.  A padding column evaluates to
// a + b + kPadCost with a, b <= DPSO_COST_MAX = 2^29, at most 2^31 - 1, so the
// int32 sum cannot wrap; its delta (that minus the row's own edge, <= 2^29)
// is at least 2^29 - 1 > 0, so padding never supplies an improving move.
constexpr int kPadCost = (1 << 30) - 1;

static_assert(2LL * DPSO_COST_MAX + kPadCost <= INT_MAX, "padding column overflows");
static_assert(static_cast<long long>(kPadCost) - DPSO_COST_MAX > 0, "padding column improves");

// Barrier over the WPT warps that own one tour: the whole block when a CTA
// holds one tour, else named barrier 1 + group (WPT * 32 threads).
template <int TPC>
__device__ __forceinline__ void group_sync(int grp) {
    constexpr int kCount = kThreads / TPC;
    if constexpr (TPC == 1) {
        __syncthreads();
    } else {
        // constant barrier ids (grp is uniform per warp), so only TPC + 1 of
        // the 16 hardware barriers are reserved
        switch (grp) {
            case 0: asm volatile("bar.sync 1, %0;\n" ::"n"(kCount) : "memory"); break;
            case 1: asm volatile("bar.sync 2, %0;\n" ::"n"(kCount) : "memory"); break;
            case 2: asm volatile("bar.sync 3, %0;\n" ::"n"(kCount) : "memory"); break;
            default: asm volatile("bar.sync 4, %0;\n" ::"n"(kCount) : "memory"); break;
        }
    }
}

// Barrier over the 8 warps of tile subgroup `half` of a tour that two
// subgroups share (TG = 2; the tour owns the whole CTA): named barrier
// 1 + half.  With TG = 1 it is the tour's barrier.
template <int TPC, int TG>
__device__ __forceinline__ void half_sync(int grp, int half) {
    if constexpr (TG == 1) {
        group_sync<TPC>(grp);
    } else if (half == 0) {
        asm volatile("bar.sync 1, %0;\n" ::"n"(kThreads) : "memory");
    } else {
        asm volatile("bar.sync 2, %0;\n" ::"n"(kThreads) : "memory");
    }
}

// ROWS: tile height (positions per tile, one per lane).  TPC: tours per CTA;
// the 8 warps split into TPC groups of 8 / TPC warps, each solving its own
// tour in its own slice of shared memory (`group_words` ints, 128-byte
// aligned), so short tours still give every warp a long column range.
// TG: tile subgroups per tour (TPC = 1 only): with TG = 2 the CTA has 16
// warps and evaluates two tiles of the same pass at once, each 8-warp
// subgroup with its own tile buffer and barrier, so a tour's passes take
// about half as long (a shorter tail when tours need very different pass
// counts) for the same shared memory and warps per SM as two CTAs.
// Resident CTAs per SM the register budget is sized for: two for the
// 16-warp shapes and for one long tour per CTA (16- and 8-row tiles, where
// shared memory holds at most two CTAs), four for 30-row tiles, else three.
template <int ROWS, int TPC, int TG>
constexpr int tiled_min_blocks() {
    return TG == 2 || (TPC == 1 && ROWS <= 16) ? 2 : (ROWS == 30 ? 4 : 3);
}

// SEG: segment tiles (launches whose longest tour has n >= kSegmentMinN;
// one tour per CTA), else partial tiles.  Each kernel holds only its own
// mode's code: with both compiled in, short tours ran 6-10 % slower.
// PITCH: 0, or (8-row segment tiles, one tour per CTA) the staged rows' pitch
// in words as a compile-time constant (a class at least the tour's row size,
// PITCH/4 odd).  Nine rows at such a pitch need no word shift for conflict-
// free columns (rows 0..7, and rows 1..8, each fall on distinct bank quads;
// row 8 only ever serves as a lane's second row), so a lane's second row is
// its first plus a constant and both gathers of a label share one address:
// C[x_i][y] at r1 + 4y and C[x_i+1][y] at r1 + 4y + 4 PITCH.
template <int ROWS, int TPC, int TG, bool SEG, int PITCH = 0>
__global__ void __launch_bounds__(kThreads * TG, (tiled_min_blocks<ROWS, TPC, TG>()))
    two_opt_tiled_kernel(TwoOptBatch b, int group_words) {
    static_assert(!SEG || TPC == 1, "segment tiles are instantiated for one tour per CTA");
    static_assert(TG == 1 || TPC == 1, "two tile subgroups need the whole CTA");
    static_assert(PITCH == 0 || (SEG && ROWS == 8 && TPC == 1 && TG == 1 && PITCH % 8 == 4),
                  "a compile-time pitch is for 8-row segment tiles, 4 times an odd number");
    constexpr int kPB = PITCH * 4;     // bytes from a staged row to the next (PITCH > 0)
    constexpr int kRows = ROWS;        // positions per tile, one per lane
    constexpr int kStaged = ROWS + 1;  // cost rows staged per tile
    // Tiles of 16 or 8 rows (long tours) split each warp into 2 or 4 lane
    // groups that evaluate the same rows over different column ranges, so no
    // lane idles; the groups' minima per row meet by shuffles.
    constexpr int SPLIT = ROWS == 8 ? 4 : (ROWS == 16 ? 2 : 1);
    constexpr int WPT = kWarps * TG / TPC;  // warps per tour
    constexpr int WSG = WPT / TG;           // warps per tile subgroup
    constexpr int GT = WPT * 32;            // threads per tour
    // A group's shared slice seen through three element types (all alias its
    // start): TG tile buffers of kStaged x (staged pitch) ints, then the column records
    // (n + 4 int2, the last four padding), then the tour (n + 1 uint16).
    // Offsets depend on the tour's n; slices are sized for the largest n.
    extern __shared__ __align__(128) int sm_all[];
    __shared__ unsigned long long s_best[TPC];
    __shared__ unsigned int s_next[TPC];     // tiles taken in this pass (TG = 2)
    __shared__ int s_tile[TPC * TG * 2];     // a subgroup's next tile, by parity
    // s_part: the tour's work item, then each pass's need-tile count, then
    // the winning column (each read after a barrier, before the next write)
    __shared__ int s_part[TPC], s_e0[TPC], s_e1[TPC], s_p[TPC];
    __shared__ int s_mode[TPC * TG];         // short tours: 1 when the subgroup's tile is full
    __shared__ long long s_pf[TPC], s_f[TPC];
    // The tour's task descriptor, its running cost and the subgroups' counts of
    // evaluated pairs live in shared memory rather than registers: they are
    // read once per pass, tile or tour, and registers are what limits this
    // kernel to 64 per thread.
    __shared__ TwoOptTask s_task[TPC];
    __shared__ unsigned long long s_evals[TPC * TG];
    // tile-arrival barrier per tile subgroup; a subgroup whose tile copy did
    // not complete sets its own abort flag (read by its own threads after its
    // barrier, by the whole tour after a tour barrier)
    __shared__ __align__(8) unsigned long long s_mbar[TPC * TG];
    __shared__ int s_abort[TPC * TG];

    const int lane = threadIdx.x & 31;
    const int grp = (threadIdx.x >> 5) / WPT;  // tour group
    const int warp = (threadIdx.x >> 5) % WPT; // warp within the group
    const int half = warp / WSG;               // tile subgroup within the tour
    const int wsg = warp % WSG;                // warp within the tile subgroup
    const int tid = threadIdx.x % GT;          // thread within the group
    int* smi = sm_all + static_cast<size_t>(grp) * group_words;
    int2* smi2 = reinterpret_cast<int2*>(smi);
    const int4* smi4 = reinterpret_cast<const int4*>(smi);
    uint16_t* smu = reinterpret_cast<uint16_t*>(smi);

    const int sg = grp * TG + half;  // this thread's tile subgroup slot
    const unsigned mbar = smem_addr(&s_mbar[sg]);
    unsigned phase = 0;  // parity of the tile-arrival phase to wait for
    if (tid % (WSG * 32) == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_abort[sg] = 0;
    }
    auto tour_aborted = [&]() {  // after a tour barrier: uniform over the tour
        bool ab = false;
#pragma unroll
        for (int h = 0; h < TG; ++h) ab = ab || s_abort[grp * TG + h] != 0;
        return ab;
    };
    for (;;) {
        if (tid == 0) s_part[grp] = static_cast<int>(atomicAdd(b.queue, 1u));
        group_sync<TPC>(grp);
        const int g = s_part[grp];
        if (g >= b.total) break;
        if (tid == 0) {
            const int prob = find_inst(b.off, b.nprob, g);
            s_task[grp] = b.tasks[prob];
            const int* order = b.tasks[prob].order;
            s_p[grp] = order ? order[g - b.off[prob]] : g - b.off[prob];
        }
        group_sync<TPC>(grp);
        const TwoOptTask& a = s_task[grp];
        const int p = s_p[grp];
        if (a.gate && *a.gate == 0) {  // this problem does not exchange edges now
            group_sync<TPC>(grp);
            continue;
        }
        const int n = a.n;
        const int ldq = shifted_ld(n);                 // the row-shifted copies' pitch
        const int spitch = PITCH > 0 ? PITCH : ldq;    // the staged rows' pitch
        const int buf_words = kStaged * spitch;
        const int rec2 = TG * buf_words / 2;    // int2 index of record 0 (even)
        const int xs16 = (rec2 + n + 4) * 4;    // uint16 index of x_0
        // u64 index of the row cache, after the tour (n + 1 uint16, padded)
        const int rk64 = (xs16 + (n + 1 + 7) / 8 * 8 + 3) / 4;
        const int ntiles = grid_tiles(n, kRows);  // grid tiles start at I <= n-3
        // the pass's need-tile bitmask (u32 index) and list (uint16 index)
        const int nb32 = 2 * (rk64 + ((n + 1) & ~1));
        const int nl16 = 2 * (nb32 + (ntiles + 63) / 64 * 2);
        const int guard = 1000 + 100 * n;
        // segment tiles in launches holding long tours, whose rows are long
        // enough that staging them costs more than the passes' fixed overhead
        // (GB300 measurements: partial tiles 10-25 % faster below n = 400,
        // 3 % slower at 600, 27 % slower at 1992); every tour of such a
        // launch takes them, so the partial-tile path is not compiled in
        constexpr bool segmode = SEG;

        // The subgroup stages the `count` cost rows of the tile starting at I:
        // warp w posts the kPerWarp rows of slot w - 1 (warp 0 the last slot,
        // empty for most tile heights), one bulk copy per lane (row r from
        // shifted copy (r>>3)&3), so the copies are issued by several warps at
        // once rather than one after another by one warp.  Lane 0 of one warp
        // arms the barrier with the tile's bytes afterwards (a copy that lands
        // before that only takes the transaction count below zero: the phase
        // still waits for that one arrival).  Offsets into the shifted copies
        // fit 32 bits (4 n ldq words < 2^30).
        constexpr int kPerWarp = (kStaged + WSG - 1) / WSG;
        const unsigned tile_s = smem_addr(smi + half * buf_words);
        const unsigned row_bytes = static_cast<unsigned>(ldq) * 4u;
        const unsigned slot_bytes = static_cast<unsigned>(spitch) * 4u;
        auto stage = [&](int I, int count) {
            // the subgroup barrier before this ordered the generic reads of
            // the previous tile; this orders them before the async writes
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            const int r = ((wsg + WSG - 1) % WSG) * kPerWarp + lane;
            if (lane < kPerWarp && r < count) {
                const unsigned k = PITCH > 0 ? 0u : (r >> 3) & 3;
                const unsigned off = (k * static_cast<unsigned>(n) + smu[xs16 + I + r]) * row_bytes;
                bulk_row(tile_s + r * slot_bytes, reinterpret_cast<const char*>(a.Cs) + off,
                         row_bytes, mbar);
            }
        };
        // Every thread waits for the tile's bytes, at most ~2 s of clock; a
        // copy that never lands sets the group's abort flag and the status.
        auto stage_wait = [&]() {
            unsigned done = 0;
            const long long t0 = clock64();
            while (!done) {
                asm volatile(
                    "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
                    "selp.u32 %0, 1, 0, p; }\n"
                    : "=r"(done) : "r"(mbar), "r"(phase) : "memory");
                if (!done && clock64() - t0 > (1ll << 32)) {
                    s_abort[sg] = 1;
                    if (a.status) atomicExch(a.status, DPSO_ERR_TIMEOUT);
                    break;
                }
            }
            phase ^= 1u;
        };

        {
            const uint16_t* tour = a.tours + static_cast<size_t>(p) * a.ldt;
            for (int i = tid; i < n; i += GT) smu[xs16 + i] = tour[i];
            if (tid == 0) smu[xs16 + n] = tour[0];
        }
        group_sync<TPC>(grp);
        for (int c = tid; c < n; c += GT) {
            const int u = smu[xs16 + c], v = smu[xs16 + c + 1];
            smi2[rec2 + c] = make_int2(4 * v, -a.C[static_cast<size_t>(u) * a.ldc + v]);
        }
        if (tid < 4) smi2[rec2 + n + tid] = make_int2(0, kPadCost);
        if (tid == 0) s_f[grp] = a.cost[p];
        if (wsg == 0 && lane == 0) s_evals[sg] = 0;
        int moves = 0, passes = 0;
        group_sync<TPC>(grp);

        // Row cache: rowkey[i] is the smallest (delta, i, column) of row i
        // over all its columns when that delta is negative (an improving
        // move), else ~0, as of the last pass that evaluated the row.  A move
        // that reverses positions pa+1..pb changes the pairs of rows pa..pb
        // and, for rows below pa, only columns pa..pb; rows above pb keep
        // theirs.  The warps fold their keys into it with shared atomicMin.
        unsigned long long* const rowkey = reinterpret_cast<unsigned long long*>(smi) + rk64;
        unsigned* const needbits = reinterpret_cast<unsigned*>(smi) + nb32;
        uint16_t* const needlist = smu + nl16;
        int pa = -1, pb = -1;  // the previous move; pb < 0: evaluate every pair
        if (tid == 0) {
            s_best[grp] = ~0ull;
            s_next[grp] = 0;
        }
        for (int w = tid; w < (ntiles + 31) / 32; w += GT) needbits[w] = 0;
        group_sync<TPC>(grp);

        for (;;) {
            if (a.max_moves > 0 && moves >= a.max_moves) break;
            if (moves >= guard) {
                if (tid == 0 && a.status) atomicExch(a.status, DPSO_ERR_INTERNAL);
                break;
            }
            const bool first = pb < 0;
            // The pass's tiles.  First pass: every grid tile, in full.  After a
            // move (pa, pb), long tours (segment mode): nseg segment tiles of
            // rows pa.., starting at pa, whose staged rows pa..pb+1 also serve
            // every row below pa over columns pa..pb (C is symmetric:
            // C[x_i][x_j] = C[x_j][x_i]); then the grid tiles holding a row
            // below pa whose cached improving move lay in a group touching
            // pa..pb (its row is evaluated afresh in full).  Keys of the rows
            // evaluated in full are reset first.  Short tours (rows of a few
            // hundred bytes, cheap to stage): the grid tiles up to pb, last
            // first; a tile holding rows of pa..pb, or a row whose cached move
            // lay in a group touching pa..pb, in full, the others only in the
            // groups of columns covering pa..pb.
            int nseg = 0;
            if (segmode && first) {
                for (int r = tid; r <= n - 3; r += GT) rowkey[r] = ~0ull;
            } else if (segmode) {
                nseg = (pb - pa + kRows) / kRows;
                for (int r = tid; r <= min(pb, n - 3); r += GT) {
                    if (r >= pa) {
                        rowkey[r] = ~0ull;
                    } else {
                        const unsigned long long k = rowkey[r];
                        const int cmc = static_cast<int>(k & 0xffffu);
                        if (k != ~0ull && cmc + 3 >= pa && cmc <= pb) {
                            rowkey[r] = ~0ull;
                            atomicOr(&needbits[(r / kRows) >> 5], 1u << ((r / kRows) & 31));
                        }
                    }
                }
            }
            if (segmode) group_sync<TPC>(grp);  // (short tours: full tiles reset their own rows)
            if (!first && segmode && warp == 0) {
                // compact the need bitmask into a list (one warp; at most 32
                // words: n <= 4145 tours have at most 518 grid tiles) and clear it
                const int nw = (ntiles + 31) / 32;
                const unsigned bits = lane < nw ? needbits[lane] : 0u;
                const int cnt = __popc(bits);
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                int pos = incl - cnt;
                for (unsigned b = bits; b; b &= b - 1) needlist[pos++] = static_cast<uint16_t>(32 * lane + __ffs(b) - 1);
                if (lane < nw) needbits[lane] = 0u;
                if (lane == 31) s_part[grp] = incl;  // (the work item is no longer needed this tour)
            }
            if (segmode && !first) group_sync<TPC>(grp);
            const int tlast = first ? ntiles - 1 : min(ntiles - 1, pb / kRows);
            const int ntot = first || !segmode ? tlast + 1 : nseg + s_part[grp];
            // Tiles are taken in order (segment tiles first; short tours: the
            // grid tiles from the last one down); with two
            // subgroups each takes the next one when it finishes its own
            // (s_tile, double-buffered by tile parity, published before the
            // subgroup barrier that the readers pass).
            int par = 0, taken = 0;
            if (TG == 2 && wsg == 0 && lane == 0)
                s_tile[sg * 2] = static_cast<int>(atomicAdd(&s_next[grp], 1u));
            for (;;) {
                half_sync<TPC, TG>(grp, half);  // the previous tile is no longer read
                if (s_abort[sg]) break;  // read after the barrier: the subgroup agrees
                const int t = TG == 1 ? taken : s_tile[sg * 2 + par];
                if (t >= ntot) break;
                ++taken;
                const bool seg = segmode && !first && t < nseg;
                const int I = !segmode || first ? (tlast - t) * kRows
                                                : (seg ? pa + t * kRows : needlist[t - nseg] * kRows);
                // staged rows I..I+count-1; rows evaluated I..rlast
                const int count = seg ? min(kStaged, pb + 2 - I) : min(kStaged, n - 1 - I);
                const int rlast = seg ? min(min(I + kRows - 1, pb), n - 3)
                                      : (first || !segmode ? n - 3 : min(pa - 1, n - 3));
                stage(I, count);
                // the barrier is armed by warp 0 for short tours (which first
                // decides the tile's mode) and by the last warp for long ones
                if (wsg == (segmode ? WSG - 1 : 0)) {
                    if (!segmode) {
                        // short tours: the tile's mode; a full tile starts its
                        // rows' keys afresh.  Both before the barrier arrival
                        // that the other warps acquire.
                        bool full = first || (I <= pb && I + kRows - 1 >= pa);
                        const int i = I + lane;
                        const bool row_ok = lane < kRows && i <= n - 3;
                        if (!full) {
                            bool need = false;
                            if (row_ok) {
                                const unsigned long long k = rowkey[i];
                                const int cmc = static_cast<int>(k & 0xffffu);
                                need = k != ~0ull && cmc + 3 >= pa && cmc <= pb;
                            }
                            full = __any_sync(0xffffffffu, need);
                        }
                        if (full && row_ok) rowkey[i] = ~0ull;
                        if (lane == 0) s_mode[sg] = full ? 1 : 0;
                    }
                    __syncwarp();
                    if (lane == 0) mbar_expect(mbar, static_cast<unsigned>(count) * row_bytes);
                }
                stage_wait();
                const bool full = segmode || s_mode[sg] != 0;
                // the row this lane evaluates (lanes past the tile height idle
                // on a valid row unless the tile splits the warp); byte offsets
                // of its two staged rows (row start plus its 0..3 word shift)
                const int lrow = SPLIT > 1 ? (lane & (kRows - 1)) : min(lane, kRows - 1);
                const int part = SPLIT > 1 ? lane / kRows : 0;
                const int ie = I + lrow;
                const bool eval_ok = (SPLIT > 1 || lane < kRows) && ie <= rlast;
                const int ra = lrow, rb1 = lrow + 1;
                const int shift1 = PITCH > 0 ? 0 : (ra >> 3) & 3;
                const int shift2 = PITCH > 0 ? 0 : (rb1 >> 3) & 3;
                const int p1 = half * buf_words + ra * spitch + shift1;
                const int p2 = half * buf_words + rb1 * spitch + shift2;
                const char* const r1 = reinterpret_cast<const char*>(smi + p1);
                const char* const r2 = reinterpret_cast<const char*>(smi + p2);
                auto at = [](const char* row, int off) {
                    return *reinterpret_cast<const int*>(row + off);
                };
                // the lane's second row at byte offset off (with a compile-time
                // pitch: the first row's address of that label plus kPB)
                auto at2 = [&](int off) {
                    if constexpr (PITCH > 0)
                        return *reinterpret_cast<const int*>((r1 + off) + kPB);
                    else
                        return at(r2, off);
                };
                // (a) the tile's rows over every column: groups of four from
                // the even column at or below I+2 (records are read in pairs),
                // contiguous per warp; the records past n are padding
                // (partial tiles of short tours: the groups of the tile's
                // grid that hold pa..pb)
                int cstart = (I + 2) & ~1, cstop = n;
                if (!full) {
                    cstart = I + 2 + ((max(pa, I + 2) - I - 2) & ~3);
                    cstop = min(n, pb + 1);
                }
                const int ngroups = cstop > cstart ? (cstop - cstart + 3) >> 2 : 0;
                // groups starting below I+kStaged hold the diagonal triangle
                // (masked).  Where a warp splits into lane groups (8/16-row
                // tiles) they go one per lane group, so that none runs them
                // alone while the rest of its warp waits; the other groups are
                // split evenly, contiguous per warp and per lane group.  With
                // one row per lane they stay at the start of warp 0's range
                // (a warp runs its masked groups instead of as many unmasked ones).
                const int nmask =
                    SPLIT > 1 ? min(ngroups, max(0, (I + kStaged - cstart + 3) >> 2)) : 0;
                const int nrest = ngroups - nmask;
                const int cs2 = cstart + 4 * nmask;
                const int g0 = (nrest * wsg) / WSG, g1 = (nrest * (wsg + 1)) / WSG;
                // (the counting rotates over the warps, tile by tile)
                if (wsg == t % WSG) {
                    // pairs (i, j), i+2 <= j <= n-1, (i, j) != (0, n-1), of the rows
                    // evaluated (in the columns cstart..E-1), and of the rows
                    // below pa against the segment's columns (segment tiles)
                    const int i = I + lane;
                    const bool row_ok = lane < kRows && i <= rlast;
                    const int E = min(cstart + 4 * ngroups, n);
                    int cnt = row_ok ? max(0, E - max(cstart, i + 2)) : 0;
                    cnt -= (i == 0 && E == n && cnt > 0) ? 1 : 0;
                    if (seg && pa > 0 && lane < kRows && I + lane <= pb) {
                        const int j = I + lane;
                        cnt += pa - (j == pa ? 1 : 0) - (j == n - 1 ? 1 : 0);
                    }
                    const unsigned tc = __reduce_add_sync(0xffffffffu, static_cast<unsigned>(cnt));
                    if (lane == 0) s_evals[sg] += tc;
                }
                {
                    // this lane group's share of the warp's groups
                    int h0 = g0, h1 = g1;
                    if constexpr (SPLIT > 1) {
                        h0 = g0 + ((g1 - g0) * part) / SPLIT;
                        h1 = g0 + ((g1 - g0) * (part + 1)) / SPLIT;
                    }
                    // first valid column of this lane's row (rows past rlast have none)
                    const int lim = eval_ok ? ie + 2 : INT_MAX;
                    int m = INT_MAX, cm = 0;
                    int c = 0, q = 0;
                    const int4* rp = smi4;
                    auto group = [&](bool masked) {
                        const int4 ra4 = rp[0], rb4 = rp[1];
                        int v0 = at(r1, q) + at2(ra4.x) + ra4.y;
                        int v1 = at(r1, ra4.x) + at2(ra4.z) + ra4.w;
                        int v2 = at(r1, ra4.z) + at2(rb4.x) + rb4.y;
                        int v3 = at(r1, rb4.x) + at2(rb4.z) + rb4.w;
                        if (masked) {
                            v0 = c >= lim ? v0 : INT_MAX;
                            v1 = c + 1 >= lim ? v1 : INT_MAX;
                            v2 = c + 2 >= lim ? v2 : INT_MAX;
                            v3 = c + 3 >= lim ? v3 : INT_MAX;
                        }
                        const int mv = min(min(v0, v1), min(v2, v3));
                        cm = mv < m ? c : cm;  // first group holding the lane minimum
                        m = min(m, mv);
                        q = rb4.z;
                        c += 4;
                        rp += 2;
                    };
                    // this lane group's triangle groups first (its lowest
                    // columns: the scan stays in increasing column order)
                    constexpr int kGroups = WSG * SPLIT;
                    for (int k = wsg * SPLIT + part; k < nmask; k += kGroups) {
                        c = cstart + 4 * k;
                        q = smi2[rec2 + c - 1].x;  // 4 x_c (c >= I + 1 >= 1)
                        rp = smi4 + ((rec2 + c) >> 1);
                        group(true);
                    }
                    c = cs2 + 4 * h0;
                    const int cend = cs2 + 4 * h1;
                    q = h0 < h1 ? smi2[rec2 + c - 1].x : 0;  // 4 x_c
                    rp = smi4 + ((rec2 + c) >> 1);           // records c .. c+3
                    if constexpr (SPLIT == 1) {
                        const int cmask = min(cend, I + kStaged);
                        while (c < cmask) group(true);
                    }
                    // two groups at a time (sixteen gathers in flight) where the
                    // register budget allows it: one long tour per 8-warp CTA
                    constexpr bool kPairs = TPC == 1 && TG == 1 && ROWS <= 16;
                    while (kPairs && c + 4 < cend) {
                        const int4 ra4 = rp[0], rb4 = rp[1], rc4 = rp[2], rd4 = rp[3];
                        const int v0 = at(r1, q) + at2(ra4.x) + ra4.y;
                        const int v1 = at(r1, ra4.x) + at2(ra4.z) + ra4.w;
                        const int v2 = at(r1, ra4.z) + at2(rb4.x) + rb4.y;
                        const int v3 = at(r1, rb4.x) + at2(rb4.z) + rb4.w;
                        const int v4 = at(r1, rb4.z) + at2(rc4.x) + rc4.y;
                        const int v5 = at(r1, rc4.x) + at2(rc4.z) + rc4.w;
                        const int v6 = at(r1, rc4.z) + at2(rd4.x) + rd4.y;
                        const int v7 = at(r1, rd4.x) + at2(rd4.z) + rd4.w;
                        const int ma = min(min(v0, v1), min(v2, v3));
                        const int mb = min(min(v4, v5), min(v6, v7));
                        cm = ma < m ? c : cm;
                        m = min(m, ma);
                        cm = mb < m ? c + 4 : cm;
                        m = min(m, mb);
                        q = rd4.z;
                        c += 8;
                        rp += 4;
                    }
                    while (c < cend) group(false);
                    // only improving moves enter the cache (m + the row's own
                    // edge term < 0; no overflow: m <= 2^31 - 1 - 2^29 on a valid column)
                    const int dl = m != INT_MAX ? m + smi2[rec2 + ie].y : 0;
                    unsigned long long key = eval_ok && dl < 0 ? pack_key(dl, ie, cm) : ~0ull;
                    if constexpr (SPLIT > 1) {  // the lane groups sharing a row
                        key = min(key, __shfl_xor_sync(0xffffffffu, key, 16));
                        if constexpr (SPLIT == 4) key = min(key, __shfl_xor_sync(0xffffffffu, key, 8));
                    }
                    if (part == 0 && key != ~0ull) atomicMin(&rowkey[ie], key);
                }
                if (SPLIT == 1 && seg && pa > 0) {
                    // (b) rows i < pa against this tile's segment columns
                    // j = I + lane, one column j per lane (its staged rows
                    // C[x_j], C[x_j+1], read at x_i, x_i+1: the same column on
                    // every lane, so conflict-free), rows i in groups of four,
                    // contiguous per warp:
                    //   delta(i, j) = C[x_j][x_i] + C[x_j+1][x_i+1] - C[x_i][x_i+1]
                    //                 - C[x_j][x_j+1],
                    // each row's minimum over the lanes by one warp reduction; a
                    // negative one goes to the cache with its first j.  The pairs
                    // (pa - 1, pa) and (0, n - 1) are not 2-opt moves; their delta
                    // is exactly 0 for a symmetric C, so they never enter it.
                    const int j = I + lane;
                    const bool jok = lane < kRows && j <= pb;
                    const int tj = jok ? smi2[rec2 + j].y : 0;
                    const int ngb = (pa + 3) >> 2;
                    const int b0 = (ngb * wsg) / WSG, b1 = (ngb * (wsg + 1)) / WSG;
                    int q = b0 < b1 ? smi2[rec2 + (b0 > 0 ? 4 * b0 - 1 : n - 1)].x : 0;  // 4 x_i
                    const int4* rq = smi4 + ((rec2 + 4 * b0) >> 1);
                    for (int gi = b0; gi < b1; ++gi) {
                        const int i0 = 4 * gi;
                        const int4 ra4 = rq[0], rb4 = rq[1];
                        rq += 2;
                        int d0 = at(r1, q) + at2(ra4.x) + ra4.y + tj;
                        int d1 = at(r1, ra4.x) + at2(ra4.z) + ra4.w + tj;
                        int d2 = at(r1, ra4.z) + at2(rb4.x) + rb4.y + tj;
                        int d3 = at(r1, rb4.x) + at2(rb4.z) + rb4.w + tj;
                        q = rb4.z;
                        d0 = jok ? d0 : INT_MAX;
                        d1 = jok && i0 + 1 < pa ? d1 : INT_MAX;
                        d2 = jok && i0 + 2 < pa ? d2 : INT_MAX;
                        d3 = jok && i0 + 3 < pa ? d3 : INT_MAX;
                        const int m0 = __reduce_min_sync(0xffffffffu, d0);
                        const int m1 = __reduce_min_sync(0xffffffffu, d1);
                        const int m2 = __reduce_min_sync(0xffffffffu, d2);
                        const int m3 = __reduce_min_sync(0xffffffffu, d3);
                        if (min(min(m0, m1), min(m2, m3)) < 0) {
                            const int dd[4] = {d0, d1, d2, d3}, mmv[4] = {m0, m1, m2, m3};
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const unsigned bal = __ballot_sync(0xffffffffu, dd[k] == mmv[k]);
                                if (mmv[k] < 0 && lane == __ffs(bal) - 1)
                                    atomicMin(&rowkey[i0 + k], pack_key(mmv[k], i0 + k, j));
                            }
                        }
                    }
                }
                if (SPLIT > 1 && seg && pa > 0) {
                    // (b) rows i < pa against this tile's segment columns
                    // j = I + r, one row i per lane (blocks of 32 rows), r over
                    // the tile:
                    //   delta(i, j) = C[x_j][x_i] + C[x_j+1][x_i+1] - C[x_i][x_i+1]
                    //                 - C[x_j][x_j+1]
                    // read from the staged rows r, r + 1 (their bases are the
                    // same on every lane), the lane keeping its smallest
                    // negative delta and first r.  The (block, r) units are split
                    // evenly over the warps (a block's r range may be split
                    // between two warps; both fold into the cache).  The pairs
                    // (pa - 1, pa) and (0, n - 1) are not 2-opt moves; their
                    // delta is exactly 0 for a symmetric C, so they never enter
                    // the cache.
                    const int jn = min(kRows, pb - I + 1);
                    const int* const tb = smi + half * buf_words;
                    const int nblk = (pa + 31) >> 5;
                    int tjr[kRows];  // -C[x_j][x_j+1] of the tile's columns
#pragma unroll
                    for (int r = 0; r < kRows; ++r) tjr[r] = r < jn ? smi2[rec2 + I + r].y : 0;
                    const int nu = nblk * jn;
                    int u = (nu * wsg) / WSG;
                    const int u1 = (nu * (wsg + 1)) / WSG;
                    while (u < u1) {
                        const int blk = u / jn;
                        const int r0 = u - blk * jn;
                        const int re = min(jn, r0 + (u1 - u));
                        const int i = (blk << 5) + lane;
                        const int ic = min(i, pa - 1);  // lanes past pa: a valid row, not kept
                        const int qi = smi2[rec2 + (ic > 0 ? ic - 1 : n - 1)].x;  // 4 x_i
                        const int2 ri = smi2[rec2 + ic];  // {4 x_i+1, -C[x_i][x_i+1]}
                        // kept while below -ri.y, i.e. while the delta is negative
                        int best = -ri.y, br = 0;
                        // (with a compile-time pitch: two addresses per lane,
                        // every staged row at a constant offset from them)
                        const char* const bq = reinterpret_cast<const char*>(tb) + qi;
                        const char* const bx = reinterpret_cast<const char*>(tb) + ri.x;
#pragma unroll
                        for (int r = 0; r < kRows; ++r) {
                            if (r >= r0 && r < re) {
                                int d;
                                if constexpr (PITCH > 0) {
                                    d = *reinterpret_cast<const int*>(bq + r * kPB) +
                                        *reinterpret_cast<const int*>(bx + (r + 1) * kPB) + tjr[r];
                                } else {
                                    const char* const ra_ = reinterpret_cast<const char*>(
                                        tb + r * spitch + ((r >> 3) & 3));
                                    const char* const rb_ = reinterpret_cast<const char*>(
                                        tb + (r + 1) * spitch + (((r + 1) >> 3) & 3));
                                    d = at(ra_, qi) + at(rb_, ri.x) + tjr[r];
                                }
                                br = d < best ? r : br;
                                best = min(best, d);
                            }
                        }
                        if (i < pa && best < -ri.y)
                            atomicMin(&rowkey[i], pack_key(best + ri.y, i, I + br));
                        u += re - r0;
                    }
                }
                if (TG == 2 && wsg == 0 && lane == 0)
                    s_tile[sg * 2 + (par ^ 1)] = static_cast<int>(atomicAdd(&s_next[grp], 1u));
                par ^= 1;
            }
            ++passes;
            group_sync<TPC>(grp);
            if (tour_aborted()) break;  // no move from a pass with a missing tile
            {
                unsigned long long kl = ~0ull;
                for (int r = tid; r <= n - 3; r += GT) kl = min(kl, rowkey[r]);
                kl = warp_min_u64(kl);
                if (lane == 0 && kl != ~0ull) atomicMin(&s_best[grp], kl);
            }
            group_sync<TPC>(grp);
            const unsigned long long best = s_best[grp];
            if (best == ~0ull) break;
            const int bd = static_cast<int>(static_cast<uint32_t>(best >> 32) ^ 0x80000000u);
            if (bd >= 0) break;
            const int bi = static_cast<int>((best >> 16) & 0xffffu);
            if (warp == 0) {
                // the winning group's first column of delta bd, with the two
                // costs of the new edges, from C: lanes 0..3 test one column each
                const int j = static_cast<int>(best & 0xffffu) + lane;
                bool match = false;
                int e0 = 0, e1 = 0;
                if (lane < 4 && j >= bi + 2 && j <= n - 1) {
                    const int xi = smu[xs16 + bi], xi1 = smu[xs16 + bi + 1];
                    const int xj = smu[xs16 + j], xj1 = smu[xs16 + j + 1];
                    const int* C = a.C;
                    const size_t ldc = static_cast<size_t>(a.ldc);
                    e0 = C[xi * ldc + xj];
                    e1 = C[xi1 * ldc + xj1];
                    match = e0 + e1 + smi2[rec2 + j].y + smi2[rec2 + bi].y == bd;
                }
                const unsigned mm = __ballot_sync(0xffffffffu, match);
                if (lane == (mm ? __ffs(mm) - 1 : 0)) {
                    s_part[grp] = mm ? j : -1;  // (the work item is no longer needed this tour)
                    s_e0[grp] = e0;
                    s_e1[grp] = e1;
                }
            }
            group_sync<TPC>(grp);
            const int bj = s_part[grp];
            const int ei = s_e0[grp], ej = s_e1[grp];
            if (bj < 0) {  // cannot happen: the cache and C disagree
                if (tid == 0 && a.status) atomicExch(a.status, DPSO_ERR_INTERNAL);
                break;
            }
            if (tid == 0) {  // every thread has read them; the next pass starts afresh
                s_best[grp] = ~0ull;
                s_next[grp] = 0;
            }
            // reverse x[bi+1..bj] and the edge terms strictly between bi and bj
            for (int q2 = tid; q2 < (bj - bi) / 2; q2 += GT) {
                const uint16_t t0 = smu[xs16 + bi + 1 + q2];
                smu[xs16 + bi + 1 + q2] = smu[xs16 + bj - q2];
                smu[xs16 + bj - q2] = t0;
            }
            for (int q2 = tid; q2 < (bj - bi - 1) / 2; q2 += GT) {
                const int t0 = smi2[rec2 + bi + 1 + q2].y;
                smi2[rec2 + bi + 1 + q2].y = smi2[rec2 + bj - 1 - q2].y;
                smi2[rec2 + bj - 1 - q2].y = t0;
            }
            group_sync<TPC>(grp);
            for (int cc = bi + tid; cc <= bj; cc += GT)
                smi2[rec2 + cc] = make_int2(4 * smu[xs16 + cc + 1],
                                            cc == bi ? -ei : (cc == bj ? -ej : smi2[rec2 + cc].y));
            if (tid == 0) s_f[grp] += bd;
            ++moves;
            pa = bi;
            pb = bj;
            group_sync<TPC>(grp);
        }

        if (wsg == 0 && lane == 0 && a.evals && s_evals[sg]) atomicAdd(a.evals, s_evals[sg]);
        {
            uint16_t* tour = a.tours + static_cast<size_t>(p) * a.ldt;
            for (int i = tid; i < n; i += GT) tour[i] = smu[xs16 + i];
        }
        if (tid == 0) {
            a.cost[p] = s_f[grp];
            if (a.tour_passes) {
                a.tour_passes[p] = static_cast<unsigned int>(passes);
                a.tour_moves[p] = static_cast<unsigned int>(moves);
            } else {
                const long long npairs = static_cast<long long>(n) * (n - 3) / 2;
                atomicAdd(a.pairs, static_cast<unsigned long long>(passes) * npairs);
                atomicAdd(a.moves, static_cast<unsigned long long>(moves));
            }
            s_pf[grp] = a.pbest ? a.pcost[p] : LLONG_MIN;
        }
        group_sync<TPC>(grp);
        const long long f = s_f[grp];
        if (a.pbest && f < s_pf[grp]) {
            uint16_t* pb = a.pbest + static_cast<size_t>(p) * a.ldt;
            for (int i = tid; i < n; i += GT) pb[i] = smu[xs16 + i];
            if (tid == 0) a.pcost[p] = f;
        }
        group_sync<TPC>(grp);
        if (tour_aborted()) break;  // copies are not completing: the group stops
    }
}

// Shared bytes of one tour group (TG tile buffers), rounded to 128 bytes.
size_t group_bytes(int n, int rows, int tg) {
    return (two_opt_tiled_smem(n, rows, tg) + 127) / 128 * 128;
}

template <int ROWS, int TPC, int TG, bool SEG, int PITCH = 0>
cudaError_t launch_cfg(const TwoOptBatch& b, int num_sms, cudaStream_t st) {
    const size_t gb = group_bytes(b.max_n, ROWS, TG);
    const size_t smem = gb * TPC;
    auto* kern = two_opt_tiled_kernel<ROWS, TPC, TG, SEG, PITCH>;
    cudaError_t e = raise_smem_limit(kern, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads * TG, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = max(1, min((b.total + TPC - 1) / TPC, per_sm * num_sms));
    kern<<<grid, kThreads * TG, smem, st>>>(b, static_cast<int>(gb / sizeof(int)));
    return cudaGetLastError();
}

// 8-row segment tiles, one tour per CTA: the instantiation of the launch's
// pitch class (the runtime pitch when the tours are longer than every class).
template <int K>
cudaError_t launch_pitch(const TwoOptBatch& b, int pitch, int num_sms, cudaStream_t st) {
    if (pitch == kPitchStep * K + 4) return launch_cfg<8, 1, 1, true, kPitchStep * K + 4>(b, num_sms, st);
    if constexpr (K < kPitchMax) {
        return launch_pitch<K + 1>(b, pitch, num_sms, st);
    } else {
        return launch_cfg<8, 1, 1, true>(b, num_sms, st);
    }
}

// Launches with segment tiles (for every tour) when the launch holds a tour
// of at least kSegmentMinN viewpoints and the shape has one tour per CTA;
// other shapes use partial tiles for every tour.  Results are the same
// either way.
template <int ROWS>
cudaError_t launch_rows(const TwoOptBatch& b, int tpc, int tg, int num_sms, cudaStream_t st) {
    const bool seg = b.max_n >= kSegmentMinN;
    if (tg == 2) {
        if (tpc != 1) return cudaErrorInvalidValue;
        return seg ? launch_cfg<ROWS, 1, 2, true>(b, num_sms, st)
                   : launch_cfg<ROWS, 1, 2, false>(b, num_sms, st);
    }
    switch (tpc) {
        case 1:
            if constexpr (ROWS == 8) {
                if (seg) return launch_pitch<kPitchMin>(b, staged_pitch(b.max_n, 8, 1), num_sms, st);
            }
            return seg ? launch_cfg<ROWS, 1, 1, true>(b, num_sms, st)
                       : launch_cfg<ROWS, 1, 1, false>(b, num_sms, st);
        case 2: return launch_cfg<ROWS, 2, 1, false>(b, num_sms, st);
        case 4: return launch_cfg<ROWS, 4, 1, false>(b, num_sms, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// Resident CTAs per SM for a shape: shared memory (228 KB per SM; per CTA
// 1 KB reserved by the system and under 1 KB of the kernel's static shared
// variables) against the register budget of tiled_min_blocks.
int two_opt_tiled_ctas(int n, int rows, int tpc, int tg) {
    const int by_smem =
        static_cast<int>((228 * 1024) / (group_bytes(n, rows, tg) * tpc + 2048));
    const int by_regs = tg == 2 || (tpc == 1 && rows <= 16) ? 2 : (rows == 30 ? 4 : 3);
    return min(by_smem, by_regs);
}

// Default launch shape for tours of n viewpoints, from sweeps on GB300 of
// steady-state DPSO generations (1024 tours, n = 64 .. 1992): up to n = 256,
// 32-row tiles with 2 tours per CTA; beyond that, one tour per CTA and the
// tile height and tile subgroups that keep the most tile rows in flight per
// SM (rows x subgroups x resident CTAs), ties to the taller tile and to one
// subgroup.  With the row cache most tiles of a pass re-evaluate a few
// columns, so a pass costs about its staged rows, and more rows in flight
// hide more of each tile's copy.  two_opt_tiled_rows returns 0 when no tile
// height fits.
int two_opt_tiled_tg(int n, int rows, int tpc) {
    if (tpc != 1 || n <= 256 || !two_opt_tiled_fits(n, rows, 1, 2)) return 1;
    return 2 * two_opt_tiled_ctas(n, rows, 1, 2) > two_opt_tiled_ctas(n, rows, 1, 1) ? 2 : 1;
}

int two_opt_tiled_rows(int n) {
    if (n < 3 || n > 65535) return 0;
    if (n <= 256) return 32;
    int best = 0, best_score = 0;
    for (int rows : {32, 30, 24, 16, 8}) {
        if (!two_opt_tiled_fits(n, rows, 1, 1)) continue;
        const int tg = two_opt_tiled_tg(n, rows, 1);
        const int score = rows * tg * two_opt_tiled_ctas(n, rows, 1, tg);
        if (score > best_score) {
            best = rows;
            best_score = score;
        }
    }
    return best;
}

int two_opt_tiled_tpc(int n, int rows) {
    return n <= 256 && two_opt_tiled_fits(n, rows, 2, 1) ? 2 : 1;
}

// The launch shape used when none is pinned.  Long tours whose tallest
// fitting tile has 16 rows or fewer take 8-row tiles, one tour per CTA, when
// two such CTAs fit on an SM and the launch has at least two tours per SM:
// two tours in flight per SM, each with eight warps (2.34 s against 2.76 s
// with two 4-warp tours per CTA and 3.07 s with 16-row tiles, per
// steady-state generation of 4096 tours at n = 1992); with fewer tours the
// tallest tile is kept.
void two_opt_default_shape(int n, int count, int num_sms, int* rows, int* tpc, int* tg) {
    *rows = two_opt_tiled_rows(n);
    *tpc = *rows > 0 ? two_opt_tiled_tpc(n, *rows) : 0;
    *tg = *rows > 0 ? two_opt_tiled_tg(n, *rows, *tpc) : 0;
    if (*rows > 0 && *rows <= 16 && n > 256 && count >= 2 * num_sms &&
        two_opt_tiled_fits(n, 8, 1, 1) && two_opt_tiled_ctas(n, 8, 1, 1) >= 2) {
        *rows = 8;
        *tpc = 1;
        *tg = 1;
    }
}

cudaError_t build_shifted_copies(const int* C, int ldc, int n, int* Cs, cudaStream_t st) {
    dim3 grid(n, 4);
    shift_copies_kernel<<<grid, 128, 0, st>>>(C, ldc, n, shifted_ld(n), Cs);
    return cudaGetLastError();
}

bool two_opt_tiled_fits(int n, int rows, int tpc, int tg) {
    // (one warp compacts the need-tile bitmask: at most 32 words of grid tiles)
    return n >= 3 && n <= 65535 && grid_tiles(n, rows > 0 ? rows : 1) <= 1024 &&
           (rows == 32 || rows == 30 || rows == 24 || rows == 16 || rows == 8) &&
           (tpc == 1 || tpc == 2 || tpc == 4) && (tg == 1 || (tg == 2 && tpc == 1)) &&
           group_bytes(n, rows, tg) * tpc <= 220 * 1024;
}

cudaError_t launch_two_opt_tiled(const TwoOptBatch& b, int rows, int tpc, int tg, int num_sms,
                                 cudaStream_t st) {
    if (!b.shifted || !two_opt_tiled_fits(b.max_n, rows, tpc, tg)) return cudaErrorInvalidValue;
    switch (rows) {
        case 32: return launch_rows<32>(b, tpc, tg, num_sms, st);
        case 30: return launch_rows<30>(b, tpc, tg, num_sms, st);
        case 24: return launch_rows<24>(b, tpc, tg, num_sms, st);
        case 16: return launch_rows<16>(b, tpc, tg, num_sms, st);
        case 8: return launch_rows<8>(b, tpc, tg, num_sms, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace dpso
