// Edge exchange of Sec. 3.2.3 (best-improvement 2-opt to 2-optimality), the
// pipelined tiled variant for tours whose 33-row tiles fit in shared memory.
//
// Same mathematics and tie order as two_opt.cu:
//   delta(i, j) = C[x_i][x_j] + C[x_i+1][x_j+1] - C[x_i][x_i+1] - C[x_j][x_j+1],
//   the applied move is the smallest (delta, i, j) with delta < 0.
//
// Layout and mapping:
//  * One CTA per tour (persistent grid, work queue), 8 warps.
//  * A tile is 32 positions I..I+31, one per lane; its 33 cost rows
//    C[x_I..x_I+32] are staged in shared memory with 16-byte cp.async copies
//    issued by all threads, in a STAGES-deep pipeline (commit / wait groups),
//    so the next tiles load while the current one is evaluated.
//  * 16-byte copies need 16-byte-aligned rows, which alone would put rows a,
//    a+8, a+16, a+24 in the same bank.  The cost matrix is therefore kept in
//    four copies whose rows are shifted right by 0..3 words; row a of a tile is
//    taken from copy (a>>3)&3 into a row pitch ldq with ldq/4 odd, so the 32
//    lanes reading one column hit 32 distinct banks.
//  * Column records rec[c] = {x_c+1, -C[x_c][x_c+1]} give the second gather's
//    column and the edge term in one broadcast load; the first gather's column
//    x_c is the previous record's.
//  * Each lane tracks, over its columns in increasing order, the first minimum
//    of C[x_i][x_c] + C[x_i+1][x_c+1] - C[x_c][x_c+1] and the two gathered
//    costs there.  Subtracting C[x_i][x_i+1] gives a candidate (delta, i, j);
//    a packed 64-bit key keeps the lexicographically smallest across tiles.
//    One block reduction per pass yields (delta*, i*, j*), and the winning
//    lane publishes C[x_i*][x_j*] and C[x_i*+1][x_j*+1], the two new edges.
//  * Pairs with j = i+1 and (0, n-1) have delta = 0 for a symmetric C and
//    never win, so only the triangle at the start of each tile is masked.
#include <climits>

#include "common.cuh"

namespace dpso {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// (delta, i, j) -> order-preserving 64-bit key: biased delta, then i, then j.
__device__ __forceinline__ unsigned long long pack_key(int delta, int i, int j) {
    return (static_cast<unsigned long long>(static_cast<uint32_t>(delta) ^ 0x80000000u) << 32) |
           (static_cast<unsigned long long>(static_cast<uint32_t>(i)) << 16) |
           static_cast<uint32_t>(j);
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

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

// Row pitch (words) of the shifted copies and of the staged rows: room for a
// shift of up to 3 words, a multiple of 4 words (16-byte rows), ldq/4 odd.
__host__ __device__ int shifted_ld(int n) {
    int q = (n + 3 + 3) / 4 * 4;
    if (((q / 4) & 1) == 0) q += 4;
    return q;
}

size_t two_opt_tiled_smem(int n, int rows_per_tile, int stages) {
    const size_t rows =
        static_cast<size_t>(stages) * (rows_per_tile + 1) * shifted_ld(n) * sizeof(int);
    const size_t rec = static_cast<size_t>(n + 4) * sizeof(int2);
    const size_t xs = static_cast<size_t>((n + 1 + 7) / 8 * 8) * sizeof(uint16_t);
    return rows + rec + xs;
}

namespace {

// Record cost of the padding columns past n: larger than any real column
// value (at most 2^30), so padding never supplies an improving move.
constexpr int kPadCost = (1 << 30) + 1;

template <int ROWS, int STAGES>
__global__ void __launch_bounds__(kThreads) two_opt_tiled_kernel(TwoOptBatch b) {
    constexpr int kRows = ROWS;           // positions per tile, one per lane
    constexpr int kStaged = ROWS + 1;     // cost rows staged per tile
    // One dynamic shared block seen through three element types (all arrays
    // alias its start): STAGES tile buffers of kStaged x ldq ints, then the
    // column records (n + 4 int2, the last four padding), then the tour
    // (n + 1 uint16).  Offsets depend on the tour's n; the block is sized for
    // the largest n of the launch.
    extern __shared__ __align__(128) int smi[];
    extern __shared__ __align__(128) int2 smi2[];
    extern __shared__ __align__(128) int4 smi4[];
    extern __shared__ __align__(128) uint16_t smu[];
    __shared__ unsigned long long s_key[kWarps];
    __shared__ unsigned long long s_best;
    __shared__ int s_part, s_e0, s_e1;
    __shared__ long long s_pf;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (;;) {
        if (tid == 0) s_part = static_cast<int>(atomicAdd(b.queue, 1u));
        __syncthreads();
        const int g = s_part;
        if (g >= b.total) break;
        const int prob = find_inst(b.off, b.nprob, g);
        const int p = g - b.off[prob];
        const TwoOptTask a = b.tasks[prob];
        if (a.gate && *a.gate == 0) {  // this problem does not exchange edges now
            __syncthreads();
            continue;
        }
        const int n = a.n;
        const int ldq = shifted_ld(n);
        const int q16 = ldq / 4;
        const int buf_words = kStaged * ldq;
        const int rec2 = STAGES * buf_words / 2;  // int2 index of record 0 (even)
        const int xs16 = (rec2 + n + 4) * 4;      // uint16 index of x_0
        const int* __restrict__ C = a.C;
        const int* __restrict__ Cs = a.Cs;
        const int ldc = a.ldc;
        const long long npairs = static_cast<long long>(n) * (n - 3) / 2;
        const int ntiles = (n - 2 + kRows - 1) / kRows;  // tiles start at I <= n-3
        const int guard = 1000 + 100 * n;

        // All threads: copy the cost rows of tile t into buffer t % STAGES.
        auto stage = [&](int t) {
            const int I = t * kRows;
            const int count = min(kStaged, n - 1 - I);
            const int boff = (t % STAGES) * buf_words;
            for (int r = warp; r < count; r += kWarps) {
                const int k = (r >> 3) & 3;
                const char* src =
                    reinterpret_cast<const char*>(
                        Cs + (static_cast<size_t>(k) * n + smu[xs16 + I + r]) * ldq) +
                    lane * 16;
                int* dst = smi + boff + r * ldq + lane * 4;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (j * 32 + lane < q16) cp_async16(dst + j * 128, src + j * 512);
                for (int j = 4; j * 32 + lane < q16; ++j) cp_async16(dst + j * 128, src + j * 512);
            }
        };

        uint16_t* tour = a.tours + static_cast<size_t>(p) * a.ldt;
        for (int i = tid; i < n; i += kThreads) smu[xs16 + i] = tour[i];
        if (tid == 0) smu[xs16 + n] = tour[0];
        __syncthreads();
        for (int c = tid; c < n; c += kThreads) {
            const int u = smu[xs16 + c], v = smu[xs16 + c + 1];
            smi2[rec2 + c] = make_int2(v, -C[static_cast<size_t>(u) * ldc + v]);
        }
        if (tid < 4) smi2[rec2 + n + tid] = make_int2(0, kPadCost);
        long long f = a.cost[p];
        int moves = 0, passes = 0;
        __syncthreads();

        for (;;) {
            if (a.max_moves > 0 && moves >= a.max_moves) break;
            if (moves >= guard) {
                if (tid == 0 && a.status) atomicExch(a.status, DPSO_ERR_INTERNAL);
                break;
            }
            if constexpr (STAGES > 1) {
#pragma unroll
                for (int s = 0; s < STAGES - 1; ++s) {
                    if (s < ntiles) stage(s);
                    cp_async_commit();
                }
            }
            unsigned long long key = ~0ull;
            int ke0 = 0, ke1 = 0;
            for (int t = 0; t < ntiles; ++t) {
                if constexpr (STAGES == 1) {
                    __syncthreads();
                    stage(t);
                    cp_async_commit();
                    cp_async_wait<0>();
                    __syncthreads();
                } else {
                    cp_async_wait<STAGES - 2>();
                    __syncthreads();
                    if (t + STAGES - 1 < ntiles) stage(t + STAGES - 1);
                    cp_async_commit();
                }
                const int I = t * kRows;
                const int boff = (t % STAGES) * buf_words;
                // lanes past the tile height idle on a valid row
                const int ra = min(lane, kRows - 1), rb1 = min(lane + 1, kRows);
                const int p1 = boff + ra * ldq + ((ra >> 3) & 3);
                const int p2 = boff + rb1 * ldq + ((rb1 >> 3) & 3);
                // columns in groups of four, contiguous per warp; the records
                // past n are padding
                const int cbeg = I + 2;
                const int ngroups = (n - cbeg + 3) >> 2;
                const int g0 = (ngroups * warp) / kWarps, g1 = (ngroups * (warp + 1)) / kWarps;
                // first valid column of this lane's row (rows past n-3 have none)
                const int lim = (lane < kRows && I + lane <= n - 3) ? I + lane + 2 : INT_MAX;
                int m = INT_MAX, cm = 0, e0 = 0, e1 = 0;
                int c = cbeg + 4 * g0;
                const int cend = cbeg + 4 * g1;
                int q = g0 < g1 ? smi2[rec2 + c - 1].x : 0;  // x_c
                auto group = [&](bool masked) {
                    const int4 ra = smi4[(rec2 + c) >> 1], rb = smi4[(rec2 + c + 2) >> 1];
                    const int a0 = smi[p1 + q], b0 = smi[p2 + ra.x];
                    const int a1 = smi[p1 + ra.x], b1 = smi[p2 + ra.z];
                    const int a2 = smi[p1 + ra.z], b2 = smi[p2 + rb.x];
                    const int a3 = smi[p1 + rb.x], b3 = smi[p2 + rb.z];
                    int v0 = a0 + b0 + ra.y, v1 = a1 + b1 + ra.w;
                    int v2 = a2 + b2 + rb.y, v3 = a3 + b3 + rb.w;
                    if (masked) {
                        v0 = c >= lim ? v0 : INT_MAX;
                        v1 = c + 1 >= lim ? v1 : INT_MAX;
                        v2 = c + 2 >= lim ? v2 : INT_MAX;
                        v3 = c + 3 >= lim ? v3 : INT_MAX;
                    }
                    const int mv = min(min(v0, v1), min(v2, v3));
                    if (mv < m) {  // rare: a new first minimum in this lane's columns
                        if (v0 == mv) {
                            cm = c;
                            e0 = a0;
                            e1 = b0;
                        } else if (v1 == mv) {
                            cm = c + 1;
                            e0 = a1;
                            e1 = b1;
                        } else if (v2 == mv) {
                            cm = c + 2;
                            e0 = a2;
                            e1 = b2;
                        } else {
                            cm = c + 3;
                            e0 = a3;
                            e1 = b3;
                        }
                        m = mv;
                    }
                    q = rb.z;
                    c += 4;
                };
                // groups starting below I+33 hold the diagonal triangle
                const int cmask = min(cend, I + kStaged);
                while (c < cmask) group(true);
                while (c < cend) group(false);
                if (m != INT_MAX && lim != INT_MAX) {  // idle lanes own no row
                    const unsigned long long k =
                        pack_key(m + smi2[rec2 + I + lane].y, I + lane, cm);
                    if (k < key) {
                        key = k;
                        ke0 = e0;
                        ke1 = e1;
                    }
                }
            }
            ++passes;
            const unsigned long long kw = warp_min_u64(key);
            if (lane == 0) s_key[warp] = kw;
            __syncthreads();
            if (warp == 0) {
                unsigned long long kk = lane < kWarps ? s_key[lane] : ~0ull;
                kk = warp_min_u64(kk);
                if (lane == 0) s_best = kk;
            }
            __syncthreads();
            const unsigned long long best = s_best;
            if (best == ~0ull) break;
            const int bd = static_cast<int>(static_cast<uint32_t>(best >> 32) ^ 0x80000000u);
            if (bd >= 0) break;
            if (key == best) {  // exactly one lane evaluated (i*, j*)
                s_e0 = ke0;
                s_e1 = ke1;
            }
            __syncthreads();
            const int bi = static_cast<int>((best >> 16) & 0xffffu);
            const int bj = static_cast<int>(best & 0xffffu);
            const int ei = s_e0, ej = s_e1;
            // reverse x[bi+1..bj] and the edge terms strictly between bi and bj
            for (int q2 = tid; q2 < (bj - bi) / 2; q2 += kThreads) {
                const uint16_t t0 = smu[xs16 + bi + 1 + q2];
                smu[xs16 + bi + 1 + q2] = smu[xs16 + bj - q2];
                smu[xs16 + bj - q2] = t0;
            }
            for (int q2 = tid; q2 < (bj - bi - 1) / 2; q2 += kThreads) {
                const int t0 = smi2[rec2 + bi + 1 + q2].y;
                smi2[rec2 + bi + 1 + q2].y = smi2[rec2 + bj - 1 - q2].y;
                smi2[rec2 + bj - 1 - q2].y = t0;
            }
            __syncthreads();
            for (int cc = bi + tid; cc <= bj; cc += kThreads)
                smi2[rec2 + cc] = make_int2(smu[xs16 + cc + 1],
                                            cc == bi ? -ei : (cc == bj ? -ej : smi2[rec2 + cc].y));
            f += bd;
            ++moves;
            __syncthreads();
        }

        for (int i = tid; i < n; i += kThreads) tour[i] = smu[xs16 + i];
        if (tid == 0) {
            a.cost[p] = f;
            if (a.tour_passes) {
                a.tour_passes[p] = static_cast<unsigned int>(passes);
                a.tour_moves[p] = static_cast<unsigned int>(moves);
            } else {
                atomicAdd(a.pairs, static_cast<unsigned long long>(passes) * npairs);
                atomicAdd(a.moves, static_cast<unsigned long long>(moves));
            }
            s_pf = a.pbest ? a.pcost[p] : LLONG_MIN;
        }
        __syncthreads();
        if (a.pbest && f < s_pf) {
            uint16_t* pb = a.pbest + static_cast<size_t>(p) * a.ldt;
            for (int i = tid; i < n; i += kThreads) pb[i] = smu[xs16 + i];
            if (tid == 0) a.pcost[p] = f;
        }
        __syncthreads();
    }
}

template <int ROWS, int STAGES>
cudaError_t launch_cfg(const TwoOptBatch& b, int num_sms, cudaStream_t st) {
    const size_t smem = two_opt_tiled_smem(b.max_n, ROWS, STAGES);
    cudaError_t e = cudaFuncSetAttribute(two_opt_tiled_kernel<ROWS, STAGES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, two_opt_tiled_kernel<ROWS, STAGES>,
                                                      kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = max(1, min(b.total, per_sm * num_sms));
    two_opt_tiled_kernel<ROWS, STAGES><<<grid, kThreads, smem, st>>>(b);
    return cudaGetLastError();
}

}  // namespace

// Tile height for n (0 = no height fits): the tallest of 32 / 24 / 16 / 8 rows
// whose single-stage tile fits in 220 KB of shared memory.  One stage is used:
// at the sizes measured, more resident CTAs beat deeper pipelines.
int two_opt_tiled_rows(int n) {
    if (n < 3 || n > 65535) return 0;
    for (int rows : {32, 24, 16, 8})
        if (two_opt_tiled_smem(n, rows, 1) <= 220 * 1024) return rows;
    return 0;
}

cudaError_t build_shifted_copies(const int* C, int ldc, int n, int* Cs, cudaStream_t st) {
    dim3 grid(n, 4);
    shift_copies_kernel<<<grid, 128, 0, st>>>(C, ldc, n, shifted_ld(n), Cs);
    return cudaGetLastError();
}

cudaError_t launch_two_opt_tiled(const TwoOptBatch& b, int rows, int num_sms, cudaStream_t st) {
    if (!b.shifted || two_opt_tiled_smem(b.max_n, rows, 1) > 220 * 1024)
        return cudaErrorInvalidValue;
    switch (rows) {
        case 32: return launch_cfg<32, 1>(b, num_sms, st);
        case 24: return launch_cfg<24, 1>(b, num_sms, st);
        case 16: return launch_cfg<16, 1>(b, num_sms, st);
        case 8: return launch_cfg<8, 1>(b, num_sms, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace dpso
