// Node-swap exchange: the "swap nodes(i,j) and evaluate fitness" reading of
// the edge exchange in the paper's GPU listing (Sec. 3.2.3, Fig. "pseudocode"
// GPU kernels).  Every pair of positions i < j of the cyclic tour is
// evaluated; the swap of x_i and x_j with the most improvement is applied,
// repeatedly, until no swap improves (ties: smallest (delta, i, j)).
//
// With a = x_i-1, b = x_i, c = x_i+1, d = x_j-1, e = x_j, f = x_j+1 (indices
// mod n) and d_k = C[x_k][x_k+1]:
//   general:      delta = C[a][e] + C[e][c] + C[d][b] + C[b][f]
//                         - d_i-1 - d_i - d_j-1 - d_j
//   j = i + 1:    the general value + 2 d_i  (the edge b-e stays)
//   (0, n - 1):   C[x_n-2][x_0] + C[x_n-1][x_1] - d_n-2 - d_0
//
// Layout follows the tiled 2-opt: one CTA per tour from a persistent grid and
// a work queue; a tile is R positions I..I+R-1, one per lane; its R+2 cost
// rows C[x_I-1 .. x_I+R] (position I-1 wrapping to n-1) arrive by one bulk
// copy per row from the four row-shifted copies, so the lanes reading rows
// l, l+1, l+2 at one column hit distinct banks.  Per column a lane gathers
// C[a][e], C[c][e] and C[b][x_j+1]; C[b][x_j-1] is the latter of two columns
// before, so a pair costs three gathers.  Column records are those of the
// 2-opt, {4 x_c+1, -d_c}.  Entries of C must be at most 2^28 so that every
// sum stays inside int32 (checked by the callers).
#include <climits>

#include "tiled_common.cuh"

namespace dpso {
namespace {

using namespace tiled;

template <int ROWS>
__global__ void __launch_bounds__(kThreads, 3) node_swap_tiled_kernel(TwoOptBatch b) {
    constexpr int kRows = ROWS;        // positions per tile, one per lane
    constexpr int kStaged = ROWS + 2;  // cost rows staged per tile
    // Shared block: the tile buffer (kStaged x ldq ints), the column records
    // (n + 4 int2, the last four padding), the tour (n + 1 uint16).
    extern __shared__ __align__(128) int smi[];
    int2* smi2 = reinterpret_cast<int2*>(smi);
    const int4* smi4 = reinterpret_cast<const int4*>(smi);
    uint16_t* smu = reinterpret_cast<uint16_t*>(smi);
    __shared__ unsigned long long s_key[kWarps];
    __shared__ unsigned long long s_best;
    __shared__ int s_part, s_abort;
    __shared__ long long s_pf;
    __shared__ __align__(8) unsigned long long s_mbar;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned mbar = smem_addr(&s_mbar);
    unsigned phase = 0;
    if (tid == 0) {
        mbar_init(mbar);
        s_abort = 0;
    }
    for (;;) {
        if (tid == 0) s_part = static_cast<int>(atomicAdd(b.queue, 1u));
        __syncthreads();
        const int g = s_part;
        if (g >= b.total) break;
        const int prob = find_inst(b.off, b.nprob, g);
        const TwoOptTask a = b.tasks[prob];
        const int p = a.order ? a.order[g - b.off[prob]] : g - b.off[prob];
        if (a.gate && *a.gate == 0) {  // this problem does not exchange now
            __syncthreads();
            continue;
        }
        const int n = a.n;
        const int ldq = shifted_ld(n);
        const int buf_words = kStaged * ldq;
        const int rec2 = buf_words / 2;       // int2 index of record 0 (even)
        const int xs16 = (rec2 + n + 4) * 4;  // uint16 index of x_0
        const int* __restrict__ C = a.C;
        const int ldc = a.ldc;
        const long long npairs = static_cast<long long>(n) * (n - 1) / 2;
        const int ntiles = (n - 1 + kRows - 1) / kRows;  // rows i <= n-2
        const int guard = 1000 + 100 * n;
        const char* const cs0 = reinterpret_cast<const char*>(a.Cs);
        const unsigned tile_s = smem_addr(smi);
        const unsigned row_bytes = static_cast<unsigned>(ldq) * 4u;

        // The block stages rows of positions I-1 .. I+R (I-1 wrapping), staged
        // row r from shifted copy (r>>3)&3: each warp posts kPerWarp rows, one
        // bulk copy per lane, so the copies are issued by all warps at once;
        // lane 0 of warp 0 arms the barrier (a copy that lands first only
        // takes the transaction count below zero until that one arrival).
        constexpr int kPerWarp = (kStaged + kWarps - 1) / kWarps;
        auto stage = [&](int I) {
            const int count = min(kStaged, n + 1 - I);
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            if (warp == 0 && lane == 0) mbar_expect(mbar, static_cast<unsigned>(count) * row_bytes);
            const int r = warp * kPerWarp + lane;
            if (lane < kPerWarp && r < count) {
                int pos = I - 1 + r;
                if (pos < 0) pos += n;
                const unsigned k = (r >> 3) & 3;
                const unsigned off = (k * static_cast<unsigned>(n) + smu[xs16 + pos]) * row_bytes;
                bulk_row(tile_s + r * row_bytes, cs0 + off, row_bytes, mbar);
            }
        };
        auto at = [](const char* row, int off) { return *reinterpret_cast<const int*>(row + off); };

        uint16_t* tour = a.tours + static_cast<size_t>(p) * a.ldt;
        for (int i = tid; i < n; i += kThreads) smu[xs16 + i] = tour[i];
        if (tid == 0) smu[xs16 + n] = tour[0];
        __syncthreads();
        for (int c = tid; c < n; c += kThreads) {
            const int u = smu[xs16 + c], v = smu[xs16 + c + 1];
            smi2[rec2 + c] = make_int2(4 * v, -C[static_cast<size_t>(u) * ldc + v]);
        }
        if (tid < 4) smi2[rec2 + n + tid] = make_int2(0, 0);  // padding: masked below
        long long f = a.cost[p];
        int moves = 0, passes = 0;
        __syncthreads();

        for (;;) {
            if (a.max_moves > 0 && moves >= a.max_moves) break;
            if (moves >= guard) {
                if (tid == 0 && a.status) atomicExch(a.status, DPSO_ERR_INTERNAL);
                break;
            }
            unsigned long long key = ~0ull;
            for (int t = 0; t < ntiles; ++t) {
                const int I = t * kRows;
                __syncthreads();  // the previous tile is no longer read
                if (s_abort) break;
                stage(I);
                if (!mbar_wait(mbar, phase)) {
                    s_abort = 1;
                    if (a.status) atomicExch(a.status, DPSO_ERR_TIMEOUT);
                }
                phase ^= 1u;
                // this lane's rows: positions i-1, i, i+1 = staged rows ra..ra+2
                const int ra = min(lane, kRows - 1);
                const char* const rm = reinterpret_cast<const char*>(smi + ra * ldq + ((ra >> 3) & 3));
                const char* const r0 =
                    reinterpret_cast<const char*>(smi + (ra + 1) * ldq + (((ra + 1) >> 3) & 3));
                const char* const rp =
                    reinterpret_cast<const char*>(smi + (ra + 2) * ldq + (((ra + 2) >> 3) & 3));
                const int i = I + lane;
                const bool row_ok = lane < kRows && i <= n - 2;
                const int lim = row_ok ? i + 1 : INT_MAX;  // first column of this row
                const int e_i = row_ok ? smi2[rec2 + i].y : 0;
                const int e_im1 = row_ok ? smi2[rec2 + (i == 0 ? n - 1 : i - 1)].y : 0;
                // columns in groups of four from I (even, so that the 16-byte
                // record loads are aligned; column I itself is always masked),
                // contiguous per warp
                const int cbeg = I;
                const int ngroups = (n - cbeg + 3) >> 2;
                const int g0 = (ngroups * warp) / kWarps, g1 = (ngroups * (warp + 1)) / kWarps;
                int m = INT_MAX, cm = 0;
                int c = cbeg + 4 * g0;
                const int cend = cbeg + 4 * g1;
                // carries: byte offsets of x_c-1 and x_c, their row-i costs, e_c-1
                int q_m1 = 0, q_0 = 0, M_m1 = 0, M_0 = 0, e_m1 = 0;
                if (g0 < g1) {
                    const int cm1 = c == 0 ? n - 1 : c - 1;
                    q_m1 = 4 * smu[xs16 + cm1];
                    q_0 = 4 * smu[xs16 + c];
                    M_m1 = at(r0, q_m1);
                    M_0 = at(r0, q_0);
                    e_m1 = smi2[rec2 + cm1].y;
                }
                const int4* rp4 = smi4 + ((rec2 + c) >> 1);  // records c .. c+3
                // v(i, col) = C[a][e] + C[c][e] + C[b][x_col-1] + C[b][x_col+1]
                //             - d_col-1 - d_col; delta = v - d_i-1 - d_i
                auto group = [&](bool masked) {
                    const int4 ra4 = rp4[0], rb4 = rp4[1];
                    const int X1 = ra4.x, X2 = ra4.z, X3 = rb4.x, X4 = rb4.z;  // 4 x_c+1..c+4
                    const int M1 = at(r0, X1), M2 = at(r0, X2), M3 = at(r0, X3), M4 = at(r0, X4);
                    int v0 = at(rm, q_0) + at(rp, q_0) + M_m1 + M1 + e_m1 + ra4.y;
                    int v1 = at(rm, X1) + at(rp, X1) + M_0 + M2 + ra4.y + ra4.w;
                    int v2 = at(rm, X2) + at(rp, X2) + M1 + M3 + ra4.w + rb4.y;
                    int v3 = at(rm, X3) + at(rp, X3) + M2 + M4 + rb4.y + rb4.w;
                    if (masked) {
                        // columns before i+1, past n-1, and (0, n-1) are not
                        // general pairs; j = i+1 keeps the edge b-e: + 2 d_i
                        auto fix = [&](int v, int col) {
                            if (col < lim || col >= n || (i == 0 && col == n - 1)) return INT_MAX;
                            return col == i + 1 ? v - 2 * e_i : v;
                        };
                        v0 = fix(v0, c);
                        v1 = fix(v1, c + 1);
                        v2 = fix(v2, c + 2);
                        v3 = fix(v3, c + 3);
                    }
                    const int mv = min(min(v0, v1), min(v2, v3));
                    cm = mv < m ? c : cm;  // first group holding the lane minimum
                    m = min(m, mv);
                    q_m1 = X3;
                    q_0 = X4;
                    M_m1 = M3;
                    M_0 = M4;
                    e_m1 = rb4.w;
                    c += 4;
                    rp4 += 2;
                };
                // masked: the groups that hold columns before I+kStaged (the
                // triangle and the adjacent pairs) and the last warp's last
                // group (padding and the pair (0, n-1))
                const int cmask = min(cend, I + kStaged);
                const int clast = (warp == kWarps - 1 && g1 > g0) ? cend - 4 : cend;
                while (c < cmask) group(true);
                while (c < clast) group(false);
                if (c < cend) group(true);
                if (m != INT_MAX && row_ok) {
                    const int dl = m + e_im1 + e_i;
                    if (pack_key(dl, i, cm) < key) {  // find the column in group cm
                        const int cm1 = cm == 0 ? n - 1 : cm - 1;
                        int xm = 4 * smu[xs16 + cm1], x0 = 4 * smu[xs16 + cm];
                        int em = smi2[rec2 + cm1].y;
                        int jx = -1;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int2 r = smi2[rec2 + cm + u];  // {4 x_col+1, e_col}
                            int v = at(rm, x0) + at(rp, x0) + at(r0, xm) + at(r0, r.x) + em + r.y;
                            const int col = cm + u;
                            if (col < lim || col >= n || (i == 0 && col == n - 1)) v = INT_MAX;
                            else if (col == i + 1) v -= 2 * e_i;
                            if (jx < 0 && v == m) jx = col;
                            xm = x0;
                            x0 = r.x;
                            em = r.y;
                        }
                        key = pack_key(dl, i, jx);
                    }
                }
                // the wrap pair (0, n-1), from rows x_n-1 (staged row 0) and x_0
                if (I == 0 && lane == 0 && n >= 3) {
                    const int dw = at(rm, smi2[rec2].x) + at(r0, smi2[rec2 + n - 3].x) +
                                   smi2[rec2 + n - 2].y + smi2[rec2].y;
                    const unsigned long long kw = pack_key(dw, 0, n - 1);
                    if (kw < key) key = kw;
                }
            }
            ++passes;
            const unsigned long long kwarp = warp_min_u64(key);
            if (lane == 0) s_key[warp] = kwarp;
            __syncthreads();
            if (s_abort) break;  // no move from a pass with a missing tile
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
            const int bi = static_cast<int>((best >> 16) & 0xffffu);
            const int bj = static_cast<int>(best & 0xffffu);
            if (tid == 0) {
                const uint16_t t0 = smu[xs16 + bi];
                smu[xs16 + bi] = smu[xs16 + bj];
                smu[xs16 + bj] = t0;
                smu[xs16 + n] = smu[xs16];
            }
            __syncthreads();
            if (tid < 4) {  // records of the edges that start at i-1, i, j-1, j
                const int ks[4] = {bi == 0 ? n - 1 : bi - 1, bi, bj - 1, bj};
                const int k = ks[tid];
                const int u = smu[xs16 + k], v = smu[xs16 + k + 1];
                smi2[rec2 + k] = make_int2(4 * v, -C[static_cast<size_t>(u) * ldc + v]);
            }
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
            if (a.evals) atomicAdd(a.evals, static_cast<unsigned long long>(passes) * npairs);
            s_pf = a.pbest ? a.pcost[p] : LLONG_MIN;
        }
        __syncthreads();
        if (a.pbest && f < s_pf) {
            uint16_t* pb = a.pbest + static_cast<size_t>(p) * a.ldt;
            for (int i = tid; i < n; i += kThreads) pb[i] = smu[xs16 + i];
            if (tid == 0) a.pcost[p] = f;
        }
        __syncthreads();
        if (s_abort) break;  // copies are not completing: this CTA stops
    }
}

template <int ROWS>
cudaError_t launch_ns(const TwoOptBatch& b, int num_sms, cudaStream_t st) {
    const size_t smem = node_swap_tiled_smem(b.max_n, ROWS);
    cudaError_t e = raise_smem_limit(node_swap_tiled_kernel<ROWS>, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, node_swap_tiled_kernel<ROWS>,
                                                      kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = max(1, min(b.total, per_sm * num_sms));
    node_swap_tiled_kernel<ROWS><<<grid, kThreads, smem, st>>>(b);
    return cudaGetLastError();
}

}  // namespace

size_t node_swap_tiled_smem(int n, int rows) {
    // rows + 2 staged cost rows, the column records (n + 4 int2), the tour
    // (n + 1 uint16, padded to 8)
    const size_t staged = static_cast<size_t>(rows + 2) * shifted_ld(n) * sizeof(int);
    const size_t rec = static_cast<size_t>(n + 4) * sizeof(int2);
    const size_t xs = static_cast<size_t>((n + 1 + 7) / 8 * 8) * sizeof(uint16_t);
    return staged + rec + xs;
}

int node_swap_tiled_rows(int n) {
    if (n < 3 || n > 65535) return 0;
    for (int rows : {32, 24, 16, 8})
        if (node_swap_tiled_smem(n, rows) <= 220 * 1024) return rows;
    return 0;
}

cudaError_t launch_node_swap_tiled(const TwoOptBatch& b, int num_sms, cudaStream_t st) {
    const int rows = node_swap_tiled_rows(b.max_n);
    if (!b.shifted || rows == 0) return cudaErrorInvalidValue;
    switch (rows) {
        case 32: return launch_ns<32>(b, num_sms, st);
        case 24: return launch_ns<24>(b, num_sms, st);
        case 16: return launch_ns<16>(b, num_sms, st);
        default: return launch_ns<8>(b, num_sms, st);
    }
}

}  // namespace dpso
