// Edge exchange of Sec. 3.2.3: best-improvement 2-opt, repeated until no
// exchange of two non-adjacent edges shortens the tour.
//
// For a tour x (positions 0..n-1, x_n = x_0) and edges e_i = (x_i, x_i+1),
//   delta(i, j) = C[x_i][x_j] + C[x_i+1][x_j+1] - C[x_i][x_i+1] - C[x_j][x_j+1]
// over 0 <= i, i+2 <= j <= n-1, (i, j) != (0, n-1).  The applied move is the
// lexicographically smallest (delta, i, j) with delta < 0; it reverses
// x[i+1..j].
//
// GPU mapping: one CTA per tour (a persistent grid pulls tours from a queue).
// The tour and its edge costs live in shared memory.  A pass walks row tiles
// of R positions I..I+R-1: the R+1 cost rows C[x_I..x_I+R] are staged in
// shared memory with an odd row stride, so the R lanes that share a column
// read R distinct banks.  Each lane keeps the minimum of
//   C[x_i][x_c] + C[x_i+1][x_c+1] - C[x_c][x_c+1]
// over its columns; the per-row minimum minus C[x_i][x_i+1] is delta's row
// minimum.  The pass's smallest row minimum gives (delta*, i*); one rescan of
// row i* finds the smallest j*.  Only pairs with delta < 0 matter, so the
// exact lexicographic argmin is recovered.
#include <climits>

#include "common.cuh"

namespace dpso {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 8;

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

__host__ __device__ constexpr int row_stride(int n) { return n | 1; }

__host__ __device__ inline size_t two_opt_smem(int n, int R) {
    const size_t rows = static_cast<size_t>(R + 1) * row_stride(n) * sizeof(int);
    const size_t dd = static_cast<size_t>((n + 3) / 4 * 4) * sizeof(int);
    const size_t xs = static_cast<size_t>((n + 1 + 7) / 8 * 8) * sizeof(uint16_t);
    return rows + dd + xs;
}

template <int R>
__global__ void __launch_bounds__(kWarps * 32) two_opt_kernel(TwoOptBatch b) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_rowmin[R];
    __shared__ int s_part, s_bd, s_bi, s_bj, s_ei, s_ej;
    __shared__ long long s_pf;

    constexpr int kStreams = 32 / R;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int arow = lane % R, stream = lane / R;

    for (;;) {
        if (tid == 0) s_part = static_cast<int>(atomicAdd(b.queue, 1u));
        __syncthreads();
        const int g = s_part;
        if (g >= b.total) break;
        const int prob = find_inst(b.off, b.nprob, g);
        const TwoOptTask a = b.tasks[prob];
        const int p = a.order ? a.order[g - b.off[prob]] : g - b.off[prob];
        if (a.gate && *a.gate == 0) {  // this problem does not exchange edges now
            __syncthreads();
            continue;
        }
        const int n = a.n;
        const int ldr = row_stride(n);
        int* rows = reinterpret_cast<int*>(smraw);
        int* dd = rows + static_cast<size_t>(R + 1) * ldr;
        uint16_t* xs = reinterpret_cast<uint16_t*>(dd + (n + 3) / 4 * 4);
        const int* __restrict__ C = a.C;
        const int ldc = a.ldc;
        const long long npairs = static_cast<long long>(n) * (n - 3) / 2;
        uint16_t* tour = a.tours + static_cast<size_t>(p) * a.ldt;
        for (int i = tid; i < n; i += blockDim.x) xs[i] = tour[i];
        __syncthreads();
        for (int i = tid; i < n; i += blockDim.x)
            dd[i] = C[static_cast<size_t>(xs[i]) * ldc + xs[i + 1 == n ? 0 : i + 1]];
        if (tid == 0) xs[n] = xs[0];
        long long f = a.cost[p];
        int moves = 0, passes = 0;
        __syncthreads();

        // Each move lowers the integer cost, so the loop ends; the guard only
        // turns an impossible runaway into an error status instead of a hang.
        const int guard = 1000 + 100 * n;
        for (;;) {
            if (a.max_moves > 0 && moves >= a.max_moves) break;
            if (moves >= guard) {
                if (tid == 0 && a.status) atomicExch(a.status, DPSO_ERR_INTERNAL);
                break;
            }
            int best_d = INT_MAX, best_i = INT_MAX;  // meaningful in thread 0
            for (int I = 0; I <= n - 3; I += R) {
                const int nrows = min(R, n - 2 - I);
                for (int r = warp; r <= nrows; r += kWarps) {
                    const int* src = C + static_cast<size_t>(xs[I + r]) * ldc;
                    int* dst = rows + static_cast<size_t>(r) * ldr;
                    for (int c = lane; c < n; c += 32) cp_async4(dst + c, src + c);
                }
                if (tid < R) s_rowmin[tid] = INT_MAX;
                cp_async_wait_all();
                __syncthreads();

                int m = INT_MAX;
                const int rowi = I + arow;
                const bool row_ok = arow < nrows;
                const int* r0 = rows + static_cast<size_t>(arow) * ldr;
                const int* r1 = r0 + ldr;
                for (int c = I + 2 + warp * kStreams + stream; c < n; c += kWarps * kStreams) {
                    if (row_ok && c >= rowi + 2 && !(rowi == 0 && c == n - 1)) {
                        const int v = r0[xs[c]] + r1[xs[c + 1]] - dd[c];
                        m = min(m, v);
                    }
                }
#pragma unroll
                for (int o = R; o < 32; o <<= 1) m = min(m, __shfl_xor_sync(kFull, m, o));
                if (stream == 0 && row_ok && m != INT_MAX) atomicMin(&s_rowmin[arow], m);
                __syncthreads();
                if (tid == 0) {
                    for (int r = 0; r < nrows; ++r) {
                        const int mm = s_rowmin[r];
                        if (mm == INT_MAX) continue;
                        const int dl = mm - dd[I + r];
                        if (dl < best_d) {
                            best_d = dl;
                            best_i = I + r;
                        }
                    }
                }
                __syncthreads();
            }
            ++passes;
            if (tid == 0) {
                s_bd = best_d;
                s_bi = best_i;
                s_bj = INT_MAX;
            }
            __syncthreads();
            const int bd = s_bd;
            if (bd >= 0) break;
            const int bi = s_bi;
            {
                const size_t ra = static_cast<size_t>(xs[bi]) * ldc;
                const size_t rb = static_cast<size_t>(xs[bi + 1]) * ldc;
                for (int j = bi + 2 + tid; j < n; j += blockDim.x) {
                    if (bi == 0 && j == n - 1) continue;
                    const int dl = C[ra + xs[j]] + C[rb + xs[j + 1]] - dd[bi] - dd[j];
                    if (dl == bd) atomicMin(&s_bj, j);
                }
            }
            __syncthreads();
            const int bj = s_bj;
            if (tid == 0) {
                s_ei = C[static_cast<size_t>(xs[bi]) * ldc + xs[bj]];
                s_ej = C[static_cast<size_t>(xs[bi + 1]) * ldc + xs[bj + 1]];
            }
            __syncthreads();
            // reverse x[bi+1..bj] and the edge costs in between
            const int lx = bj - bi, le = bj - bi - 1;
            for (int q = tid; q < lx / 2; q += blockDim.x) {
                const uint16_t t0 = xs[bi + 1 + q];
                xs[bi + 1 + q] = xs[bj - q];
                xs[bj - q] = t0;
            }
            for (int q = tid; q < le / 2; q += blockDim.x) {
                const int t0 = dd[bi + 1 + q];
                dd[bi + 1 + q] = dd[bj - 1 - q];
                dd[bj - 1 - q] = t0;
            }
            __syncthreads();
            if (tid == 0) {
                dd[bi] = s_ei;
                dd[bj] = s_ej;
            }
            f += bd;
            ++moves;
            __syncthreads();
        }

        for (int i = tid; i < n; i += blockDim.x) tour[i] = xs[i];
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
            for (int i = tid; i < n; i += blockDim.x) pb[i] = xs[i];
            if (tid == 0) a.pcost[p] = f;
        }
        __syncthreads();
    }
}

template <int R>
cudaError_t launch_r(const TwoOptBatch& b, int num_sms, cudaStream_t st) {
    const size_t smem = two_opt_smem(b.max_n, R);
    cudaError_t e = raise_smem_limit(two_opt_kernel<R>, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, two_opt_kernel<R>, kWarps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = max(1, min(b.total, per_sm * num_sms));
    two_opt_kernel<R><<<grid, kWarps * 32, smem, st>>>(b);
    return cudaGetLastError();
}

}  // namespace

int two_opt_rows(int n) {
    const size_t budget = 220 * 1024;
    for (int R = 32; R >= 4; R /= 2)
        if (two_opt_smem(n, R) <= budget) return R;
    return 0;
}

cudaError_t launch_two_opt_general(const TwoOptBatch& b, int num_sms, cudaStream_t st) {
    switch (two_opt_rows(b.max_n)) {
        case 32: return launch_r<32>(b, num_sms, st);
        case 16: return launch_r<16>(b, num_sms, st);
        case 8: return launch_r<8>(b, num_sms, st);
        case 4: return launch_r<4>(b, num_sms, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_two_opt(const TwoOptBatch& b, int num_sms, cudaStream_t st) {
    if (b.total <= 0) return cudaSuccess;
    if (b.kind == 1) return launch_node_swap_tiled(b, num_sms, st);
    if (b.shifted && two_opt_tiled_rows(b.max_n) > 0) {
        int rows = b.rows, tpc = b.tpc, tg = b.tg;
        if (rows <= 0) {  // no pinned shape
            two_opt_default_shape(b.max_n, b.total, num_sms, &rows, &tpc, &tg);
        } else {
            if (tpc <= 0) tpc = two_opt_tiled_tpc(b.max_n, rows);
            if (tg <= 0) tg = two_opt_tiled_tg(b.max_n, rows, tpc);
        }
        return launch_two_opt_tiled(b, rows, tpc, tg, num_sms, st);
    }
    return launch_two_opt_general(b, num_sms, st);
}

}  // namespace dpso
