// Edge exchange of Sec. 3.2.3 (best-improvement 2-opt to 2-optimality), the
// TMA-staged variant for tours whose 33-row tiles fit in shared memory.
//
// Same mathematics and tie order as two_opt.cu:
//   delta(i, j) = C[x_i][x_j] + C[x_i+1][x_j+1] - C[x_i][x_i+1] - C[x_j][x_j+1],
//   the applied move is the smallest (delta, i, j) with delta < 0.
//
// Layout and mapping:
//  * One CTA per tour (persistent grid, work queue), 8 warps.
//  * A tile is 32 positions I..I+31, one per lane; its 33 cost rows
//    C[x_I..x_I+32] are staged into shared memory by TMA bulk copies (one
//    instruction per row), double-buffered behind an mbarrier per buffer.
//  * Bulk copies need 16-byte-aligned rows, which alone would put rows a,
//    a+8, a+16, a+24 in the same bank.  The cost matrix is therefore kept in
//    four copies whose rows are shifted right by 0..3 words; row a of a tile is
//    taken from copy (a>>3)&3 into a row pitch ldq with ldq/4 odd, so the 32
//    lanes reading one column hit 32 distinct banks.
//  * Column records rec[c] = {x_c+1, -C[x_c][x_c+1]} give the second gather's
//    column and the edge term in one broadcast load; the first gather's column
//    x_c is the previous record's.
//  * Each lane keeps min over its columns of C[x_i][x_c] + C[x_i+1][x_c+1] -
//    C[x_c][x_c+1]; subtracting C[x_i][x_i+1] gives its row's best delta, which
//    enters a packed 64-bit (delta, i) key kept across all tiles of the pass.
//    One block reduction per pass yields (delta*, i*); a scan of row i*
//    yields the smallest j*.  Pairs with j = i+1 or (0, n-1) have delta = 0
//    for a symmetric C and never win, so only the triangle of each tile is
//    masked.
#include <climits>

#include "common.cuh"

namespace dpso {
namespace {

constexpr int kRows = 32;
constexpr int kStaged = kRows + 1;
constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kWaitSpins = 1 << 20;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity; false after kWaitSpins tries.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity) {
    for (int it = 0; it < kWaitSpins; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ unsigned long long pack_key(int delta, int i) {
    return (static_cast<unsigned long long>(static_cast<uint32_t>(delta) ^ 0x80000000u) << 32) |
           static_cast<uint32_t>(i);
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

}  // namespace

// Row pitch (words) of the shifted copies and of the staged rows: room for a
// shift of up to 3 words, a multiple of 4 words (16-byte rows), ldq/4 odd.
__host__ __device__ int shifted_ld(int n) {
    int q = (n + 3 + 3) / 4 * 4;
    if (((q / 4) & 1) == 0) q += 4;
    return q;
}

size_t two_opt_tma_smem(int n, int stages) {
    const size_t rows = static_cast<size_t>(stages) * kStaged * shifted_ld(n) * sizeof(int);
    const size_t rec = static_cast<size_t>(n + 1) * sizeof(int2);
    const size_t xs = static_cast<size_t>((n + 1 + 7) / 8 * 8) * sizeof(uint16_t);
    return rows + rec + xs;
}

namespace {

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

__global__ void __launch_bounds__(kThreads) two_opt_tma_kernel(TwoOptArgs a, int stages) {
    if (a.gate && *a.gate == 0) return;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ unsigned long long s_bar[2];
    __shared__ unsigned long long s_key[kWarps];
    __shared__ unsigned long long s_best;
    __shared__ int s_part, s_bj;
    __shared__ long long s_pf;

    const int n = a.n;
    const int ldq = shifted_ld(n);
    const size_t buf_words = static_cast<size_t>(kStaged) * ldq;
    int* rows = reinterpret_cast<int*>(sm);
    int2* rec = reinterpret_cast<int2*>(sm + stages * buf_words * sizeof(int));
    uint16_t* xs = reinterpret_cast<uint16_t*>(rec + (n + 1));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int* __restrict__ C = a.C;
    const int* __restrict__ Cs = a.Cs;
    const int ldc = a.ldc;
    const long long npairs = static_cast<long long>(n) * (n - 3) / 2;
    const int ntiles = (n - 2 + kRows - 1) / kRows;  // tiles start at I <= n-3
    const int guard = 1000 + 100 * n;

    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    uint32_t uses[2] = {0u, 0u};    // phases consumed per buffer (every thread)
    uint32_t issued[2] = {0u, 0u};  // phases issued per buffer (thread 0)

    // Thread 0: stage the rows of tile t into buffer t % stages.
    auto issue = [&](int t) {
        const int b = t % stages;
        const int I = t * kRows;
        const int count = min(kStaged, n - 1 - I);
        int* dst = rows + b * buf_words;
        mbar_expect_tx(&s_bar[b], static_cast<uint32_t>(count * ldq * sizeof(int)));
        for (int r = 0; r < count; ++r) {
            const int k = (r >> 3) & 3;
            const int* src = Cs + (static_cast<size_t>(k) * n + xs[I + r]) * ldq;
            bulk_g2s(dst + static_cast<size_t>(r) * ldq, src, ldq * sizeof(int), &s_bar[b]);
        }
        ++issued[b];
    };
    auto abort_kernel = [&]() {
        if (tid == 0) {
            for (int b = 0; b < 2; ++b)
                while (uses[b] < issued[b]) {
                    mbar_wait(&s_bar[b], uses[b] & 1u);
                    ++uses[b];
                }
            if (a.status) atomicExch(a.status, DPSO_ERR_TIMEOUT);
        }
        __syncthreads();
    };

    for (;;) {
        if (tid == 0) s_part = static_cast<int>(atomicAdd(a.queue, 1u));
        __syncthreads();
        const int p = s_part;
        if (p >= a.count) break;
        uint16_t* tour = a.tours + static_cast<size_t>(p) * a.ldt;
        for (int i = tid; i < n; i += kThreads) xs[i] = tour[i];
        if (tid == 0) xs[n] = tour[0];
        __syncthreads();
        for (int c = tid; c < n; c += kThreads) {
            const int u = xs[c], v = xs[c + 1];
            rec[c] = make_int2(v, -C[static_cast<size_t>(u) * ldc + v]);
        }
        long long f = a.cost[p];
        int moves = 0, passes = 0;
        __syncthreads();

        for (;;) {
            if (a.max_moves > 0 && moves >= a.max_moves) break;
            if (moves >= guard) {
                if (tid == 0 && a.status) atomicExch(a.status, DPSO_ERR_INTERNAL);
                break;
            }
            if (tid == 0) {
                fence_proxy_async();
                for (int t = 0; t < stages && t < ntiles; ++t) issue(t);
            }
            unsigned long long key = ~0ull;
            for (int t = 0; t < ntiles; ++t) {
                const int b = t % stages;
                bool ok = mbar_wait(&s_bar[b], uses[b] & 1u);
                if (ok) {
                    ++uses[b];
                    const int I = t * kRows;
                    const int* buf = rows + b * buf_words;
                    const int* P1 = buf + static_cast<size_t>(lane) * ldq + ((lane >> 3) & 3);
                    const int* P2 = buf + static_cast<size_t>(lane + 1) * ldq + (((lane + 1) >> 3) & 3);
                    const int cbeg = I + 2, total = n - cbeg;
                    const int c0 = cbeg + static_cast<int>((static_cast<long long>(total) * warp) / kWarps);
                    const int c1 = cbeg + static_cast<int>((static_cast<long long>(total) * (warp + 1)) / kWarps);
                    int m = INT_MAX;
                    int c = c0;
                    if (c < c1) {
                        int q = rec[c - 1].x;  // x_c
                        // columns where lanes beyond the diagonal are masked
                        const int tri_end = min(c1, I + kRows + 2);
                        for (; c < tri_end; ++c) {
                            const int2 r = rec[c];
                            const int v = P1[q] + P2[r.x] + r.y;
                            q = r.x;
                            if (lane <= c - I - 2) m = min(m, v);
                        }
                        for (; c + 4 <= c1; c += 4) {
                            const int2 r0 = rec[c], r1 = rec[c + 1], r2 = rec[c + 2], r3 = rec[c + 3];
                            const int v0 = P1[q] + P2[r0.x] + r0.y;
                            const int v1 = P1[r0.x] + P2[r1.x] + r1.y;
                            const int v2 = P1[r1.x] + P2[r2.x] + r2.y;
                            const int v3 = P1[r2.x] + P2[r3.x] + r3.y;
                            m = min(m, min(min(v0, v1), min(v2, v3)));
                            q = r3.x;
                        }
                        for (; c < c1; ++c) {
                            const int2 r = rec[c];
                            m = min(m, P1[q] + P2[r.x] + r.y);
                            q = r.x;
                        }
                    }
                    if (m != INT_MAX) key = min(key, pack_key(m + rec[I + lane].y, I + lane));
                }
                ok = __syncthreads_and(ok);
                if (!ok) {
                    abort_kernel();
                    return;
                }
                if (tid == 0 && t + stages < ntiles) {
                    fence_proxy_async();
                    issue(t + stages);
                }
            }
            ++passes;
            key = warp_min_u64(key);
            if (lane == 0) s_key[warp] = key;
            __syncthreads();
            if (warp == 0) {
                unsigned long long kk = lane < kWarps ? s_key[lane] : ~0ull;
                kk = warp_min_u64(kk);
                if (lane == 0) {
                    s_best = kk;
                    s_bj = INT_MAX;
                }
            }
            __syncthreads();
            const unsigned long long best = s_best;
            if (best == ~0ull) break;
            const int bd = static_cast<int>(static_cast<uint32_t>(best >> 32) ^ 0x80000000u);
            if (bd >= 0) break;
            const int bi = static_cast<int>(best & 0xffffffffu);
            {
                const size_t ra = static_cast<size_t>(xs[bi]) * ldc;
                const size_t rb = static_cast<size_t>(xs[bi + 1]) * ldc;
                const int ndi = rec[bi].y;
                for (int j = bi + 2 + tid; j < n; j += kThreads) {
                    const int dl = C[ra + xs[j]] + C[rb + xs[j + 1]] + ndi + rec[j].y;
                    if (dl == bd) atomicMin(&s_bj, j);
                }
            }
            __syncthreads();
            const int bj = s_bj;
            const int ei = C[static_cast<size_t>(xs[bi]) * ldc + xs[bj]];
            const int ej = C[static_cast<size_t>(xs[bi + 1]) * ldc + xs[bj + 1]];
            __syncthreads();
            // reverse x[bi+1..bj] and the edge terms strictly between bi and bj
            for (int q = tid; q < (bj - bi) / 2; q += kThreads) {
                const uint16_t t0 = xs[bi + 1 + q];
                xs[bi + 1 + q] = xs[bj - q];
                xs[bj - q] = t0;
            }
            for (int q = tid; q < (bj - bi - 1) / 2; q += kThreads) {
                const int t0 = rec[bi + 1 + q].y;
                rec[bi + 1 + q].y = rec[bj - 1 - q].y;
                rec[bj - 1 - q].y = t0;
            }
            __syncthreads();
            for (int c = bi + tid; c <= bj; c += kThreads)
                rec[c] = make_int2(xs[c + 1], c == bi ? -ei : (c == bj ? -ej : rec[c].y));
            f += bd;
            ++moves;
            __syncthreads();
        }

        for (int i = tid; i < n; i += kThreads) tour[i] = xs[i];
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
            for (int i = tid; i < n; i += kThreads) pb[i] = xs[i];
            if (tid == 0) a.pcost[p] = f;
        }
        __syncthreads();
    }
}

}  // namespace

// Stages (0 = not eligible) and CTAs per SM the TMA variant uses for n.
int two_opt_tma_stages(int n, int* ctas_per_sm) {
    const size_t two = two_opt_tma_smem(n, 2), one = two_opt_tma_smem(n, 1);
    if (two <= 110 * 1024) { *ctas_per_sm = 2; return 2; }
    if (two <= 220 * 1024) { *ctas_per_sm = 1; return 2; }
    if (one <= 220 * 1024) { *ctas_per_sm = 1; return 1; }
    *ctas_per_sm = 0;
    return 0;
}

cudaError_t build_shifted_copies(const int* C, int ldc, int n, int* Cs, cudaStream_t st) {
    dim3 grid(n, 4);
    shift_copies_kernel<<<grid, 128, 0, st>>>(C, ldc, n, shifted_ld(n), Cs);
    return cudaGetLastError();
}

cudaError_t launch_two_opt_tma(const TwoOptArgs& a, int num_sms, cudaStream_t st) {
    int per_sm_target = 0;
    const int stages = two_opt_tma_stages(a.n, &per_sm_target);
    if (stages == 0 || !a.Cs) return cudaErrorInvalidValue;
    const size_t smem = two_opt_tma_smem(a.n, stages);
    cudaError_t e = cudaFuncSetAttribute(two_opt_tma_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, two_opt_tma_kernel, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = max(1, min(a.count, per_sm * num_sms));
    two_opt_tma_kernel<<<grid, kThreads, smem, st>>>(a, stages);
    return cudaGetLastError();
}

}  // namespace dpso
