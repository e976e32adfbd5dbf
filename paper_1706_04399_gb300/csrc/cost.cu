// Edge-cost matrix of the extended TSP (Sec. 2.3): straight-segment Euclidean
// length in millimetres, rounded to nearest in FP64, plus a penalty when the
// closed segment meets an obstacle box grown by the UAV radius.
//
// Every FP64 step is an explicit round-to-nearest intrinsic, so nothing is
// contracted into an FMA and sqrt / divide are the correctly rounded IEEE
// operations; the file is also built with -fmad=false.
#include <math.h>

#include "common.cuh"

namespace dpso {
namespace {

// Closed segment p + t (q - p), t in [0, 1], against the closed box
// [lo - r, hi + r] (slab test, axes x, y, z in order).
__device__ bool segment_blocked(const double p[3], const double q[3], const double* box,
                                double r) {
    double tmin = 0.0, tmax = 1.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double lo = __dsub_rn(box[k], r);
        const double hi = __dadd_rn(box[3 + k], r);
        const double d = __dsub_rn(q[k], p[k]);
        if (d == 0.0) {
            if (p[k] < lo || p[k] > hi) return false;
        } else {
            double t1 = __ddiv_rn(__dsub_rn(lo, p[k]), d);
            double t2 = __ddiv_rn(__dsub_rn(hi, p[k]), d);
            if (t1 > t2) {
                const double tt = t1;
                t1 = t2;
                t2 = tt;
            }
            if (t1 > tmin) tmin = t1;
            if (t2 < tmax) tmax = t2;
        }
    }
    return tmin <= tmax;
}

constexpr int kTile = 32;

// One thread per (i, j) with i < j inside 32 x 32 tiles of the upper triangle;
// boxes are staged in shared memory in chunks.
__global__ void __launch_bounds__(kTile * 8) cost_matrix_kernel(
    const double* __restrict__ xyz, int n, const double* __restrict__ boxes, int m, double r,
    int penalty, int* __restrict__ C, int ldc, int* err) {
    const int bi = blockIdx.y * kTile, bj = blockIdx.x * kTile;
    if (bj + kTile <= bi) return;  // strictly below the diagonal
    __shared__ double sbox[256 * 6];
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    long long base[4];
    bool blocked[4];
    int ii[4], jj[4];
    double p[4][3], q[4][3];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        ii[s] = bi + ty + 8 * s;
        jj[s] = bj + tx;
        blocked[s] = false;
        base[s] = 0;
        if (ii[s] < n && jj[s] < n && ii[s] < jj[s]) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                p[s][k] = xyz[3 * (size_t)ii[s] + k];
                q[s][k] = xyz[3 * (size_t)jj[s] + k];
            }
            const double dx = __dsub_rn(q[s][0], p[s][0]);
            const double dy = __dsub_rn(q[s][1], p[s][1]);
            const double dz = __dsub_rn(q[s][2], p[s][2]);
            double acc = __dmul_rn(dx, dx);
            acc = __dadd_rn(acc, __dmul_rn(dy, dy));
            acc = __dadd_rn(acc, __dmul_rn(dz, dz));
            base[s] = __double2ll_rn(__dmul_rn(1000.0, __dsqrt_rn(acc)));
        }
    }
    for (int b0 = 0; b0 < m; b0 += 256) {
        const int cnt = min(256, m - b0);
        __syncthreads();
        for (int e = ty * kTile + tx; e < cnt * 6; e += kTile * 8) sbox[e] = boxes[6 * (size_t)b0 + e];
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (ii[s] < n && jj[s] < n && ii[s] < jj[s]) {
                for (int b = 0; b < cnt && !blocked[s]; ++b)
                    blocked[s] = segment_blocked(p[s], q[s], sbox + 6 * b, r);
            }
        }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int i = ii[s], j = jj[s];
        if (i >= n || j >= n) continue;
        if (i == j) {
            C[(size_t)i * ldc + i] = 0;
            continue;
        }
        if (i > j) continue;
        long long v = base[s] + (blocked[s] ? (long long)penalty : 0LL);
        if (v > DPSO_COST_MAX) {
            atomicOr(err, 2);
            v = DPSO_COST_MAX;
        }
        C[(size_t)i * ldc + j] = static_cast<int>(v);
        C[(size_t)j * ldc + i] = static_cast<int>(v);
    }
}

// Flags non-finite coordinates and inverted boxes (bit 0 of *err).
__global__ void check_inputs_kernel(const double* __restrict__ xyz, int n,
                                    const double* __restrict__ boxes, int m, int* err) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 3 * n && !isfinite(xyz[k])) atomicOr(err, 1);
    if (k < m) {
        for (int a = 0; a < 6; ++a)
            if (!isfinite(boxes[6 * (size_t)k + a])) atomicOr(err, 1);
        for (int a = 0; a < 3; ++a)
            if (boxes[6 * (size_t)k + a] > boxes[6 * (size_t)k + 3 + a]) atomicOr(err, 1);
    }
}

// Flags an asymmetric matrix or a non-zero diagonal (bit 0) and entries outside
// [0, limit] (bit 1).
__global__ void check_cost_kernel(const int* __restrict__ C, int n, int ldc, int limit, int* err) {
    const int i = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int v = C[(size_t)i * ldc + j];
        if (v < 0 || v > limit) atomicOr(err, 2);
        if (i == j ? v != 0 : v != C[(size_t)j * ldc + i]) atomicOr(err, 1);
    }
}

}  // namespace

cudaError_t launch_cost_matrix(const double* xyz, int n, const double* boxes, int m, double radius,
                               int penalty, int* C, int ldc, int* err, cudaStream_t st) {
    const int tiles = (n + kTile - 1) / kTile;
    dim3 grid(tiles, tiles), block(kTile, 8);
    cost_matrix_kernel<<<grid, block, 0, st>>>(xyz, n, boxes, m, radius, penalty, C, ldc, err);
    return cudaGetLastError();
}

cudaError_t launch_check_inputs(const double* xyz, int n, const double* boxes, int m, int* err,
                                cudaStream_t st) {
    const int work = max(3 * n, m);
    check_inputs_kernel<<<(work + 255) / 256, 256, 0, st>>>(xyz, n, boxes, m, err);
    return cudaGetLastError();
}

cudaError_t launch_check_cost(const int* C, int n, int ldc, int* err, cudaStream_t st) {
    return launch_check_cost_limit(C, n, ldc, DPSO_COST_MAX, err, st);
}

cudaError_t launch_check_cost_limit(const int* C, int n, int ldc, int limit, int* err,
                                    cudaStream_t st) {
    dim3 grid((n + 255) / 256, n);
    check_cost_kernel<<<grid, 256, 0, st>>>(C, n, ldc, limit, err);
    return cudaGetLastError();
}

}  // namespace dpso

using namespace dpso;

extern "C" int dpso_cost_matrix(const double* xyz_dev, int32_t n, const double* boxes_dev,
                                int32_t m, const dpso_cost_params* cp, int32_t* C_dev,
                                void* stream) {
    if (!xyz_dev || !C_dev || !cp || n < 1 || m < 0 || (m > 0 && !boxes_dev)) return DPSO_ERR_ARG;
    if (n > DPSO_MAX_N) return DPSO_ERR_RANGE;
    if (!(cp->uav_radius_m >= 0.0) || !isfinite(cp->uav_radius_m) || cp->blocked_penalty_mm < 0 ||
        cp->reserved != 0)
        return DPSO_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* err = nullptr;
    if (cudaMallocAsync(&err, sizeof(int), st) != cudaSuccess) return DPSO_ERR_NO_MEMORY;
    int herr = 0;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_check_inputs(xyz_dev, n, boxes_dev, m, err, st);
    if (e == cudaSuccess)
        e = launch_cost_matrix(xyz_dev, n, boxes_dev, m, cp->uav_radius_m, cp->blocked_penalty_mm,
                               C_dev, n, err, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(err, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return DPSO_ERR_CUDA;
    if (herr & 1) return DPSO_ERR_ARG;
    if (herr & 2) return DPSO_ERR_RANGE;
    return DPSO_OK;
}
