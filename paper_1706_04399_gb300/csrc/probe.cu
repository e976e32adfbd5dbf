// Measurement aids for the rooflines (the paper has no counterpart; these only
// measure the device): the L2 read bandwidth that bounds staging cost rows
// from the L2-resident cost matrix in the 2-opt kernel, and the rate of
// independent 4-byte random gathers from an L2-resident matrix that bounds the
// tour-fitness kernel (each C[x_k][x_k+1] is one such gather).
#include "common.cuh"

namespace dpso {
namespace {

// Every thread reads 16-byte words of the buffer in a grid-stride loop, `reps`
// times; the xor of everything read is stored only if it hits a sentinel, so
// the loads cannot be dropped.
__global__ void l2_read_kernel(const uint4* __restrict__ buf, size_t words, int reps,
                               unsigned int* sink) {
    unsigned int acc = 0;
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    for (int r = 0; r < reps; ++r)
        for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < words;
             i += stride) {
            const uint4 v = buf[i];
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (acc == 0x9E3779B9u) sink[0] = acc;
}

// Every thread issues `reps` rounds of eight independent 4-byte loads at
// pseudo-random word indices of the buffer (a 32-bit LCG per thread, index by
// multiply-shift), the same access shape as a fitness gather.  The xor of the
// loaded words is stored only if it hits a sentinel.
__global__ void l2_gather_kernel(const int* __restrict__ buf, unsigned words, int reps,
                                 unsigned int* sink) {
    unsigned s = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
    int acc = 0;
    for (int r = 0; r < reps; ++r) {
        unsigned idx[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            s = s * 1664525u + 1013904223u;
            idx[k] = static_cast<unsigned>((static_cast<unsigned long long>(s) * words) >> 32);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) acc ^= buf[idx[k]];
    }
    if (static_cast<unsigned>(acc) == 0x9E3779B9u) sink[0] = acc;
}

// Best-of-five CUDA-event time of `launch(reps)` after one warm-up launch.
template <typename F>
int best_of_five(cudaStream_t st, F launch, double* best_ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int status = DPSO_OK;
    *best_ms = 1e30;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        status = DPSO_ERR_CUDA;
    } else {
        launch(true);
        for (int trial = 0; trial < 5 && status == DPSO_OK; ++trial) {
            float ms = 0.f;
            if (cudaEventRecord(e0, st) != cudaSuccess) status = DPSO_ERR_CUDA;
            launch(false);
            if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
                cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                status = DPSO_ERR_CUDA;
            else if (ms < *best_ms)
                *best_ms = ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return status;
}

}  // namespace
}  // namespace dpso

using namespace dpso;

extern "C" int dpso_probe_l2_gather_gbs(size_t bytes, int32_t reps, double* gbs, void* stream) {
    if (!gbs || bytes < 4096 || bytes > (static_cast<size_t>(1) << 33) || reps < 1)
        return DPSO_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DPSO_ERR_CUDA;
    const unsigned words = static_cast<unsigned>(bytes / 4);
    void* buf = nullptr;
    if (cudaMalloc(&buf, static_cast<size_t>(words) * 4 + 16) != cudaSuccess) {
        cudaGetLastError();
        return DPSO_ERR_NO_MEMORY;
    }
    unsigned int* sink =
        reinterpret_cast<unsigned int*>(static_cast<char*>(buf) + static_cast<size_t>(words) * 4);
    const int grid = sms * 8, block = 256;
    double best_ms = 0.0;
    int status = DPSO_OK;
    if (cudaMemsetAsync(buf, 1, static_cast<size_t>(words) * 4, st) != cudaSuccess) {
        status = DPSO_ERR_CUDA;
    } else {
        // the warm-up launch reads the whole buffer once, so it is L2-resident
        l2_read_kernel<<<grid, block, 0, st>>>(static_cast<const uint4*>(buf), words / 4, 1, sink);
        status = best_of_five(st, [&](bool warm) {
            l2_gather_kernel<<<grid, block, 0, st>>>(static_cast<const int*>(buf), words,
                                                     warm ? 1 : reps, sink);
        }, &best_ms);
    }
    cudaFree(buf);
    if (status != DPSO_OK) return status;
    *gbs = 4.0 * 8.0 * static_cast<double>(grid) * block * reps / (best_ms * 1e-3) / 1e9;
    return DPSO_OK;
}

extern "C" int dpso_probe_l2_read_gbs(size_t bytes, int32_t reps, double* gbs, void* stream) {
    if (!gbs || bytes < 4096 || reps < 1) return DPSO_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DPSO_ERR_CUDA;
    const size_t words = bytes / 16;
    void* buf = nullptr;
    if (cudaMalloc(&buf, words * 16 + 16) != cudaSuccess) {
        cudaGetLastError();
        return DPSO_ERR_NO_MEMORY;
    }
    unsigned int* sink = reinterpret_cast<unsigned int*>(static_cast<char*>(buf) + words * 16);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int status = DPSO_OK;
    double best_ms = 1e30;
    if (cudaMemsetAsync(buf, 1, words * 16, st) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        status = DPSO_ERR_CUDA;
    } else {
        const int grid = sms * 8;
        l2_read_kernel<<<grid, 256, 0, st>>>(static_cast<const uint4*>(buf), words, 1, sink);
        for (int trial = 0; trial < 5 && status == DPSO_OK; ++trial) {
            float ms = 0.f;
            if (cudaEventRecord(e0, st) != cudaSuccess) status = DPSO_ERR_CUDA;
            l2_read_kernel<<<grid, 256, 0, st>>>(static_cast<const uint4*>(buf), words, reps, sink);
            if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
                cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                status = DPSO_ERR_CUDA;
            else if (ms < best_ms)
                best_ms = ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (status != DPSO_OK) return status;
    *gbs = static_cast<double>(words) * 16.0 * reps / (best_ms * 1e-3) / 1e9;
    return DPSO_OK;
}
