// Measurement aid for the roofline of the 2-opt kernel: the L2 read bandwidth
// that bounds staging cost rows from the L2-resident cost matrix.  (The paper
// has no counterpart; this only measures the device.)
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

}  // namespace
}  // namespace dpso

using namespace dpso;

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
