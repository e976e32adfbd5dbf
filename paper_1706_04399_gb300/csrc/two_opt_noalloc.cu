// dpso_two_opt_noalloc: the standalone 2-opt entry point without any device
// allocation.  Its scratch (error word, work queue, totals and per-tour pass /
// move counts) lives in one fixed array inside the library.  It runs the
// general (untiled) 2-opt kernel: the tiled kernel stages rows from four
// row-shifted copies of the cost matrix, which would need an allocation.
//
// Who needs it: callers that must not allocate device memory while they run,
// e.g. an on-board re-planning loop whose GPU memory is reserved once at
// start-up (cudaMalloc / cudaFree can synchronise the device and can fail under
// fragmentation mid-mission), or a host process whose device memory belongs to
// another allocator (a framework's caching pool) that does not expect
// allocations made behind its back.
#include "common.cuh"

namespace dpso {
namespace {

// Scratch layout (32-bit words): [0] error word, [1] work queue, [2..3] pairs
// total, [4..5] moves total, [6..15] unused, [16..63] the task descriptor,
// [64..65] its tour offsets, then `count` pass counts followed by `count` move
// counts.
constexpr int kTaskWord = 16;
constexpr int kOffWord = 64;
constexpr int kHeaderWords = 68;
constexpr size_t kScratchBytes = 128 * 1024;
static_assert(sizeof(TwoOptTask) <= (kOffWord - kTaskWord) * 4, "task descriptor does not fit");
static_assert((kScratchBytes / 4 - kHeaderWords) / 2 == DPSO_NOALLOC_MAX_TOURS,
              "DPSO_NOALLOC_MAX_TOURS must match the scratch array");

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned int g_scratch[kScratchBytes / 4];

// Device address of g_scratch on the current device (the host-side symbol is
// only a stand-in, not a device address).  Looked up on every call, with the
// caller's device current: the lookup allocates nothing, and an address kept
// from an earlier call would be stale after the context were reset.
int scratch_address(unsigned int** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return DPSO_ERR_CUDA;
    *out = static_cast<unsigned int*>(p);
    return DPSO_OK;
}

// Sums the per-tour counts into the totals (one block, deterministic order
// per thread, integer sums).
__global__ void noalloc_totals_kernel(unsigned int* scratch, int count, long long npairs) {
    __shared__ unsigned long long sp[256], sm[256];
    const unsigned int* passes = scratch + kHeaderWords;
    const unsigned int* moves = passes + count;
    unsigned long long a = 0, b = 0;
    for (int p = threadIdx.x; p < count; p += blockDim.x) {
        a += static_cast<unsigned long long>(passes[p]) * static_cast<unsigned long long>(npairs);
        b += moves[p];
    }
    sp[threadIdx.x] = a;
    sm[threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sp[threadIdx.x] += sp[threadIdx.x + o];
            sm[threadIdx.x] += sm[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        reinterpret_cast<unsigned long long*>(scratch + 2)[0] = sp[0];
        reinterpret_cast<unsigned long long*>(scratch + 4)[0] = sm[0];
    }
}

}  // namespace
}  // namespace dpso

using namespace dpso;

extern "C" int dpso_two_opt_noalloc(const int32_t* C_dev, int32_t n, uint16_t* tours_dev,
                                    int32_t count, int64_t* cost_dev, int32_t max_moves,
                                    int64_t* pairs_host, int64_t* moves_host, void* stream) {
    if (!C_dev || !tours_dev || !cost_dev || n < 3 || count < 0 || max_moves < 0)
        return DPSO_ERR_ARG;
    if (n > DPSO_MAX_N || count > DPSO_NOALLOC_MAX_TOURS) return DPSO_ERR_RANGE;
    if (pairs_host) *pairs_host = 0;
    if (moves_host) *moves_host = 0;
    if (count == 0) return DPSO_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DPSO_ERR_CUDA;
    unsigned int* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    int* err = reinterpret_cast<int*>(scratch);
    const size_t used = sizeof(unsigned int) * (kHeaderWords + 2 * static_cast<size_t>(count));
    unsigned int header[6] = {0, 0, 0, 0, 0, 0};

    // The array keeps the previous call's contents: clear what must start at 0.
    cudaError_t e = cudaMemsetAsync(scratch, 0, used, st);
    if (e == cudaSuccess) e = launch_check_cost(C_dev, n, n, err, st);
    if (e == cudaSuccess) {
        tours_valid_kernel<<<count, 256, n, st>>>(tours_dev, n, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(header, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return DPSO_ERR_CUDA;
    if (header[0] & 1u) return DPSO_ERR_ARG;
    if (header[0] & 2u) return DPSO_ERR_RANGE;

    e = launch_fitness(C_dev, n, n, tours_dev, n, count, reinterpret_cast<long long*>(cost_dev), st);
    TwoOptTask a{};
    a.C = C_dev;
    a.ldc = n;
    a.n = n;
    a.tours = tours_dev;
    a.ldt = n;
    a.count = count;
    a.cost = reinterpret_cast<long long*>(cost_dev);
    a.max_moves = max_moves;
    a.pairs = reinterpret_cast<unsigned long long*>(scratch + 2);
    a.moves = reinterpret_cast<unsigned long long*>(scratch + 4);
    a.status = err;
    a.tour_passes = scratch + kHeaderWords;
    a.tour_moves = scratch + kHeaderWords + count;
    TwoOptTask* task = reinterpret_cast<TwoOptTask*>(scratch + kTaskWord);
    int* toff = reinterpret_cast<int*>(scratch + kOffWord);
    const int host_off[2] = {0, count};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(task, &a, sizeof(TwoOptTask), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(toff, host_off, sizeof(host_off), cudaMemcpyHostToDevice, st);
    const TwoOptBatch tb{task, toff, 1, count, n, false, 0, scratch + 1};
    if (e == cudaSuccess) e = launch_two_opt(tb, sms, st);
    if (e == cudaSuccess) {
        noalloc_totals_kernel<<<1, 256, 0, st>>>(scratch, count,
                                                 static_cast<long long>(n) * (n - 3) / 2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(header, scratch, sizeof(header), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return DPSO_ERR_CUDA;
    if (static_cast<int>(header[0]) == DPSO_ERR_INTERNAL) return DPSO_ERR_INTERNAL;
    unsigned long long pairs = header[2] | (static_cast<unsigned long long>(header[3]) << 32);
    unsigned long long moves = header[4] | (static_cast<unsigned long long>(header[5]) << 32);
    if (pairs_host) *pairs_host = static_cast<int64_t>(pairs);
    if (moves_host) *moves_host = static_cast<int64_t>(moves);
    return DPSO_OK;
}
