// Device helpers shared by the tiled exchange kernels (2-opt, node swap):
// shared-memory addresses, one bulk copy per staged cost row counted on an
// mbarrier with a clock-bounded wait, and the order-preserving (delta, i, j)
// keys of the exact lexicographic argmin.
#pragma once

#include "common.cuh"

namespace dpso {
namespace tiled {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// One row of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory by the bulk-copy engine; completion is
// counted in bytes on the mbarrier at `mbar`.
__device__ __forceinline__ void bulk_row(unsigned dst, const void* src, unsigned bytes,
                                         unsigned mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_init(unsigned mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Arms the barrier for `bytes` of copies (one arrival: the calling thread).
__device__ __forceinline__ void mbar_expect(unsigned mbar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes)
                 : "memory");
}

// Waits for the phase of parity `phase` to complete, at most ~2 s of clock.
// Returns false when it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned phase) {
    unsigned done = 0;
    const long long t0 = clock64();
    while (!done) {
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
            "selp.u32 %0, 1, 0, p; }\n"
            : "=r"(done) : "r"(mbar), "r"(phase) : "memory");
        if (!done && clock64() - t0 > (1ll << 32)) return false;
    }
    return true;
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

}  // namespace tiled
}  // namespace dpso
