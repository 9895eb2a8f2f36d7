// Shared-memory barriers (mbarrier) and the bulk global -> shared copy of the
// tensor memory accelerator (cp.async.bulk), in inline PTX.
//
// A bulk copy moves a contiguous, 16-byte aligned block whose size is a
// multiple of 16 bytes into shared memory without passing through registers;
// its completion is counted in bytes on an mbarrier (expect_tx / complete_tx).
// The tensor-core MMAs (tcgen05.cuh) signal their completion on the same kind
// of barrier.  Every wait here is bounded: it returns false after max_polls
// unsuccessful polls, and the caller records the failure instead of hanging.
#pragma once
#include <cstdint>

namespace afem {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes an initialised barrier visible to the asynchronous proxy (the bulk
// copy engine) before a copy that completes on it is issued.
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Bounded wait for the completion of the barrier phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int max_polls) {
    uint32_t done = 0;
    for (int i = 0; i < max_polls && !done; ++i) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
    }
    return done != 0;
}

// One thread: arrive on the barrier and announce `bytes` of bulk-copy data
// that will complete on it.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// One thread: bulk copy of `bytes` (multiple of 16) from global src to shared
// dst (both 16-byte aligned), completing on bar.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

}  // namespace tc
}  // namespace afem
