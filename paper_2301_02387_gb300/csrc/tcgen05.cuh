// Fifth-generation tensor cores (tcgen05, sm_100-family incl. sm_103a) in
// inline PTX: tensor-memory allocation, the single-thread MMA issued from
// shared-memory operand descriptors, its completion through an mbarrier, and
// the warp-wide loads of the FP32 accumulators from tensor memory.
//
// Only the forms this library uses are wrapped: kind::tf32, cta_group::1,
// M = 128, operands K-major without swizzling.  An operand tile of R rows
// (M or N) and KT columns (the contraction index) is stored as 8-row x
// 16-byte core matrices, 128 contiguous bytes each (row r of a core matrix at
// byte 16 r); core matrix (row group g, column group c) sits at byte
// g * (KT / 4) * 128 + c * 128.  The descriptor of the K-slice that starts at
// column 8 s then has start = tile + 256 s, leading-dimension byte offset
// 128 (the next core matrix along K) and stride byte offset (KT / 4) * 128
// (the next row group).
//
// The accumulator D (M = 128 rows x N FP32 columns) occupies tensor-memory
// lanes 0..127 (row = lane) and N consecutive columns; warp w of a warpgroup
// reads lanes 32 (w % 4) .. 32 (w % 4) + 31.
#pragma once
#include <cstdint>

#include "mbarrier.cuh"

namespace afem {
namespace tc {

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset, stride byte offset (each in 16-byte units), the fixed field value 1
// at bit 46, base offset 0, no swizzling.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(lbo_bytes >> 4) << 16) |
           (static_cast<uint64_t>(sbo_bytes >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D in FP32 (bits 4-5 = 1), A and B
// TF32 (bits 7-9 and 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at
// bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

// Warp-wide: allocate ncols (a power of two, 32..512) tensor-memory columns;
// the base address is written to *dst (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Warp-wide (the allocating warp): free the columns.
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// One thread: D (tensor memory) = A B^T (+ D when accumulate).
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate ? 1u : 0u)
        : "memory");
}

// One thread: the mbarrier receives one arrival when every MMA this thread
// issued before has completed.
__device__ __forceinline__ void commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Generic-proxy writes to shared memory made visible to the tensor cores.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Warp-wide: 16 consecutive FP32 columns of this thread's lane.
__device__ __forceinline__ void ld_x16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// TF32 part of a float (10 explicit significand bits, rounded to nearest on
// the magnitude): the tensor cores read only those bits of an operand, so the
// part is exact there.  Finite inputs below 2^127 in magnitude.
__device__ __forceinline__ float tf32_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Byte offset of element (row, k) in an operand tile with KT columns laid out
// as described at the top of this file.
__host__ __device__ constexpr uint32_t tile_offset(int row, int k, int KT) {
    return static_cast<uint32_t>((row >> 3) * (KT / 4) * 128 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

}  // namespace tc
}  // namespace afem
