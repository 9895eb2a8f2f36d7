// Column reductions over DoF-major [rows][k] arrays and a grow-only device
// workspace.  Reductions are two-stage with a fixed order (per-block partials,
// then one finalize block), so results do not depend on scheduling.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "afem_internal.h"

namespace afem {

constexpr int kRedThreads = 256;

// Conversions between binary32 and binary64 written from the IEEE-754 bit
// layout, so that they run on the integer pipe: on GB300 the hardware
// conversions issue on the FP64 pipe, which is the bound of the Gram-Schmidt
// passes.
// binary32 -> binary64: exact for zeros, normal numbers, infinities and NaNs;
// binary32 subnormals (below 1.18e-38) become zeros of the same sign.
__device__ __forceinline__ double widen_f32(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    uint64_t bits = uint64_t(u & 0x80000000u) << 32;
    if (e != 0u) {
        const uint64_t E = e == 0xFFu ? 0x7FFull : uint64_t(e) + 896ull;   // rebias 127 -> 1023
        bits |= (E << 52) | (uint64_t(u & 0x7FFFFFu) << 29);
    }
    return __longlong_as_double(static_cast<long long>(bits));
}
// binary64 -> binary32, rounded to nearest with ties to even on the 29
// dropped significand bits (a carry out of the significand raises the
// exponent, as it should); results below the binary32 normal range become
// zeros of the same sign, results above it infinities; NaNs stay NaNs.
__device__ __forceinline__ float narrow_f64(double d) {
    const uint64_t b = static_cast<uint64_t>(__double_as_longlong(d));
    const uint32_t sign = uint32_t(b >> 32) & 0x80000000u;
    const int e = int((b >> 52) & 0x7FFull);
    const uint64_t m = b & 0xFFFFFFFFFFFFFull;
    if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));
    const int ef = e - 896;   // binary32 biased exponent
    if (ef <= 0) return __uint_as_float(sign);
    if (ef >= 255) return __uint_as_float(sign | 0x7F800000u);
    const uint32_t keep = uint32_t(m >> 29);
    const uint32_t rest = uint32_t(m & 0x1FFFFFFFull);
    uint32_t r = (uint32_t(ef) << 23) | keep;
    if (rest > 0x10000000u || (rest == 0x10000000u && (keep & 1u))) r += 1u;
    return __uint_as_float(sign | r);
}
// narrow_f64(d * 2^k) with k added to the exponent field before rounding (no
// floating-point multiply); zeros, infinities and NaNs as in narrow_f64.
__device__ __forceinline__ float narrow_f64_scaled(double d, int k) {
    const uint64_t b = static_cast<uint64_t>(__double_as_longlong(d));
    const uint32_t sign = uint32_t(b >> 32) & 0x80000000u;
    const int e = int((b >> 52) & 0x7FFull);
    const uint64_t m = b & 0xFFFFFFFFFFFFFull;
    if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));
    if (e == 0) return __uint_as_float(sign);
    const int ef = e - 896 + k;
    if (ef <= 0) return __uint_as_float(sign);
    if (ef >= 255) return __uint_as_float(sign | 0x7F800000u);
    const uint32_t keep = uint32_t(m >> 29);
    const uint32_t rest = uint32_t(m & 0x1FFFFFFFull);
    uint32_t r = (uint32_t(ef) << 23) | keep;
    if (rest > 0x10000000u || (rest == 0x10000000u && (keep & 1u))) r += 1u;
    return __uint_as_float(sign | r);
}
// widen_f32(f) * 2^k through the exponent field: exact unless the result
// leaves the binary64 normal range (zero or infinity then).
__device__ __forceinline__ double widen_f32_scaled(float f, int k) {
    const uint32_t u = __float_as_uint(f);
    const int e = int((u >> 23) & 0xFFu);
    uint64_t bits = uint64_t(u & 0x80000000u) << 32;
    if (e == 0xFF) {
        bits |= (0x7FFull << 52) | (uint64_t(u & 0x7FFFFFu) << 29);
    } else if (e != 0) {
        const int E = e + 896 + k;
        if (E >= 0x7FF) bits |= 0x7FFull << 52;
        else if (E > 0) bits |= (uint64_t(E) << 52) | (uint64_t(u & 0x7FFFFFu) << 29);
    }
    return __longlong_as_double(static_cast<long long>(bits));
}
// Streaming multiprocessors of the current device, looked up once per device.
inline int device_sms() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c < 1) return 1;
    cache[dev].store(c, std::memory_order_relaxed);
    return c;
}
// Blocks of the reductions with one partial row per block: 4 per SM, at most
// kRedBlocksMax (the size of the partial-row buffers).
constexpr int kRedBlocksMax = 1024;
inline int red_blocks() {
    const int g = 4 * device_sms();
    return g < kRedBlocksMax ? g : kRedBlocksMax;
}

// Threads (r, c) = (t / k, t % k) for t < k * (256 / k); the rest idle.
struct ColLayout {
    int k, R, used;
    __device__ __forceinline__ ColLayout(int k_) : k(k_), R(kRedThreads / k_), used(k_ * (kRedThreads / k_)) {}
};

// Sum s[c + k*r] over r into out[c] for c < k (fixed order).  s has kRedThreads entries.
__device__ __forceinline__ void reduce_columns(double* s, int k, int R, double* out_block) {
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double acc = 0.0;
        for (int r = 0; r < R; ++r) acc += s[c + k * r];
        out_block[c] = acc;
    }
}

// Last-block reduction: every block has written its row partial[blockIdx][0..kout)
// (kout <= blockDim).  All threads of all blocks call this; it returns true only
// in the block that finishes last, where s_sum[0..kout) then holds the column
// sums over all blocks.  The sums are formed in a fixed order (thread j of a
// column adds blocks j, j+J, ..., then a fixed tree), independent of which block
// finishes last.  *counter must be 0 before the launch; the last block resets it.
__device__ __forceinline__ bool last_block_sum(const double* partial, int kout, unsigned* counter,
                                               double* s_sum /* >= blockDim doubles */) {
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    const int J = blockDim.x / kout;
    const int t = threadIdx.x;
    double acc = 0.0;
    if (t < J * kout) {
        const int c = t % kout, j = t / kout;
        for (unsigned b = j; b < gridDim.x; b += J) acc += __ldcg(partial + size_t(b) * kout + c);
    }
    s_sum[t] = acc;
    __syncthreads();
    if (t < kout) {
        double s = 0.0;
        for (int j = 0; j < J; ++j) s += s_sum[t + j * kout];
        acc = s;
    }
    __syncthreads();
    if (t < kout) s_sum[t] = acc;
    __syncthreads();
    if (t == 0) *counter = 0u;
    return true;
}

// Sum partial[b][c] over blocks b into out[c] (one block, fixed order).
__global__ void finalize_columns_kernel(const double* __restrict__ partial, int nblk, int k,
                                        double* __restrict__ out);

// Carve 256-byte-aligned sub-buffers out of one allocation.  A Carver built
// with a null base only measures: run the same sequence of take() calls once
// to size the allocation, then again on the real base, so the two can never
// disagree.
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <typename T>
    T* take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
    size_t size() const { return off + 256; }
};

// Blocks for n items at `block` threads, at most per_sm blocks per SM.
inline unsigned grid_for(int64_t n, int block = 256, int per_sm = 16) {
    int64_t g = (n + block - 1) / block;
    const int64_t cap = int64_t(per_sm) * device_sms();
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return unsigned(g);
}

}  // namespace afem
