// Column reductions over DoF-major [rows][k] arrays and a grow-only device
// workspace.  Reductions are two-stage with a fixed order (per-block partials,
// then one finalize block), so results do not depend on scheduling.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "afem_internal.h"

namespace afem {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 152 * 4;   // 4 blocks per SM on a 152-SM GB300

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

inline unsigned grid_for(int64_t n, int block = 256, int64_t cap = 152 * 16) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return unsigned(g);
}

}  // namespace afem
