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
