// Arithmetic peaks of the device (library instrumentation with no counterpart
// in the paper): FP64 and FP32 fused multiply-add throughput, the
// denominators of the rooflines of the FP64-bound kernels.
//
// Every thread runs 8 independent multiply-add chains x <- x a + b; the
// blocks fill the device (4 blocks of 256 threads per SM).  The chains'
// sum is compared with a value it cannot take, so the compiler keeps them.
#include <cmath>

#include "afem_internal.h"
#include "vec_common.cuh"

namespace afem {

constexpr int kPeakChains = 8;
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(int64_t iters, T a, T b, T* __restrict__ sink) {
    T x[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) x[k] = fma(x[k], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s += x[k];
    if (s == T(-1.25e30)) *sink = s;
}

template <typename T>
static int time_fma(int64_t iters, unsigned grid, T* sink, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
    AFEM_CUDA_TRY(cudaEventRecord(e0, s));
    AFEM_LAUNCH((fma_peak_kernel<T>), grid, kPeakThreads, 0, s, iters, T(0.999999), T(1e-6), sink);
    AFEM_CUDA_TRY(cudaGetLastError());
    AFEM_CUDA_TRY(cudaEventRecord(e1, s));
    AFEM_CUDA_TRY(cudaEventSynchronize(e1));
    AFEM_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
    return AFEM_OK;
}

template <typename T>
static int fma_peak(double target_ms, double* flops, cudaStream_t s) {
    const unsigned grid = unsigned(4 * device_sms());
    T* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(T));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int rc = e == cudaSuccess ? AFEM_OK : cuda_error(e, "afem_fma_peak");
    float ms = 0.f;
    int64_t iters = 1024;
    // calibrate: grow the loop until one launch takes at least a tenth of the target
    while (rc == AFEM_OK) {
        rc = time_fma<T>(iters, grid, sink, s, e0, e1, &ms);
        if (rc || ms >= 0.1 * target_ms || iters >= (int64_t(1) << 40)) break;
        iters *= 4;
    }
    if (rc == AFEM_OK) {
        if (ms > 0.f) iters = int64_t(double(iters) * target_ms / ms) + 1;
        double best = 0.0;
        for (int r = 0; r < 3 && rc == AFEM_OK; ++r) {
            rc = time_fma<T>(iters, grid, sink, s, e0, e1, &ms);
            if (rc == AFEM_OK && ms > 0.f) {
                const double f = 2.0 * kPeakChains * double(iters) * grid * kPeakThreads / (1e-3 * ms);
                if (f > best) best = f;
            }
        }
        *flops = best;
    }
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (sink) cudaFree(sink);
    return rc;
}

}  // namespace afem

using namespace afem;

extern "C" int afem_fma_peak(int kind, double target_ms, double* flops_per_s, void* stream) {
    if (!flops_per_s) return set_error(AFEM_EINVAL, "afem_fma_peak: null output");
    if (!(target_ms > 0.0) || target_ms > 1e4) return set_error(AFEM_EINVAL, "afem_fma_peak: target_ms out of range");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (kind == AFEM_PEAK_FP64) return fma_peak<double>(target_ms, flops_per_s, s);
    if (kind == AFEM_PEAK_FP32) return fma_peak<float>(target_ms, flops_per_s, s);
    return set_error(AFEM_EINVAL, "afem_fma_peak: kind must be AFEM_PEAK_FP64 or AFEM_PEAK_FP32");
}
