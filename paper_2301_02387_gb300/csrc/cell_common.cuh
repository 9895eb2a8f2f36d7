// Device helpers shared by the cell kernels: real/complex value ops and the
// constrained gather / scatter of one cell node (Sec. 3.1, bridged functions).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "afem_internal.h"

namespace afem {

struct BasisParams {
    double xi[kMaxP1];
    double w[kMaxP1];
    double K[kMaxP1 * kMaxP1];
    double S[kMaxP1 * kMaxP1];   // skew part of int L_i L_j' (velocity gauge)
};

struct CellArgs {
    const int32_t* cell_node;   // [ncell][(p+1)^3]: >= 0 master, < 0 -(hanging)-1
    const double4* geom;        // (corner, h)
    const int32_t* hp;          // hanging rows (CSR)
    const int32_t* hm;
    const double* hw;
    const double* v_master;
    const double* v_hang;
    const double* f_master;     // [N][3] nuclear force (with_pot == 3)
    const double* f_hang;       // [nh][3]
    int64_t n_interior;
    BasisParams B;
    double E[3];
    double c_kin;               // factor of the stiffness term
    int with_pot;               // pointwise term: 1 F[V + E.r], 2 F[E.r], 3 F[E.force]
    int masked;                 // treat surface masters (>= n_interior) as zero, in and out
    int vg;                     // velocity gauge: the term -i A . G with A in Avec (complex data only)
    double Avec[3];
};

CellArgs make_cell_args(const afem_mesh* m);

template <typename T> __device__ __forceinline__ T vzero();
template <> __device__ __forceinline__ double vzero<double>() { return 0.0; }
template <> __device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float vzero<float>() { return 0.0f; }
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.0f, 0.0f); }

__device__ __forceinline__ void vfma(double& acc, double s, double v) { acc = fma(s, v, acc); }
__device__ __forceinline__ void vfma(double2& acc, double s, double2 v) {
    acc.x = fma(s, v.x, acc.x);
    acc.y = fma(s, v.y, acc.y);
}
__device__ __forceinline__ void vfma(float& acc, float s, float v) { acc = fmaf(s, v, acc); }
__device__ __forceinline__ void vfma(float2& acc, float s, float2 v) {
    acc.x = fmaf(s, v.x, acc.x);
    acc.y = fmaf(s, v.y, acc.y);
}

__device__ __forceinline__ double vscale(double v, double s) { return v * s; }
__device__ __forceinline__ double2 vscale(double2 v, double s) { return make_double2(v.x * s, v.y * s); }
__device__ __forceinline__ float vscale(float v, double s) { return v * float(s); }
__device__ __forceinline__ float2 vscale(float2 v, double s) {
    return make_float2(v.x * float(s), v.y * float(s));
}

__device__ __forceinline__ void vatomic_add(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void vatomic_add(double2* p, double2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}
__device__ __forceinline__ void vatomic_add(float* p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void vatomic_add(float2* p, float2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

// Value of vector component v at cell node `idx` (master or hanging).
template <typename T>
__device__ __forceinline__ T gather_value(const CellArgs& a, int idx, const T* __restrict__ x, int nv,
                                          int v) {
    T val = vzero<T>();
    if (idx >= 0) {
        if (!(a.masked && idx >= a.n_interior)) val = x[int64_t(idx) * nv + v];
    } else {
        const int hh = -idx - 1;
        const int e1 = a.hp[hh + 1];
        for (int e = a.hp[hh]; e < e1; ++e) {
            const int m = a.hm[e];
            if (a.masked && m >= a.n_interior) continue;
            vfma(val, a.hw[e], x[int64_t(m) * nv + v]);
        }
    }
    return val;
}

// Scatter-add r into the masters that cell node `idx` depends on (C^T).
template <typename T>
__device__ __forceinline__ void scatter_value(const CellArgs& a, int idx, T* __restrict__ y, int nv,
                                              int v, T r) {
    if (idx >= 0) {
        if (!(a.masked && idx >= a.n_interior)) vatomic_add(&y[int64_t(idx) * nv + v], r);
    } else {
        const int hh = -idx - 1;
        const int e1 = a.hp[hh + 1];
        for (int e = a.hp[hh]; e < e1; ++e) {
            const int m = a.hm[e];
            if (a.masked && m >= a.n_interior) continue;
            vatomic_add(&y[int64_t(m) * nv + v], vscale(r, a.hw[e]));
        }
    }
}

}  // namespace afem
