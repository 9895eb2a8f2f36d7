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

// Exterior complex scaling of the kinetic energy (afem_mesh_set_ecs): per cell
// the axes along which it lies outside the inner box, the factors e^{i m theta}
// (m = -2..3) of its stiffness terms J / eta_d^2, and per master
// rho = M_L / M_theta, which turns the assembled scaled stiffness into
// M_L M_theta^-1 A_theta before the common M_L^-1.
struct EcsArgs {
    const uint8_t* flags;   // [ncell] bit d: scaled along axis d
    const double2* rho;     // [N]
    double2 e[6];           // e^{i m theta}, m = -2..3
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

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
    // G pass: the mean fields at the hanging points, [nh][n^2] rows (C U,
    // formed once per propagation); null: interpolated from the masters here
    const double2* u_hang;
    EcsArgs ecs;                // complex scaling (the ECS kernel variants only)
};

// The stiffness factors J / eta_d^2 of cell `cell` (k scaled axes:
// J = e^{i k theta}, eta_d = e^{i theta} on a scaled axis).
__device__ __forceinline__ void ecs_factors(const EcsArgs& e, int64_t cell, double2& sx, double2& sy, double2& sz) {
    const int f = e.flags[cell];
    const int k = (f & 1) + ((f >> 1) & 1) + ((f >> 2) & 1);
    sx = e.e[k - 2 * (f & 1) + 2];
    sy = e.e[k - 2 * ((f >> 1) & 1) + 2];
    sz = e.e[k - 2 * ((f >> 2) & 1) + 2];
}

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
        // a hanging point's constraint row, four entries per round: the index
        // loads, then the value loads, issued together (masked rows not read)
        const int hh = -idx - 1;
        const int e1 = a.hp[hh + 1];
        int e = a.hp[hh];
        for (; e + 4 <= e1; e += 4) {
            const int m0 = a.hm[e], m1 = a.hm[e + 1], m2 = a.hm[e + 2], m3 = a.hm[e + 3];
            const T x0 = (a.masked && m0 >= a.n_interior) ? vzero<T>() : x[int64_t(m0) * nv + v];
            const T x1 = (a.masked && m1 >= a.n_interior) ? vzero<T>() : x[int64_t(m1) * nv + v];
            const T x2 = (a.masked && m2 >= a.n_interior) ? vzero<T>() : x[int64_t(m2) * nv + v];
            const T x3 = (a.masked && m3 >= a.n_interior) ? vzero<T>() : x[int64_t(m3) * nv + v];
            vfma(val, a.hw[e], x0);
            vfma(val, a.hw[e + 1], x1);
            vfma(val, a.hw[e + 2], x2);
            vfma(val, a.hw[e + 3], x3);
        }
        for (; e < e1; ++e) {
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
        // four entries per round: index and weight loads before the round's atomics
        const int hh = -idx - 1;
        const int e1 = a.hp[hh + 1];
        int e = a.hp[hh];
        for (; e + 4 <= e1; e += 4) {
            int mm[4];
            double ww[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                mm[u] = a.hm[e + u];
                ww[u] = a.hw[e + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (!(a.masked && mm[u] >= a.n_interior)) vatomic_add(&y[int64_t(mm[u]) * nv + v], vscale(r, ww[u]));
        }
        for (; e < e1; ++e) {
            const int m = a.hm[e];
            if (a.masked && m >= a.n_interior) continue;
            vatomic_add(&y[int64_t(m) * nv + v], vscale(r, a.hw[e]));
        }
    }
}

// Scatter of a scaled cell's output: the kinetic part rk enters master m as
// rho_m rk, the pointwise part rp unchanged (both through C^T).
__device__ __forceinline__ void scatter_ecs(const CellArgs& a, int idx, double2* __restrict__ y, int nv, int v,
                                            double2 rk, double2 rp) {
    if (idx >= 0) {
        if (!(a.masked && idx >= a.n_interior)) {
            const double2 t = cmul(a.ecs.rho[idx], rk);
            vatomic_add(&y[int64_t(idx) * nv + v], make_double2(t.x + rp.x, t.y + rp.y));
        }
    } else {
        const int hh = -idx - 1;
        const int e1 = a.hp[hh + 1];
        for (int e = a.hp[hh]; e < e1; ++e) {
            const int m = a.hm[e];
            if (a.masked && m >= a.n_interior) continue;
            const double2 t = cmul(a.ecs.rho[m], rk);
            vatomic_add(&y[int64_t(m) * nv + v], vscale(make_double2(t.x + rp.x, t.y + rp.y), a.hw[e]));
        }
    }
}

}  // namespace afem
