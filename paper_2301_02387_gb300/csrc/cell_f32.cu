// FP32 forms of the fused cell operators (precision form of the hot path).
//
// Same operators as the FP64 kernels (Sec. 3.1: GLL sum-factorised cell
// stiffness, pointwise potential, hanging-node gather/scatter; Eq.
// discretized_eom): the per-cell data and the arithmetic are in float /
// complex64, reading float copies of the mesh tables, so no FP64 instruction
// runs inside the cell loop.  Callers keep the accuracy-critical parts in FP64
// (Krylov Gram-Schmidt, residuals of the Poisson refinement).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "afem_internal.h"
#include "cell_common.cuh"
#include "mbarrier.cuh"
#include "vec_common.cuh"

namespace afem {

// Entries of a hanging point's constraint row loaded together by the
// four-lane gather (1: one at a time).
#ifndef AFEM_HANG_UNROLL
#define AFEM_HANG_UNROLL 4
#endif

struct CellArgs32 {
    const int32_t* cell_node;
    const float4* geom;       // (corner, h)
    const int32_t* hp;
    const int32_t* hm;
    const float* hw;
    const float* v_master;
    const float* v_hang;
    const float* v_cell;      // [ncell][(p+1)^3] potential at the cell nodes
    // stiffness only (null: off): p.Ap of the conjugate-gradient sweep per column,
    // added in FP64 to slot (block % kPapSlots) of [kPapSlots][columns]
    double* pap_slots;
    int64_t ncell;
    int64_t n_interior;
    float xi[kMaxP1], w[kMaxP1], K[kMaxP1 * kMaxP1];
    float S[kMaxP1 * kMaxP1];   // skew part of int L_i L_j' (velocity gauge)
    float E[3];
    float Avec[3];              // vector potential (vg != 0)
    int masked;
    int vg;                     // velocity gauge: -i A . grad in the G pass (generic kernel only)
    // G pass: the mean fields at the hanging points, [nh][n^2] complex64 rows
    // (C U, formed once per propagation); null: interpolated from the masters
    const float2* u_hang;
    // complex scaling of the kinetic term (the ECS variant of the generic kernel)
    const uint8_t* ecs_flags;   // [ncell] bit d: scaled along axis d
    const float2* ecs_rho;      // [N] M_L / M_theta
    float2 ecs_e[6];            // e^{i m theta}, m = -2..3
};

__device__ __forceinline__ float2 cmul32(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

template <typename T>
__device__ __forceinline__ T gather32(const CellArgs32& a, int idx, const T* __restrict__ x, int nv, int v) {
    T val = vzero<T>();
    if (idx >= 0) {
        if (!(a.masked && idx >= a.n_interior)) val = x[int64_t(idx) * nv + v];
    } else {
        const int hh = -idx - 1;
        for (int e = a.hp[hh]; e < a.hp[hh + 1]; ++e) {
            const int m = a.hm[e];
            if (a.masked && m >= a.n_interior) continue;
            vfma(val, a.hw[e], x[int64_t(m) * nv + v]);
        }
    }
    return val;
}

__device__ __forceinline__ float2 fscale(float2 v, float s) { return make_float2(v.x * s, v.y * s); }
__device__ __forceinline__ float fscale(float v, float s) { return v * s; }

template <typename T>
__device__ __forceinline__ void scatter32(const CellArgs32& a, int idx, T* __restrict__ y, int nv, int v, T r) {
    if (idx >= 0) {
        if (!(a.masked && idx >= a.n_interior)) vatomic_add(&y[int64_t(idx) * nv + v], r);
    } else {
        const int hh = -idx - 1;
        for (int e = a.hp[hh]; e < a.hp[hh + 1]; ++e) {
            const int m = a.hm[e];
            if (a.masked && m >= a.n_interior) continue;
            vatomic_add(&y[int64_t(m) * nv + v], fscale(r, a.hw[e]));
        }
    }
}

// Scatter of a complex-scaled cell's output: the kinetic part rk enters master
// m as rho_m rk, the pointwise part rp unchanged (both through C^T).
__device__ __forceinline__ void scatter32_ecs(const CellArgs32& a, int idx, float2* __restrict__ y, int nv, int v,
                                              float2 rk, float2 rp) {
    if (idx >= 0) {
        if (!(a.masked && idx >= a.n_interior)) {
            const float2 t = cmul32(a.ecs_rho[idx], rk);
            vatomic_add(&y[int64_t(idx) * nv + v], make_float2(t.x + rp.x, t.y + rp.y));
        }
    } else {
        const int hh = -idx - 1;
        for (int e = a.hp[hh]; e < a.hp[hh + 1]; ++e) {
            const int m = a.hm[e];
            if (a.masked && m >= a.n_interior) continue;
            const float2 t = cmul32(a.ecs_rho[m], rk);
            vatomic_add(&y[int64_t(m) * nv + v], fscale(make_float2(t.x + rp.x, t.y + rp.y), a.hw[e]));
        }
    }
}

// y += A x for nv real columns (c_kin = 1), or the G-operator cell pass for
// complex columns: z_p = H1~ v_p + sum_q (C U_pq) o (C v_q) weighted (U may be null).
// ECS (complex columns, G): the kinetic term complex-scaled (afem_mesh_set_ecs).
template <int P, typename T, bool G, bool VG = false, bool ECS = false>
__global__ void __launch_bounds__(256) cell32_kernel(CellArgs32 a, const T* __restrict__ x,
                                                     const float2* __restrict__ U, T* __restrict__ y, int nv) {
    constexpr int P1 = P + 1;
    constexpr int NN = P1 * P1 * P1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s_u = reinterpret_cast<T*>(smem_raw);
    float2* s_U = reinterpret_cast<float2*>(s_u + NN * nv);
    __shared__ int s_idx[NN];
    __shared__ float s_pot[NN];
    __shared__ float s_wq[NN];
    __shared__ float s_K[P1 * P1];
    __shared__ float s_w[P1];
    const int64_t cell = blockIdx.x;
    const int tid = threadIdx.x, bs = blockDim.x;
    const float4 g = a.geom[cell];
    for (int i = tid; i < NN; i += bs) s_idx[i] = a.cell_node[cell * NN + i];
    if (tid < P1 * P1) s_K[tid] = a.K[tid];
    if (tid < P1) s_w[tid] = a.w[tid];
    __syncthreads();
    for (int it = tid; it < NN * nv; it += bs) {
        const int i = it / nv, q = it - i * nv;
        s_u[it] = gather32<T>(a, s_idx[i], x, nv, q);
    }
    const int nn2 = nv * nv;
    if (G) {
        if (U) {
            CellArgs32 au = a;
            au.masked = 0;
            for (int it = tid; it < NN * nn2; it += bs) {
                const int i = it / nn2, pq = it - i * nn2;
                const int idx = s_idx[i];
                s_U[it] = (idx < 0 && a.u_hang) ? a.u_hang[int64_t(-idx - 1) * nn2 + pq]
                                                : gather32<float2>(au, idx, U, nn2, pq);
            }
        }
        const float h3 = g.w * g.w * g.w;
        for (int i = tid; i < NN; i += bs) {
            const int ia = i % P1, ib = (i / P1) % P1, ic = i / (P1 * P1);
            const int idx = s_idx[i];
            const float V = idx >= 0 ? a.v_master[idx] : a.v_hang[-idx - 1];
            const float px = g.x + g.w * a.xi[ia], py = g.y + g.w * a.xi[ib], pz = g.z + g.w * a.xi[ic];
            const float wq = h3 * s_w[ia] * s_w[ib] * s_w[ic];
            s_wq[i] = wq;
            s_pot[i] = wq * (V + a.E[0] * px + a.E[1] * py + a.E[2] * pz);
        }
    }
    __syncthreads();
    const float ck = (G ? 0.5f : 1.0f) * g.w;
    for (int it = tid; it < NN * nv; it += bs) {
        const int i = it / nv, p = it - i * nv;
        const int ia = i % P1, ib = (i / P1) % P1, ic = i / (P1 * P1);
        T ax = vzero<T>(), ay = vzero<T>(), az = vzero<T>();
#pragma unroll
        for (int m = 0; m < P1; ++m) {
            vfma(ax, s_K[ia * P1 + m], s_u[(m + P1 * (ib + P1 * ic)) * nv + p]);
            vfma(ay, s_K[ib * P1 + m], s_u[(ia + P1 * (m + P1 * ic)) * nv + p]);
            vfma(az, s_K[ic * P1 + m], s_u[(ia + P1 * (ib + P1 * m)) * nv + p]);
        }
        T r = vzero<T>();
        float2 rk = make_float2(0.f, 0.f);
        if constexpr (ECS && G && sizeof(T) == sizeof(float2)) {
            // the cell's stiffness factors J / eta_d^2 (k scaled axes: J = e^{i k theta})
            const int f = a.ecs_flags[cell];
            const int k = (f & 1) + ((f >> 1) & 1) + ((f >> 2) & 1);
            const float cx = ck * s_w[ib] * s_w[ic], cy = ck * s_w[ia] * s_w[ic], cz = ck * s_w[ia] * s_w[ib];
            const float2 tx = cmul32(a.ecs_e[k - 2 * (f & 1) + 2], make_float2(cx * ax.x, cx * ax.y));
            const float2 ty = cmul32(a.ecs_e[k - 2 * ((f >> 1) & 1) + 2], make_float2(cy * ay.x, cy * ay.y));
            const float2 tz = cmul32(a.ecs_e[k - 2 * ((f >> 2) & 1) + 2], make_float2(cz * az.x, cz * az.y));
            rk = make_float2(tx.x + ty.x + tz.x, tx.y + ty.y + tz.y);
        } else {
            vfma(r, ck * s_w[ib] * s_w[ic], ax);
            vfma(r, ck * s_w[ia] * s_w[ic], ay);
            vfma(r, ck * s_w[ia] * s_w[ib], az);
        }
        if constexpr (G) {
            vfma(r, s_pot[i], s_u[it]);
            if constexpr (VG && sizeof(T) == sizeof(float2)) {
                {   // -i h^2 (A_x w_b w_c (S u)_x + A_y w_a w_c (S u)_y + A_z w_a w_b (S u)_z)
                    float2 gx = make_float2(0.f, 0.f), gy = gx, gz = gx;
#pragma unroll
                    for (int m = 0; m < P1; ++m) {
                        vfma(gx, a.S[ia * P1 + m], s_u[(m + P1 * (ib + P1 * ic)) * nv + p]);
                        vfma(gy, a.S[ib * P1 + m], s_u[(ia + P1 * (m + P1 * ic)) * nv + p]);
                        vfma(gz, a.S[ic * P1 + m], s_u[(ia + P1 * (ib + P1 * m)) * nv + p]);
                    }
                    const float h2 = g.w * g.w;
                    float2 t = make_float2(0.f, 0.f);
                    vfma(t, h2 * a.Avec[0] * s_w[ib] * s_w[ic], gx);
                    vfma(t, h2 * a.Avec[1] * s_w[ia] * s_w[ic], gy);
                    vfma(t, h2 * a.Avec[2] * s_w[ia] * s_w[ib], gz);
                    r.x += t.y;
                    r.y -= t.x;
                }
            }
            if (U) {
                float2 mf = make_float2(0.0f, 0.0f);
                const float2* Ui = s_U + i * nn2 + p * nv;
                const T* ui = s_u + i * nv;
                for (int q = 0; q < nv; ++q) {
                    mf.x = fmaf(Ui[q].x, ui[q].x, fmaf(-Ui[q].y, ui[q].y, mf.x));
                    mf.y = fmaf(Ui[q].x, ui[q].y, fmaf(Ui[q].y, ui[q].x, mf.y));
                }
                vfma(r, s_wq[i], mf);
            }
        }
        if constexpr (ECS && G && sizeof(T) == sizeof(float2)) scatter32_ecs(a, s_idx[i], y, nv, p, rk, r);
        else scatter32<T>(a, s_idx[i], y, nv, p, r);
    }
}

// Four-lane form of the same cell pass: every node's columns are handled as
// float4 quads (4 real columns, or 2 complex orbitals), so gathers are 16-byte
// loads and the scatter is one vector atomic per quad instead of four.  The
// stiffness and potential terms act on every float lane alike; the mean-field
// term of G mixes the orbitals of a node (complex products per orbital pair).
__device__ __forceinline__ void f4fma(float4& acc, float s, const float4 v) {
    acc.x = fmaf(s, v.x, acc.x);
    acc.y = fmaf(s, v.y, acc.y);
    acc.z = fmaf(s, v.z, acc.z);
    acc.w = fmaf(s, v.w, acc.w);
}

__device__ __forceinline__ float4 gather32v(const CellArgs32& a, int idx, const float4* __restrict__ x, int L4,
                                            int q) {
    float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
    if (idx >= 0) {
        if (!(a.masked && idx >= a.n_interior)) val = x[int64_t(idx) * L4 + q];
    } else {
        // a hanging point: its constraint row (17 masters on average at degree 4)
        // walked AFEM_HANG_UNROLL entries at a time, the index loads and then the
        // row loads issued together, so the walk waits on a fraction of the
        // dependent index -> value latencies; masked masters add zero
        const int hh = -idx - 1;
        const int e1 = a.hp[hh + 1];
        int e = a.hp[hh];
#if AFEM_HANG_UNROLL >= 4
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (; e + 4 <= e1; e += 4) {
            const int m0 = a.hm[e], m1 = a.hm[e + 1], m2 = a.hm[e + 2], m3 = a.hm[e + 3];
            // masked (surface) masters are not read: their rows may hold anything
            const float4 x0 = (a.masked && m0 >= a.n_interior) ? z4 : x[int64_t(m0) * L4 + q];
            const float4 x1 = (a.masked && m1 >= a.n_interior) ? z4 : x[int64_t(m1) * L4 + q];
            const float4 x2 = (a.masked && m2 >= a.n_interior) ? z4 : x[int64_t(m2) * L4 + q];
            const float4 x3 = (a.masked && m3 >= a.n_interior) ? z4 : x[int64_t(m3) * L4 + q];
            f4fma(val, a.hw[e], x0);
            f4fma(val, a.hw[e + 1], x1);
            f4fma(val, a.hw[e + 2], x2);
            f4fma(val, a.hw[e + 3], x3);
        }
#elif AFEM_HANG_UNROLL >= 2
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (; e + 2 <= e1; e += 2) {
            const int m0 = a.hm[e], m1 = a.hm[e + 1];
            const float4 x0 = (a.masked && m0 >= a.n_interior) ? z4 : x[int64_t(m0) * L4 + q];
            const float4 x1 = (a.masked && m1 >= a.n_interior) ? z4 : x[int64_t(m1) * L4 + q];
            f4fma(val, a.hw[e], x0);
            f4fma(val, a.hw[e + 1], x1);
        }
#endif
        for (; e < e1; ++e) {
            const int m = a.hm[e];
            if (a.masked && m >= a.n_interior) continue;
            f4fma(val, a.hw[e], x[int64_t(m) * L4 + q]);
        }
    }
    return val;
}

__device__ __forceinline__ void scatter32v(const CellArgs32& a, int idx, float4* __restrict__ y, int L4, int q,
                                           float4 r) {
    if (idx >= 0) {
        if (!(a.masked && idx >= a.n_interior)) atomicAdd(&y[int64_t(idx) * L4 + q], r);
    } else {
        // the constraint row four entries per round: its index and weight loads
        // issued before the round's atomics (which the loads may not pass)
        const int hh = -idx - 1;
        const int e1 = a.hp[hh + 1];
        int e = a.hp[hh];
        for (; e + 4 <= e1; e += 4) {
            int mm[4];
            float ww[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                mm[u] = a.hm[e + u];
                ww[u] = a.hw[e + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (!(a.masked && mm[u] >= a.n_interior))
                    atomicAdd(&y[int64_t(mm[u]) * L4 + q],
                              make_float4(ww[u] * r.x, ww[u] * r.y, ww[u] * r.z, ww[u] * r.w));
        }
        for (; e < e1; ++e) {
            const int m = a.hm[e];
            if (a.masked && m >= a.n_interior) continue;
            const float w = a.hw[e];
            atomicAdd(&y[int64_t(m) * L4 + q], make_float4(w * r.x, w * r.y, w * r.z, w * r.w));
        }
    }
}

// 16-byte global -> shared copy that does not pass through registers
// (cp.async): a thread issues all of its copies back to back and waits once,
// so the gather of a cell's node rows keeps several loads in flight per
// thread.  Both addresses are 16-byte aligned (float4 rows).
__device__ __forceinline__ void cp_async16(float4* smem_dst, const float4* gmem_src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Slots of the fused p.Ap sums (spread over slots to keep the FP64 atomics of
// the cell blocks off a single address per column).
constexpr int kPapSlots = 64;

// Compile-time quad counts of the four-lane pass (others run with L4C = 0).
__host__ __device__ constexpr int quads_c32(int L4) { return (L4 >= 1 && L4 <= 4) ? L4 : 0; }

// Cells per work item of the four-lane pass: as many cells as fill 256 threads
// with one (node, quad) item each, so that small cells (p <= 3, few quads) do
// not leave most of a block idle; one cell where a cell's items already fill
// the block (and with a run-time quad count).
__host__ __device__ constexpr int cells_per_item32(int P, int L4C) {
    return L4C <= 0 ? 1
                    : ((P + 1) * (P + 1) * (P + 1) * L4C >= 256 ? 1 : 256 / ((P + 1) * (P + 1) * (P + 1) * L4C));
}

// Dynamic shared memory of one four-lane work item: the cell tiles of the
// input (and of the mean fields when with_u), then the cells' geometry,
// potential and quadrature weights and node indices.
__host__ __device__ constexpr size_t cell32v_smem(int P, int L4, int n, bool with_u) {
    return cells_per_item32(P, quads_c32(L4)) == 1
               ? size_t((P + 1) * (P + 1) * (P + 1)) * (size_t(L4) * 16 + (with_u ? size_t((n * n / 2) | 1) * 16 : 0))
               : size_t(cells_per_item32(P, quads_c32(L4))) *
                     (size_t((P + 1) * (P + 1) * (P + 1)) *
                          (size_t(L4) * 16 + (with_u ? size_t((n * n / 2) | 1) * 16 : 0) + 12) +
                      16);
}

// The four-lane cell pass of work item `item` -- cells item * CPB ..
// item * CPB + CPB - 1 that exist, CPB = cells_per_item32(P, L4C) -- by the
// whole block (any block size): the body of cell32v_kernel, also called per
// (instance, item) by the batched kernels.  Uses the block's shared memory; a
// caller looping over items synchronises the block between two calls.
// L4C > 0 fixes the quad count at compile time (no integer division per item);
// L4C = 0 takes it from L4rt.
template <int P, bool G, int L4C, bool PAP = false>
__device__ __forceinline__ void cell32v_body(const CellArgs32& a, int64_t item, const float4* __restrict__ x,
                                             const float2* __restrict__ U, float4* __restrict__ y, int L4rt,
                                             int n) {
    constexpr int P1 = P + 1;
    constexpr int NN = P1 * P1 * P1;
    constexpr int CPB = cells_per_item32(P, L4C);
    const int L4 = L4C > 0 ? L4C : L4rt;
    const int64_t cell0 = item * CPB;
    const int nc = int(a.ncell - cell0 < CPB ? a.ncell - cell0 : CPB);
    // with the quad count fixed, the orbital count n = 2 L4 is too
    const int nn2 = (G && L4C > 0) ? 4 * L4C * L4C : n * n;
    // float4 pairs of a node's n^2 complex fields sit SU = (n^2/2) | 1 quads apart
    // in shared memory: an odd stride puts the rows that the 8 lanes of a quarter
    // warp read (4 nodes x 2 orbital pairs) on distinct banks
    const int SU = (nn2 / 2) | 1;
    // dynamic shared memory, laid out as cell32v_smem counts it: the tiles,
    // then (several cells per item) the per-cell arrays, which one-cell items
    // keep in static shared memory (constant addresses, no registers)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* s_u = reinterpret_cast<float4*>(smem_raw);            // [CPB][NN][L4]
    float4* s_U4 = s_u + CPB * NN * L4;                           // [CPB][NN][SU] (G with U)
    float4* s_g;                                                  // [CPB] cell corner, side
    float* s_pot;                                                 // [CPB][NN]
    float* s_wq;                                                  // [CPB][NN]
    int* s_idx;                                                   // [CPB][NN]
    if constexpr (CPB == 1) {
        __shared__ float4 st_g[1];
        __shared__ float st_pot[NN], st_wq[NN];
        __shared__ int st_idx[NN];
        s_g = st_g;
        s_pot = st_pot;
        s_wq = st_wq;
        s_idx = st_idx;
    } else {
        s_g = s_U4 + ((G && U) ? CPB * NN * SU : 0);
        s_pot = reinterpret_cast<float*>(s_g + CPB);
        s_wq = s_pot + CPB * NN;
        s_idx = reinterpret_cast<int*>(s_wq + CPB * NN);
    }
    __shared__ float s_K[P1 * P1];
    __shared__ float s_w[P1];
    const int tid = threadIdx.x, bs = blockDim.x;
    for (int j = tid; j < nc * NN; j += bs) s_idx[j] = a.cell_node[cell0 * NN + j];
    for (int c = tid; c < nc; c += bs) s_g[c] = a.geom[cell0 + c];
    if (tid < P1 * P1) s_K[tid] = a.K[tid];
    if (tid < P1) s_w[tid] = a.w[tid];
    __syncthreads();
    // j = cell slot * NN + node.  In the G pass the rows of masters are copied
    // asynchronously, hanging points (weighted sums) and masked surface masters
    // (zero) go through registers; the stiffness pass (fewer rows per thread,
    // and its p.Ap epilogue at the 32-register limit) loads all in registers
    for (int it = tid; it < nc * NN * L4; it += bs) {
        const int j = it / L4, q = it - j * L4;
        const int idx = s_idx[j];
        if (G && idx >= 0 && !(a.masked && idx >= a.n_interior)) cp_async16(s_u + it, x + int64_t(idx) * L4 + q);
        else s_u[it] = gather32v(a, idx, x, L4, q);
    }
    if (G) {
        if (U) {
            // the n^2 complex fields of a node as float4 pairs (n = 2 L4 is even)
            CellArgs32 au = a;
            au.masked = 0;
            const int h2 = nn2 / 2;
            const float4* U4 = reinterpret_cast<const float4*>(U);
            for (int it = tid; it < nc * NN * h2; it += bs) {
                const int j = it / h2, c = it - j * h2;
                const int idx = s_idx[j];
                if (idx >= 0) cp_async16(s_U4 + j * SU + c, U4 + int64_t(idx) * h2 + c);
                else if (a.u_hang)
                    cp_async16(s_U4 + j * SU + c, reinterpret_cast<const float4*>(a.u_hang) + int64_t(-idx - 1) * h2 + c);
                else s_U4[j * SU + c] = gather32v(au, idx, U4, h2, c);
            }
        }
        const float* vc = a.v_cell + cell0 * NN;
        for (int j = tid; j < nc * NN; j += bs) {
            const int cc = j / NN, i = j - cc * NN;
            const int ia = i % P1, ib = (i / P1) % P1, ic = i / (P1 * P1);
            const float4 g = s_g[cc];
            const float px = g.x + g.w * a.xi[ia], py = g.y + g.w * a.xi[ib], pz = g.z + g.w * a.xi[ic];
            const float wq = g.w * g.w * g.w * s_w[ia] * s_w[ib] * s_w[ic];
            s_wq[j] = wq;
            s_pot[j] = wq * (vc[j] + a.E[0] * px + a.E[1] * py + a.E[2] * pz);
        }
    }
    if constexpr (G) cp_async_wait_all();
    __syncthreads();
    float4 pap = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int it = tid; it < nc * NN * L4; it += bs) {
        const int j = it / L4, q = it - j * L4;
        const int cc = j / NN, i = j - cc * NN;
        const int ia = i % P1, ib = (i / P1) % P1, ic = i / (P1 * P1);
        const float4* u0 = s_u + cc * NN * L4 + q;   // this cell's tile, quad q
        float4 ax = make_float4(0.f, 0.f, 0.f, 0.f), ay = ax, az = ax;
#pragma unroll
        for (int m = 0; m < P1; ++m) {
            f4fma(ax, s_K[ia * P1 + m], u0[(m + P1 * (ib + P1 * ic)) * L4]);
            f4fma(ay, s_K[ib * P1 + m], u0[(ia + P1 * (m + P1 * ic)) * L4]);
            f4fma(az, s_K[ic * P1 + m], u0[(ia + P1 * (ib + P1 * m)) * L4]);
        }
        const float ck = (G ? 0.5f : 1.0f) * s_g[cc].w;
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        f4fma(r, ck * s_w[ib] * s_w[ic], ax);
        f4fma(r, ck * s_w[ia] * s_w[ic], ay);
        f4fma(r, ck * s_w[ia] * s_w[ib], az);
        if constexpr (G) {
            f4fma(r, s_pot[j], s_u[it]);
            if (U) {
                // orbitals p0 = 2q (lanes x, y) and p1 = 2q + 1 (lanes z, w); the
                // node's orbitals and the two field rows are read as 16-byte quads
                // (orbitals 2c, 2c + 1 with U[p][2c], U[p][2c + 1])
                float2 m0 = make_float2(0.f, 0.f), m1 = m0;
                const int nl = L4C > 0 ? 2 * L4C : n;
                const int hl = nl / 2;   // quads per field row
                const float4* Ur = s_U4 + j * SU + q * nl;
#pragma unroll
                for (int c = 0; c < (L4C > 0 ? L4C : 64); ++c) {
                    if (L4C == 0 && c >= hl) break;
                    const float4 u = s_u[j * L4 + c];
                    const float4 a0 = Ur[c];
                    const float4 a1 = Ur[hl + c];
                    m0.x = fmaf(a0.x, u.x, fmaf(-a0.y, u.y, m0.x));
                    m0.y = fmaf(a0.x, u.y, fmaf(a0.y, u.x, m0.y));
                    m0.x = fmaf(a0.z, u.z, fmaf(-a0.w, u.w, m0.x));
                    m0.y = fmaf(a0.z, u.w, fmaf(a0.w, u.z, m0.y));
                    m1.x = fmaf(a1.x, u.x, fmaf(-a1.y, u.y, m1.x));
                    m1.y = fmaf(a1.x, u.y, fmaf(a1.y, u.x, m1.y));
                    m1.x = fmaf(a1.z, u.z, fmaf(-a1.w, u.w, m1.x));
                    m1.y = fmaf(a1.z, u.w, fmaf(a1.w, u.z, m1.y));
                }
                const float wq = s_wq[j];
                r.x = fmaf(wq, m0.x, r.x);
                r.y = fmaf(wq, m0.y, r.y);
                r.z = fmaf(wq, m1.x, r.z);
                r.w = fmaf(wq, m1.y, r.w);
            }
        }
        scatter32v(a, s_idx[j], y, L4, q, r);
        if constexpr (!G && PAP) {   // the cell's part of p.Ap: p (gathered, zero on the surface) times A_K p
            const float4 u = s_u[it];
            pap.x = fmaf(u.x, r.x, pap.x);
            pap.y = fmaf(u.y, r.y, pap.y);
            pap.z = fmaf(u.z, r.z, pap.z);
            pap.w = fmaf(u.w, r.w, pap.w);
        }
    }
    if constexpr (!G && PAP && L4C > 0 && 32 % L4C == 0) {
        // p.Ap = sum over cells of u_K . A_K u_K (p vanishes on the surface, so
        // the masked scatter drops nothing): lanes with the same quad summed by
        // shuffles, the 8 warps in FP64, one FP64 atomic per column and block
        {
#pragma unroll
            for (int off = L4C; off < 32; off <<= 1) {
                pap.x += __shfl_xor_sync(0xffffffffu, pap.x, off);
                pap.y += __shfl_xor_sync(0xffffffffu, pap.y, off);
                pap.z += __shfl_xor_sync(0xffffffffu, pap.z, off);
                pap.w += __shfl_xor_sync(0xffffffffu, pap.w, off);
            }
            __shared__ float4 s_pap[8][L4C];
            const int lane = tid & 31, warp = tid >> 5;
            if (lane < L4C && warp < 8) s_pap[warp][lane] = pap;
            __syncthreads();
            if (tid < 4 * L4C) {
                const int q = tid >> 2, comp = tid & 3;
                double xs = 0.0;
                for (int w8 = 0; w8 < 8 && w8 * 32 < bs; ++w8) {
                    const float4 v = s_pap[w8][q];
                    xs += widen_f32(comp == 0 ? v.x : comp == 1 ? v.y : comp == 2 ? v.z : v.w);
                }
                atomicAdd(&a.pap_slots[int64_t(item % kPapSlots) * (4 * L4C) + tid], xs);
            }
        }
    }
}

// PAP: the stiffness pass also forms p.Ap (into a.pap_slots) for the
// conjugate-gradient sweep.
template <int P, bool G, int L4C, bool PAP>
__global__ void __launch_bounds__(256) cell32v_kernel(const __grid_constant__ CellArgs32 a,
                                                      const float4* __restrict__ x, const float2* __restrict__ U,
                                                      float4* __restrict__ y, int L4rt, int n) {
    cell32v_body<P, G, L4C, PAP>(a, blockIdx.x, x, U, y, L4rt, n);
}

// Degree 4 (the largest cells): held to 32 registers so that 8 blocks of 256
// threads share an SM.
template <bool G, int L4C, bool PAP>
__global__ void __launch_bounds__(256, 8) cell32v_kernel_q4(const __grid_constant__ CellArgs32 a,
                                                            const float4* __restrict__ x,
                                                            const float2* __restrict__ U, float4* __restrict__ y,
                                                            int L4rt, int n) {
    cell32v_body<4, G, L4C, PAP>(a, blockIdx.x, x, U, y, L4rt, n);
}

template <int P, bool G, int L4C, bool PAP>
constexpr auto cell32v_pick() {
    if constexpr (P == 4) return cell32v_kernel_q4<G, L4C, PAP>;
    else return cell32v_kernel<P, G, L4C, PAP>;
}

// ------------------------------------------------ frozen per-cell blocks
// Within one orbital propagation (Sec. 3.2: phi, U and E frozen over the
// step) the pointwise part of the G cell pass does not change between its
// Krylov applications: at every cell node it is the n x n complex matrix
//   B_pq = m_node (U_pq(node) + delta_pq (V(node) + E . x_node)),
// m_node the node's quadrature weight h^3 w_a w_b w_c.  It is formed once per
// propagation, cell by cell in node order ([ncell][(p+1)^3][SU] float4, each
// node's n^2 complex entries row by row as float4 pairs, SU = (n^2/2) | 1
// quads per node: the odd stride keeps the rows that a quarter warp reads on
// distinct banks), so each cell's block is one contiguous, 16-byte aligned
// run that the cell pass stages into shared memory with a single bulk copy of
// the tensor memory accelerator (cp.async.bulk) instead of one gather per
// node row; hanging nodes take the mean fields interpolated through C.
__host__ __device__ constexpr int gblock_quads(int n) { return ((n * n) / 2) | 1; }

// One float4 of B per thread: (cell, node, quad k); row p = k / (n/2), columns
// 2 (k % (n/2)) and + 1; the padding quad is zero.
__global__ void gcell_blocks32_kernel(const CellArgs32 a, const float2* __restrict__ U,
                                      const float2* __restrict__ U_hang, int n, int P1, float4* __restrict__ B) {
    const int NN = P1 * P1 * P1;
    const int SU = gblock_quads(n), half = n / 2, nn = n * n;
    const int64_t total = a.ncell * NN * SU;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < total;
         o += int64_t(gridDim.x) * blockDim.x) {
        const int k = int(o % SU);
        const int64_t cj = o / SU;                 // cell * NN + node
        const int64_t cell = cj / NN;
        const int j = int(cj - cell * NN);
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < nn / 2) {
            const int p = k / half, q0 = 2 * (k - p * half);
            const int ia = j % P1, ib = (j / P1) % P1, ic = j / (P1 * P1);
            const float4 g = a.geom[cell];
            const float px = g.x + g.w * a.xi[ia], py = g.y + g.w * a.xi[ib], pz = g.z + g.w * a.xi[ic];
            const float wq = g.w * g.w * g.w * a.w[ia] * a.w[ib] * a.w[ic];
            const float pot = a.v_cell[cj] + a.E[0] * px + a.E[1] * py + a.E[2] * pz;
            const int idx = a.cell_node[cj];
            const float2* row = idx >= 0 ? U + int64_t(idx) * nn : U_hang + int64_t(-idx - 1) * nn;
            float2 u0 = row[p * n + q0], u1 = row[p * n + q0 + 1];
            if (q0 == p) u0.x += pot;
            if (q0 + 1 == p) u1.x += pot;
            out = make_float4(wq * u0.x, wq * u0.y, wq * u1.x, wq * u1.y);
        }
        B[o] = out;
    }
}

constexpr int kBulkMaxPolls = 1 << 20;   // polls of a cell's block copy before the pass gives up

// The degree-4 G cell pass on staged per-cell blocks: one cell per block of
// 256 threads, L4C = n/2 complex orbital pairs per node (n = 2, 4, 6, 8).
// Thread 0 starts the bulk copy of the cell's block first; the gathers of the
// Krylov vector (asynchronous 16-byte copies for masters, the constraint walk
// for hanging points) overlap it.  The kinetic term is the node-per-thread
// sum factorisation of cell32v_body; the pointwise part is sum_q B_pq v_q.
// A copy that does not complete within the poll limit sets *err (a value the
// host reads with every substep's results) and the cell is skipped.
template <int L4C>
__global__ void __launch_bounds__(256, 8) gcell32b_kernel(const __grid_constant__ CellArgs32 a,
                                                          const float4* __restrict__ x,
                                                          const float4* __restrict__ B, float4* __restrict__ y,
                                                          double* __restrict__ err) {
    constexpr int P1 = 5, NN = 125, L4 = L4C, n = 2 * L4C;
    constexpr int SU = gblock_quads(n);
    constexpr uint32_t kBytes = uint32_t(NN * SU * 16);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4* s_B = reinterpret_cast<float4*>(smem_raw);   // [NN][SU]
    float4* s_u = s_B + NN * SU;                         // [NN][L4]
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_idx[NN];
    __shared__ float4 s_g;
    __shared__ float s_K[P1 * P1];
    __shared__ float s_w[P1];
    const int64_t cell = blockIdx.x;
    const int tid = threadIdx.x;
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_fence_init();
        tc::mbar_arrive_expect_tx(&bar, kBytes);
        tc::bulk_copy_g2s(s_B, B + cell * (NN * SU), kBytes, &bar);
        s_g = a.geom[cell];
    }
    for (int i = tid; i < NN; i += 256) s_idx[i] = a.cell_node[cell * NN + i];
    if (tid < P1 * P1) s_K[tid] = a.K[tid];
    if (tid < P1) s_w[tid] = a.w[tid];
    __syncthreads();
    for (int it = tid; it < NN * L4; it += 256) {
        const int j = it / L4, q = it - j * L4;
        const int idx = s_idx[j];
        if (idx >= 0 && !(a.masked && idx >= a.n_interior)) cp_async16(s_u + it, x + int64_t(idx) * L4 + q);
        else s_u[it] = gather32v(a, idx, x, L4, q);
    }
    cp_async_wait_all();
    const bool got = tc::mbar_wait(&bar, 0u, kBulkMaxPolls);
    if (__syncthreads_or(!got)) {
        // the copy may still be in flight: wait once more (bounded) before the
        // block's shared memory is released
        if (tid == 0) {
            *err = 1.0;
            tc::mbar_wait(&bar, 0u, kBulkMaxPolls);
        }
        __syncthreads();
        return;
    }
    const float ck = 0.5f * s_g.w;
    for (int it = tid; it < NN * L4; it += 256) {
        const int j = it / L4, q = it - j * L4;
        const int ia = j % P1, ib = (j / P1) % P1, ic = j / (P1 * P1);
        const float4* u0 = s_u + q;
        float4 ax = make_float4(0.f, 0.f, 0.f, 0.f), ay = ax, az = ax;
#pragma unroll
        for (int m = 0; m < P1; ++m) {
            f4fma(ax, s_K[ia * P1 + m], u0[(m + P1 * (ib + P1 * ic)) * L4]);
            f4fma(ay, s_K[ib * P1 + m], u0[(ia + P1 * (m + P1 * ic)) * L4]);
            f4fma(az, s_K[ic * P1 + m], u0[(ia + P1 * (ib + P1 * m)) * L4]);
        }
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        f4fma(r, ck * s_w[ib] * s_w[ic], ax);
        f4fma(r, ck * s_w[ia] * s_w[ic], ay);
        f4fma(r, ck * s_w[ia] * s_w[ib], az);
        // rows p0 = 2q (lanes x, y) and p1 = 2q + 1 (lanes z, w) of the node's
        // block against its orbitals, read as 16-byte quads
        const float4* Br = s_B + j * SU + q * n;
        float2 m0 = make_float2(0.f, 0.f), m1 = m0;
#pragma unroll
        for (int c = 0; c < L4C; ++c) {
            const float4 u = s_u[j * L4 + c];
            const float4 a0 = Br[c];
            const float4 a1 = Br[L4C + c];
            m0.x = fmaf(a0.x, u.x, fmaf(-a0.y, u.y, m0.x));
            m0.y = fmaf(a0.x, u.y, fmaf(a0.y, u.x, m0.y));
            m0.x = fmaf(a0.z, u.z, fmaf(-a0.w, u.w, m0.x));
            m0.y = fmaf(a0.z, u.w, fmaf(a0.w, u.z, m0.y));
            m1.x = fmaf(a1.x, u.x, fmaf(-a1.y, u.y, m1.x));
            m1.y = fmaf(a1.x, u.y, fmaf(a1.y, u.x, m1.y));
            m1.x = fmaf(a1.z, u.z, fmaf(-a1.w, u.w, m1.x));
            m1.y = fmaf(a1.z, u.w, fmaf(a1.w, u.z, m1.y));
        }
        r.x += m0.x;
        r.y += m0.y;
        r.z += m1.x;
        r.w += m1.y;
        scatter32v(a, s_idx[j], y, L4, q, r);
    }
}

// Complex64 quads of v at the hanging points, C v (interior masters only: the
// G pass is Dirichlet-masked), [nh][L4]; formed once per application so that
// the pipelined pass below gathers every node row by an asynchronous copy.
__global__ void hang_expand32v_kernel(const int32_t* __restrict__ hp, const int32_t* __restrict__ hm,
                                      const float* __restrict__ hw, int64_t nh, int64_t n_interior,
                                      const float4* __restrict__ x, int L4, float4* __restrict__ xh) {
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < nh * L4;
         o += int64_t(gridDim.x) * blockDim.x) {
        const int64_t h = o / L4;
        const int q = int(o - h * L4);
        float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int e = hp[h]; e < hp[h + 1]; ++e) {
            const int m = hm[e];
            if (m < n_interior) f4fma(val, hw[e], x[int64_t(m) * L4 + q]);
        }
        xh[o] = val;
    }
}

// Pipelined form of gcell32b_kernel (n = 2 or 4): a block walks the cells
// blockIdx.x, + gridDim.x, ... with two shared-memory buffers; while it
// computes one cell, the next cell's block (one bulk copy) and node rows
// (16-byte asynchronous copies of v, or of C v at hanging nodes; zeros at
// surface masters) are already in flight into the other buffer.  One block
// barrier per cell.
template <int L4C>
__global__ void __launch_bounds__(256, 4) gcell32p_kernel(const __grid_constant__ CellArgs32 a,
                                                          const float4* __restrict__ x,
                                                          const float4* __restrict__ xh,
                                                          const float4* __restrict__ B, float4* __restrict__ y,
                                                          double* __restrict__ err) {
    constexpr int P1 = 5, NN = 125, L4 = L4C, n = 2 * L4C;
    constexpr int SU = gblock_quads(n);
    constexpr uint32_t kBytes = uint32_t(NN * SU * 16);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4* s_B = reinterpret_cast<float4*>(smem_raw);   // [2][NN][SU]
    float4* s_u = s_B + 2 * NN * SU;                     // [2][NN][L4]
    int* s_idx = reinterpret_cast<int*>(s_u + 2 * NN * L4);   // [2][NN]
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float4 s_g[2];
    __shared__ float s_K[P1 * P1];
    __shared__ float s_w[P1];
    const int tid = threadIdx.x;
    if (tid == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::mbar_fence_init();
    }
    if (tid < P1 * P1) s_K[tid] = a.K[tid];
    if (tid < P1) s_w[tid] = a.w[tid];
    __syncthreads();
    auto stage = [&](int64_t c, int b) {
        if (tid == 0) {
            tc::mbar_arrive_expect_tx(&bar[b], kBytes);
            tc::bulk_copy_g2s(s_B + b * NN * SU, B + c * (NN * SU), kBytes, &bar[b]);
            s_g[b] = a.geom[c];
        }
        for (int it = tid; it < NN * L4; it += 256) {
            const int j = it / L4, q = it - j * L4;
            const int idx = a.cell_node[c * NN + j];
            if (q == 0) s_idx[b * NN + j] = idx;
            float4* dst = s_u + b * NN * L4 + it;
            if (idx < 0) cp_async16(dst, xh + int64_t(-idx - 1) * L4 + q);
            else if (idx < a.n_interior) cp_async16(dst, x + int64_t(idx) * L4 + q);
            else *dst = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    int64_t cell = blockIdx.x;
    if (cell < a.ncell) stage(cell, 0);
    uint32_t parity = 0u;   // bit b: phase parity of buffer b's barrier
    int b = 0;
    for (; cell < a.ncell; cell += gridDim.x, b ^= 1) {
        cp_async_wait_all();
        const uint32_t ph = (parity >> b) & 1u;
        const bool got = tc::mbar_wait(&bar[b], ph, kBulkMaxPolls);
        parity ^= 1u << b;
        if (__syncthreads_or(!got)) {
            // the block copy may still be in flight: wait once more (bounded)
            // before the block's shared memory is released
            if (tid == 0) {
                *err = 1.0;
                tc::mbar_wait(&bar[b], ph, kBulkMaxPolls);
            }
            __syncthreads();
            return;
        }
        const int64_t next = cell + gridDim.x;
        if (next < a.ncell) stage(next, b ^ 1);
        const float4* ub = s_u + b * NN * L4;
        const float4* Bb = s_B + b * NN * SU;
        const int* ib_ = s_idx + b * NN;
        const float ck = 0.5f * s_g[b].w;
        for (int it = tid; it < NN * L4; it += 256) {
            const int j = it / L4, q = it - j * L4;
            const int ia = j % P1, ib = (j / P1) % P1, ic = j / (P1 * P1);
            const float4* u0 = ub + q;
            float4 ax = make_float4(0.f, 0.f, 0.f, 0.f), ay = ax, az = ax;
#pragma unroll
            for (int m = 0; m < P1; ++m) {
                f4fma(ax, s_K[ia * P1 + m], u0[(m + P1 * (ib + P1 * ic)) * L4]);
                f4fma(ay, s_K[ib * P1 + m], u0[(ia + P1 * (m + P1 * ic)) * L4]);
                f4fma(az, s_K[ic * P1 + m], u0[(ia + P1 * (ib + P1 * m)) * L4]);
            }
            float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
            f4fma(r, ck * s_w[ib] * s_w[ic], ax);
            f4fma(r, ck * s_w[ia] * s_w[ic], ay);
            f4fma(r, ck * s_w[ia] * s_w[ib], az);
            const float4* Br = Bb + j * SU + q * n;
            float2 m0 = make_float2(0.f, 0.f), m1 = m0;
#pragma unroll
            for (int c = 0; c < L4C; ++c) {
                const float4 u = ub[j * L4 + c];
                const float4 a0 = Br[c];
                const float4 a1 = Br[L4C + c];
                m0.x = fmaf(a0.x, u.x, fmaf(-a0.y, u.y, m0.x));
                m0.y = fmaf(a0.x, u.y, fmaf(a0.y, u.x, m0.y));
                m0.x = fmaf(a0.z, u.z, fmaf(-a0.w, u.w, m0.x));
                m0.y = fmaf(a0.z, u.w, fmaf(a0.w, u.z, m0.y));
                m1.x = fmaf(a1.x, u.x, fmaf(-a1.y, u.y, m1.x));
                m1.y = fmaf(a1.x, u.y, fmaf(a1.y, u.x, m1.y));
                m1.x = fmaf(a1.z, u.z, fmaf(-a1.w, u.w, m1.x));
                m1.y = fmaf(a1.z, u.w, fmaf(a1.w, u.z, m1.y));
            }
            r.x += m0.x;
            r.y += m0.y;
            r.z += m1.x;
            r.w += m1.y;
            scatter32v(a, ib_[j], y, L4, q, r);
        }
    }
}

// Line-ordered form of the four-lane pass: the three 1D contractions run as
// whole lines (each thread loads the P1 values of one line once and writes P1
// outputs), accumulated direction by direction in shared memory, which cuts
// the shared-memory loads per cell from 3 (p+1) per output to about 3 per
// output.  Node-local terms (potential, mean field) are added with the first
// direction.  128 threads per cell.
template <int P, bool G>
__global__ void __launch_bounds__(128) cell32L_kernel(CellArgs32 a, const float4* __restrict__ x,
                                                      const float2* __restrict__ U, float4* __restrict__ y, int L4,
                                                      int n) {
    constexpr int P1 = P + 1;
    constexpr int NN = P1 * P1 * P1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* s_u = reinterpret_cast<float4*>(smem_raw);          // [NN][L4]
    float4* s_acc = s_u + NN * L4;                              // [NN][L4]
    float2* s_U = reinterpret_cast<float2*>(s_acc + NN * L4);   // [NN][n*n] (G with U)
    __shared__ int s_idx[NN];
    __shared__ float s_pot[NN];
    __shared__ float s_wq[NN];
    __shared__ float s_K[P1 * P1];
    __shared__ float s_w[P1];
    const int64_t cell = blockIdx.x;
    const int tid = threadIdx.x, bs = blockDim.x;
    const float4 g = a.geom[cell];
    for (int i = tid; i < NN; i += bs) s_idx[i] = a.cell_node[cell * NN + i];
    if (tid < P1 * P1) s_K[tid] = a.K[tid];
    if (tid < P1) s_w[tid] = a.w[tid];
    __syncthreads();
    for (int it = tid; it < NN * L4; it += bs) {
        const int i = it / L4, q = it - i * L4;
        s_u[it] = gather32v(a, s_idx[i], x, L4, q);
    }
    const int nn2 = n * n;
    if (G) {
        if (U) {
            CellArgs32 au = a;
            au.masked = 0;
            for (int it = tid; it < NN * nn2; it += bs) {
                const int i = it / nn2, pq = it - i * nn2;
                const int idx = s_idx[i];
                s_U[it] = (idx < 0 && a.u_hang) ? a.u_hang[int64_t(-idx - 1) * nn2 + pq]
                                                : gather32<float2>(au, idx, U, nn2, pq);
            }
        }
        const float h3 = g.w * g.w * g.w;
        for (int i = tid; i < NN; i += bs) {
            const int ia = i % P1, ib = (i / P1) % P1, ic = i / (P1 * P1);
            const int idx = s_idx[i];
            const float V = idx >= 0 ? a.v_master[idx] : a.v_hang[-idx - 1];
            const float px = g.x + g.w * a.xi[ia], py = g.y + g.w * a.xi[ib], pz = g.z + g.w * a.xi[ic];
            const float wq = h3 * s_w[ia] * s_w[ib] * s_w[ic];
            s_wq[i] = wq;
            s_pot[i] = wq * (V + a.E[0] * px + a.E[1] * py + a.E[2] * pz);
        }
    }
    __syncthreads();
    const float ck = (G ? 0.5f : 1.0f) * g.w;
    constexpr int NL = P1 * P1;   // lines per direction
    // direction 0 (x): line (b, c), nodes a + P1 (b + P1 c); stores
    for (int it = tid; it < NL * L4; it += bs) {
        const int line = it / L4, q = it - line * L4;
        const int b = line % P1, c = line / P1;
        float4 u[P1];
#pragma unroll
        for (int m = 0; m < P1; ++m) u[m] = s_u[(m + P1 * (b + P1 * c)) * L4 + q];
        const float sc = ck * s_w[b] * s_w[c];
#pragma unroll
        for (int aa = 0; aa < P1; ++aa) {
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int m = 0; m < P1; ++m) f4fma(acc, s_K[aa * P1 + m], u[m]);
            const int node = aa + P1 * (b + P1 * c);
            float4 r = make_float4(sc * acc.x, sc * acc.y, sc * acc.z, sc * acc.w);
            if constexpr (G) {
                f4fma(r, s_pot[node], u[aa]);
                if (U) {
                    const float2* ui = reinterpret_cast<const float2*>(s_u + node * L4);
                    const float2* U0 = s_U + node * nn2 + (2 * q) * n;
                    const float2* U1 = U0 + n;
                    float2 m0 = make_float2(0.f, 0.f), m1 = m0;
                    for (int rr = 0; rr < n; ++rr) {
                        const float2 uu = ui[rr];
                        m0.x = fmaf(U0[rr].x, uu.x, fmaf(-U0[rr].y, uu.y, m0.x));
                        m0.y = fmaf(U0[rr].x, uu.y, fmaf(U0[rr].y, uu.x, m0.y));
                        m1.x = fmaf(U1[rr].x, uu.x, fmaf(-U1[rr].y, uu.y, m1.x));
                        m1.y = fmaf(U1[rr].x, uu.y, fmaf(U1[rr].y, uu.x, m1.y));
                    }
                    const float wq = s_wq[node];
                    r.x = fmaf(wq, m0.x, r.x);
                    r.y = fmaf(wq, m0.y, r.y);
                    r.z = fmaf(wq, m1.x, r.z);
                    r.w = fmaf(wq, m1.y, r.w);
                }
            }
            s_acc[node * L4 + q] = r;
        }
    }
    __syncthreads();
    // direction 1 (y): line (a, c)
    for (int it = tid; it < NL * L4; it += bs) {
        const int line = it / L4, q = it - line * L4;
        const int aa = line % P1, c = line / P1;
        float4 u[P1];
#pragma unroll
        for (int m = 0; m < P1; ++m) u[m] = s_u[(aa + P1 * (m + P1 * c)) * L4 + q];
        const float sc = ck * s_w[aa] * s_w[c];
#pragma unroll
        for (int b = 0; b < P1; ++b) {
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int m = 0; m < P1; ++m) f4fma(acc, s_K[b * P1 + m], u[m]);
            float4& o = s_acc[(aa + P1 * (b + P1 * c)) * L4 + q];
            f4fma(o, sc, acc);
        }
    }
    __syncthreads();
    // direction 2 (z): line (a, b)
    for (int it = tid; it < NL * L4; it += bs) {
        const int line = it / L4, q = it - line * L4;
        const int aa = line % P1, b = line / P1;
        float4 u[P1];
#pragma unroll
        for (int m = 0; m < P1; ++m) u[m] = s_u[(aa + P1 * (b + P1 * m)) * L4 + q];
        const float sc = ck * s_w[aa] * s_w[b];
#pragma unroll
        for (int c = 0; c < P1; ++c) {
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int m = 0; m < P1; ++m) f4fma(acc, s_K[c * P1 + m], u[m]);
            float4& o = s_acc[(aa + P1 * (b + P1 * c)) * L4 + q];
            f4fma(o, sc, acc);
        }
    }
    __syncthreads();
    for (int it = tid; it < NN * L4; it += bs) {
        const int i = it / L4, q = it - i * L4;
        scatter32v(a, s_idx[i], y, L4, q, s_acc[it]);
    }
}

CellArgs32 make_cell_args32(const afem_mesh* m) {
    CellArgs32 a{};
    const DeviceMesh& D = m->dev;
    a.cell_node = D.cell_node;
    a.geom = D.cell_geom32;
    a.hp = D.hang_ptr;
    a.hm = D.hang_master;
    a.hw = D.hang_w32;
    a.v_master = D.v_master32;
    a.v_hang = D.v_hang32;
    a.v_cell = D.v_cell32;
    a.ncell = D.ncell;
    a.n_interior = D.n_interior;
    const Basis1D& b = m->basis;
    const int p1 = b.p + 1;
    for (int i = 0; i < p1; ++i) {
        a.xi[i] = float(b.xi[i]);
        a.w[i] = float(b.w[i]);
        for (int j = 0; j < p1; ++j) {
            a.K[i * p1 + j] = float(b.K[i][j]);
            a.S[i * p1 + j] = float(b.S[i][j]);
        }
    }
    return a;
}

template <typename T, bool G>
static int launch32(const afem_mesh* m, const CellArgs32& a, const T* x, const float2* U, T* y, int nv,
                    cudaStream_t s) {
    const int p = m->dev.p;
    const int nn = (p + 1) * (p + 1) * (p + 1);
    const size_t smem = size_t(nn) * nv * sizeof(T) + ((G && U) ? size_t(nn) * nv * nv * sizeof(float2) : 0);
    const unsigned grid = unsigned(m->dev.ncell);
    AFEM_CUDA_TRY(cudaMemsetAsync(y, 0, size_t(m->dev.n_master) * nv * sizeof(T), s));
    if (grid == 0) return AFEM_OK;
    switch (p) {
#define AFEM_CASE(PP)                                                                          \
    case PP: {                                                                                 \
        auto k = cell32_kernel<PP, T, G, false>;                                               \
        if constexpr (G && sizeof(T) == sizeof(float2)) {                                      \
            if (a.vg) k = cell32_kernel<PP, T, G, true>;                                       \
            if (a.ecs_flags) k = cell32_kernel<PP, T, G, false, true>;                         \
        }                                                                                      \
        if (smem > 48 * 1024)                                                                  \
            AFEM_CUDA_TRY(allow_dyn_smem(k));                                    \
        AFEM_LAUNCH((k), grid, 256, smem, s, a, x, U, y, nv);                                  \
        break;                                                                                 \
    }
        AFEM_CASE(1)
        AFEM_CASE(2)
        AFEM_CASE(3)
        AFEM_CASE(4)
#undef AFEM_CASE
        default:
            return set_error(AFEM_EINVAL, "degree out of range");
    }
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

// The four-lane kernel for a quad count (compile-time for 1..4), with the p.Ap
// epilogue when asked (stiffness, 1, 2 or 4 quads).
// Column-pair line pass of the stiffness (AFEM_OPT_CELL32_VARIANT = 2): the
// three 1D contractions of the sum factorisation each run over whole lines of
// a cell, one thread per (line, column pair): it reads the p+1 values of its
// line once, forms the p+1 outputs in registers (the 1D matrix is read from the
// kernel's parameters), and accumulates them in shared memory, which the next
// direction re-reads along its own lines.  Shared-memory traffic per output is
// one load and one store per direction instead of 3 (p+1) loads, and the
// float2 granularity keeps the line in p+1 register pairs.  Small cells are
// grouped so that a direction's items fill the block.
__host__ __device__ constexpr int cells_per_itemT(int P, int L2) {
    return (P + 1) * (P + 1) * L2 >= 256 ? 1 : 256 / ((P + 1) * (P + 1) * L2);
}

__host__ __device__ constexpr size_t cell32T_smem(int P, int L2) {
    return size_t(cells_per_itemT(P, L2)) *
           (16 + size_t((P + 1) * (P + 1) * (P + 1)) * (size_t(L2) * 16 + sizeof(int)));
}

template <int P, int L2, bool PAP>
__global__ void __launch_bounds__(256, 8) cell32T_kernel(const __grid_constant__ CellArgs32 a,
                                                         const float4* __restrict__ x, float4* __restrict__ y) {
    constexpr int P1 = P + 1;
    constexpr int NN = P1 * P1 * P1;
    constexpr int NL = P1 * P1;
    constexpr int L4 = L2 / 2;
    constexpr int CB = cells_per_itemT(P, L2);
    static_assert(L2 % 2 == 0 && CB * NL * L2 <= 256, "one direction's items must fit the block");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* s_g = reinterpret_cast<float4*>(smem_raw);        // [CB] corner, side
    float2* s_u = reinterpret_cast<float2*>(s_g + CB);        // [CB][NN][L2] the gathered input
    float2* s_acc = s_u + CB * NN * L2;                       // [CB][NN][L2] the cell outputs
    int* s_idx = reinterpret_cast<int*>(s_acc + CB * NN * L2);   // [CB][NN]
    const int64_t cell0 = int64_t(blockIdx.x) * CB;
    const int nc = int(a.ncell - cell0 < CB ? a.ncell - cell0 : CB);
    const int tid = threadIdx.x;
    for (int j = tid; j < nc * NN; j += blockDim.x) s_idx[j] = a.cell_node[cell0 * NN + j];
    if (tid < nc) s_g[tid] = a.geom[cell0 + tid];
    __syncthreads();
    float4* s_u4 = reinterpret_cast<float4*>(s_u);
    for (int it = tid; it < nc * NN * L4; it += blockDim.x) {
        const int j = it / L4, q = it - j * L4;
        s_u4[it] = gather32v(a, s_idx[j], x, L4, q);
    }
    __syncthreads();
    // this thread's item in every direction: (cell slot, line, column pair)
    const int c2 = tid % L2;
    const int line = (tid / L2) % NL;
    const int cb = tid / (L2 * NL);
    const bool act = cb < nc;
    const int l0 = line % P1, l1 = line / P1;
    const float2* ub = s_u + (cb * NN) * L2 + c2;
    float2* ab = s_acc + (cb * NN) * L2 + c2;
    const float sc = act ? s_g[cb].w * a.w[l0] * a.w[l1] : 0.0f;
    float2 u[P1];
    // direction x: line (b, c) = (l0, l1), nodes m + P1 line
    if (act) {
#pragma unroll
        for (int m = 0; m < P1; ++m) u[m] = ub[(m + P1 * line) * L2];
#pragma unroll
        for (int o = 0; o < P1; ++o) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 0; m < P1; ++m) vfma(acc, a.K[o * P1 + m], u[m]);
            ab[(o + P1 * line) * L2] = make_float2(sc * acc.x, sc * acc.y);
        }
    }
    __syncthreads();
    // direction y: line (a, c) = (l0, l1), nodes l0 + P1 (m + P1 l1)
    if (act) {
#pragma unroll
        for (int m = 0; m < P1; ++m) u[m] = ub[(l0 + P1 * (m + P1 * l1)) * L2];
#pragma unroll
        for (int o = 0; o < P1; ++o) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 0; m < P1; ++m) vfma(acc, a.K[o * P1 + m], u[m]);
            float2& r = ab[(l0 + P1 * (o + P1 * l1)) * L2];
            r.x = fmaf(sc, acc.x, r.x);
            r.y = fmaf(sc, acc.y, r.y);
        }
    }
    __syncthreads();
    // direction z: line (a, b) = (l0, l1), nodes line + NL m
    if (act) {
#pragma unroll
        for (int m = 0; m < P1; ++m) u[m] = ub[(line + NL * m) * L2];
#pragma unroll
        for (int o = 0; o < P1; ++o) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 0; m < P1; ++m) vfma(acc, a.K[o * P1 + m], u[m]);
            float2& r = ab[(line + NL * o) * L2];
            r.x = fmaf(sc, acc.x, r.x);
            r.y = fmaf(sc, acc.y, r.y);
        }
    }
    __syncthreads();
    const float4* s_acc4 = reinterpret_cast<const float4*>(s_acc);
    float4 pap = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int it = tid; it < nc * NN * L4; it += blockDim.x) {
        const int j = it / L4, q = it - j * L4;
        const float4 r = s_acc4[it];
        scatter32v(a, s_idx[j], y, L4, q, r);
        if constexpr (PAP) {   // the cell's part of p.Ap (p is zero on the surface)
            const float4 v = s_u4[it];
            pap.x = fmaf(v.x, r.x, pap.x);
            pap.y = fmaf(v.y, r.y, pap.y);
            pap.z = fmaf(v.z, r.z, pap.z);
            pap.w = fmaf(v.w, r.w, pap.w);
        }
    }
    if constexpr (PAP) {
        static_assert(32 % L4 == 0, "the p.Ap lanes of one column quad are L4 apart");
        // blockDim is a multiple of 32 and of L4, so a lane's quad is tid % L4 in every iteration
#pragma unroll
        for (int off = L4; off < 32; off <<= 1) {
            pap.x += __shfl_xor_sync(0xffffffffu, pap.x, off);
            pap.y += __shfl_xor_sync(0xffffffffu, pap.y, off);
            pap.z += __shfl_xor_sync(0xffffffffu, pap.z, off);
            pap.w += __shfl_xor_sync(0xffffffffu, pap.w, off);
        }
        __shared__ float4 s_pap[8][L4];
        const int lane = tid & 31, warp = tid >> 5;
        if (lane < L4 && warp < 8) s_pap[warp][lane] = pap;
        __syncthreads();
        if (tid < 4 * L4) {
            const int q = tid >> 2, comp = tid & 3;
            double xs = 0.0;
            for (int w8 = 0; w8 < 8 && w8 * 32 < int(blockDim.x); ++w8) {
                const float4 v = s_pap[w8][q];
                xs += widen_f32(comp == 0 ? v.x : comp == 1 ? v.y : comp == 2 ? v.z : v.w);
            }
            atomicAdd(&a.pap_slots[int64_t(blockIdx.x % kPapSlots) * (4 * L4) + tid], xs);
        }
    }
}

template <int PP, int L2>
static int launch32T_l(const afem_mesh* m, const CellArgs32& a, const float4* x, float4* y, cudaStream_t s) {
    constexpr int CB = cells_per_itemT(PP, L2);
    const size_t smem = cell32T_smem(PP, L2);
    auto k = a.pap_slots ? cell32T_kernel<PP, L2, true> : cell32T_kernel<PP, L2, false>;
    if (smem > 48 * 1024)
        AFEM_CUDA_TRY(allow_dyn_smem(k));
    const unsigned items = unsigned((m->dev.ncell + CB - 1) / CB);
    AFEM_LAUNCH((k), items, 256, smem, s, a, x, y);
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

// The column-pair line pass of the stiffness for 1, 2 or 4 column quads.
template <int PP>
static int launch32T(const afem_mesh* m, const CellArgs32& a, const float4* x, float4* y, int L4, cudaStream_t s) {
    if (L4 == 1) return launch32T_l<PP, 2>(m, a, x, y, s);
    if (L4 == 2) return launch32T_l<PP, 4>(m, a, x, y, s);
    return launch32T_l<PP, 8>(m, a, x, y, s);
}

template <int PP, bool G>
static auto pick32v(int L4, bool pap) {
    if constexpr (!G) {
        if (pap)
            return L4 == 1 ? cell32v_pick<PP, G, 1, true>()
                           : L4 == 2 ? cell32v_pick<PP, G, 2, true>() : cell32v_pick<PP, G, 4, true>();
    }
    return L4 == 1   ? cell32v_pick<PP, G, 1, false>()
           : L4 == 2 ? cell32v_pick<PP, G, 2, false>()
           : L4 == 3 ? cell32v_pick<PP, G, 3, false>()
           : L4 == 4 ? cell32v_pick<PP, G, 4, false>()
                     : cell32v_pick<PP, G, 0, false>();
}

// L = float lanes per node (multiple of 4); n = orbitals (G only).
template <bool G>
static int launch32v(const afem_mesh* m, const CellArgs32& a, const float* x, const float2* U, float* y, int L,
                     int n, cudaStream_t s) {
    const int p = m->dev.p;
    const int nn = (p + 1) * (p + 1) * (p + 1);
    const int L4 = L / 4;
    const unsigned grid = unsigned(m->dev.ncell);
    AFEM_CUDA_TRY(cudaMemsetAsync(y, 0, size_t(m->dev.n_master) * L * sizeof(float), s));
    if (grid == 0) return AFEM_OK;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    float4* y4 = reinterpret_cast<float4*>(y);
    if (!G && m->cell32_variant == 2 && (L4 == 1 || L4 == 2 || L4 == 4)) {
        switch (p) {
            case 1: return launch32T<1>(m, a, x4, y4, L4, s);
            case 2: return launch32T<2>(m, a, x4, y4, L4, s);
            case 3: return launch32T<3>(m, a, x4, y4, L4, s);
            case 4: return launch32T<4>(m, a, x4, y4, L4, s);
            default: return set_error(AFEM_EINVAL, "degree out of range");
        }
    }
    if (m->cell32_variant == 1) {
        const size_t smemL =
            2 * size_t(nn) * L4 * sizeof(float4) + ((G && U) ? size_t(nn) * n * n * sizeof(float2) : 0);
        switch (p) {
#define AFEM_CASE(PP)                                                                          \
    case PP: {                                                                                 \
        auto k = cell32L_kernel<PP, G>;                                                        \
        if (smemL > 48 * 1024)                                                                 \
            AFEM_CUDA_TRY(allow_dyn_smem(k));                                   \
        AFEM_LAUNCH((k), grid, 128, smemL, s, a, x4, U, y4, L4, n);                            \
        break;                                                                                 \
    }
            AFEM_CASE(1)
            AFEM_CASE(2)
            AFEM_CASE(3)
            AFEM_CASE(4)
#undef AFEM_CASE
            default:
                return set_error(AFEM_EINVAL, "degree out of range");
        }
        AFEM_CUDA_TRY(cudaGetLastError());
        return AFEM_OK;
    }
    // several small cells per block (cells_per_item32); the mean fields sit
    // (n^2/2) | 1 quads apart per node (see cell32v_body)
    const int cpb = cells_per_item32(p, quads_c32(L4));
    const unsigned items = unsigned((m->dev.ncell + cpb - 1) / cpb);
    const size_t smem = cell32v_smem(p, L4, n, G && U);
    switch (p) {
#define AFEM_CASE(PP)                                                                          \
    case PP: {                                                                                 \
        auto k = pick32v<PP, G>(L4, a.pap_slots != nullptr);                                   \
        if (smem > 48 * 1024)                                                                  \
            AFEM_CUDA_TRY(allow_dyn_smem(k));                                    \
        AFEM_LAUNCH((k), items, 256, smem, s, a, x4, U, y4, L4, n);                            \
        break;                                                                                 \
    }
        AFEM_CASE(1)
        AFEM_CASE(2)
        AFEM_CASE(3)
        AFEM_CASE(4)
#undef AFEM_CASE
        default:
            return set_error(AFEM_EINVAL, "degree out of range");
    }
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// pap_slots (optional): [kPapSlots][nv] FP64 sums that receive p.Ap per column
// (x = p, masked), for nv in {4, 8, 16} on the four-lane path; returns
// AFEM_EINVAL when they are asked for outside it.
int launch_stiffness32(const afem_mesh* m, const float* x, float* y, int nv, int masked, cudaStream_t s,
                       double* pap_slots) {
    CellArgs32 a = make_cell_args32(m);
    a.masked = masked;
    const bool quads = nv % 4 == 0 && aligned16(x) && aligned16(y);
    if (pap_slots) {
        if (!quads || !(nv == 4 || nv == 8 || nv == 16) || m->cell32_variant == 1)
            return set_error(AFEM_EINVAL, "stiffness: fused p.Ap needs 4, 8 or 16 aligned columns");
        a.pap_slots = pap_slots;
    }
    if (quads) return launch32v<false>(m, a, x, nullptr, y, nv, 0, s);
    return launch32<float, false>(m, a, x, nullptr, y, nv, s);
}

// z = H1~ v + mean field (complex64), Dirichlet-masked.
// velocity != 0: E holds the vector potential A (velocity gauge), applied by
// the generic (two-lane) kernel.
int launch_g_cell32(const afem_mesh* m, const double* E, const float2* v, const float2* U, float2* z, int n,
                    cudaStream_t s, int velocity, const float2* U_hang) {
    CellArgs32 a = make_cell_args32(m);
    a.masked = 1;
    a.u_hang = U ? U_hang : nullptr;
    for (int i = 0; i < 3; ++i) a.E[i] = (E && !velocity) ? float(E[i]) : 0.0f;
    if (m->ecs_on) {   // complex-scaled kinetic term: the generic (two-lane) kernel
        if (velocity) return set_error(AFEM_EINVAL, "complex scaling is built for the length gauge");
        a.ecs_flags = m->ecs_flags;
        a.ecs_rho = m->ecs_rho32;
        for (int k = -2; k <= 3; ++k)
            a.ecs_e[k + 2] = make_float2(float(std::cos(k * m->ecs_theta)), float(std::sin(k * m->ecs_theta)));
        return launch32<float2, true>(m, a, v, U, z, n, s);
    }
    if (velocity && E) {
        a.vg = 1;
        for (int i = 0; i < 3; ++i) a.Avec[i] = float(E[i]);
        return launch32<float2, true>(m, a, v, U, z, n, s);
    }
    if (n % 2 == 0 && aligned16(v) && aligned16(z))
        return launch32v<true>(m, a, reinterpret_cast<const float*>(v), U, reinterpret_cast<float*>(z), 2 * n, n, s);
    return launch32<float2, true>(m, a, v, U, z, n, s);
}

// Whether the G cell pass of this mesh and orbital count runs on frozen
// per-cell blocks (degree 4, n even, length gauge, no complex scaling, the
// option on).
bool gcell_blocks_apply(const afem_mesh* m, int n, int velocity) {
    return m->gcell_blocks && m->dev.p == 4 && n % 2 == 0 && n <= 8 && !velocity && !m->ecs_on;
}

size_t gcell_blocks_bytes(const afem_mesh* m, int n) {
    return size_t(m->dev.ncell) * 125 * gblock_quads(n) * sizeof(float4);
}

// B of every cell (see gcell_blocks32_kernel) from the complex64 mean fields at
// the masters (U) and at the hanging points (U_hang), field E.
int build_gcell_blocks32(const afem_mesh* m, const double* E, const float2* U, const float2* U_hang, int n,
                         float4* B, cudaStream_t s) {
    if (m->dev.n_hanging > 0 && !U_hang) return set_error(AFEM_EINVAL, "G cell blocks: hanging mean fields missing");
    CellArgs32 a = make_cell_args32(m);
    for (int i = 0; i < 3; ++i) a.E[i] = E ? float(E[i]) : 0.0f;
    const int64_t total = m->dev.ncell * 125 * gblock_quads(n);
    AFEM_LAUNCH((gcell_blocks32_kernel), grid_for(total), 256, 0, s, a, U, U_hang, n, m->dev.p + 1, B);
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

// z = H1~ v + mean field (complex64, Dirichlet-masked) on the frozen blocks B;
// err: a double that becomes 1 if a block copy did not complete.
int launch_g_cell32_blocks(const afem_mesh* m, const float2* v, const float4* B, float2* z, int n, double* err,
                           float4* vh, cudaStream_t s) {
    if (!aligned16(v) || !aligned16(z) || !aligned16(B))
        return set_error(AFEM_EINVAL, "G cell blocks: vectors must be 16-byte aligned");
    CellArgs32 a = make_cell_args32(m);
    a.masked = 1;
    const int64_t N = m->dev.n_master;
    AFEM_CUDA_TRY(cudaMemsetAsync(z, 0, size_t(N) * n * sizeof(float2), s));
    if (m->dev.ncell == 0) return AFEM_OK;
    const unsigned grid = unsigned(m->dev.ncell);
    const float4* x4 = reinterpret_cast<const float4*>(v);
    float4* y4 = reinterpret_cast<float4*>(z);
    if (vh && n <= 4 && m->gcell_blocks == 2) {
        // pipelined persistent form: C v at the hanging points first
        const int L4 = n / 2;
        const int64_t nh = m->dev.n_hanging;
        if (nh > 0) {
            AFEM_LAUNCH((hang_expand32v_kernel), grid_for(nh * L4), 256, 0, s, m->dev.hang_ptr, m->dev.hang_master,
                        m->dev.hang_w32, nh, m->dev.n_interior, x4, L4, vh);
        }
        const size_t smem = size_t(2) * 125 * (gblock_quads(n) + L4) * sizeof(float4) + size_t(2) * 125 * sizeof(int);
        auto k = n == 2 ? gcell32p_kernel<1> : gcell32p_kernel<2>;
        if (smem > 48 * 1024)
            AFEM_CUDA_TRY(allow_dyn_smem(k));
        int per_sm = 0;
        AFEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem));
        if (per_sm < 1) per_sm = 1;
        int64_t g = int64_t(per_sm) * device_sms();
        if (g > m->dev.ncell) g = m->dev.ncell;
        AFEM_LAUNCH((k), unsigned(g), 256, smem, s, a, x4, vh, B, y4, err);
        AFEM_CUDA_TRY(cudaGetLastError());
        return AFEM_OK;
    }
    switch (n) {
#define AFEM_GB_CASE(NO)                                                                                      \
    case NO: {                                                                                                \
        const size_t smem = size_t(125) * (gblock_quads(NO) + NO / 2) * sizeof(float4);                       \
        if (smem > 48 * 1024)                                                                                 \
            AFEM_CUDA_TRY(allow_dyn_smem(gcell32b_kernel<NO / 2>));                                                   \
        AFEM_LAUNCH((gcell32b_kernel<NO / 2>), grid, 256, smem, s, a, x4, B, y4, err);                        \
        break;                                                                                                \
    }
        AFEM_GB_CASE(2)
        AFEM_GB_CASE(4)
        AFEM_GB_CASE(6)
        AFEM_GB_CASE(8)
#undef AFEM_GB_CASE
        default:
            return set_error(AFEM_EINVAL, "G cell blocks: n must be 2, 4, 6 or 8");
    }
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

// ---------------------------------------------------------------- batching
// One instance of a batched FP32 cell pass (the batching form: many meshes of
// uneven size and degree in one persistent launch).  Kept in device memory and
// read by the batched kernels, so a captured graph holds no instance pointer.
struct BatchInst32 {
    CellArgs32 a;             // mesh tables; masked and E set per apply
    const float4* x;          // [N][4 L4] input
    float4* y;                // [N][4 L4] output
    const double* ml_inv;     // M_L^-1 for the orbital operator, null for the stiffness
    int64_t cell0;            // first global work item of the instance
    int64_t n_rows;           // masters
    int p, L4;
};

size_t batch32_inst_bytes() { return sizeof(BatchInst32); }

// Fills the instance record for mesh m: kind AFEM_OP_H1_C64 (nvec complex
// orbitals, nvec even) or AFEM_OP_STIFF_F32 (nvec real columns, nvec % 4 == 0).
int batch32_fill(const afem_mesh* m, int kind, const double* E, const void* x, void* y, int nvec, int64_t cell0,
                 void* out) {
    if (m->ecs_on) return set_error(AFEM_EINVAL, "afem_batch: not built for a complex-scaled mesh");
    BatchInst32 b{};
    b.a = make_cell_args32(m);
    const int L = kind == AFEM_OP_H1_C64 ? 2 * nvec : nvec;
    if (L % 4 != 0 || !aligned16(x) || !aligned16(y))
        return set_error(AFEM_EINVAL, "afem_batch_op_apply: needs 16-byte aligned buffers and 4 float lanes per "
                                      "quad (an even orbital count, or real columns in multiples of 4)");
    b.a.masked = kind == AFEM_OP_H1_C64 ? 1 : 0;
    for (int i = 0; i < 3; ++i) b.a.E[i] = (kind == AFEM_OP_H1_C64 && E) ? float(E[i]) : 0.0f;
    b.x = static_cast<const float4*>(x);
    b.y = static_cast<float4*>(y);
    b.ml_inv = kind == AFEM_OP_H1_C64 ? m->dev.ml_inv : nullptr;
    b.cell0 = cell0;
    b.n_rows = m->dev.n_master;
    b.p = m->dev.p;
    b.L4 = L / 4;
    std::memcpy(out, &b, sizeof(b));
    return AFEM_OK;
}

constexpr int kBatchMaxInst = 256;

// Out-of-line copies of the cell-pass bodies: each keeps its own register
// budget instead of the batched kernel taking the largest of all of them.
template <int P, bool G, int L4C>
__device__ __noinline__ void cell32v_body_call(const BatchInst32& b, int64_t cell) {
    cell32v_body<P, G, L4C>(b.a, cell, b.x, nullptr, b.y, b.L4, 2 * b.L4);
}

// The cell pass of one work item (instance, group of cells_per_item32 cells)
// by the whole block.
template <bool G>
__device__ __forceinline__ void batch_item(const BatchInst32& b, int64_t cell) {
    switch (b.p * 8 + quads_c32(b.L4)) {
#define AFEM_BI(PP, LL)                          \
    case PP * 8 + LL:                            \
        cell32v_body_call<PP, G, LL>(b, cell);   \
        break;
        AFEM_BI(1, 0) AFEM_BI(1, 1) AFEM_BI(1, 2) AFEM_BI(1, 3) AFEM_BI(1, 4)
        AFEM_BI(2, 0) AFEM_BI(2, 1) AFEM_BI(2, 2) AFEM_BI(2, 3) AFEM_BI(2, 4)
        AFEM_BI(3, 0) AFEM_BI(3, 1) AFEM_BI(3, 2) AFEM_BI(3, 3) AFEM_BI(3, 4)
        AFEM_BI(4, 0) AFEM_BI(4, 1) AFEM_BI(4, 2) AFEM_BI(4, 3) AFEM_BI(4, 4)
#undef AFEM_BI
        default:
            break;
    }
}

// Persistent batched cell pass: block b takes work items b, b + grid, ... of
// the concatenated work-item lists (all instances' cell groups, instance by
// instance).
// The current instance's record is staged in shared memory (its tables, 1D
// matrices and field are then read from there, as the single-instance kernel
// reads them from its parameters), refreshed only when the instance changes.
template <bool G>
__global__ void batch_cell32_kernel(const BatchInst32* __restrict__ inst, int count, int64_t total) {
    __shared__ int64_t s_off[kBatchMaxInst + 1];
    __shared__ BatchInst32 s_inst;
    static_assert(sizeof(BatchInst32) % 8 == 0, "instance record is copied as 8-byte words");
    for (int i = threadIdx.x; i <= count; i += blockDim.x)
        s_off[i] = i < count ? inst[i].cell0 : total;
    __syncthreads();
    int lo = 0, cur = -1;
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        while (lo + 1 < count && s_off[lo + 1] <= g) ++lo;   // items ascend within a block
        if (lo != cur) {   // the same for every thread of the block
            const auto* src = reinterpret_cast<const unsigned long long*>(inst + lo);
            auto* dst = reinterpret_cast<unsigned long long*>(&s_inst);
            for (int i = threadIdx.x; i < int(sizeof(BatchInst32) / 8); i += blockDim.x) dst[i] = src[i];
            cur = lo;
            __syncthreads();
        }
        batch_item<G>(s_inst, g - s_off[lo]);
        __syncthreads();
    }
}

// y_i = 0 for every instance before the scatter.
__global__ void batch_zero_kernel(const BatchInst32* __restrict__ inst, int count) {
    for (int i = 0; i < count; ++i) {
        float4* y = inst[i].y;
        const int64_t total = inst[i].n_rows * inst[i].L4;
        for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < total;
             o += int64_t(gridDim.x) * blockDim.x)
            y[o] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// y_i[k] *= M_L^-1[k] (the orbital operator).
__global__ void batch_scale_kernel(const BatchInst32* __restrict__ inst, int count) {
    for (int i = 0; i < count; ++i) {
        const double* s = inst[i].ml_inv;
        if (!s) continue;
        float4* y = inst[i].y;
        const int L4 = inst[i].L4;
        const int64_t total = inst[i].n_rows * L4;
        for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < total;
             o += int64_t(gridDim.x) * blockDim.x) {
            const float f = float(s[o / L4]);
            float4 v = y[o];
            v.x *= f;
            v.y *= f;
            v.z *= f;
            v.w *= f;
            y[o] = v;
        }
    }
}

// Dynamic shared memory of the batched cell pass: the largest instance's
// [cells per item][(p+1)^3][L4] float4 tile.
size_t batch32_smem(const std::vector<int>& p, const std::vector<int>& L4) {
    size_t mx = 0;
    for (size_t i = 0; i < p.size(); ++i) {
        mx = std::max(mx, cell32v_smem(p[i], L4[i], 2 * L4[i], false));
    }
    return mx;
}

// Work items of one instance: its cells in groups of cells_per_item32.
int64_t batch32_items(int p, int L4, int64_t ncell) {
    const int cpb = cells_per_item32(p, quads_c32(L4));
    return (ncell + cpb - 1) / cpb;
}

int batch32_occupancy(int kind, int block, size_t smem, int* per_sm) {
    const void* k = kind == AFEM_OP_H1_C64 ? reinterpret_cast<const void*>(batch_cell32_kernel<true>)
                                           : reinterpret_cast<const void*>(batch_cell32_kernel<false>);
    if (smem > 48 * 1024) AFEM_CUDA_TRY(allow_dyn_smem(k));
    AFEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, block, smem));
    if (*per_sm < 1) return set_error(AFEM_EINVAL, "afem_batch: the batched cell pass does not fit on an SM");
    return AFEM_OK;
}

// zero, persistent cell pass over all instances, M_L^-1 (orbital operator).
int batch32_launch(int kind, const void* d_inst, int count, int64_t total, int block, unsigned grid, size_t smem,
                   cudaStream_t s) {
    if (count < 1 || count > kBatchMaxInst) return set_error(AFEM_EINVAL, "afem_batch: 1..256 instances");
    const auto* inst = static_cast<const BatchInst32*>(d_inst);
    AFEM_LAUNCH((batch_zero_kernel), 8 * device_sms(), 256, 0, s, inst, count);
    if (kind == AFEM_OP_H1_C64) {
        AFEM_LAUNCH((batch_cell32_kernel<true>), grid, block, smem, s, inst, count, total);
        AFEM_LAUNCH((batch_scale_kernel), 8 * device_sms(), 256, 0, s, inst, count);
    } else {
        AFEM_LAUNCH((batch_cell32_kernel<false>), grid, block, smem, s, inst, count, total);
    }
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

}  // namespace afem
