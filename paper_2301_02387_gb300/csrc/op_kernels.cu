// Matrix-free finite-element operators on the hanging-node octree mesh.
//
// Sec. 3.1: with the tensor-product GLL basis and collocated GLL quadrature,
// the cell stiffness of a cube of side h is
//     A_K = h (Khat (x) W (x) W + W (x) Khat (x) W + W (x) W (x) Khat)
// (Khat the 1D stiffness, W the diagonal of 1D weights), the cell mass is the
// diagonal h^3 W (x) W (x) W and a pointwise potential f contributes
// h^3 (w (x) w (x) w) f at the nodes.  Each output node therefore needs only
// three 1D line contractions, so one kernel pass per cell does
//   gather (with hanging-node interpolation, the "bridged" functions)
//   -> sum-factorised contraction in shared memory
//   -> scatter-add through C^T (atomics) ,
// and the one-body operator of Eq. discretized_eom, H1~ = 1/2 A + F[V + E.r],
// is this pass followed by the inverse lumped mass.
#include <cmath>

#include "afem_internal.h"
#include "cell_common.cuh"
#include "vec_common.cuh"

namespace afem {

// ------------------------------------------------------------------ kernels
// Velocity-gauge term of one output node (Sec. 2: -i A(t) . grad): with the
// skew-symmetric cell matrix h^2 (W (x) W (x) S) per direction,
// r += -i h^2 (A_x w_b w_c (S u)_x + A_y w_a w_c (S u)_y + A_z w_a w_b (S u)_z).
__device__ __forceinline__ void add_velocity_term(double2& r, const double* s_S, const double* s_w,
                                                  const double2* s_u, int ia, int ib, int ic, int nv, int v,
                                                  double h2, const double* A, int P1) {
    double2 gx = make_double2(0.0, 0.0), gy = gx, gz = gx;
    for (int m = 0; m < P1; ++m) {
        vfma(gx, s_S[ia * P1 + m], s_u[(m + P1 * (ib + P1 * ic)) * nv + v]);
        vfma(gy, s_S[ib * P1 + m], s_u[(ia + P1 * (m + P1 * ic)) * nv + v]);
        vfma(gz, s_S[ic * P1 + m], s_u[(ia + P1 * (ib + P1 * m)) * nv + v]);
    }
    double2 t = make_double2(0.0, 0.0);
    vfma(t, h2 * A[0] * s_w[ib] * s_w[ic], gx);
    vfma(t, h2 * A[1] * s_w[ia] * s_w[ic], gy);
    vfma(t, h2 * A[2] * s_w[ia] * s_w[ib], gz);
    r.x += t.y;   // -i t
    r.y -= t.x;
}

// The kinetic part of a complex-scaled cell: ck (sx w_b w_c ax + sy w_a w_c ay
// + sz w_a w_b az) with the cell's complex factors (afem_mesh_set_ecs).
__device__ __forceinline__ double2 ecs_kinetic(double2 sx, double2 sy, double2 sz, double cx, double cy,
                                               double cz, double2 ax, double2 ay, double2 az) {
    const double2 tx = cmul(sx, make_double2(cx * ax.x, cx * ax.y));
    const double2 ty = cmul(sy, make_double2(cy * ay.x, cy * ay.y));
    const double2 tz = cmul(sz, make_double2(cz * az.x, cz * az.y));
    return make_double2(tx.x + ty.x + tz.x, tx.y + ty.y + tz.y);
}

// VG: with the velocity-gauge term (complex data; a.vg set), a separate
// instantiation so that the plain operator keeps its register budget.
// ECS: complex-scaled kinetic term (complex data; the mesh's scaling set).
template <int P, typename T, bool VG = false, bool ECS = false>
__global__ void __launch_bounds__(256) cell_op_kernel(CellArgs a, const T* __restrict__ x,
                                                      T* __restrict__ y, int nv) {
    constexpr int P1 = P + 1;
    constexpr int NN = P1 * P1 * P1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s_u = reinterpret_cast<T*>(smem_raw);
    __shared__ int s_idx[NN];
    __shared__ double s_pot[NN];
    __shared__ double s_K[P1 * P1];
    __shared__ double s_S[P1 * P1];
    __shared__ double s_w[P1];

    const int64_t cell = blockIdx.x;
    const int tid = threadIdx.x;
    const int bs = blockDim.x;
    const double4 g = a.geom[cell];
    for (int n = tid; n < NN; n += bs) s_idx[n] = a.cell_node[cell * NN + n];
    if (tid < P1 * P1) {
        s_K[tid] = a.B.K[tid];
        s_S[tid] = a.B.S[tid];
    }
    if (tid < P1) s_w[tid] = a.B.w[tid];
    __syncthreads();

    const int total = NN * nv;
    for (int it = tid; it < total; it += bs) {
        const int n = it / nv;
        const int v = it - n * nv;
        s_u[it] = gather_value<T>(a, s_idx[n], x, nv, v);
    }
    if (a.with_pot) {
        const double h3 = g.w * g.w * g.w;
        for (int n = tid; n < NN; n += bs) {
            const int ia = n % P1, ib = (n / P1) % P1, ic = n / (P1 * P1);
            const int idx = s_idx[n];
            // with_pot == 2: the field term E.r alone (the position operator);
            // with_pot == 3: E.force (the nuclear force along E)
            double f;
            if (a.with_pot == 3) {
                const double* F = idx >= 0 ? a.f_master + 3 * int64_t(idx) : a.f_hang + 3 * int64_t(-idx - 1);
                f = a.E[0] * F[0] + a.E[1] * F[1] + a.E[2] * F[2];
            } else {
                const double V = a.with_pot == 2 ? 0.0 : (idx >= 0 ? a.v_master[idx] : a.v_hang[-idx - 1]);
                const double px = g.x + g.w * a.B.xi[ia];
                const double py = g.y + g.w * a.B.xi[ib];
                const double pz = g.z + g.w * a.B.xi[ic];
                f = V + a.E[0] * px + a.E[1] * py + a.E[2] * pz;
            }
            s_pot[n] = h3 * s_w[ia] * s_w[ib] * s_w[ic] * f;
        }
    }
    __syncthreads();

    const double ck = a.c_kin * g.w;
    for (int it = tid; it < total; it += bs) {
        const int n = it / nv;
        const int v = it - n * nv;
        const int ia = n % P1, ib = (n / P1) % P1, ic = n / (P1 * P1);
        T ax = vzero<T>(), ay = vzero<T>(), az = vzero<T>();
#pragma unroll
        for (int m = 0; m < P1; ++m) {
            vfma(ax, s_K[ia * P1 + m], s_u[(m + P1 * (ib + P1 * ic)) * nv + v]);
            vfma(ay, s_K[ib * P1 + m], s_u[(ia + P1 * (m + P1 * ic)) * nv + v]);
            vfma(az, s_K[ic * P1 + m], s_u[(ia + P1 * (ib + P1 * m)) * nv + v]);
        }
        if constexpr (ECS) {
            double2 sx, sy, sz;
            ecs_factors(a.ecs, cell, sx, sy, sz);
            const double2 rk = ecs_kinetic(sx, sy, sz, ck * s_w[ib] * s_w[ic], ck * s_w[ia] * s_w[ic],
                                           ck * s_w[ia] * s_w[ib], ax, ay, az);
            double2 rp = make_double2(0.0, 0.0);
            if (a.with_pot) vfma(rp, s_pot[n], s_u[it]);
            scatter_ecs(a, s_idx[n], y, nv, v, rk, rp);
        } else {
            T r = vzero<T>();
            vfma(r, ck * s_w[ib] * s_w[ic], ax);
            vfma(r, ck * s_w[ia] * s_w[ic], ay);
            vfma(r, ck * s_w[ia] * s_w[ib], az);
            if (a.with_pot) vfma(r, s_pot[n], s_u[it]);
            if constexpr (VG) add_velocity_term(r, s_S, s_w, s_u, ia, ib, ic, nv, v, g.w * g.w, a.Avec, P1);
            scatter_value<T>(a, s_idx[n], y, nv, v, r);
        }
    }
}

// Packed orbital operator before projection and inverse mass (Eqs. orb_eom,
// discretized_eom):  z_p = H1~ v_p + C^T diag(m_f) sum_q (C U_pq) o (C v_q),
// for all n orbitals of one cell at once.  U: complex [N][n][n] nodal fields.
template <int P, bool VG = false, bool ECS = false>
__global__ void __launch_bounds__(256) g_cell_kernel(CellArgs a, const double2* __restrict__ v,
                                                     const double2* __restrict__ U, double2* __restrict__ z,
                                                     int n) {
    constexpr int P1 = P + 1;
    constexpr int NN = P1 * P1 * P1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* s_u = reinterpret_cast<double2*>(smem_raw);   // [NN][n]
    double2* s_U = s_u + NN * n;                            // [NN][n*n]
    __shared__ int s_idx[NN];
    __shared__ double s_pot[NN];
    __shared__ double s_wq[NN];
    __shared__ double s_K[P1 * P1];
    __shared__ double s_S[P1 * P1];
    __shared__ double s_w[P1];

    const int64_t cell = blockIdx.x;
    const int tid = threadIdx.x;
    const int bs = blockDim.x;
    const double4 g = a.geom[cell];
    for (int i = tid; i < NN; i += bs) s_idx[i] = a.cell_node[cell * NN + i];
    if (tid < P1 * P1) {
        s_K[tid] = a.B.K[tid];
        s_S[tid] = a.B.S[tid];
    }
    if (tid < P1) s_w[tid] = a.B.w[tid];
    __syncthreads();
    const int nn2 = n * n;
    for (int it = tid; it < NN * n; it += bs) {
        const int i = it / n, q = it - i * n;
        s_u[it] = gather_value<double2>(a, s_idx[i], v, n, q);
    }
    if (U) {
        CellArgs au = a;
        au.masked = 0;   // the mean fields are defined on all masters
        for (int it = tid; it < NN * nn2; it += bs) {
            const int i = it / nn2, pq = it - i * nn2;
            const int idx = s_idx[i];
            s_U[it] = (idx < 0 && a.u_hang) ? a.u_hang[int64_t(-idx - 1) * nn2 + pq]
                                            : gather_value<double2>(au, idx, U, nn2, pq);
        }
    }
    {
        const double h3 = g.w * g.w * g.w;
        for (int i = tid; i < NN; i += bs) {
            const int ia = i % P1, ib = (i / P1) % P1, ic = i / (P1 * P1);
            const int idx = s_idx[i];
            const double V = idx >= 0 ? a.v_master[idx] : a.v_hang[-idx - 1];
            const double px = g.x + g.w * a.B.xi[ia];
            const double py = g.y + g.w * a.B.xi[ib];
            const double pz = g.z + g.w * a.B.xi[ic];
            const double wq = h3 * s_w[ia] * s_w[ib] * s_w[ic];
            s_wq[i] = wq;
            s_pot[i] = wq * (V + a.E[0] * px + a.E[1] * py + a.E[2] * pz);
        }
    }
    __syncthreads();
    const double ck = 0.5 * g.w;
    for (int it = tid; it < NN * n; it += bs) {
        const int i = it / n, p = it - i * n;
        const int ia = i % P1, ib = (i / P1) % P1, ic = i / (P1 * P1);
        double2 ax = vzero<double2>(), ay = vzero<double2>(), az = vzero<double2>();
#pragma unroll
        for (int m = 0; m < P1; ++m) {
            vfma(ax, s_K[ia * P1 + m], s_u[(m + P1 * (ib + P1 * ic)) * n + p]);
            vfma(ay, s_K[ib * P1 + m], s_u[(ia + P1 * (m + P1 * ic)) * n + p]);
            vfma(az, s_K[ic * P1 + m], s_u[(ia + P1 * (ib + P1 * m)) * n + p]);
        }
        double2 r = vzero<double2>();
        double2 rk = vzero<double2>();
        if constexpr (ECS) {   // kinetic part apart (scaled at the scatter); r keeps the pointwise terms
            double2 sx, sy, sz;
            ecs_factors(a.ecs, cell, sx, sy, sz);
            rk = ecs_kinetic(sx, sy, sz, ck * s_w[ib] * s_w[ic], ck * s_w[ia] * s_w[ic], ck * s_w[ia] * s_w[ib], ax,
                             ay, az);
        } else {
            vfma(r, ck * s_w[ib] * s_w[ic], ax);
            vfma(r, ck * s_w[ia] * s_w[ic], ay);
            vfma(r, ck * s_w[ia] * s_w[ib], az);
        }
        vfma(r, s_pot[i], s_u[it]);
        if constexpr (VG) add_velocity_term(r, s_S, s_w, s_u, ia, ib, ic, n, p, g.w * g.w, a.Avec, P1);
        if (U) {
            double2 mf = vzero<double2>();
            const double2* Ui = s_U + i * nn2 + p * n;
            const double2* ui = s_u + i * n;
            for (int q = 0; q < n; ++q) {
                mf.x = fma(Ui[q].x, ui[q].x, fma(-Ui[q].y, ui[q].y, mf.x));
                mf.y = fma(Ui[q].x, ui[q].y, fma(Ui[q].y, ui[q].x, mf.y));
            }
            vfma(r, s_wq[i], mf);
        }
        if constexpr (ECS) scatter_ecs(a, s_idx[i], z, n, p, rk, r);
        else scatter_value<double2>(a, s_idx[i], z, n, p, r);
    }
}

// velocity != 0: E holds the vector potential A of the velocity gauge (the
// field term is then -i A . grad instead of E . r).
int launch_g_cell(const afem_mesh* m, const double* E, const double2* v, const double2* U, double2* z, int n,
                  cudaStream_t s, int velocity, const double2* U_hang) {
    CellArgs a = make_cell_args(m);
    a.u_hang = U ? U_hang : nullptr;
    a.c_kin = 0.5;
    a.with_pot = 1;
    a.masked = 1;
    for (int i = 0; i < 3; ++i) a.E[i] = (E && !velocity) ? E[i] : 0.0;
    if (velocity && m->ecs_on)
        return set_error(AFEM_EINVAL, "complex scaling is built for the length gauge");
    if (velocity && E) {
        a.vg = 1;
        for (int i = 0; i < 3; ++i) a.Avec[i] = E[i];
    }
    const int p = m->dev.p;
    const int nn = (p + 1) * (p + 1) * (p + 1);
    const size_t smem = size_t(nn) * n * sizeof(double2) + (U ? size_t(nn) * n * n * sizeof(double2) : 0);
    const unsigned grid = unsigned(m->dev.ncell);
    AFEM_CUDA_TRY(cudaMemsetAsync(z, 0, size_t(m->dev.n_master) * n * sizeof(double2), s));
    if (grid == 0) return AFEM_OK;
    switch (p) {
#define AFEM_CASE(PP)                                                                          \
    case PP: {                                                                                 \
        auto k = a.vg ? g_cell_kernel<PP, true> : g_cell_kernel<PP, false>;                    \
        if (m->ecs_on) k = g_cell_kernel<PP, false, true>;                                     \
        if (smem > 48 * 1024)                                                                  \
            AFEM_CUDA_TRY(allow_dyn_smem(k));                                    \
        AFEM_LAUNCH((k), grid, 256, smem, s, a, v, U, z, n);                                              \
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

template <typename T>
__global__ void scale_rows_kernel(T* __restrict__ y, const double* __restrict__ s, int64_t n, int nv) {
    const int64_t total = n * nv;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        y[i] = vscale(y[i], s[i / nv]);
    }
}

// ------------------------------------------------------------------ host
CellArgs make_cell_args(const afem_mesh* m) {
    CellArgs a{};
    const DeviceMesh& D = m->dev;
    a.cell_node = D.cell_node;
    a.geom = D.cell_geom;
    a.hp = D.hang_ptr;
    a.hm = D.hang_master;
    a.hw = D.hang_w;
    a.v_master = D.v_master;
    a.v_hang = D.v_hang;
    a.f_master = D.f_master;
    a.f_hang = D.f_hang;
    a.n_interior = D.n_interior;
    if (m->ecs_on) {
        a.ecs.flags = m->ecs_flags;
        a.ecs.rho = m->ecs_rho;
        for (int k = -2; k <= 3; ++k)
            a.ecs.e[k + 2] = make_double2(std::cos(k * m->ecs_theta), std::sin(k * m->ecs_theta));
    }
    const Basis1D& b = m->basis;
    const int p1 = b.p + 1;
    for (int i = 0; i < p1; ++i) {
        a.B.xi[i] = b.xi[i];
        a.B.w[i] = b.w[i];
        for (int j = 0; j < p1; ++j) {
            a.B.K[i * p1 + j] = b.K[i][j];
            a.B.S[i * p1 + j] = b.S[i][j];
        }
    }
    return a;
}

template <typename T>
static int launch_cell_op(const afem_mesh* m, const CellArgs& a, const T* x, T* y, int nv,
                          cudaStream_t s) {
    const int p = m->dev.p;
    const int p1 = p + 1;
    const size_t smem = size_t(p1) * p1 * p1 * nv * sizeof(T);
    const unsigned grid = unsigned(m->dev.ncell);
    if (grid == 0) return AFEM_OK;
    const int block = 256;
    switch (p) {
#define AFEM_CASE(PP)                                                                          \
    case PP: {                                                                                 \
        auto k = cell_op_kernel<PP, T, false>;                                                 \
        if constexpr (sizeof(T) == sizeof(double2)) {                                          \
            if (a.vg) k = cell_op_kernel<PP, T, true>;                                         \
            if (a.ecs.flags) k = cell_op_kernel<PP, T, false, true>;                           \
        }                                                                                      \
        if (smem > 48 * 1024)                                                                  \
            AFEM_CUDA_TRY(allow_dyn_smem(k));                                    \
        AFEM_LAUNCH((k), grid, block, smem, s, a, x, y, nv);                                              \
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

template <typename T>
static int launch_scale_rows(T* y, const double* s, int64_t n, int nv, cudaStream_t st) {
    if (n == 0) return AFEM_OK;
    const int64_t total = n * nv;
    const int block = 256;
    const unsigned grid = unsigned(std::min<int64_t>((total + block - 1) / block, int64_t(32) * device_sms()));
    AFEM_LAUNCH((scale_rows_kernel<T>), grid, block, 0, st, y, s, n, nv);
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

int launch_stiffness(const afem_mesh* m, const double* x, double* y, int nv, int masked, cudaStream_t s) {
    CellArgs a = make_cell_args(m);
    a.c_kin = 1.0;
    a.with_pot = 0;
    a.masked = masked;
    AFEM_CUDA_TRY(cudaMemsetAsync(y, 0, size_t(m->dev.n_master) * nv * sizeof(double), s));
    return launch_cell_op<double>(m, a, x, y, nv, s);
}

int launch_stiffness32(const afem_mesh* m, const float* x, float* y, int nv, int masked, cudaStream_t s,
                       double* pap_slots = nullptr);
int launch_g_cell32(const afem_mesh* m, const double* E, const float2* v, const float2* U, float2* z, int n,
                    cudaStream_t s, int velocity = 0, const float2* U_hang = nullptr);

int launch_op_apply(afem_mesh* m, int kind, const double* E, const void* x, void* y, int nv,
                    cudaStream_t s) {
    CellArgs a = make_cell_args(m);
    const int64_t N = m->dev.n_master;
    if (kind == AFEM_OP_H1) {
        a.c_kin = 0.5;
        a.with_pot = 1;
        a.masked = 1;
        for (int i = 0; i < 3; ++i) a.E[i] = E ? E[i] : 0.0;
        auto* yy = static_cast<double2*>(y);
        AFEM_CUDA_TRY(cudaMemsetAsync(yy, 0, size_t(N) * nv * sizeof(double2), s));
        int rc = launch_cell_op<double2>(m, a, static_cast<const double2*>(x), yy, nv, s);
        if (rc) return rc;
        return launch_scale_rows<double2>(yy, m->dev.ml_inv, N, nv, s);
    }
    if ((kind == AFEM_OP_H1_VG || kind == AFEM_OP_H1_VG_C64) && m->ecs_on)
        return set_error(AFEM_EINVAL, "afem_op_apply: complex scaling is built for the length gauge");
    if (kind == AFEM_OP_H1_VG) {   // velocity gauge: E holds A
        a.c_kin = 0.5;
        a.with_pot = 1;
        a.masked = 1;
        a.vg = E ? 1 : 0;
        for (int i = 0; i < 3; ++i) a.Avec[i] = E ? E[i] : 0.0;
        auto* yy = static_cast<double2*>(y);
        AFEM_CUDA_TRY(cudaMemsetAsync(yy, 0, size_t(N) * nv * sizeof(double2), s));
        int rc = launch_cell_op<double2>(m, a, static_cast<const double2*>(x), yy, nv, s);
        if (rc) return rc;
        return launch_scale_rows<double2>(yy, m->dev.ml_inv, N, nv, s);
    }
    if (kind == AFEM_OP_STIFF) {
        a.c_kin = 1.0;
        a.with_pot = 0;
        a.masked = 0;
        auto* yy = static_cast<double*>(y);
        AFEM_CUDA_TRY(cudaMemsetAsync(yy, 0, size_t(N) * nv * sizeof(double), s));
        return launch_cell_op<double>(m, a, static_cast<const double*>(x), yy, nv, s);
    }
    if (kind == AFEM_OP_POS || kind == AFEM_OP_FORCE) {   // y = M_L^-1 F[e.r] x or M_L^-1 F[e.force] x, masked
        a.c_kin = 0.0;
        a.with_pot = kind == AFEM_OP_POS ? 2 : 3;
        a.masked = 1;
        for (int i = 0; i < 3; ++i) a.E[i] = E ? E[i] : 0.0;
        auto* yy = static_cast<double2*>(y);
        AFEM_CUDA_TRY(cudaMemsetAsync(yy, 0, size_t(N) * nv * sizeof(double2), s));
        int rc = launch_cell_op<double2>(m, a, static_cast<const double2*>(x), yy, nv, s);
        if (rc) return rc;
        return launch_scale_rows<double2>(yy, m->dev.ml_inv, N, nv, s);
    }
    if (kind == AFEM_OP_STIFF_F32)
        return launch_stiffness32(m, static_cast<const float*>(x), static_cast<float*>(y), nv, 0, s);
    if (kind == AFEM_OP_H1_C64 || kind == AFEM_OP_H1_VG_C64) {
        auto* yy = static_cast<float2*>(y);
        int rc = launch_g_cell32(m, E, static_cast<const float2*>(x), nullptr, yy, nv, s, kind == AFEM_OP_H1_VG_C64);
        if (rc) return rc;
        return launch_scale_rows<float2>(yy, m->dev.ml_inv, N, nv, s);
    }
    return set_error(AFEM_EINVAL, "afem_op_apply: unknown operator kind");
}

}  // namespace afem
