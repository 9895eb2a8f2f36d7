// One-electron limit of the orbital step and its derivatives (Sec. 2 and
// Sec. 3.2 with one orbital and one configuration: the mean fields and the
// projector vanish, and the orbital equation is the time-dependent
// Schroedinger equation with the length-gauge H1~ of Sec. 3.1).
//
//   phi_{k+1} = P_k phi_k,   P_k = exp(-i dt H~(E_k)),   H~(E) = M_L^-1 H1~(E e)
//   d_k       = <phi_k, O phi_k>_M,  O = Z~ = M_L^-1 F[e.r] = dH~/dE (dipole) or
//               O = M_L^-1 F[e.f], f = -grad V (the potential part of the Ehrenfest acceleration)
//
// Derivatives with respect to the field samples E_k use the block identity
//   exp([[X, Y], [0, X]]) = [[exp X, L(X, Y)], [0, exp X]],
// L the Frechet derivative of exp at X in the direction Y.  With the packed
// G cell pass on two stacked vectors and the mean-field slot U_pq set to e.r
// (Eq. packed_orb_eom with n = 2 and no projector):
//   tangent:  exp(-i dt [[H~, v_k Z~], [0, H~]]) [dphi_k; phi_k] = [dphi_{k+1}; phi_{k+1}]
//   adjoint:  exp(+i dt [[H~, 0], [Z~, H~]]) [lam_{k+1}; 0] = [P_k^+ lam_{k+1}; L_k^+ lam_{k+1}]
// where ^+ is the adjoint in <.,.>_M; so each backward step is one Arnoldi
// propagation of a two-column vector, which yields both the propagated adjoint
// state and the field gradient dJ/dE_k = 2 Re <L_k^+ lam_{k+1}, phi_k>_M; the
// signal's operator O enters only the seeds g_k O phi_k of the adjoint state.
#include <vector>

#include "afem_internal.h"
#include "arnoldi.cuh"
#include "vec_common.cuh"

namespace afem {

// U[k] = [[0, c01 e.r_k], [c10 e.r_k, 0]] (complex128 [N][2][2]) from the
// master coordinates.
__global__ void fill_pos_field_kernel(double2* __restrict__ U, const double* __restrict__ xyz, double e0, double e1,
                                      double e2, double c01, double c10, int64_t n) {
    for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const double r = e0 * xyz[3 * k] + e1 * xyz[3 * k + 1] + e2 * xyz[3 * k + 2];
        U[4 * k + 0] = make_double2(0.0, 0.0);
        U[4 * k + 1] = make_double2(c01 * r, 0.0);
        U[4 * k + 2] = make_double2(c10 * r, 0.0);
        U[4 * k + 3] = make_double2(0.0, 0.0);
    }
}

// X[k] = [a[k][0] + g b[k], 0]: the next two-column adjoint state from the
// first column of the two-column a (null reads as 0) and the one-column b.
__global__ void adjoint_seed_kernel(double2* __restrict__ X, const double2* a, const double2* __restrict__ b,
                                    double g, int64_t n) {
    for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const double2 v = a ? a[2 * k] : make_double2(0.0, 0.0);
        const double2 w = b[k];
        X[2 * k] = make_double2(fma(g, w.x, v.x), fma(g, w.y, v.y));
        X[2 * k + 1] = make_double2(0.0, 0.0);
    }
}

namespace {

struct TdseWork {
    double2* X;       // [N][2] two-column state
    double2* Xn;      // [N][2]
    double2* Y;       // [N][2] Z~ applied to the state
    double2* U;       // [N][2][2] position field of the block operator
    double2* phis;    // [seg + 1][N] one recomputed segment (adjoint)
    double2* dots;    // [rows][4] inner products, read once at the end
    double2* part;    // reduction partials
    unsigned* cnt;    // reduction counter
};

int tdse_reserve(afem_mesh* m, int64_t dot_rows, int seg, TdseWork& w) {
    const size_t N = size_t(m->dev.n_master);
    auto carve = [&](Carver& cv) {
        w.X = cv.take<double2>(2 * N);
        w.Xn = cv.take<double2>(2 * N);
        w.Y = cv.take<double2>(2 * N);
        w.U = cv.take<double2>(4 * N);
        w.phis = cv.take<double2>(size_t(seg + 1) * N);
        w.dots = cv.take<double2>(size_t(dot_rows) * 4);
        w.part = cv.take<double2>(size_t(kRedBlocksMax) * 256);
        w.cnt = cv.take<unsigned>(4);
    };
    Carver measure(nullptr);
    carve(measure);
    int rc = m->ws_tdse.reserve(measure.size());
    if (rc) return rc;
    Carver cv(m->ws_tdse.ptr);
    carve(cv);
    return AFEM_OK;
}

struct Stepper {
    afem_mesh* m;
    double e[3];
    double dt, tol;
    int mk, mixed;
    cudaStream_t s;
    int obs;   // operator kind of the signal: AFEM_OP_POS (dipole) or AFEM_OP_FORCE
    int step(double Ek, const double2* in, const double2* U, int n, double2* out, int flags) const {
        const double E[3] = {Ek * e[0], Ek * e[1], Ek * e[2]};
        return arnoldi_step(m, E, in, U, nullptr, n, mk, dt, mixed, tol, out, nullptr, nullptr, nullptr, nullptr, s,
                            flags | kArnNoProjector);
    }
    // y = O x for nv columns of x, O the signal's operator (Z~ for the dipole)
    int pos(const double2* x, double2* y, int nv) const { return launch_op_apply(m, obs, e, x, y, nv, s); }
};

int check_common(afem_mesh* m, const double* e_dir, const double* E, int K, double dt, int mk, double tol,
                 int precision, int observable, const char* who) {
    const std::string w(who);
    if (observable != AFEM_OP_POS && observable != AFEM_OP_FORCE)
        return set_error(AFEM_EINVAL, w + ": observable must be AFEM_OP_POS or AFEM_OP_FORCE");
    if (!m || !e_dir || (K > 0 && !E)) return set_error(AFEM_EINVAL, w + ": null argument");
    if (m->ecs_on)   // the adjoint sweep takes the operator as self-adjoint, which complex scaling breaks
        return set_error(AFEM_EINVAL, w + ": not built for a complex-scaled mesh");
    if (K < 0) return set_error(AFEM_EINVAL, w + ": n_steps must be >= 0");
    if (!(dt > 0.0)) return set_error(AFEM_EINVAL, w + ": dt must be > 0");
    if (mk < 1 || mk > kMaxKrylov) return set_error(AFEM_EINVAL, w + ": krylov_m must be 1..16");
    if (!(tol >= 0.0)) return set_error(AFEM_EINVAL, w + ": tol must be >= 0");
    if (precision != AFEM_PREC_FP64 && precision != AFEM_PREC_MIXED)
        return set_error(AFEM_EINVAL, w + ": unknown precision");
    if (m->host_only) return set_error(AFEM_EINVAL, w + ": mesh was built host-only");
    return AFEM_OK;
}

}  // namespace

int tdse_forward(afem_mesh* m, const double* e_dir, const double* E, int K, double dt, int mk, double tol,
                 int precision, int observable, const double2* phi0, double2* phi_end, double* d, double2* ckpt,
                 int every, cudaStream_t s) {
    int rc = check_common(m, e_dir, E, K, dt, mk, tol, precision, observable, "afem_tdse_forward");
    if (rc) return rc;
    if (!phi0 || !d) return set_error(AFEM_EINVAL, "afem_tdse_forward: null argument");
    if (ckpt && every < 1) return set_error(AFEM_EINVAL, "afem_tdse_forward: checkpoint interval must be >= 1");
    const DeviceMesh& D = m->dev;
    const int64_t N = D.n_master;
    TdseWork w{};
    if ((rc = tdse_reserve(m, int64_t(K) + 1, 1, w))) return rc;
    AFEM_CUDA_TRY(cudaMemsetAsync(w.cnt, 0, 4 * sizeof(unsigned), s));
    const Stepper st{m, {e_dir[0], e_dir[1], e_dir[2]}, dt, tol, mk, precision == AFEM_PREC_MIXED, s, observable};
    double2* cur = w.phis;        // ping-pong between the two segment slots
    double2* nxt = w.phis + N;
    AFEM_CUDA_TRY(cudaMemcpyAsync(cur, phi0, N * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    for (int k = 0;; ++k) {
        if (ckpt && k < K && k % every == 0)
            AFEM_CUDA_TRY(cudaMemcpyAsync(ckpt + int64_t(k / every) * N, cur, N * sizeof(double2),
                                          cudaMemcpyDeviceToDevice, s));
        // d_k = <phi_k, O phi_k>_M
        if ((rc = st.pos(cur, w.Y, 1))) return rc;
        if ((rc = cdot(cur, 1, w.Y, 1, D.ml, D.n_interior, 0, w.part, w.dots + k, w.cnt, s))) return rc;
        if (k == K) break;
        if ((rc = st.step(E[k], cur, nullptr, 1, nxt, 0))) return rc;
        std::swap(cur, nxt);
    }
    if (phi_end) AFEM_CUDA_TRY(cudaMemcpyAsync(phi_end, cur, N * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    std::vector<double2> h(size_t(K) + 1);
    AFEM_CUDA_TRY(cudaMemcpyAsync(h.data(), w.dots, h.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
    AFEM_CUDA_TRY(cudaStreamSynchronize(s));
    for (int k = 0; k <= K; ++k) d[k] = h[k].x;
    return AFEM_OK;
}

int tdse_jvp(afem_mesh* m, const double* e_dir, const double* E, int K, double dt, int mk, double tol,
             int precision, int observable, const double2* phi0, const double* v, double* d, double* dd,
             cudaStream_t s) {
    int rc = check_common(m, e_dir, E, K, dt, mk, tol, precision, observable, "afem_tdse_jvp");
    if (rc) return rc;
    if (!phi0 || (K > 0 && !v) || !d || !dd) return set_error(AFEM_EINVAL, "afem_tdse_jvp: null argument");
    const DeviceMesh& D = m->dev;
    const int64_t N = D.n_master;
    TdseWork w{};
    if ((rc = tdse_reserve(m, int64_t(K) + 1, 0, w))) return rc;
    AFEM_CUDA_TRY(cudaMemsetAsync(w.cnt, 0, 4 * sizeof(unsigned), s));
    const Stepper st{m, {e_dir[0], e_dir[1], e_dir[2]}, dt, tol, mk, precision == AFEM_PREC_MIXED, s, observable};
    // [dphi_0; phi_0] = [0; phi_0]
    AFEM_CUDA_TRY(cudaMemsetAsync(w.X, 0, 2 * N * sizeof(double2), s));
    AFEM_CUDA_TRY(cudaMemcpy2DAsync(w.X + 1, 2 * sizeof(double2), phi0, sizeof(double2), sizeof(double2), N,
                                    cudaMemcpyDeviceToDevice, s));
    double2* cur = w.X;
    double2* nxt = w.Xn;
    for (int k = 0;; ++k) {
        // S[a][b] = <X_a, O X_b>_M: d_k = S[1][1], dd_k = 2 Re S[0][1]
        if ((rc = st.pos(cur, w.Y, 2))) return rc;
        if ((rc = cdot(cur, 2, w.Y, 2, D.ml, D.n_interior, 0, w.part, w.dots + 4 * int64_t(k), w.cnt, s))) return rc;
        if (k == K) break;
        AFEM_LAUNCH((fill_pos_field_kernel), grid_for(N), 256, 0, s, w.U, D.master_xyz, st.e[0], st.e[1], st.e[2],
                    v[k], 0.0, N);
        AFEM_CUDA_TRY(cudaGetLastError());
        if ((rc = st.step(E[k], cur, w.U, 2, nxt, 0))) return rc;
        std::swap(cur, nxt);
    }
    std::vector<double2> h(4 * (size_t(K) + 1));
    AFEM_CUDA_TRY(cudaMemcpyAsync(h.data(), w.dots, h.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
    AFEM_CUDA_TRY(cudaStreamSynchronize(s));
    for (int k = 0; k <= K; ++k) {
        d[k] = h[4 * k + 3].x;
        dd[k] = 2.0 * h[4 * k + 1].x;
    }
    return AFEM_OK;
}

int tdse_vjp(afem_mesh* m, const double* e_dir, const double* E, int K, double dt, int mk, double tol,
             int precision, int observable, const double2* ckpt, int every, const double* g, double* grad_E,
             double2* lam0, cudaStream_t s) {
    int rc = check_common(m, e_dir, E, K, dt, mk, tol, precision, observable, "afem_tdse_vjp");
    if (rc) return rc;
    if (K < 1) return set_error(AFEM_EINVAL, "afem_tdse_vjp: n_steps must be >= 1");
    if (!ckpt || !g || !grad_E) return set_error(AFEM_EINVAL, "afem_tdse_vjp: null argument");
    if (every < 1) return set_error(AFEM_EINVAL, "afem_tdse_vjp: checkpoint interval must be >= 1");
    const DeviceMesh& D = m->dev;
    const int64_t N = D.n_master;
    const int seg = every < K ? every : K;
    TdseWork w{};
    if ((rc = tdse_reserve(m, 2 * int64_t(K), seg, w))) return rc;
    AFEM_CUDA_TRY(cudaMemsetAsync(w.cnt, 0, 4 * sizeof(unsigned), s));
    const Stepper st{m, {e_dir[0], e_dir[1], e_dir[2]}, dt, tol, mk, precision == AFEM_PREC_MIXED, s, observable};
    // [[H~, 0], [Z~, H~]]: the position field in slot (1, 0), the same for every step
    AFEM_LAUNCH((fill_pos_field_kernel), grid_for(N), 256, 0, s, w.U, D.master_xyz, st.e[0], st.e[1], st.e[2], 0.0,
                1.0, N);
    AFEM_CUDA_TRY(cudaGetLastError());
    double2* zphi = w.Y;   // Z~ phi_j (one column)
    const int n_seg = (K + every - 1) / every;
    for (int sg = n_seg - 1; sg >= 0; --sg) {
        const int a = sg * every;
        const int b = a + every < K ? a + every : K;
        // recompute phi_a..phi_b from the checkpoint (the forward's values up to
        // the order of the cell passes' atomic sums)
        AFEM_CUDA_TRY(cudaMemcpyAsync(w.phis, ckpt + int64_t(sg) * N, N * sizeof(double2), cudaMemcpyDeviceToDevice,
                                      s));
        for (int j = a; j < b; ++j)
            if ((rc = st.step(E[j], w.phis + int64_t(j - a) * N, nullptr, 1, w.phis + int64_t(j - a + 1) * N, 0)))
                return rc;
        if (b == K) {   // lam_K = g_K Z~ phi_K
            if ((rc = st.pos(w.phis + int64_t(b - a) * N, zphi, 1))) return rc;
            AFEM_LAUNCH((adjoint_seed_kernel), grid_for(N), 256, 0, s, w.X, nullptr, zphi, g[K], N);
            AFEM_CUDA_TRY(cudaGetLastError());
        }
        for (int j = b - 1; j >= a; --j) {
            const double2* phij = w.phis + int64_t(j - a) * N;
            if ((rc = st.step(E[j], w.X, w.U, 2, w.Xn, kArnBackward))) return rc;
            // <L_j^+ lam_{j+1}, phi_j>_M in slot 1 of the pair
            if ((rc = cdot(w.Xn, 2, phij, 1, D.ml, D.n_interior, 0, w.part, w.dots + 2 * int64_t(j), w.cnt, s)))
                return rc;
            // lam_j = P_j^+ lam_{j+1} + g_j O phi_j
            if ((rc = st.pos(phij, zphi, 1))) return rc;
            AFEM_LAUNCH((adjoint_seed_kernel), grid_for(N), 256, 0, s, w.X, w.Xn, zphi, g[j], N);
            AFEM_CUDA_TRY(cudaGetLastError());
        }
    }
    if (lam0)
        AFEM_CUDA_TRY(cudaMemcpy2DAsync(lam0, sizeof(double2), w.X, 2 * sizeof(double2), sizeof(double2), N,
                                        cudaMemcpyDeviceToDevice, s));
    std::vector<double2> h(2 * size_t(K));
    AFEM_CUDA_TRY(cudaMemcpyAsync(h.data(), w.dots, h.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
    AFEM_CUDA_TRY(cudaStreamSynchronize(s));
    for (int j = 0; j < K; ++j) grad_E[j] = 2.0 * h[2 * j + 1].x;
    return AFEM_OK;
}

}  // namespace afem
