// Exterior complex scaling of the kinetic energy (Sec. 4 absorbs the outgoing
// flux by ECS outside an inner box, [-35,35] x [-10,10] x [-10,10] in its water
// run; the construction itself is left to the cited literature).
//
// Reading built here: Cartesian scaling with a sharp onset at the faces of the
// inner box |x_d| <= R_d, x_d -> +-R_d + e^{i theta} (x_d -+ R_d) outside.  The
// mesh has to keep every cell wholly inside or outside the box along each axis
// (the box faces lie on cell faces).  A cell scaled along the axes with flag
// f_d = 1 has eta_d = e^{i theta f_d} and J = prod_d eta_d; in the weak form its
// stiffness becomes h sum_d (J / eta_d^2) (d-th Kronecker term) and its mass
// J h^3 W (x) W (x) W.  With M_theta = C^T (J m_f) the kinetic operator on nodal
// vectors is 1/2 M_theta^-1 A_theta; the pointwise terms (nuclear potential,
// E . r, mean fields) keep their real weights and the orbital inner product
// stays u^H M_L v.  The cell kernels form the scaled stiffness per cell and
// scatter it multiplied by rho = M_L / M_theta per master, so that the common
// M_L^-1 that follows yields M_theta^-1 A_theta.
//
// This file holds the host set-up: per-cell axis flags and rho per master.
#include <cmath>
#include <complex>
#include <vector>

#include "afem_internal.h"

namespace afem {

void mesh_free_ecs(afem_mesh* m) {
    cudaFree(m->ecs_flags);
    cudaFree(m->ecs_rho);
    cudaFree(m->ecs_rho32);
    m->ecs_flags = nullptr;
    m->ecs_rho = nullptr;
    m->ecs_rho32 = nullptr;
    m->ecs_on = 0;
    m->ecs_theta = 0.0;
    for (double& r : m->ecs_half_width) r = 0.0;
}

template <typename T>
static int upload_ecs(T*& dst, const std::vector<T>& v) {
    cudaError_t e = cudaMalloc(&dst, v.size() * sizeof(T));
    if (e != cudaSuccess) {
        dst = nullptr;
        return set_error(AFEM_ENOMEM, "afem_mesh_set_ecs: cudaMalloc failed");
    }
    AFEM_CUDA_TRY(cudaMemcpy(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return AFEM_OK;
}

int mesh_set_ecs(afem_mesh* m, double theta, const double half_width[3]) {
    if (!(theta >= 0.0) || !(theta < 0.5 * M_PI))
        return set_error(AFEM_EINVAL, "afem_mesh_set_ecs: theta must lie in [0, pi/2)");
    if (theta == 0.0) {
        mesh_free_ecs(m);
        return AFEM_OK;
    }
    if (!half_width) return set_error(AFEM_EINVAL, "afem_mesh_set_ecs: null half widths");
    for (int d = 0; d < 3; ++d)
        if (!(half_width[d] > 0.0) || !std::isfinite(half_width[d]))
            return set_error(AFEM_EINVAL, "afem_mesh_set_ecs: half widths must be positive");
    const HostMesh& H = m->host;
    const int64_t ncell = int64_t(H.lev.size());
    const int p1 = H.p + 1;
    const int nn = p1 * p1 * p1;
    const double tol = 1e-9 * (H.hi - H.lo);
    // the axes along which each cell lies outside the inner box
    std::vector<uint8_t> flags(size_t(ncell), 0);
    for (int64_t c = 0; c < ncell; ++c) {
        for (int d = 0; d < 3; ++d) {
            const double lo = H.corner[3 * c + d], hi = lo + H.h[c], R = half_width[d];
            const bool inside = lo >= -R - tol && hi <= R + tol;
            const bool outside = lo >= R - tol || hi <= -R + tol;
            if (!inside && !outside)
                return set_error(AFEM_EMESH, "afem_mesh_set_ecs: a face of the scaling box cuts a cell");
            if (outside) flags[size_t(c)] |= uint8_t(1u << d);
        }
    }
    // M_theta = C^T (J m_f): each cell's GLL weights times its Jacobian, through
    // the constraints; masters that no scaled cell touches keep rho = 1 exactly
    const std::complex<double> eta = std::polar(1.0, theta);
    std::vector<std::complex<double>> Mt(size_t(H.n_master), 0.0);
    std::vector<uint8_t> touched(size_t(H.n_master), 0);
    const Basis1D& B = m->basis;
    for (int64_t c = 0; c < ncell; ++c) {
        const int f = flags[size_t(c)];
        const int k = (f & 1) + ((f >> 1) & 1) + ((f >> 2) & 1);
        const std::complex<double> J = std::pow(eta, k);
        const double h3 = H.h[c] * H.h[c] * H.h[c];
        for (int i = 0; i < nn; ++i) {
            const int ia = i % p1, ib = (i / p1) % p1, ic = i / (p1 * p1);
            const std::complex<double> wq = h3 * B.w[ia] * B.w[ib] * B.w[ic] * J;
            const int32_t idx = H.cell_node[size_t(c) * nn + i];
            if (idx >= 0) {
                Mt[size_t(idx)] += wq;
                if (f) touched[size_t(idx)] = 1;
            } else {
                const int32_t h = -idx - 1;
                for (int32_t e = H.hang_ptr[h]; e < H.hang_ptr[h + 1]; ++e) {
                    Mt[size_t(H.hang_master[e])] += H.hang_w[e] * wq;
                    if (f) touched[size_t(H.hang_master[e])] = 1;
                }
            }
        }
    }
    std::vector<double2> rho(size_t(H.n_master));
    std::vector<float2> rho32(size_t(H.n_master));
    for (int64_t i = 0; i < H.n_master; ++i) {
        std::complex<double> r = 1.0;
        if (touched[size_t(i)]) r = H.ml[size_t(i)] / Mt[size_t(i)];
        rho[size_t(i)] = make_double2(r.real(), r.imag());
        rho32[size_t(i)] = make_float2(float(r.real()), float(r.imag()));
    }
    mesh_free_ecs(m);
    int rc;
    if ((rc = upload_ecs(m->ecs_flags, flags)) || (rc = upload_ecs(m->ecs_rho, rho)) ||
        (rc = upload_ecs(m->ecs_rho32, rho32))) {
        mesh_free_ecs(m);
        return rc;
    }
    m->ecs_on = 1;
    m->ecs_theta = theta;
    for (int d = 0; d < 3; ++d) m->ecs_half_width[d] = half_width[d];
    return AFEM_OK;
}

}  // namespace afem
