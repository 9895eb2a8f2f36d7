// Batched Poisson solves for the pair mean fields (Sec. 3.1, Eq. mean-field).
//
// Delta W^r_s = -4 pi phi_r^* phi_s with Dirichlet data equal to the direct
// integral on the box surface.  Weak form with GLL quadrature:
//     A W = 4 pi C^T (m_f o rho_f),  rho_f = conj(phi_r) phi_s at all support points,
// solved on the interior masters with the surface masters fixed to g.  The
// surface data is the direct integral as a multipole expansion about the box
// centre, l <= 12 (the paper leaves the evaluation open):
//     g(x) = sum_lm 4 pi/(2l+1) q_lm R_lm(x) / r^(2l+1),
//     q_lm = sum_f m_f rho_f R_lm(x_f),   R_lm = r^l Y_lm (real, orthonormal Y).
// All n^2 real right-hand sides (|phi_r|^2, and Re / Im of conj(phi_r) phi_s
// for r < s) are solved together by Jacobi-preconditioned CG (the paper uses
// CG with algebraic multigrid from Trilinos); each column has its own alpha,
// beta and stopping test ||r|| <= rtol ||b - A_IB g||.
#include <cmath>
#include <vector>

#include "afem_internal.h"
#include "cell_common.cuh"
#include "vec_common.cuh"

namespace afem {

constexpr int kLmax = 12;
constexpr int kNlm = (kLmax + 1) * (kLmax + 1);
constexpr int kMomTile = 32;
constexpr int kMomBlocks = 152 * 2;
__constant__ double c_sh_norm[kNlm];       // factor applied to C_lm / S_lm at index l*l + l + |m|
__constant__ double c_sh_irreg[kLmax + 1];  // 4 pi / (2l + 1)

static int ensure_sh_tables() {
    static bool done[64] = {false};
    int dev = 0;
    AFEM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 64 && done[dev]) return AFEM_OK;
    double norm[kNlm], irr[kLmax + 1];
    for (int l = 0; l <= kLmax; ++l) {
        irr[l] = 4.0 * M_PI / (2 * l + 1);
        for (int m = -l; m <= l; ++m) {
            const int am = m < 0 ? -m : m;
            double ratio = 1.0;   // (l-|m|)! / (l+|m|)!
            for (int t = l - am + 1; t <= l + am; ++t) ratio /= t;
            double N = std::sqrt((2 * l + 1) / (4.0 * M_PI) * ratio);
            norm[l * l + l + m] = am == 0 ? N : std::sqrt(2.0) * N;
        }
    }
    AFEM_CUDA_TRY(cudaMemcpyToSymbol(c_sh_norm, norm, sizeof(norm)));
    AFEM_CUDA_TRY(cudaMemcpyToSymbol(c_sh_irreg, irr, sizeof(irr)));
    if (dev < 64) done[dev] = true;
    return AFEM_OK;
}

// Real regular solid harmonics R[l*l + l + m] = r^l Y_lm(x^), l <= kLmax.
// With C_lm + i S_lm = r^l P_l^m(cos t) e^{i m p}:
//   C_mm + i S_mm = -(2m-1) (x + i y) (C_{m-1,m-1} + i S_{m-1,m-1}),
//   C_{m+1,m} = (2m+1) z C_mm,
//   C_lm = ((2l-1) z C_{l-1,m} - (l+m-1) r^2 C_{l-2,m}) / (l - m),
// and Y_l0 = N_l0 C_l0, Y_lm = sqrt2 N_lm C_lm, Y_l,-m = sqrt2 N_lm S_lm.
__device__ void regular_solid_harmonics(double x, double y, double z, double* R) {
    const double r2 = x * x + y * y + z * z;
    double cmm = 1.0, smm = 0.0;
    for (int m = 0; m <= kLmax; ++m) {
        double c2 = 0.0, s2 = 0.0, c1 = cmm, s1 = smm;
        {
            const int i = m * m + m;
            R[i + m] = c_sh_norm[i + m] * cmm;
            if (m > 0) R[i - m] = c_sh_norm[i + m] * smm;
        }
        for (int l = m + 1; l <= kLmax; ++l) {
            double c, s;
            if (l == m + 1) {
                c = (2 * m + 1) * z * c1;
                s = (2 * m + 1) * z * s1;
            } else {
                c = ((2 * l - 1) * z * c1 - (l + m - 1) * r2 * c2) / (l - m);
                s = ((2 * l - 1) * z * s1 - (l + m - 1) * r2 * s2) / (l - m);
            }
            const int i = l * l + l;
            R[i + m] = c_sh_norm[i + m] * c;
            if (m > 0) R[i - m] = c_sh_norm[i + m] * s;
            c2 = c1;
            s2 = s1;
            c1 = c;
            s1 = s;
        }
        const double nc = -(2 * m + 1) * (x * cmm - y * smm);
        const double ns = -(2 * m + 1) * (x * smm + y * cmm);
        cmm = nc;
        smm = ns;
    }
}

// One order m of the same harmonics (l = m..kLmax): C_mm, S_mm by the same
// recurrence in m, then the recurrence in l; lets several threads share a point.
__device__ void solid_harmonics_order(double x, double y, double z, int m, double* R) {
    const double r2 = x * x + y * y + z * z;
    double cmm = 1.0, smm = 0.0;
    for (int q = 0; q < m; ++q) {
        const double nc = -(2 * q + 1) * (x * cmm - y * smm);
        const double ns = -(2 * q + 1) * (x * smm + y * cmm);
        cmm = nc;
        smm = ns;
    }
    double c2 = 0.0, s2 = 0.0, c1 = cmm, s1 = smm;
    {
        const int i = m * m + m;
        R[i + m] = c_sh_norm[i + m] * cmm;
        if (m > 0) R[i - m] = c_sh_norm[i + m] * smm;
    }
    for (int l = m + 1; l <= kLmax; ++l) {
        double c, s;
        if (l == m + 1) {
            c = (2 * m + 1) * z * c1;
            s = (2 * m + 1) * z * s1;
        } else {
            c = ((2 * l - 1) * z * c1 - (l + m - 1) * r2 * c2) / (l - m);
            s = ((2 * l - 1) * z * s1 - (l + m - 1) * r2 * s2) / (l - m);
        }
        const int i = l * l + l;
        R[i + m] = c_sh_norm[i + m] * c;
        if (m > 0) R[i - m] = c_sh_norm[i + m] * s;
        c2 = c1;
        s2 = s1;
        c1 = c;
        s1 = s;
    }
}

// Column c of the pair-density right-hand sides from orbital values at one point.
// Order: c < n: |phi_c|^2; then for r < s: Re(conj(phi_r) phi_s), Im(...).
__device__ __forceinline__ void pair_columns(const double2* ph, int n, double* rho) {
    for (int r = 0; r < n; ++r) rho[r] = ph[r].x * ph[r].x + ph[r].y * ph[r].y;
    int c = n;
    for (int r = 0; r < n; ++r)
        for (int s = r + 1; s < n; ++s) {
            rho[c++] = ph[r].x * ph[s].x + ph[r].y * ph[s].y;
            rho[c++] = ph[r].x * ph[s].y - ph[r].y * ph[s].x;
        }
}

struct PointArgs {
    const double2* phi;     // [N][n]
    int n;
    int ncol;
    int64_t N, n_int, nh;
    const double* xyz_m;    // [N][3]
    const double* xyz_h;    // [nh][3]
    const double* mf_m;
    const double* mf_h;
    const int32_t* hp;
    const int32_t* hm;
    const double* hw;
    double cx, cy, cz;      // expansion centre
};

// RHS b = 4 pi C^T (m_f o rho) (atomics into zeroed b) and per-block moment partials.
__global__ void __launch_bounds__(256) pair_rhs_moments_kernel(PointArgs a, double* __restrict__ b,
                                                               double* __restrict__ qpart) {
    extern __shared__ __align__(16) double smem_d[];
    double* s_R = smem_d;                          // [kMomTile][kNlm]
    double* s_w = s_R + kMomTile * kNlm;           // [kMomTile][ncol]
    double* s_Q = s_w + kMomTile * a.ncol;         // [kNlm][ncol]
    __shared__ double4 s_pt[kMomTile];             // point relative to the centre, valid flag
    const int ncol = a.ncol;
    const int tid = threadIdx.x;
    for (int o = tid; o < kNlm * ncol; o += blockDim.x) s_Q[o] = 0.0;
    const int64_t npts = a.N + a.nh;
    const int64_t ntiles = (npts + kMomTile - 1) / kMomTile;
    double2 ph[8];
    double rho[64];
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        if (tid < kMomTile) {
            const int64_t f = tile * kMomTile + tid;
            double* Rrow = s_R + tid * kNlm;
            double* wrow = s_w + tid * ncol;
            if (f < npts) {
                double mf, x, y, z;
                if (f < a.N) {
                    const bool inner = f < a.n_int;
                    for (int r = 0; r < a.n; ++r)
                        ph[r] = inner ? a.phi[f * a.n + r] : make_double2(0.0, 0.0);
                    mf = a.mf_m[f];
                    x = a.xyz_m[3 * f];
                    y = a.xyz_m[3 * f + 1];
                    z = a.xyz_m[3 * f + 2];
                } else {
                    const int64_t h = f - a.N;
                    for (int r = 0; r < a.n; ++r) ph[r] = make_double2(0.0, 0.0);
                    for (int e = a.hp[h]; e < a.hp[h + 1]; ++e) {
                        const int m = a.hm[e];
                        if (m >= a.n_int) continue;
                        for (int r = 0; r < a.n; ++r) vfma(ph[r], a.hw[e], a.phi[int64_t(m) * a.n + r]);
                    }
                    mf = a.mf_h[h];
                    x = a.xyz_h[3 * h];
                    y = a.xyz_h[3 * h + 1];
                    z = a.xyz_h[3 * h + 2];
                }
                pair_columns(ph, a.n, rho);
                for (int c = 0; c < ncol; ++c) wrow[c] = mf * rho[c];
                // right-hand side through C^T
                const double fpi = 4.0 * M_PI;
                if (!b) {
                    // moments only
                } else if (f < a.N) {
                    for (int c = 0; c < ncol; ++c) atomicAdd(&b[f * ncol + c], fpi * wrow[c]);
                } else {
                    const int64_t h = f - a.N;
                    for (int e = a.hp[h]; e < a.hp[h + 1]; ++e) {
                        const int64_t m = a.hm[e];
                        for (int c = 0; c < ncol; ++c) atomicAdd(&b[m * ncol + c], fpi * a.hw[e] * wrow[c]);
                    }
                }
                s_pt[tid] = make_double4(x - a.cx, y - a.cy, z - a.cz, 1.0);
            } else {
                for (int c = 0; c < ncol; ++c) wrow[c] = 0.0;
                s_pt[tid] = make_double4(0.0, 0.0, 0.0, 0.0);
            }
            (void)Rrow;
        }
        __syncthreads();
        // harmonics of the tile: 8 threads per point, orders m and m + 8
        for (int it = tid; it < kMomTile * 8; it += blockDim.x) {
            const int tp = it >> 3, j = it & 7;
            const double4 q = s_pt[tp];
            double* Rr = s_R + tp * kNlm;
            for (int m = j; m <= kLmax; m += 8) {
                if (q.w != 0.0) {
                    solid_harmonics_order(q.x, q.y, q.z, m, Rr);
                } else {
                    for (int l = m; l <= kLmax; ++l) {
                        Rr[l * l + l + m] = 0.0;
                        if (m > 0) Rr[l * l + l - m] = 0.0;
                    }
                }
            }
        }
        __syncthreads();
        for (int o = tid; o < kNlm * ncol; o += blockDim.x) {
            const int lm = o / ncol, c = o - lm * ncol;
            double acc = s_Q[o];
            for (int t = 0; t < kMomTile; ++t) acc = fma(s_R[t * kNlm + lm], s_w[t * ncol + c], acc);
            s_Q[o] = acc;
        }
    }
    __syncthreads();
    for (int o = tid; o < kNlm * ncol; o += blockDim.x) qpart[int64_t(blockIdx.x) * kNlm * ncol + o] = s_Q[o];
}

__global__ void finalize_columns_kernel(const double* __restrict__ partial, int nblk, int k,
                                        double* __restrict__ out) {
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double acc = 0.0;
        for (int b = 0; b < nblk; ++b) acc += partial[int64_t(b) * k + c];
        out[c] = acc;
    }
}

// Dirichlet data g at the surface masters from the moments; written into x.
__global__ void multipole_bc_kernel(const double* __restrict__ q, int ncol, const double* __restrict__ xyz,
                                    int64_t n_int, int64_t N, double cx, double cy, double cz,
                                    double* __restrict__ x) {
    extern __shared__ __align__(16) double s_q[];   // [kNlm][ncol]
    for (int o = threadIdx.x; o < kNlm * ncol; o += blockDim.x) s_q[o] = q[o];
    __syncthreads();
    double R[kNlm];
    for (int64_t k = n_int + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < N;
         k += int64_t(gridDim.x) * blockDim.x) {
        const double dx = xyz[3 * k] - cx, dy = xyz[3 * k + 1] - cy, dz = xyz[3 * k + 2] - cz;
        regular_solid_harmonics(dx, dy, dz, R);
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double rinv = 1.0 / sqrt(r2);
        double fac[kLmax + 1];
        double t = rinv;                      // 1 / r^(2l+1)
        for (int l = 0; l <= kLmax; ++l) {
            fac[l] = c_sh_irreg[l] * t;
            t *= rinv * rinv;
        }
        for (int c = 0; c < ncol; ++c) {
            double g = 0.0;
            for (int l = 0; l <= kLmax; ++l) {
                double gl = 0.0;
                for (int m = -l; m <= l; ++m) {
                    const int i = l * l + l + m;
                    gl = fma(s_q[i * ncol + c], R[i], gl);
                }
                g = fma(fac[l], gl, g);
            }
            x[k * ncol + c] = g;
        }
    }
}

// ----------------------------------------------------------------- PCG
struct PcgState {
    double* alpha;   // [k]
    double* beta;
    double* rz;
    double* bb;      // ||b_eff||^2
    double* rr;
    int* active;     // [k]
    int* n_active;   // [1]
    double rtol2;
};

// Column partial sums of a*b over interior rows: partial[block][c].
__global__ void col_dot_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n, int k,
                               double* __restrict__ partial) {
    __shared__ double s[kRedThreads];
    const int R = kRedThreads / k, used = R * k;
    const int t = threadIdx.x;
    double acc = 0.0;
    if (t < used) {
        const int c = t % k, r = t / k;
        for (int64_t i = int64_t(blockIdx.x) * R + r; i < n; i += int64_t(gridDim.x) * R)
            acc = fma(a[i * k + c], b[i * k + c], acc);
    }
    s[t] = acc;
    reduce_columns(s, k, R, partial + int64_t(blockIdx.x) * k);
}

// r = b - t - Ap0 (interior rows), z = Dinv r, p = z; partials of (b-t)^2, r.z, r.r.
__global__ void pcg_init_kernel(const double* __restrict__ b, const double* __restrict__ t,
                                const double* __restrict__ Ax, const double* __restrict__ dinv,
                                double* __restrict__ r, double* __restrict__ z, double* __restrict__ p,
                                int64_t n, int k, double* __restrict__ partial /*[blk][3k]*/) {
    __shared__ double s[kRedThreads];
    const int R = kRedThreads / k, used = R * k;
    const int tid = threadIdx.x;
    double abb = 0.0, arz = 0.0, arr = 0.0;
    if (tid < used) {
        const int c = tid % k, rr0 = tid / k;
        for (int64_t i = int64_t(blockIdx.x) * R + rr0; i < n; i += int64_t(gridDim.x) * R) {
            const int64_t o = i * k + c;
            const double be = b[o] - t[o];
            const double ri = be - Ax[o];
            const double zi = dinv[i] * ri;
            r[o] = ri;
            z[o] = zi;
            p[o] = zi;
            abb = fma(be, be, abb);
            arz = fma(ri, zi, arz);
            arr = fma(ri, ri, arr);
        }
    }
    double* out = partial + int64_t(blockIdx.x) * 3 * k;
    s[tid] = abb;
    reduce_columns(s, k, R, out);
    __syncthreads();
    s[tid] = arz;
    reduce_columns(s, k, R, out + k);
    __syncthreads();
    s[tid] = arr;
    reduce_columns(s, k, R, out + 2 * k);
}

__global__ void pcg_init_finalize_kernel(const double* __restrict__ partial, int nblk, int k, PcgState st) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double bb = 0.0, rz = 0.0, rr = 0.0;
        for (int b = 0; b < nblk; ++b) {
            bb += partial[int64_t(b) * 3 * k + c];
            rz += partial[int64_t(b) * 3 * k + k + c];
            rr += partial[int64_t(b) * 3 * k + 2 * k + c];
        }
        st.bb[c] = bb;
        st.rz[c] = rz;
        st.rr[c] = rr;
        st.alpha[c] = 0.0;
        st.beta[c] = 0.0;
        const int act = (bb > 0.0 && rr > st.rtol2 * bb) ? 1 : 0;
        st.active[c] = act;
        if (act) atomicAdd(&cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *st.n_active = cnt;
}

__global__ void pcg_alpha_kernel(const double* __restrict__ partial, int nblk, int k, PcgState st) {
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double pAp = 0.0;
        for (int b = 0; b < nblk; ++b) pAp += partial[int64_t(b) * k + c];
        st.alpha[c] = (st.active[c] && pAp > 0.0) ? st.rz[c] / pAp : 0.0;
    }
}

// x += alpha p, r -= alpha Ap, z = Dinv r; partials of r.z and r.r.
__global__ void pcg_update_kernel(double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
                                  const double* __restrict__ p, const double* __restrict__ Ap,
                                  const double* __restrict__ dinv, int64_t n, int k, PcgState st,
                                  double* __restrict__ partial /*[blk][2k]*/) {
    __shared__ double s[kRedThreads];
    const int R = kRedThreads / k, used = R * k;
    const int tid = threadIdx.x;
    double arz = 0.0, arr = 0.0;
    if (tid < used) {
        const int c = tid % k, rr0 = tid / k;
        const double al = st.alpha[c];
        for (int64_t i = int64_t(blockIdx.x) * R + rr0; i < n; i += int64_t(gridDim.x) * R) {
            const int64_t o = i * k + c;
            x[o] = fma(al, p[o], x[o]);
            const double ri = fma(-al, Ap[o], r[o]);
            const double zi = dinv[i] * ri;
            r[o] = ri;
            z[o] = zi;
            arz = fma(ri, zi, arz);
            arr = fma(ri, ri, arr);
        }
    }
    double* out = partial + int64_t(blockIdx.x) * 2 * k;
    s[tid] = arz;
    reduce_columns(s, k, R, out);
    __syncthreads();
    s[tid] = arr;
    reduce_columns(s, k, R, out + k);
}

__global__ void pcg_beta_kernel(const double* __restrict__ partial, int nblk, int k, PcgState st) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double rz = 0.0, rr = 0.0;
        for (int b = 0; b < nblk; ++b) {
            rz += partial[int64_t(b) * 2 * k + c];
            rr += partial[int64_t(b) * 2 * k + k + c];
        }
        if (st.active[c]) {
            st.beta[c] = st.rz[c] != 0.0 ? rz / st.rz[c] : 0.0;
            st.rz[c] = rz;
            st.rr[c] = rr;
            if (!(rr > st.rtol2 * st.bb[c])) st.active[c] = 0;
            if (!isfinite(rr)) st.active[c] = 0;
        } else {
            st.beta[c] = 0.0;
        }
        if (st.active[c]) atomicAdd(&cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *st.n_active = cnt;
}

__global__ void pcg_p_kernel(double* __restrict__ p, const double* __restrict__ z, int64_t n, int k,
                             PcgState st) {
    const int64_t total = n * k;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < total;
         o += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(o % k);
        if (st.active[c]) p[o] = fma(st.beta[c], p[o], z[o]);
    }
}

// ---- fused CG kernels: block partials + last-block finalize (alpha or beta)
// p.Ap per column; the last block sets alpha = rz / pAp for active columns.
template <typename T>
__global__ void dot_alpha_kernel(const T* __restrict__ p, const T* __restrict__ Ap, int64_t n, int k,
                                 double* __restrict__ partial, unsigned* __restrict__ counter, PcgState st) {
    __shared__ double s[kRedThreads];
    const int R = kRedThreads / k, used = R * k;
    const int t = threadIdx.x;
    double acc = 0.0;
    if (t < used) {
        const int c = t % k, r = t / k;
        for (int64_t i = int64_t(blockIdx.x) * R + r; i < n; i += int64_t(gridDim.x) * R)
            acc += double(p[i * k + c]) * double(Ap[i * k + c]);
    }
    s[t] = acc;
    reduce_columns(s, k, R, partial + int64_t(blockIdx.x) * k);
    if (!last_block_sum(partial, k, counter, s)) return;
    for (int c = t; c < k; c += blockDim.x) {
        const double pAp = s[c];
        st.alpha[c] = (st.active[c] && pAp > 0.0) ? st.rz[c] / pAp : 0.0;
    }
}

// x += alpha p, r -= alpha Ap; partials of r.(Dinv r) and r.r; the last block
// sets beta, rz, rr and, with reliable updates (rr_upd != null), the number of
// columns due for a float64 residual replacement in flags[1]; without them it
// retires converged columns (rr <= rtol2 bb) and counts the active ones in
// *st.n_active.
template <typename T>
__global__ void update_beta_kernel(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                   const T* __restrict__ Ap, const T* __restrict__ dinv, int64_t n, int k, PcgState st,
                                   double* __restrict__ partial, unsigned* __restrict__ counter,
                                   const double* __restrict__ scale, const double* __restrict__ rr_upd,
                                   const double* __restrict__ bb64, double rtol2, double delta2,
                                   int* __restrict__ flags) {
    __shared__ double s[kRedThreads];
    const int R = kRedThreads / k, used = R * k;
    const int tid = threadIdx.x;
    double arz = 0.0, arr = 0.0;
    if (tid < used) {
        const int c = tid % k, r0 = tid / k;
        const T al = T(st.alpha[c]);
        for (int64_t i = int64_t(blockIdx.x) * R + r0; i < n; i += int64_t(gridDim.x) * R) {
            const int64_t o = i * k + c;
            x[o] = x[o] + al * p[o];
            const T ri = r[o] - al * Ap[o];
            r[o] = ri;
            const double rd = double(ri);
            arz += rd * double(dinv[i] * ri);
            arr += rd * rd;
        }
    }
    double* out = partial + int64_t(blockIdx.x) * 2 * k;
    s[tid] = arz;
    reduce_columns(s, k, R, out);
    __syncthreads();
    s[tid] = arr;
    reduce_columns(s, k, R, out + k);
    if (!last_block_sum(partial, 2 * k, counter, s)) return;
    __shared__ int s_cnt;
    if (tid == 0) s_cnt = 0;
    __syncthreads();
    for (int c = tid; c < k; c += blockDim.x) {
        const double rz = s[c], rr = s[k + c];
        if (st.active[c]) {
            st.beta[c] = st.rz[c] != 0.0 ? rz / st.rz[c] : 0.0;
            st.rz[c] = rz;
            st.rr[c] = rr;
            if (rr_upd) {
                const bool due = !(rr >= delta2 * rr_upd[c]) || scale[c] * scale[c] * rr <= rtol2 * bb64[c];
                if (due) atomicAdd(&s_cnt, 1);
            } else {
                if (!(rr > st.rtol2 * st.bb[c]) || !isfinite(rr)) st.active[c] = 0;
                if (st.active[c]) atomicAdd(&s_cnt, 1);
            }
        } else {
            st.beta[c] = 0.0;
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (rr_upd) flags[1] = s_cnt;
        else *st.n_active = s_cnt;
    }
}

// p = Dinv r + beta p (active columns)
template <typename T>
__global__ void p_update_kernel(T* __restrict__ p, const T* __restrict__ r, const T* __restrict__ dinv, int64_t n,
                                int k, PcgState st) {
    const int64_t total = n * k;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < total;
         o += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(o % k);
        if (st.active[c]) p[o] = dinv[o / k] * r[o] + T(st.beta[c]) * p[o];
    }
}

// Copy the surface rows of x into g_ext (interior rows zero).
__global__ void surface_only_kernel(const double* __restrict__ x, double* __restrict__ gext, int64_t n_int,
                                    int64_t N, int k) {
    const int64_t total = N * k;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < total;
         o += int64_t(gridDim.x) * blockDim.x)
        gext[o] = (o / k) >= n_int ? x[o] : 0.0;
}

// ------------------------------------------------------------------ host
struct PoissonWork {
    double *b, *r, *z, *p, *Ap, *t, *partial, *qpart, *q;
    double *alpha, *beta, *rz, *bb, *rr;
    int *active, *n_active;
    unsigned* counters;   // last-block reduction counters (zeroed per call)
};

int poisson_rhs_bc(afem_mesh* m, const double2* phi, int n, double* W, double* b, double* qpart, double* q,
                   cudaStream_t s) {
    int rc = ensure_sh_tables();
    if (rc) return rc;
    const DeviceMesh& D = m->dev;
    const int ncol = n * n;
    PointArgs a{};
    a.phi = phi;
    a.n = n;
    a.ncol = ncol;
    a.N = D.n_master;
    a.n_int = D.n_interior;
    a.nh = D.n_hanging;
    a.xyz_m = D.master_xyz;
    a.xyz_h = D.hang_xyz;
    a.mf_m = D.mf_master;
    a.mf_h = D.mf_hang;
    a.hp = D.hang_ptr;
    a.hm = D.hang_master;
    a.hw = D.hang_w;
    const double c0 = 0.5 * (m->desc.lo + m->desc.hi);
    a.cx = a.cy = a.cz = c0;
    AFEM_CUDA_TRY(cudaMemsetAsync(b, 0, size_t(D.n_master) * ncol * sizeof(double), s));
    const size_t smem = (size_t(kMomTile) * kNlm + size_t(kMomTile) * ncol + size_t(kNlm) * ncol) * sizeof(double);
    AFEM_CUDA_TRY(cudaFuncSetAttribute(pair_rhs_moments_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(smem)));
    const int nblk = kMomBlocks;
    AFEM_LAUNCH((pair_rhs_moments_kernel), nblk, 256, smem, s, a, b, qpart);
    AFEM_CUDA_TRY(cudaGetLastError());
    AFEM_LAUNCH((finalize_columns_kernel), 1, 256, 0, s, qpart, nblk, kNlm * ncol, q);
    AFEM_CUDA_TRY(cudaGetLastError());
    const int64_t nb = D.n_master - D.n_interior;
    if (nb > 0) {
        const size_t sm2 = size_t(kNlm) * ncol * sizeof(double);
        AFEM_CUDA_TRY(cudaFuncSetAttribute(multipole_bc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(sm2)));
        AFEM_LAUNCH((multipole_bc_kernel), grid_for(nb, 128, 152 * 8), 128, sm2, s, q, ncol, D.master_xyz, D.n_interior,
                                                                          D.n_master, c0, c0, c0, W);
        AFEM_CUDA_TRY(cudaGetLastError());
    }
    return AFEM_OK;
}

int poisson_batch(afem_mesh* m, const double2* phi, int n, double* W, double rtol, int max_it, int warm,
                  int* iters_out, double* relres_out, cudaStream_t s) {
    const DeviceMesh& D = m->dev;
    const int k = n * n;
    const int64_t N = D.n_master, Ni = D.n_interior;
    const int nblk = kRedBlocks;
    const size_t NK = size_t(N) * k;
    PoissonWork w{};
    auto carve = [&](Carver& cv) {
        w.b = cv.take<double>(NK);
        w.r = cv.take<double>(NK);
        w.z = cv.take<double>(NK);
        w.p = cv.take<double>(NK);
        w.Ap = cv.take<double>(NK);
        w.t = cv.take<double>(NK);
        w.partial = cv.take<double>(size_t(nblk) * 3 * k);
        w.qpart = cv.take<double>(size_t(kMomBlocks) * kNlm * k);
        w.q = cv.take<double>(size_t(kNlm) * k);
        w.alpha = cv.take<double>(k);
        w.beta = cv.take<double>(k);
        w.rz = cv.take<double>(k);
        w.bb = cv.take<double>(k);
        w.rr = cv.take<double>(k);
        w.active = cv.take<int>(k);
        w.n_active = cv.take<int>(1);
        w.counters = cv.take<unsigned>(4);
    };
    Carver measure(nullptr);
    carve(measure);
    int rc = m->ws_poisson.reserve(measure.size());
    if (rc) return rc;
    Carver cv(m->ws_poisson.ptr);
    carve(cv);
    PcgState st{w.alpha, w.beta, w.rz, w.bb, w.rr, w.active, w.n_active, rtol * rtol};
    AFEM_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 4 * sizeof(unsigned), s));

    if (!warm) AFEM_CUDA_TRY(cudaMemsetAsync(W, 0, NK * sizeof(double), s));
    if ((rc = poisson_rhs_bc(m, phi, n, W, w.b, w.qpart, w.q, s))) return rc;
    // t = A g_ext (surface data only), Ap = A_II x_I
    AFEM_LAUNCH((surface_only_kernel), grid_for(int64_t(NK)), 256, 0, s, W, w.z, Ni, N, k);
    AFEM_CUDA_TRY(cudaGetLastError());
    if ((rc = launch_stiffness(m, w.z, w.t, k, 0, s))) return rc;
    if ((rc = launch_stiffness(m, W, w.Ap, k, 1, s))) return rc;
    AFEM_LAUNCH((pcg_init_kernel), nblk, kRedThreads, 0, s, w.b, w.t, w.Ap, D.stiff_dinv, w.r, w.z, w.p, Ni, k, w.partial);
    AFEM_CUDA_TRY(cudaGetLastError());
    AFEM_LAUNCH((pcg_init_finalize_kernel), 1, 64, 0, s, w.partial, nblk, k, st);
    AFEM_CUDA_TRY(cudaGetLastError());

    int it = 0, n_active = 1;
    const int check_every = 4;
    while (it < max_it) {
        if (it % check_every == 0) {
            AFEM_CUDA_TRY(cudaMemcpyAsync(&n_active, w.n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
            AFEM_CUDA_TRY(cudaStreamSynchronize(s));
            if (n_active == 0) break;
        }
        if ((rc = launch_stiffness(m, w.p, w.Ap, k, 1, s))) return rc;
        AFEM_LAUNCH((dot_alpha_kernel<double>), nblk, kRedThreads, 0, s, w.p, w.Ap, Ni, k, w.partial,
                    w.counters + 0, st);
        AFEM_LAUNCH((update_beta_kernel<double>), nblk, kRedThreads, 0, s, W, w.r, w.p, w.Ap, D.stiff_dinv, Ni, k, st,
                    w.partial, w.counters + 1, static_cast<const double*>(nullptr),
                    static_cast<const double*>(nullptr), static_cast<const double*>(nullptr), 0.0, 0.0,
                    static_cast<int*>(nullptr));
        AFEM_LAUNCH((p_update_kernel<double>), grid_for(Ni * k), 256, 0, s, w.p, w.r, D.stiff_dinv, Ni, k, st);
        AFEM_CUDA_TRY(cudaGetLastError());
        ++it;
    }
    AFEM_CUDA_TRY(cudaMemcpyAsync(&n_active, w.n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
    std::vector<double> rr(k), bb(k);
    AFEM_CUDA_TRY(cudaMemcpyAsync(rr.data(), w.rr, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    AFEM_CUDA_TRY(cudaMemcpyAsync(bb.data(), w.bb, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    AFEM_CUDA_TRY(cudaStreamSynchronize(s));
    if (iters_out) *iters_out = it;
    bool finite = true;
    for (int c = 0; c < k; ++c) {
        const double rel = bb[c] > 0.0 ? std::sqrt(rr[c] / bb[c]) : 0.0;
        if (!std::isfinite(rel)) finite = false;
        if (relres_out) relres_out[c] = rel;
    }
    if (!finite) return set_error(AFEM_ENAN, "afem_poisson_batch: non-finite residual");
    if (n_active > 0)
        return set_error(AFEM_ECG_MAXIT, "afem_poisson_batch: CG reached max_it before rtol");
    return AFEM_OK;
}

// ------------------------------------------- surface data from given scratch
// Moments only (no right-hand side) with `nblk` blocks, then the Dirichlet
// data into the surface rows of W.  qpart must hold nblk * kNlm * n^2 doubles
// and q kNlm * n^2; both are overwritten completely.
int multipole_boundary(afem_mesh* m, const double2* phi, int n, double* W, double* qpart, double* q, int nblk,
                       cudaStream_t s) {
    const int ncol = n * n;
    int rc = ensure_sh_tables();
    if (rc) return rc;
    const DeviceMesh& D = m->dev;
    PointArgs a{};
    a.phi = phi;
    a.n = n;
    a.ncol = ncol;
    a.N = D.n_master;
    a.n_int = D.n_interior;
    a.nh = D.n_hanging;
    a.xyz_m = D.master_xyz;
    a.xyz_h = D.hang_xyz;
    a.mf_m = D.mf_master;
    a.mf_h = D.mf_hang;
    a.hp = D.hang_ptr;
    a.hm = D.hang_master;
    a.hw = D.hang_w;
    const double c0 = 0.5 * (m->desc.lo + m->desc.hi);
    a.cx = a.cy = a.cz = c0;
    const size_t smem = (size_t(kMomTile) * kNlm + size_t(kMomTile) * ncol + size_t(kNlm) * ncol) * sizeof(double);
    AFEM_CUDA_TRY(cudaFuncSetAttribute(pair_rhs_moments_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(smem)));
    AFEM_LAUNCH((pair_rhs_moments_kernel), nblk, 256, smem, s, a, static_cast<double*>(nullptr), qpart);
    AFEM_LAUNCH((finalize_columns_kernel), 1, 256, 0, s, qpart, nblk, kNlm * ncol, q);
    AFEM_CUDA_TRY(cudaGetLastError());
    const int64_t nb = D.n_master - D.n_interior;
    if (nb > 0) {
        const size_t sm2 = size_t(kNlm) * ncol * sizeof(double);
        AFEM_CUDA_TRY(cudaFuncSetAttribute(multipole_bc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(sm2)));
        AFEM_LAUNCH((multipole_bc_kernel), grid_for(nb, 128, 152 * 8), 128, sm2, s, q, ncol, D.master_xyz,
                    D.n_interior, D.n_master, c0, c0, c0, W);
        AFEM_CUDA_TRY(cudaGetLastError());
    }
    return AFEM_OK;
}

// ------------------------------------------------ mixed precision (FP32 inner)
// Precision form: the same Dirichlet problems are solved by iterative
// refinement.  Each outer pass forms the FP64 residual r = b - A_IB g - A_II W
// with the FP64 operator, solves A d = r / ||r|| per column by Jacobi-PCG in
// FP32 to a loose tolerance, and updates W += ||r|| d in FP64, until the FP64
// residual meets rtol.

// r = b - t - Ap (interior rows), partial r.r ; r32 filled later after scaling.
__global__ void residual64_kernel(const double* __restrict__ b, const double* __restrict__ t,
                                  const double* __restrict__ Ap, double* __restrict__ r, int64_t n, int k,
                                  double* __restrict__ partial /*[blk][2k]*/) {
    __shared__ double s[kRedThreads];
    const int R = kRedThreads / k, used = R * k;
    const int tid = threadIdx.x;
    double arr = 0.0, abb = 0.0;
    if (tid < used) {
        const int c = tid % k, r0 = tid / k;
        for (int64_t i = int64_t(blockIdx.x) * R + r0; i < n; i += int64_t(gridDim.x) * R) {
            const int64_t o = i * k + c;
            const double be = b[o] - t[o];
            const double ri = be - Ap[o];
            r[o] = ri;
            arr = fma(ri, ri, arr);
            abb = fma(be, be, abb);
        }
    }
    double* out = partial + int64_t(blockIdx.x) * 2 * k;
    s[tid] = arr;
    reduce_columns(s, k, R, out);
    __syncthreads();
    s[tid] = abb;
    reduce_columns(s, k, R, out + k);
}

// Inner FP32 PCG start: r32 = r64 / scale_c, z = Dinv r32, p = z, d = 0; partials r.z, r.r.
__global__ void pcg32_init_kernel(const double* __restrict__ r64, const double* __restrict__ scale,
                                  const float* __restrict__ dinv, float* __restrict__ r, float* __restrict__ z,
                                  float* __restrict__ p, float* __restrict__ d, int64_t n, int k,
                                  double* __restrict__ partial) {
    __shared__ double s[kRedThreads];
    const int R = kRedThreads / k, used = R * k;
    const int tid = threadIdx.x;
    double arz = 0.0, arr = 0.0;
    if (tid < used) {
        const int c = tid % k, r0 = tid / k;
        const double sc = scale[c] > 0.0 ? 1.0 / scale[c] : 0.0;
        for (int64_t i = int64_t(blockIdx.x) * R + r0; i < n; i += int64_t(gridDim.x) * R) {
            const int64_t o = i * k + c;
            const float ri = float(r64[o] * sc);
            const float zi = dinv[i] * ri;
            r[o] = ri;
            z[o] = zi;
            p[o] = zi;
            d[o] = 0.0f;
            arz += double(ri) * double(zi);
            arr += double(ri) * double(ri);
        }
    }
    double* out = partial + int64_t(blockIdx.x) * 3 * k;
    s[tid] = arr;                      // bb of the inner problem = ||r32||^2
    reduce_columns(s, k, R, out);
    __syncthreads();
    s[tid] = arz;
    reduce_columns(s, k, R, out + k);
    __syncthreads();
    s[tid] = arr;
    reduce_columns(s, k, R, out + 2 * k);
}

__global__ void col_dot32_kernel(const float* __restrict__ a, const float* __restrict__ b, int64_t n, int k,
                                 double* __restrict__ partial) {
    __shared__ double s[kRedThreads];
    const int R = kRedThreads / k, used = R * k;
    const int t = threadIdx.x;
    double acc = 0.0;
    if (t < used) {
        const int c = t % k, r = t / k;
        for (int64_t i = int64_t(blockIdx.x) * R + r; i < n; i += int64_t(gridDim.x) * R)
            acc += double(a[i * k + c]) * double(b[i * k + c]);
    }
    s[t] = acc;
    reduce_columns(s, k, R, partial + int64_t(blockIdx.x) * k);
}

__global__ void pcg32_update_kernel(float* __restrict__ x, float* __restrict__ r, float* __restrict__ z,
                                    const float* __restrict__ p, const float* __restrict__ Ap,
                                    const float* __restrict__ dinv, int64_t n, int k, PcgState st,
                                    double* __restrict__ partial) {
    __shared__ double s[kRedThreads];
    const int R = kRedThreads / k, used = R * k;
    const int tid = threadIdx.x;
    double arz = 0.0, arr = 0.0;
    if (tid < used) {
        const int c = tid % k, r0 = tid / k;
        const float al = float(st.alpha[c]);
        for (int64_t i = int64_t(blockIdx.x) * R + r0; i < n; i += int64_t(gridDim.x) * R) {
            const int64_t o = i * k + c;
            x[o] = fmaf(al, p[o], x[o]);
            const float ri = fmaf(-al, Ap[o], r[o]);
            const float zi = dinv[i] * ri;
            r[o] = ri;
            z[o] = zi;
            arz += double(ri) * double(zi);
            arr += double(ri) * double(ri);
        }
    }
    double* out = partial + int64_t(blockIdx.x) * 2 * k;
    s[tid] = arz;
    reduce_columns(s, k, R, out);
    __syncthreads();
    s[tid] = arr;
    reduce_columns(s, k, R, out + k);
}

__global__ void pcg32_p_kernel(float* __restrict__ p, const float* __restrict__ z, int64_t n, int k, PcgState st) {
    const int64_t total = n * k;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < total;
         o += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(o % k);
        if (st.active[c]) p[o] = fmaf(float(st.beta[c]), p[o], z[o]);
    }
}

// W_interior += scale_c d_c ; per-column norms of the FP64 residual in scale.
__global__ void refine_update_kernel(double* __restrict__ W, const float* __restrict__ d,
                                     const double* __restrict__ scale, int64_t n, int k) {
    const int64_t total = n * k;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < total;
         o += int64_t(gridDim.x) * blockDim.x)
        W[o] = fma(scale[o % k], double(d[o]), W[o]);
}

__global__ void finalize_residual_kernel(const double* __restrict__ partial, int nblk, int k, double rtol2,
                                         double* __restrict__ rr, double* __restrict__ bb,
                                         double* __restrict__ scale, int* __restrict__ n_active) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < nblk; ++q) {
            a += partial[int64_t(q) * 2 * k + c];
            b += partial[int64_t(q) * 2 * k + k + c];
        }
        rr[c] = a;
        bb[c] = b;
        const int act = (b > 0.0 && a > rtol2 * b && isfinite(a)) ? 1 : 0;
        scale[c] = act ? sqrt(a) : 0.0;
        if (act) atomicAdd(&cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *n_active = cnt;
}

int launch_stiffness32(const afem_mesh* m, const float* x, float* y, int nv, int masked, cudaStream_t s);

// Reliable-update form of the mixed solve: one continuous float32 CG per
// column whose correction d is folded into the float64 W, and whose residual is
// replaced by the true float64 residual (search direction rescaled), whenever
// the float32 residual has dropped by `delta` since the last replacement or
// claims convergence.  Convergence is only ever declared on the float64
// residual.

// beta, and per column whether a residual replacement is due.
__global__ void pcg32_beta_ru_kernel(const double* __restrict__ partial, int nblk, int k, PcgState st,
                                     const double* __restrict__ scale, const double* __restrict__ rr_upd,
                                     const double* __restrict__ bb64, double rtol2, double delta2,
                                     int* __restrict__ flags) {
    __shared__ int need;
    if (threadIdx.x == 0) need = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double rz = 0.0, rr = 0.0;
        for (int b = 0; b < nblk; ++b) {
            rz += partial[int64_t(b) * 2 * k + c];
            rr += partial[int64_t(b) * 2 * k + k + c];
        }
        if (st.active[c]) {
            st.beta[c] = st.rz[c] != 0.0 ? rz / st.rz[c] : 0.0;
            st.rz[c] = rz;
            st.rr[c] = rr;
            const bool due = !(rr >= delta2 * rr_upd[c]) || scale[c] * scale[c] * rr <= rtol2 * bb64[c];
            if (due) atomicAdd(&need, 1);
        } else {
            st.beta[c] = 0.0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) flags[1] = need;
}

// W += s d ; d = 0   (interior rows)
__global__ void ru_fold_kernel(double* __restrict__ W, float* __restrict__ d, const double* __restrict__ scale,
                               int64_t n, int k) {
    const int64_t total = n * k;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < total;
         o += int64_t(gridDim.x) * blockDim.x) {
        W[o] = fma(scale[o % k], double(d[o]), W[o]);
        d[o] = 0.0f;
    }
}

// rr64, bb64, new scale and activity from the float64 residual partials.
__global__ void ru_residual_finalize_kernel(const double* __restrict__ partial, int nblk, int k, double rtol2,
                                            double* __restrict__ rr64, double* __restrict__ bb64,
                                            double* __restrict__ s_new, int* __restrict__ active,
                                            int* __restrict__ flags) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < nblk; ++q) {
            a += partial[int64_t(q) * 2 * k + c];
            b += partial[int64_t(q) * 2 * k + k + c];
        }
        rr64[c] = a;
        bb64[c] = b;
        const int act = (b > 0.0 && a > rtol2 * b && isfinite(a)) ? 1 : 0;
        active[c] = act;
        s_new[c] = act ? sqrt(a) : 0.0;
        if (act) atomicAdd(&cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        flags[0] = cnt;
        flags[1] = 0;
    }
}

// r32 = r64 / s_new, z = Dinv r32, p = z (init) or p *= s_old / s_new; partials r.z, r.r.
__global__ void ru_rescale_kernel(const double* __restrict__ r64, const double* __restrict__ s_old,
                                  const double* __restrict__ s_new, const float* __restrict__ dinv,
                                  float* __restrict__ r, float* __restrict__ z, float* __restrict__ p,
                                  const int* __restrict__ active, int init, int64_t n, int k,
                                  double* __restrict__ partial) {
    __shared__ double sh[kRedThreads];
    const int R = kRedThreads / k, used = R * k;
    const int tid = threadIdx.x;
    double arz = 0.0, arr = 0.0;
    if (tid < used) {
        const int c = tid % k, r0 = tid / k;
        const bool act = active[c] != 0;
        const double inv = act ? 1.0 / s_new[c] : 0.0;
        const float pf = (act && !init && s_new[c] > 0.0) ? float(s_old[c] / s_new[c]) : 0.0f;
        for (int64_t i = int64_t(blockIdx.x) * R + r0; i < n; i += int64_t(gridDim.x) * R) {
            const int64_t o = i * k + c;
            const float ri = float(r64[o] * inv);
            const float zi = dinv[i] * ri;
            r[o] = ri;
            z[o] = zi;
            p[o] = init ? zi : (act ? p[o] * pf : 0.0f);
            arz += double(ri) * double(zi);
            arr += double(ri) * double(ri);
        }
    }
    double* out = partial + int64_t(blockIdx.x) * 2 * k;
    sh[tid] = arz;
    reduce_columns(sh, k, R, out);
    __syncthreads();
    sh[tid] = arr;
    reduce_columns(sh, k, R, out + k);
}

__global__ void ru_finalize_kernel(const double* __restrict__ partial, int nblk, int k, PcgState st,
                                   double* __restrict__ rr_upd, double* __restrict__ s_old,
                                   const double* __restrict__ s_new) {
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double rz = 0.0, rr = 0.0;
        for (int q = 0; q < nblk; ++q) {
            rz += partial[int64_t(q) * 2 * k + c];
            rr += partial[int64_t(q) * 2 * k + k + c];
        }
        st.rz[c] = rz;
        st.rr[c] = rr;
        rr_upd[c] = rr;
        s_old[c] = s_new[c];
    }
}

int poisson_batch_mixed(afem_mesh* m, const double2* phi, int n, double* W, double rtol, int max_it, int warm,
                        double delta, int* iters_out, int* outer_out, double* relres_out, cudaStream_t s) {
    const DeviceMesh& D = m->dev;
    const int k = n * n;
    const int64_t N = D.n_master, Ni = D.n_interior;
    const int nblk = kRedBlocks;
    const size_t NK = size_t(N) * k;
    PoissonWork w{};
    float *r32, *z32, *p32, *Ap32, *d32;
    double *s_old, *s_new, *rr64, *bb64, *rr_upd;
    int* flags;
    auto carve = [&](Carver& cv) {
        w.b = cv.take<double>(NK);
        w.r = cv.take<double>(NK);
        w.Ap = cv.take<double>(NK);
        w.t = cv.take<double>(NK);
        w.z = cv.take<double>(NK);
        r32 = cv.take<float>(NK);
        z32 = cv.take<float>(NK);
        p32 = cv.take<float>(NK);
        Ap32 = cv.take<float>(NK);
        d32 = cv.take<float>(NK);
        w.partial = cv.take<double>(size_t(nblk) * 3 * k);
        w.qpart = cv.take<double>(size_t(kMomBlocks) * kNlm * k);
        w.q = cv.take<double>(size_t(kNlm) * k);
        w.alpha = cv.take<double>(k);
        w.beta = cv.take<double>(k);
        w.rz = cv.take<double>(k);
        w.bb = cv.take<double>(k);
        w.rr = cv.take<double>(k);
        w.active = cv.take<int>(k);
        w.n_active = cv.take<int>(1);
        s_old = cv.take<double>(k);
        s_new = cv.take<double>(k);
        rr64 = cv.take<double>(k);
        bb64 = cv.take<double>(k);
        rr_upd = cv.take<double>(k);
        flags = cv.take<int>(2);
        w.counters = cv.take<unsigned>(4);
    };
    Carver measure(nullptr);
    carve(measure);
    int rc = m->ws_poisson.reserve(measure.size());
    if (rc) return rc;
    Carver cv(m->ws_poisson.ptr);
    carve(cv);
    PcgState st{w.alpha, w.beta, w.rz, w.bb, w.rr, w.active, w.n_active, 0.0};
    const double rtol2 = rtol * rtol, delta2 = delta * delta;
    AFEM_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 4 * sizeof(unsigned), s));

    if (!warm) AFEM_CUDA_TRY(cudaMemsetAsync(W, 0, NK * sizeof(double), s));
    if ((rc = poisson_rhs_bc(m, phi, n, W, w.b, w.qpart, w.q, s))) return rc;
    AFEM_LAUNCH((surface_only_kernel), grid_for(int64_t(NK)), 256, 0, s, W, w.z, Ni, N, k);
    if ((rc = launch_stiffness(m, w.z, w.t, k, 0, s))) return rc;   // t = A g_ext (FP64)
    AFEM_CUDA_TRY(cudaMemsetAsync(d32, 0, NK * sizeof(float), s));

    int flags_h[2] = {0, 0};
    int replacements = 0;
    // float64 residual of the current W, and the float32 state built from it
    auto replace = [&](int init) -> int {
        int r_;
        if ((r_ = launch_stiffness(m, W, w.Ap, k, 1, s))) return r_;
        AFEM_LAUNCH((residual64_kernel), nblk, kRedThreads, 0, s, w.b, w.t, w.Ap, w.r, Ni, k, w.partial);
        AFEM_LAUNCH((ru_residual_finalize_kernel), 1, 64, 0, s, w.partial, nblk, k, rtol2, rr64, bb64, s_new,
                    w.active, flags);
        AFEM_LAUNCH((ru_rescale_kernel), nblk, kRedThreads, 0, s, w.r, s_old, s_new, D.stiff_dinv32, r32, z32, p32,
                    w.active, init, Ni, k, w.partial);
        AFEM_LAUNCH((ru_finalize_kernel), 1, 64, 0, s, w.partial, nblk, k, st, rr_upd, s_old, s_new);
        AFEM_CUDA_TRY(cudaGetLastError());
        AFEM_CUDA_TRY(cudaMemcpyAsync(flags_h, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        AFEM_CUDA_TRY(cudaStreamSynchronize(s));
        ++replacements;
        return AFEM_OK;
    };
    if ((rc = replace(1))) return rc;
    int it = 0;
    const int check_every = 8;
    while (flags_h[0] > 0 && it < max_it) {
        if ((rc = launch_stiffness32(m, p32, Ap32, k, 1, s))) return rc;
        AFEM_LAUNCH((dot_alpha_kernel<float>), nblk, kRedThreads, 0, s, p32, Ap32, Ni, k, w.partial,
                    w.counters + 0, st);
        AFEM_LAUNCH((update_beta_kernel<float>), nblk, kRedThreads, 0, s, d32, r32, p32, Ap32, D.stiff_dinv32, Ni, k,
                    st, w.partial, w.counters + 1, s_old, rr_upd, bb64, rtol2, delta2, flags);
        AFEM_LAUNCH((p_update_kernel<float>), grid_for(Ni * k), 256, 0, s, p32, r32, D.stiff_dinv32, Ni, k, st);
        AFEM_CUDA_TRY(cudaGetLastError());
        ++it;
        if (it % check_every == 0 || it >= max_it) {
            AFEM_CUDA_TRY(cudaMemcpyAsync(flags_h, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
            AFEM_CUDA_TRY(cudaStreamSynchronize(s));
            if (flags_h[1] > 0 || it >= max_it) {
                AFEM_LAUNCH((ru_fold_kernel), grid_for(Ni * k), 256, 0, s, W, d32, s_old, Ni, k);
                if ((rc = replace(0))) return rc;
            }
        }
    }
    if (iters_out) *iters_out = it;
    if (outer_out) *outer_out = replacements;
    std::vector<double> rr(k), bb(k);
    AFEM_CUDA_TRY(cudaMemcpyAsync(rr.data(), rr64, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    AFEM_CUDA_TRY(cudaMemcpyAsync(bb.data(), bb64, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    AFEM_CUDA_TRY(cudaStreamSynchronize(s));
    bool finite = true;
    for (int c = 0; c < k; ++c) {
        const double rel = bb[c] > 0.0 ? std::sqrt(rr[c] / bb[c]) : 0.0;
        if (!std::isfinite(rel)) finite = false;
        if (relres_out) relres_out[c] = rel;
    }
    if (!finite) return set_error(AFEM_ENAN, "afem_poisson_batch: non-finite residual");
    if (flags_h[0] > 0)
        return set_error(AFEM_ECG_MAXIT, "afem_poisson_batch: mixed CG reached max_it before rtol");
    return AFEM_OK;
}

}  // namespace afem
