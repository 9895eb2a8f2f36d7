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
#include <mutex>
#include <vector>

#include "afem_internal.h"
#include "cell_common.cuh"
#include "vec_common.cuh"

namespace afem {

constexpr int kLmax = kMultipoleLmax;
constexpr int kNlm = kMultipoleTerms;
constexpr int kMomTile = 32;
static int mom_blocks() { return 2 * device_sms(); }   // moment partial rows: 2 blocks per SM
int mom_blocks_count() { return mom_blocks(); }
__constant__ double c_sh_norm[kNlm];       // factor applied to C_lm / S_lm at index l*l + l + |m|
__constant__ double c_sh_irreg[kLmax + 1];  // 4 pi / (2l + 1)

// Uploads the solid-harmonic normalisations once per device (synchronous
// copies; serialised across host threads).
int ensure_sh_tables() {
    static bool done[64] = {false};
    static std::mutex mu;
    int dev = 0;
    AFEM_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
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
// Per tile of kMomTile support points, every phase is spread over the block:
// (point, orbital) items stage the orbital values (hanging points through C),
// (point, column) items form m_f rho_c and the right-hand side, then the
// harmonics and the moment contraction.
__global__ void __launch_bounds__(256) pair_rhs_moments_kernel(PointArgs a, double* __restrict__ b,
                                                               double* __restrict__ qpart) {
    extern __shared__ __align__(16) double smem_d[];
    double* s_R = smem_d;                          // [kMomTile][kNlm]
    double* s_w = s_R + kMomTile * kNlm;           // [kMomTile][ncol]
    double* s_Q = s_w + kMomTile * a.ncol;         // [kNlm][ncol]
    __shared__ double4 s_pt[kMomTile];             // point relative to the centre, valid flag
    __shared__ double2 s_ph[kMomTile][8];          // orbital values at the tile's points
    __shared__ double s_mf[kMomTile];
    __shared__ int s_col[64];                      // column c -> r | s << 8 | part << 16
    const int ncol = a.ncol, n = a.n;
    const int tid = threadIdx.x;
    for (int o = tid; o < kNlm * ncol; o += blockDim.x) s_Q[o] = 0.0;
    if (tid == 0) {
        int c = 0;
        for (int r = 0; r < n; ++r) s_col[c++] = r | (r << 8);
        for (int r = 0; r < n; ++r)
            for (int t = r + 1; t < n; ++t) {
                s_col[c++] = r | (t << 8);
                s_col[c++] = r | (t << 8) | (1 << 16);
            }
    }
    const int64_t npts = a.N + a.nh;
    const int64_t ntiles = (npts + kMomTile - 1) / kMomTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        // orbital values (zero at surface masters; hanging points from interior masters)
        for (int it = tid; it < kMomTile * n; it += blockDim.x) {
            const int tp = it / n, r = it - tp * n;
            const int64_t f = tile * kMomTile + tp;
            double2 v = make_double2(0.0, 0.0);
            if (f < a.N) {
                if (f < a.n_int) v = a.phi[f * n + r];
            } else if (f < npts) {
                const int64_t h = f - a.N;
                for (int e = a.hp[h]; e < a.hp[h + 1]; ++e) {
                    const int m = a.hm[e];
                    if (m >= a.n_int) continue;
                    vfma(v, a.hw[e], a.phi[int64_t(m) * n + r]);
                }
            }
            s_ph[tp][r] = v;
        }
        for (int tp = tid; tp < kMomTile; tp += blockDim.x) {
            const int64_t f = tile * kMomTile + tp;
            if (f < a.N) {
                s_mf[tp] = a.mf_m[f];
                s_pt[tp] = make_double4(a.xyz_m[3 * f] - a.cx, a.xyz_m[3 * f + 1] - a.cy, a.xyz_m[3 * f + 2] - a.cz,
                                        1.0);
            } else if (f < npts) {
                const int64_t h = f - a.N;
                s_mf[tp] = a.mf_h[h];
                s_pt[tp] = make_double4(a.xyz_h[3 * h] - a.cx, a.xyz_h[3 * h + 1] - a.cy, a.xyz_h[3 * h + 2] - a.cz,
                                        1.0);
            } else {
                s_mf[tp] = 0.0;
                s_pt[tp] = make_double4(0.0, 0.0, 0.0, 0.0);
            }
        }
        __syncthreads();
        // m_f rho_c and the right-hand side through C^T
        for (int it = tid; it < kMomTile * ncol; it += blockDim.x) {
            const int tp = it / ncol, c = it - tp * ncol;
            const int64_t f = tile * kMomTile + tp;
            double wv = 0.0;
            if (f < npts) {
                const int code = s_col[c];
                const double2 x = s_ph[tp][code & 0xFF], y = s_ph[tp][(code >> 8) & 0xFF];
                const double rho = (code >> 16) ? x.x * y.y - x.y * y.x : x.x * y.x + x.y * y.y;
                wv = s_mf[tp] * rho;
                const double fpi = 4.0 * M_PI;
                if (!b) {
                    // moments only
                } else if (f < a.N) {
                    atomicAdd(&b[f * ncol + c], fpi * wv);
                } else {
                    const int64_t h = f - a.N;
                    for (int e = a.hp[h]; e < a.hp[h + 1]; ++e)
                        atomicAdd(&b[int64_t(a.hm[e]) * ncol + c], fpi * a.hw[e] * wv);
                }
            }
            s_w[tp * ncol + c] = wv;
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

// ---- float32 CG kernels on four columns per thread (k % 4 == 0): thread t <
// (k/4) R of a 256-thread block owns the column quad q = t % (k/4) of rows
// r = t / (k/4), r + R, ... (R = 1024 / k), loaded as float4.  Per-column
// sums go through s[r k + c] (R k = 1024 entries), the layout reduce_columns
// reads.
// GB300 issues FP64 at about 1/64 of its FP32 rate, so the per-element
// products of these kernels stay in FP32: runs of kRun rows are summed in
// FP32 and only the run sums in FP64 (random rounding of about 1e-7 per run;
// the CG scalars are formed from the FP64 totals).
constexpr int kRun = 16;
constexpr int kPapSlotsCg = 64;   // slots of the p.Ap sums of the fused stiffness pass

struct Quad {
    int q, r, R, kq;
    bool active;
    __device__ __forceinline__ Quad(int k) {
        kq = k >> 2;
        R = kRedThreads / kq;
        active = int(threadIdx.x) < kq * R;
        r = active ? int(threadIdx.x) / kq : 0;
        q = active ? int(threadIdx.x) - r * kq : 0;
    }
};

__global__ void __launch_bounds__(kRedThreads) dot_alpha4_kernel(const float4* __restrict__ p,
                                                                 const float4* __restrict__ Ap, int64_t n, int k,
                                                                 double* __restrict__ partial,
                                                                 unsigned* __restrict__ counter, PcgState st) {
    __shared__ double s[4 * kRedThreads];
    const Quad qd(k);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if (qd.active) {
        const int64_t step = int64_t(gridDim.x) * qd.R;
        int64_t i = int64_t(blockIdx.x) * qd.R + qd.r;
        while (i < n) {   // runs of kRun rows summed in FP32, the runs in FP64
            float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
            for (int run = 0; run < kRun && i < n; ++run, i += step) {
                const float4 u = p[i * qd.kq + qd.q], v = Ap[i * qd.kq + qd.q];
                f0 = fmaf(u.x, v.x, f0);
                f1 = fmaf(u.y, v.y, f1);
                f2 = fmaf(u.z, v.z, f2);
                f3 = fmaf(u.w, v.w, f3);
            }
            a0 += double(f0);
            a1 += double(f1);
            a2 += double(f2);
            a3 += double(f3);
        }
    }
    const int t = threadIdx.x;
    s[4 * t] = a0;
    s[4 * t + 1] = a1;
    s[4 * t + 2] = a2;
    s[4 * t + 3] = a3;
    reduce_columns(s, k, qd.R, partial + int64_t(blockIdx.x) * k);
    if (!last_block_sum(partial, k, counter, s)) return;
    for (int c = t; c < k; c += blockDim.x) {
        const double pAp = s[c];
        st.alpha[c] = (st.active[c] && pAp > 0.0) ? st.rz[c] / pAp : 0.0;
    }
}

// beta, rz, rr from the column sums s[c] = r.(Dinv r), s[k + c] = r.r, and the
// reliable-update count or the retirement of converged columns (last block).
__device__ __forceinline__ void cg_beta_finalize(const double* s, int k, PcgState st, const double* scale,
                                                 const double* rr_upd, const double* bb64, double rtol2, double delta2,
                                                 int* flags) {
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
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
    if (threadIdx.x == 0) {
        if (rr_upd) flags[1] = s_cnt;
        else *st.n_active = s_cnt;
    }
}

// update_beta_kernel<float> on column quads.
__global__ void __launch_bounds__(kRedThreads) update_beta4_kernel(
    float4* __restrict__ x, float4* __restrict__ r, const float4* __restrict__ p, const float4* __restrict__ Ap,
    const float* __restrict__ dinv, int64_t n, int k, PcgState st, double* __restrict__ partial,
    unsigned* __restrict__ counter, const double* __restrict__ scale, const double* __restrict__ rr_upd,
    const double* __restrict__ bb64, double rtol2, double delta2, int* __restrict__ flags,
    double* __restrict__ pap_slots) {
    __shared__ double s[4 * kRedThreads];
    __shared__ double s_alpha[64];
    // alpha = rz / p.Ap per column: from st.alpha (formed by dot_alpha4_kernel)
    // or, when the stiffness pass summed p.Ap into pap_slots, formed here
    if (pap_slots) {
        for (int c = threadIdx.x; c < k; c += blockDim.x) {
            double pAp = 0.0;
            for (int sl = 0; sl < kPapSlotsCg; ++sl) pAp += pap_slots[sl * k + c];
            s_alpha[c] = (st.active[c] && pAp > 0.0) ? st.rz[c] / pAp : 0.0;
        }
    } else {
        for (int c = threadIdx.x; c < k; c += blockDim.x) s_alpha[c] = st.alpha[c];
    }
    __syncthreads();
    const Quad qd(k);
    double z0 = 0.0, z1 = 0.0, z2 = 0.0, z3 = 0.0, r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
    if (qd.active) {
        const int c0 = 4 * qd.q;
        const float al0 = float(s_alpha[c0]), al1 = float(s_alpha[c0 + 1]), al2 = float(s_alpha[c0 + 2]),
                    al3 = float(s_alpha[c0 + 3]);
        const int64_t step = int64_t(gridDim.x) * qd.R;
        int64_t i = int64_t(blockIdx.x) * qd.R + qd.r;
        while (i < n) {   // runs of kRun rows summed in FP32, the runs in FP64
            float fz0 = 0.f, fz1 = 0.f, fz2 = 0.f, fz3 = 0.f, fr0 = 0.f, fr1 = 0.f, fr2 = 0.f, fr3 = 0.f;
            for (int run = 0; run < kRun && i < n; ++run, i += step) {
                const int64_t o = i * qd.kq + qd.q;
                const float4 pv = p[o], av = Ap[o];
                float4 xv = x[o], rv = r[o];
                const float d = dinv[i];
                xv.x = xv.x + al0 * pv.x;
                xv.y = xv.y + al1 * pv.y;
                xv.z = xv.z + al2 * pv.z;
                xv.w = xv.w + al3 * pv.w;
                rv.x = rv.x - al0 * av.x;
                rv.y = rv.y - al1 * av.y;
                rv.z = rv.z - al2 * av.z;
                rv.w = rv.w - al3 * av.w;
                x[o] = xv;
                r[o] = rv;
                fz0 = fmaf(rv.x, d * rv.x, fz0);
                fz1 = fmaf(rv.y, d * rv.y, fz1);
                fz2 = fmaf(rv.z, d * rv.z, fz2);
                fz3 = fmaf(rv.w, d * rv.w, fz3);
                fr0 = fmaf(rv.x, rv.x, fr0);
                fr1 = fmaf(rv.y, rv.y, fr1);
                fr2 = fmaf(rv.z, rv.z, fr2);
                fr3 = fmaf(rv.w, rv.w, fr3);
            }
            z0 += double(fz0);
            z1 += double(fz1);
            z2 += double(fz2);
            z3 += double(fz3);
            r0 += double(fr0);
            r1 += double(fr1);
            r2 += double(fr2);
            r3 += double(fr3);
        }
    }
    const int t = threadIdx.x;
    double* out = partial + int64_t(blockIdx.x) * 2 * k;
    s[4 * t] = z0;
    s[4 * t + 1] = z1;
    s[4 * t + 2] = z2;
    s[4 * t + 3] = z3;
    reduce_columns(s, k, qd.R, out);
    __syncthreads();
    s[4 * t] = r0;
    s[4 * t + 1] = r1;
    s[4 * t + 2] = r2;
    s[4 * t + 3] = r3;
    reduce_columns(s, k, qd.R, out + k);
    if (!last_block_sum(partial, 2 * k, counter, s)) return;
    if (pap_slots) {   // every block has read the slots: record alpha, clear them for the next sweep
        for (int c = threadIdx.x; c < k; c += blockDim.x) st.alpha[c] = s_alpha[c];
        for (int o = threadIdx.x; o < kPapSlotsCg * k; o += blockDim.x) pap_slots[o] = 0.0;
    }
    cg_beta_finalize(s, k, st, scale, rr_upd, bb64, rtol2, delta2, flags);
}

// p = Dinv r + beta p (active columns) on column quads.
__global__ void __launch_bounds__(kRedThreads) p_update4_kernel(float4* __restrict__ p, const float4* __restrict__ r,
                                                                const float* __restrict__ dinv, int64_t n, int k,
                                                                PcgState st) {
    const Quad qd(k);
    if (!qd.active) return;
    const int c0 = 4 * qd.q;
    const bool a0 = st.active[c0], a1 = st.active[c0 + 1], a2 = st.active[c0 + 2], a3 = st.active[c0 + 3];
    if (!(a0 || a1 || a2 || a3)) return;
    const float b0 = float(st.beta[c0]), b1 = float(st.beta[c0 + 1]), b2 = float(st.beta[c0 + 2]),
                b3 = float(st.beta[c0 + 3]);
    for (int64_t i = int64_t(blockIdx.x) * qd.R + qd.r; i < n; i += int64_t(gridDim.x) * qd.R) {
        const int64_t o = i * qd.kq + qd.q;
        const float d = dinv[i];
        const float4 rv = r[o];
        float4 pv = p[o];
        if (a0) pv.x = d * rv.x + b0 * pv.x;
        if (a1) pv.y = d * rv.y + b1 * pv.y;
        if (a2) pv.z = d * rv.z + b2 * pv.z;
        if (a3) pv.w = d * rv.w + b3 * pv.w;
        p[o] = pv;
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
    AFEM_CUDA_TRY(allow_dyn_smem(pair_rhs_moments_kernel));
    const int nblk = mom_blocks();
    AFEM_LAUNCH((pair_rhs_moments_kernel), nblk, 256, smem, s, a, b, qpart);
    AFEM_CUDA_TRY(cudaGetLastError());
    AFEM_LAUNCH((finalize_columns_kernel), 1, 256, 0, s, qpart, nblk, kNlm * ncol, q);
    AFEM_CUDA_TRY(cudaGetLastError());
    const int64_t nb = D.n_master - D.n_interior;
    if (nb > 0) {
        const size_t sm2 = size_t(kNlm) * ncol * sizeof(double);
        AFEM_CUDA_TRY(allow_dyn_smem(multipole_bc_kernel));
        AFEM_LAUNCH((multipole_bc_kernel), grid_for(nb, 128, 8), 128, sm2, s, q, ncol, D.master_xyz, D.n_interior,
                                                                          D.n_master, c0, c0, c0, W);
        AFEM_CUDA_TRY(cudaGetLastError());
    }
    return AFEM_OK;
}

int poisson_batch_mg(afem_mesh* m, const double2* phi, int n, double* W, double rtol, int max_it, int warm, int mixed,
                     int* iters_out, int* outer_out, double* relres_out, cudaStream_t s);

int poisson_batch(afem_mesh* m, const double2* phi, int n, double* W, double rtol, int max_it, int warm,
                  int* iters_out, double* relres_out, cudaStream_t s) {
    if (m->poisson_solver == AFEM_POISSON_MULTIGRID)
        return poisson_batch_mg(m, phi, n, W, rtol, max_it, warm, 0, iters_out, nullptr, relres_out, s);
    const DeviceMesh& D = m->dev;
    const int k = n * n;
    const int64_t N = D.n_master, Ni = D.n_interior;
    const int nblk = red_blocks();
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
        w.qpart = cv.take<double>(size_t(mom_blocks()) * kNlm * k);
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
        {
            const int p1 = D.p + 1;
            ProfScope ps(AFEM_PROF_CELL64, s, double(D.ncell) * p1 * p1 * p1 * k * (3.0 * p1 * 2.0 + 6.0));
            if ((rc = launch_stiffness(m, w.p, w.Ap, k, 1, s))) return rc;
        }
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
    AFEM_CUDA_TRY(allow_dyn_smem(pair_rhs_moments_kernel));
    AFEM_LAUNCH((pair_rhs_moments_kernel), nblk, 256, smem, s, a, static_cast<double*>(nullptr), qpart);
    AFEM_LAUNCH((finalize_columns_kernel), 1, 256, 0, s, qpart, nblk, kNlm * ncol, q);
    AFEM_CUDA_TRY(cudaGetLastError());
    const int64_t nb = D.n_master - D.n_interior;
    if (nb > 0) {
        const size_t sm2 = size_t(kNlm) * ncol * sizeof(double);
        AFEM_CUDA_TRY(allow_dyn_smem(multipole_bc_kernel));
        AFEM_LAUNCH((multipole_bc_kernel), grid_for(nb, 128, 8), 128, sm2, s, q, ncol, D.master_xyz,
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

int launch_stiffness32(const afem_mesh* m, const float* x, float* y, int nv, int masked, cudaStream_t s,
                       double* pap_slots = nullptr);

// Reliable-update form of the mixed solve: one continuous float32 CG per
// column whose correction d is folded into the float64 W, and whose residual is
// replaced by the true float64 residual (search direction rescaled), whenever
// the float32 residual has dropped by `delta` since the last replacement or
// claims convergence.  Convergence is only ever declared on the float64
// residual.

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
    if (m->poisson_solver == AFEM_POISSON_MULTIGRID)
        return poisson_batch_mg(m, phi, n, W, rtol, max_it, warm, 1, iters_out, outer_out, relres_out, s);
    const DeviceMesh& D = m->dev;
    const int k = n * n;
    const bool quads = (k % 4) == 0;   // four columns per thread in the float32 CG kernels
    // p.Ap formed by the stiffness pass itself (its four-lane form with 1, 2 or 4 quads)
    const bool fused = quads && (k == 4 || k == 8 || k == 16) && m->cell32_variant != 1;
    const int64_t N = D.n_master, Ni = D.n_interior;
    const int nblk = red_blocks();
    const size_t NK = size_t(N) * k;
    PoissonWork w{};
    float *r32, *z32, *p32, *Ap32, *d32;
    double *s_old, *s_new, *rr64, *bb64, *rr_upd;
    int* flags;
    double* pap;
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
        w.qpart = cv.take<double>(size_t(mom_blocks()) * kNlm * k);
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
        pap = cv.take<double>(size_t(kPapSlotsCg) * k);
    };
    Carver measure(nullptr);
    carve(measure);
    int rc = m->ws_poisson.reserve(measure.size());
    if (rc) return rc;
    Carver cv(m->ws_poisson.ptr);
    carve(cv);
    PcgState st{w.alpha, w.beta, w.rz, w.bb, w.rr, w.active, w.n_active, 0.0};
    AFEM_CUDA_TRY(cudaMemsetAsync(pap, 0, sizeof(double) * kPapSlotsCg * k, s));
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
        {   // algorithmic bytes: read p, write Ap (float32)
            ProfScope ps(AFEM_PROF_STIFF32, s, double(N) * k * 8.0);
            if ((rc = launch_stiffness32(m, p32, Ap32, k, 1, s, fused ? pap : nullptr))) return rc;
        }
        // algorithmic bytes: p.Ap 8 (unless the stiffness pass formed it), x/r update 24,
        // p update 12 per element (float32)
        ProfScope psv(AFEM_PROF_CGVEC32, s, double(Ni) * k * (fused ? 36.0 : 44.0));
        if (quads) {
            auto* p4 = reinterpret_cast<float4*>(p32);
            auto* r4 = reinterpret_cast<float4*>(r32);
            if (!fused)
                AFEM_LAUNCH((dot_alpha4_kernel), nblk, kRedThreads, 0, s, p4, reinterpret_cast<const float4*>(Ap32),
                            Ni, k, w.partial, w.counters + 0, st);
            AFEM_LAUNCH((update_beta4_kernel), nblk, kRedThreads, 0, s, reinterpret_cast<float4*>(d32), r4, p4,
                        reinterpret_cast<const float4*>(Ap32), D.stiff_dinv32, Ni, k, st, w.partial, w.counters + 1,
                        s_old, rr_upd, bb64, rtol2, delta2, flags, fused ? pap : nullptr);
            AFEM_LAUNCH((p_update4_kernel), nblk, kRedThreads, 0, s, p4, r4, D.stiff_dinv32, Ni, k, st);
        } else {
            AFEM_LAUNCH((dot_alpha_kernel<float>), nblk, kRedThreads, 0, s, p32, Ap32, Ni, k, w.partial,
                        w.counters + 0, st);
            AFEM_LAUNCH((update_beta_kernel<float>), nblk, kRedThreads, 0, s, d32, r32, p32, Ap32, D.stiff_dinv32, Ni,
                        k, st, w.partial, w.counters + 1, s_old, rr_upd, bb64, rtol2, delta2, flags);
            AFEM_LAUNCH((p_update_kernel<float>), grid_for(Ni * k), 256, 0, s, p32, r32, D.stiff_dinv32, Ni, k, st);
        }
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
