// Short-iterative Arnoldi propagation of all orbitals at once (Sec. 3.2).
//
// With phi, the RDMs, the mean fields and the field frozen at t, the packed
// orbital equation (Eq. packed_orb_eom) is linear, i d(phi)/dt = G phi, and
// phi(t + dt) = exp(-i G dt) phi(t).  The Krylov space of G from phi is built
// by Arnoldi (modified Gram-Schmidt, one pass) in the inner product
// <u, v> = sum_p u_p^H M_L v_p; then phi(t+dt) = beta V_m exp(-i dt H_m) e_1.
// G applied to the stacked orbitals v (Eqs. orb_eom / discretized_eom, X = 0):
//   z_p = H1~ v_p + C^T diag(m_f) sum_q (C U_pq) o (C v_q)      (one cell pass)
//   y_p = M_L^-1 z_p,   (G v)_p = y_p - sum_j phi_j (phi_j^H M_L y_p)
// and phi_j^H M_L y_p = phi_j^H z_p, so the projector needs no extra scaling.
#include <cmath>
#include <vector>

#include "afem_internal.h"
#include "arnoldi.cuh"
#include "vec_common.cuh"

namespace afem {

// S[a][b] partials: sum_k w_k conj(A[k][a]) B[k][b] over rows k < n_rows.
// diag != 0: only a == b (k_out = na), else all na*nb pairs (k_out = na*nb <= 256).
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }

template <typename TB>
__global__ void cdot_kernel(const double2* __restrict__ A, int na, const TB* __restrict__ B, int nb,
                            const double* __restrict__ w, int64_t n_rows, int diag,
                            double2* __restrict__ partial) {
    __shared__ double sx[kRedThreads], sy[kRedThreads];
    const int kout = diag ? na : na * nb;
    const int R = kRedThreads / kout, used = R * kout;
    const int t = threadIdx.x;
    double ax = 0.0, ay = 0.0;
    if (t < used) {
        const int o = t % kout, r = t / kout;
        const int ia = diag ? o : o / nb;
        const int ib = diag ? o : o - ia * nb;
        for (int64_t k = int64_t(blockIdx.x) * R + r; k < n_rows; k += int64_t(gridDim.x) * R) {
            const double2 u = A[k * na + ia];
            const double2 v = to_d2(B[k * nb + ib]);
            const double wk = w ? w[k] : 1.0;
            ax = fma(wk, fma(u.x, v.x, u.y * v.y), ax);
            ay = fma(wk, fma(u.x, v.y, -u.y * v.x), ay);
        }
    }
    sx[t] = ax;
    sy[t] = ay;
    __syncthreads();
    for (int o = t; o < kout; o += blockDim.x) {
        double x = 0.0, y = 0.0;
        for (int r = 0; r < R; ++r) {
            x += sx[o + kout * r];
            y += sy[o + kout * r];
        }
        partial[int64_t(blockIdx.x) * kout + o] = make_double2(x, y);
    }
}

// cdot with the block sums finished in the same launch (no sum_all form):
// partial rows of 2*kout doubles (re, im interleaved); the last block writes out[kout].
template <typename TB>
__global__ void cdot_fused_kernel(const double2* __restrict__ A, int na, const TB* __restrict__ B, int nb,
                                  const double* __restrict__ w, int64_t n_rows, int diag, double* __restrict__ partial,
                                  unsigned* __restrict__ counter, double2* __restrict__ out) {
    __shared__ double sx[kRedThreads], sy[kRedThreads];
    const int kout = diag ? na : na * nb;
    const int R = kRedThreads / kout, used = R * kout;
    const int t = threadIdx.x;
    double ax = 0.0, ay = 0.0;
    if (t < used) {
        const int o = t % kout, r = t / kout;
        const int ia = diag ? o : o / nb;
        const int ib = diag ? o : o - ia * nb;
        for (int64_t k = int64_t(blockIdx.x) * R + r; k < n_rows; k += int64_t(gridDim.x) * R) {
            const double2 u = A[k * na + ia];
            const double2 v = to_d2(B[k * nb + ib]);
            const double wk = w ? w[k] : 1.0;
            ax = fma(wk, fma(u.x, v.x, u.y * v.y), ax);
            ay = fma(wk, fma(u.x, v.y, -u.y * v.x), ay);
        }
    }
    sx[t] = ax;
    sy[t] = ay;
    __syncthreads();
    for (int o = t; o < kout; o += blockDim.x) {
        double x = 0.0, y = 0.0;
        for (int r = 0; r < R; ++r) {
            x += sx[o + kout * r];
            y += sy[o + kout * r];
        }
        partial[int64_t(blockIdx.x) * 2 * kout + 2 * o] = x;
        partial[int64_t(blockIdx.x) * 2 * kout + 2 * o + 1] = y;
    }
    if (!last_block_sum(partial, 2 * kout, counter, sx)) return;
    for (int o = t; o < kout; o += blockDim.x) out[o] = make_double2(sx[2 * o], sx[2 * o + 1]);
}

// out[o] = sum_b partial[b][o]; if sum_all, out[0] = sum over o as well.
__global__ void cfinalize_kernel(const double2* __restrict__ partial, int nblk, int kout, int sum_all,
                                 double2* __restrict__ out) {
    __shared__ double sx[256], sy[256];
    double tx = 0.0, ty = 0.0;
    for (int o = threadIdx.x; o < kout; o += blockDim.x) {
        double x = 0.0, y = 0.0;
        for (int b = 0; b < nblk; ++b) {
            const double2 v = partial[int64_t(b) * kout + o];
            x += v.x;
            y += v.y;
        }
        if (!sum_all) out[o] = make_double2(x, y);
        tx += x;
        ty += y;
    }
    if (!sum_all) return;
    sx[threadIdx.x] = tx;
    sy[threadIdx.x] = ty;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int i = 0; i < blockDim.x; ++i) {
            x += sx[i];
            y += sy[i];
        }
        out[0] = make_double2(x, y);
    }
}

// w[k][p] = ML^-1[k] z[k][p] - sum_j phi[k][j] S[j][p]   (interior rows; others 0)
template <typename TZ>
__global__ void project_kernel(const TZ* __restrict__ z, const double2* __restrict__ phi,
                               const double2* __restrict__ S, const double* __restrict__ ml_inv, int64_t n_int,
                               int64_t N, int n, double2* __restrict__ w) {
    const int64_t total = N * n;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < total;
         o += int64_t(gridDim.x) * blockDim.x) {
        const int64_t k = o / n;
        const int p = int(o - k * n);
        double2 r = make_double2(0.0, 0.0);
        if (k < n_int) {
            const double s = ml_inv[k];
            const double2 zo = to_d2(z[o]);
            r = make_double2(zo.x * s, zo.y * s);
            for (int j = 0; j < n; ++j) {
                const double2 f = phi[k * n + j];
                const double2 c = S[j * n + p];
                r.x -= f.x * c.x - f.y * c.y;
                r.y -= f.x * c.y + f.y * c.x;
            }
        }
        w[o] = r;
    }
}

// MGS step: w -= h_prev * V_prev (if V_prev), then partial <V_i, w>_M (or <w, w>_M if V_i null).
__global__ void mgs_kernel(double2* __restrict__ w, const double2* __restrict__ Vprev,
                           const double2* __restrict__ hprev, const double2* __restrict__ Vi,
                           const double* __restrict__ ml, int64_t n_int, int n, double2* __restrict__ partial) {
    __shared__ double sx[kRedThreads], sy[kRedThreads];
    const int64_t total = n_int * n;
    double ax = 0.0, ay = 0.0;
    const double2 h = Vprev ? *hprev : make_double2(0.0, 0.0);
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < total;
         o += int64_t(gridDim.x) * blockDim.x) {
        double2 x = w[o];
        if (Vprev) {
            const double2 v = Vprev[o];
            x.x -= h.x * v.x - h.y * v.y;
            x.y -= h.x * v.y + h.y * v.x;
            w[o] = x;
        }
        const double2 u = Vi ? Vi[o] : x;
        const double m = ml[o / n];
        ax = fma(m, fma(u.x, x.x, u.y * x.y), ax);
        ay = fma(m, fma(u.x, x.y, -u.y * x.x), ay);
    }
    sx[threadIdx.x] = ax;
    sy[threadIdx.x] = ay;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int i = 0; i < blockDim.x; ++i) {
            x += sx[i];
            y += sy[i];
        }
        partial[blockIdx.x] = make_double2(x, y);
    }
}

// The MGS step above with its reduction finished in the same launch: block
// partials (re, im) go to partial[2 * block], the last block writes *out.
__global__ void mgs_fused_kernel(double2* __restrict__ w, const double2* __restrict__ Vprev,
                                 const double2* __restrict__ hprev, const double2* __restrict__ Vi,
                                 const double* __restrict__ ml, int64_t n_int, int n, double* __restrict__ partial,
                                 unsigned* __restrict__ counter, double2* __restrict__ out) {
    __shared__ double sx[kRedThreads], sy[kRedThreads];
    const int64_t total = n_int * n;
    double ax = 0.0, ay = 0.0;
    const double2 h = Vprev ? *hprev : make_double2(0.0, 0.0);
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < total;
         o += int64_t(gridDim.x) * blockDim.x) {
        double2 x = w[o];
        if (Vprev) {
            const double2 v = Vprev[o];
            x.x -= h.x * v.x - h.y * v.y;
            x.y -= h.x * v.y + h.y * v.x;
            w[o] = x;
        }
        const double2 u = Vi ? Vi[o] : x;
        const double m = ml[o / n];
        ax = fma(m, fma(u.x, x.x, u.y * x.y), ax);
        ay = fma(m, fma(u.x, x.y, -u.y * x.x), ay);
    }
    sx[threadIdx.x] = ax;
    sy[threadIdx.x] = ay;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            sx[threadIdx.x] += sx[threadIdx.x + st];
            sy[threadIdx.x] += sy[threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = sx[0];
        partial[2 * blockIdx.x + 1] = sy[0];
    }
    if (!last_block_sum(partial, 2, counter, sx)) return;
    if (threadIdx.x == 0) *out = make_double2(sx[0], sx[1]);
}

// Sum block partials into *out (one thread, fixed order).
__global__ void sum_partials_kernel(const double2* __restrict__ partial, int nblk, double2* __restrict__ out) {
    if (threadIdx.x != 0) return;
    double x = 0.0, y = 0.0;
    for (int b = 0; b < nblk; ++b) {
        x += partial[b].x;
        y += partial[b].y;
    }
    *out = make_double2(x, y);
}

__global__ void cscale_kernel(double2* __restrict__ x, int64_t n, const double2* __restrict__ src, double s,
                              int sqrt_real_inv) {
    // x *= s, or x *= 1 / sqrt(Re *src) when sqrt_real_inv
    double f = s;
    if (sqrt_real_inv) f = 1.0 / sqrt(src->x);
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < n; o += int64_t(gridDim.x) * blockDim.x) {
        x[o].x *= f;
        x[o].y *= f;
    }
}

// phi_out = sum_i y_i V_i
__global__ void combine_kernel(const double2* __restrict__ V, int64_t stride, int m, const double2* __restrict__ y,
                               int64_t total, double2* __restrict__ out) {
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < total;
         o += int64_t(gridDim.x) * blockDim.x) {
        double x = 0.0, yy = 0.0;
        for (int i = 0; i < m; ++i) {
            const double2 v = V[i * stride + o];
            const double2 c = y[i];
            x += c.x * v.x - c.y * v.y;
            yy += c.x * v.y + c.y * v.x;
        }
        out[o] = make_double2(x, yy);
    }
}

// exp(-i dt H) for an m x m complex matrix (m <= kMaxKrylov), one block:
// scaling and squaring with a truncated Taylor series (the scaled matrix has
// 1-norm <= 1/2, and 24 terms leave a remainder below 1e-30).
// H: column-major with leading dimension ldh.  Writes E[m*m] (column-major).
__global__ void small_expm_kernel(const double2* __restrict__ H, int ldh, int m, double dt,
                                  double2* __restrict__ E) {
    __shared__ double2 A[kMaxKrylov * kMaxKrylov], P[kMaxKrylov * kMaxKrylov], S[kMaxKrylov * kMaxKrylov],
        T[kMaxKrylov * kMaxKrylov];
    __shared__ int s_sq;
    const int t = threadIdx.x;
    const int mm = m * m;
    for (int o = t; o < mm; o += blockDim.x) {
        const int i = o % m, j = o / m;
        const double2 h = H[j * ldh + i];
        A[o] = make_double2(dt * h.y, -dt * h.x);   // -i dt h
    }
    __syncthreads();
    if (t == 0) {
        double nrm = 0.0;
        for (int j = 0; j < m; ++j) {
            double c = 0.0;
            for (int i = 0; i < m; ++i) c += hypot(A[j * m + i].x, A[j * m + i].y);
            nrm = fmax(nrm, c);
        }
        int sq = 0;
        while (nrm > 0.5 && sq < 60) {
            nrm *= 0.5;
            ++sq;
        }
        s_sq = sq;
    }
    __syncthreads();
    const double sc = ldexp(1.0, -s_sq);
    for (int o = t; o < mm; o += blockDim.x) {
        A[o].x *= sc;
        A[o].y *= sc;
        const int i = o % m, j = o / m;
        S[o] = make_double2(i == j ? 1.0 : 0.0, 0.0);
        P[o] = S[o];
    }
    __syncthreads();
    for (int k = 1; k <= 24; ++k) {
        // P <- P A / k
        for (int o = t; o < mm; o += blockDim.x) {
            const int i = o % m, j = o / m;
            double x = 0.0, y = 0.0;
            for (int l = 0; l < m; ++l) {
                const double2 a = P[l * m + i], b = A[j * m + l];
                x += a.x * b.x - a.y * b.y;
                y += a.x * b.y + a.y * b.x;
            }
            T[o] = make_double2(x / k, y / k);
        }
        __syncthreads();
        for (int o = t; o < mm; o += blockDim.x) {
            P[o] = T[o];
            S[o].x += T[o].x;
            S[o].y += T[o].y;
        }
        __syncthreads();
    }
    for (int q = 0; q < s_sq; ++q) {
        for (int o = t; o < mm; o += blockDim.x) {
            const int i = o % m, j = o / m;
            double x = 0.0, y = 0.0;
            for (int l = 0; l < m; ++l) {
                const double2 a = S[l * m + i], b = S[j * m + l];
                x += a.x * b.x - a.y * b.y;
                y += a.x * b.y + a.y * b.x;
            }
            T[o] = make_double2(x, y);
        }
        __syncthreads();
        for (int o = t; o < mm; o += blockDim.x) S[o] = T[o];
        __syncthreads();
    }
    for (int o = t; o < mm; o += blockDim.x) E[o] = S[o];
}

// ------------------------------------------------------------------- host
int launch_g_cell(const afem_mesh* m, const double* E, const double2* v, const double2* U, double2* z, int n,
                  cudaStream_t s);

template <typename TB>
int cdot_t(const double2* A, int na, const TB* B, int nb, const double* w, int64_t rows, int diag,
           double2* partial, double2* out, unsigned* counter, cudaStream_t s) {
    AFEM_LAUNCH((cdot_fused_kernel<TB>), kRedBlocks, kRedThreads, 0, s, A, na, B, nb, w, rows, diag,
                reinterpret_cast<double*>(partial), counter, out);
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

int cdot(const double2* A, int na, const double2* B, int nb, const double* w, int64_t rows, int diag,
         double2* partial, double2* out, unsigned* counter, cudaStream_t s) {
    return cdot_t<double2>(A, na, B, nb, w, rows, diag, partial, out, counter, s);
}

__global__ void to_c64_kernel(const double2* __restrict__ x, float2* __restrict__ y, int64_t n) {
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < n; o += int64_t(gridDim.x) * blockDim.x)
        y[o] = make_float2(float(x[o].x), float(x[o].y));
}

int to_c64(const double2* x, float2* y, int64_t n, cudaStream_t s) {
    AFEM_LAUNCH((to_c64_kernel), grid_for(n), 256, 0, s, x, y, n);
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

int launch_g_cell32(const afem_mesh* m, const double* E, const float2* v, const float2* U, float2* z, int n,
                    cudaStream_t s);

// Mixed form: the cell pass in complex64 on a complex64 copy of v; projector
// overlaps, the projection and everything after stay FP64.
int g_apply32(afem_mesh* m, const double* E, const double2* phi, const float2* U32, int n, const double2* v,
              ArnoldiWork& w, double2* out, cudaStream_t s) {
    const DeviceMesh& D = m->dev;
    int rc = to_c64(v, w.v32, D.n_master * n, s);
    if (rc) return rc;
    if ((rc = launch_g_cell32(m, E, w.v32, U32, w.z32, n, s))) return rc;
    if ((rc = cdot_t<float2>(phi, n, w.z32, n, nullptr, D.n_interior, 0, w.cpartial, w.S, w.counters, s))) return rc;
    AFEM_LAUNCH((project_kernel<float2>), grid_for(D.n_master * n), 256, 0, s, w.z32, phi, w.S, D.ml_inv,
                D.n_interior, D.n_master, n, out);
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

int g_apply(afem_mesh* m, const double* E, const double2* phi, const double2* U, int n, const double2* v,
            double2* z, double2* out, ArnoldiWork& w, cudaStream_t s) {
    const DeviceMesh& D = m->dev;
    int rc = launch_g_cell(m, E, v, U, z, n, s);
    if (rc) return rc;
    // S[j][p] = phi_j^H z_p  (equals phi_j^H M_L y_p)
    if ((rc = cdot(phi, n, z, n, nullptr, D.n_interior, 0, w.cpartial, w.S, w.counters, s))) return rc;
    AFEM_LAUNCH((project_kernel<double2>), grid_for(D.n_master * n), 256, 0, s, z, phi, w.S, D.ml_inv, D.n_interior, D.n_master, n,
                                                            out);
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

int arnoldi_reserve(afem_mesh* m, int n, int mk, ArnoldiWork& w) {
    const size_t NV = size_t(m->dev.n_master) * n;
    auto carve = [&](Carver& cv) {
        w.V = cv.take<double2>(size_t(mk + 1) * NV);
        w.z = cv.take<double2>(NV);
        w.cpartial = cv.take<double2>(size_t(kRedBlocks) * 256);
        w.S = cv.take<double2>(64);
        w.H = cv.take<double2>(size_t(kMaxKrylov + 1) * kMaxKrylov);
        w.E = cv.take<double2>(kMaxKrylov * kMaxKrylov);
        w.y = cv.take<double2>(kMaxKrylov);
        w.beta2 = cv.take<double2>(1);
        w.v32 = cv.take<float2>(NV);
        w.z32 = cv.take<float2>(NV);
        w.U32 = cv.take<float2>(NV * n);
        w.counters = cv.take<unsigned>(4);
    };
    Carver measure(nullptr);
    carve(measure);
    int rc = m->ws_arnoldi.reserve(measure.size());
    if (rc) return rc;
    Carver cv(m->ws_arnoldi.ptr);
    carve(cv);
    w.stride = int64_t(NV);
    return AFEM_OK;
}

// Propagates phi by exp(-i G dt) with G frozen at phi (projector), U and E.
// tol <= 0: one Krylov step of dimension mk over the whole dt.  tol > 0:
// substeps tau chosen so that each substep's error estimate
// beta |h_{m+1,m}| |e_m^T exp(-i tau H_m) e_1| stays below tol * beta (the
// paper fixes the Krylov accuracy by such an estimate; here the dimension is
// fixed and the substep adapts), each from a fresh Krylov space of the same G.
int arnoldi_step(afem_mesh* m, const double* E, const double2* phi, const double2* U, const float2* U32, int n,
                 int mk, double dt, int mixed, double tol, double2* phi_out, double* err_est, int* m_used_out,
                 int* breakdown_out, int* substeps_out, cudaStream_t s) {
    const DeviceMesh& D = m->dev;
    ArnoldiWork w{};
    int rc = arnoldi_reserve(m, n, mk, w);
    if (rc) return rc;
    if (mixed && U && !U32) {
        if ((rc = to_c64(U, w.U32, D.n_master * n * n, s))) return rc;
        U32 = w.U32;
    }
    AFEM_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 4 * sizeof(unsigned), s));
    const int64_t NV = w.stride;
    const int ldh = kMaxKrylov + 1;
    const double2* src = phi;
    double remaining = dt;
    double err_sum = 0.0;
    int substeps = 0, m_used = mk, brk = 0;
    std::vector<double2> Eh(size_t(kMaxKrylov) * kMaxKrylov);
    while (remaining > 0.0) {
        if (substeps >= 4096) return set_error(AFEM_EINVAL, "arnoldi: more than 4096 substeps (tolerance too tight)");
        AFEM_CUDA_TRY(cudaMemsetAsync(w.H, 0, sizeof(double2) * ldh * kMaxKrylov, s));
        // beta^2 = <src, src>_M ; V_0 = src / beta
        AFEM_LAUNCH((mgs_fused_kernel), kRedBlocks, kRedThreads, 0, s, const_cast<double2*>(src), nullptr, nullptr,
                    nullptr, D.ml, D.n_interior, n, reinterpret_cast<double*>(w.cpartial), w.counters + 1, w.beta2);
        AFEM_CUDA_TRY(cudaMemcpyAsync(w.V, src, NV * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        AFEM_LAUNCH((cscale_kernel), grid_for(NV), 256, 0, s, w.V, NV, w.beta2, 1.0, 1);
        AFEM_CUDA_TRY(cudaGetLastError());
        double2 beta2_h;
        AFEM_CUDA_TRY(cudaMemcpyAsync(&beta2_h, w.beta2, sizeof(double2), cudaMemcpyDeviceToHost, s));
        AFEM_CUDA_TRY(cudaStreamSynchronize(s));
        const double beta = std::sqrt(beta2_h.x);
        if (!(beta > 0.0) || !std::isfinite(beta)) return set_error(AFEM_ENAN, "arnoldi: zero or non-finite norm");
        m_used = mk;
        brk = 0;
        double hlast = 0.0;
        for (int j = 0; j < mk; ++j) {
            double2* Vj = w.V + j * NV;
            double2* Wn = w.V + (j + 1) * NV;
            if (mixed) {
                if ((rc = g_apply32(m, E, phi, U32, n, Vj, w, Wn, s))) return rc;
            } else {
                if ((rc = g_apply(m, E, phi, U, n, Vj, w.z, Wn, w, s))) return rc;
            }
            // modified Gram-Schmidt against V_0..V_j
            for (int i = 0; i <= j; ++i) {
                const double2* Vprev = i > 0 ? w.V + (i - 1) * NV : nullptr;
                const double2* hprev = i > 0 ? w.H + j * ldh + (i - 1) : nullptr;
                AFEM_LAUNCH((mgs_fused_kernel), kRedBlocks, kRedThreads, 0, s, Wn, Vprev, hprev, w.V + i * NV, D.ml,
                            D.n_interior, n, reinterpret_cast<double*>(w.cpartial), w.counters + 1,
                            w.H + j * ldh + i);
            }
            // last update and the norm
            AFEM_LAUNCH((mgs_fused_kernel), kRedBlocks, kRedThreads, 0, s, Wn, w.V + j * NV, w.H + j * ldh + j,
                        nullptr, D.ml, D.n_interior, n, reinterpret_cast<double*>(w.cpartial), w.counters + 1,
                        w.beta2);
            AFEM_CUDA_TRY(cudaGetLastError());
            double2 nn2;
            AFEM_CUDA_TRY(cudaMemcpyAsync(&nn2, w.beta2, sizeof(double2), cudaMemcpyDeviceToHost, s));
            AFEM_CUDA_TRY(cudaStreamSynchronize(s));
            const double hn = std::sqrt(std::fmax(nn2.x, 0.0));
            if (!std::isfinite(hn)) return set_error(AFEM_ENAN, "arnoldi: non-finite Krylov vector");
            const double2 hv = make_double2(hn, 0.0);
            AFEM_CUDA_TRY(cudaMemcpyAsync(w.H + j * ldh + (j + 1), &hv, sizeof(double2), cudaMemcpyHostToDevice, s));
            hlast = hn;
            if (hn < 1e-14 * beta) {
                m_used = j + 1;
                brk = 1;
                break;
            }
            AFEM_LAUNCH((cscale_kernel), grid_for(NV), 256, 0, s, Wn, NV, nullptr, 1.0 / hn, 0);
            AFEM_CUDA_TRY(cudaGetLastError());
        }
        // substep length: the whole remainder, or shortened until the estimate meets tol
        double tau = remaining, err = 0.0;
        for (int tries = 0;; ++tries) {
            AFEM_LAUNCH((small_expm_kernel), 1, 256, 0, s, w.H, ldh, m_used, tau, w.E);
            AFEM_CUDA_TRY(cudaGetLastError());
            AFEM_CUDA_TRY(cudaMemcpyAsync(Eh.data(), w.E, size_t(m_used) * m_used * sizeof(double2),
                                          cudaMemcpyDeviceToHost, s));
            AFEM_CUDA_TRY(cudaStreamSynchronize(s));
            const double2 em = Eh[m_used - 1];
            err = brk ? 0.0 : beta * hlast * std::hypot(em.x, em.y);
            if (tol <= 0.0 || brk || err <= tol * beta || tries >= 40) break;
            const double shrink = 0.9 * std::pow(tol * beta / err, 1.0 / m_used);
            tau *= std::fmin(0.5, std::fmax(shrink, 0.05));
        }
        // phi_out = beta V_m exp(-i tau H_m) e_1
        std::vector<double2> yh(m_used);
        for (int i = 0; i < m_used; ++i) yh[i] = make_double2(beta * Eh[i].x, beta * Eh[i].y);
        AFEM_CUDA_TRY(cudaMemcpyAsync(w.y, yh.data(), m_used * sizeof(double2), cudaMemcpyHostToDevice, s));
        AFEM_LAUNCH((combine_kernel), grid_for(NV), 256, 0, s, w.V, NV, m_used, w.y, NV, phi_out);
        AFEM_CUDA_TRY(cudaGetLastError());
        AFEM_CUDA_TRY(cudaStreamSynchronize(s));
        err_sum += err;
        ++substeps;
        remaining = (tau >= remaining) ? 0.0 : remaining - tau;
        src = phi_out;
    }
    if (err_est) *err_est = err_sum;
    if (m_used_out) *m_used_out = m_used;
    if (breakdown_out) *breakdown_out = brk;
    if (substeps_out) *substeps_out = substeps;
    return AFEM_OK;
}

}  // namespace afem
