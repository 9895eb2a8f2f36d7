// One MCTDHF time step on the GPU (Sec. 2 and Sec. 3.2).
//
// Standard notation: E_pq = sum_s a+_{ps} a_{qs}, gamma_pq = <E_pq>,
// Gamma_pqrs = <E_pq E_rs> - delta_qr gamma_ps, h_pq = phi_p^H H1~ phi_q and
// (pq|rs) = sum_f m_f conj(phi_p) phi_q W_rs over the support points.  The
// paper's RDMs are D^p_q = gamma_qp and P^{pq}_{sr} = Gamma_{sprq}, so the
// mean-field term of Eq. orb_eom is sum_q U_pq phi_q with
//     U_pq = sum_o (gamma^-1)_po sum_rs Gamma_oqrs W_rs.
// The step, with everything frozen at t (Sec. 3.2, first order):
//   1. W_rs by the batched Poisson solve (warm-started from the last step);
//   2. h_pq and (pq|rs);  gamma, Gamma from C(t);
//   3. C(t+dt) = exp(-i dt H_CI) C(t) (Eq. ci_eom with X = 0), by a Taylor
//      series of the shifted CI Hamiltonian applied matrix-free through
//      string excitation lists;
//   4. U_pq fields;  phi(t+dt) = exp(-i G dt) phi(t) by short-iterative Arnoldi.
#include <algorithm>
#include <cmath>
#include <vector>

#include "afem_internal.h"
#include "arnoldi.cuh"
#include "vec_common.cuh"

namespace afem {

// ---------------------------------------------------------------- CI space
// Excitation lists in gather form: for string I, entries (pq = p*n+q, J, sign)
// with <I| a+_p a_q |J> = sign.
struct CiTables {
    int n = 0, na = 0, nb = 0;
    int64_t nsa = 0, nsb = 0, dim = 0;
    int32_t *a_ptr = nullptr, *a_pq = nullptr, *a_j = nullptr;
    int32_t *b_ptr = nullptr, *b_pq = nullptr, *b_j = nullptr;
    double *a_sg = nullptr, *b_sg = nullptr;
};

static std::vector<uint32_t> strings_of(int n, int k) {
    std::vector<uint32_t> out;
    for (uint32_t s = 0; s < (1u << n); ++s)
        if (__builtin_popcount(s) == k) out.push_back(s);
    return out;   // ascending bit-mask order
}

static int excite(uint32_t s, int p, int q, uint32_t& out, double& sign) {
    if (!((s >> q) & 1u)) return 0;
    int sg = __builtin_popcount(s & ((1u << q) - 1u)) & 1;
    uint32_t s1 = s & ~(1u << q);
    if ((s1 >> p) & 1u) return 0;
    sg ^= __builtin_popcount(s1 & ((1u << p) - 1u)) & 1;
    out = s1 | (1u << p);
    sign = sg ? -1.0 : 1.0;
    return 1;
}

template <typename T>
static int upload_vec(T*& dst, const std::vector<T>& v) {
    dst = nullptr;
    if (v.empty()) return AFEM_OK;
    cudaError_t e = cudaMalloc(&dst, v.size() * sizeof(T));
    if (e != cudaSuccess) return set_error(AFEM_ENOMEM, "cudaMalloc (CI tables) failed");
    AFEM_CUDA_TRY(cudaMemcpy(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return AFEM_OK;
}

static int build_lists(int n, int k, int32_t*& ptr, int32_t*& pq, int32_t*& jj, double*& sg, int64_t& nstr) {
    std::vector<uint32_t> S = strings_of(n, k);
    nstr = int64_t(S.size());
    std::vector<std::vector<std::tuple<int32_t, int32_t, double>>> lists(S.size());
    std::vector<int32_t> index(1u << n, -1);
    for (size_t i = 0; i < S.size(); ++i) index[S[i]] = int32_t(i);
    for (size_t j = 0; j < S.size(); ++j)
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                uint32_t I;
                double s;
                if (excite(S[j], p, q, I, s)) lists[index[I]].push_back({p * n + q, int32_t(j), s});
            }
    std::vector<int32_t> vptr(S.size() + 1, 0), vpq, vj;
    std::vector<double> vs;
    for (size_t i = 0; i < S.size(); ++i) {
        for (auto& e : lists[i]) {
            vpq.push_back(std::get<0>(e));
            vj.push_back(std::get<1>(e));
            vs.push_back(std::get<2>(e));
        }
        vptr[i + 1] = int32_t(vpq.size());
    }
    int rc;
    if ((rc = upload_vec(ptr, vptr))) return rc;
    if ((rc = upload_vec(pq, vpq))) return rc;
    if ((rc = upload_vec(jj, vj))) return rc;
    if ((rc = upload_vec(sg, vs))) return rc;
    return AFEM_OK;
}

// D[pq][I] = (E_pq v)[I] for all pq (thread per determinant I = ia * nsb + ib).
__global__ void ci_excite_kernel(CiTables t, const double2* __restrict__ v, double2* __restrict__ D) {
    const int nn = t.n * t.n;
    for (int64_t I = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; I < t.dim; I += int64_t(gridDim.x) * blockDim.x) {
        const int64_t ia = I / t.nsb, ib = I - ia * t.nsb;
        for (int pq = 0; pq < nn; ++pq) D[pq * t.dim + I] = make_double2(0.0, 0.0);
        for (int e = t.a_ptr[ia]; e < t.a_ptr[ia + 1]; ++e) {
            const double2 x = v[int64_t(t.a_j[e]) * t.nsb + ib];
            double2& d = D[t.a_pq[e] * t.dim + I];
            d.x += t.a_sg[e] * x.x;
            d.y += t.a_sg[e] * x.y;
        }
        for (int e = t.b_ptr[ib]; e < t.b_ptr[ib + 1]; ++e) {
            const double2 x = v[ia * t.nsb + t.b_j[e]];
            double2& d = D[t.b_pq[e] * t.dim + I];
            d.x += t.b_sg[e] * x.x;
            d.y += t.b_sg[e] * x.y;
        }
    }
}

// sigma[I] = sum_pq (E_pq Y_pq)[I]
__global__ void ci_gather_kernel(CiTables t, const double2* __restrict__ Y, double2* __restrict__ sigma) {
    for (int64_t I = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; I < t.dim; I += int64_t(gridDim.x) * blockDim.x) {
        const int64_t ia = I / t.nsb, ib = I - ia * t.nsb;
        double sx = 0.0, sy = 0.0;
        for (int e = t.a_ptr[ia]; e < t.a_ptr[ia + 1]; ++e) {
            const double2 y = Y[t.a_pq[e] * t.dim + int64_t(t.a_j[e]) * t.nsb + ib];
            sx += t.a_sg[e] * y.x;
            sy += t.a_sg[e] * y.y;
        }
        for (int e = t.b_ptr[ib]; e < t.b_ptr[ib + 1]; ++e) {
            const double2 y = Y[t.b_pq[e] * t.dim + ia * t.nsb + t.b_j[e]];
            sx += t.b_sg[e] * y.x;
            sy += t.b_sg[e] * y.y;
        }
        sigma[I] = make_double2(sx, sy);
    }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {   // conj(a) b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// Y[pq][J] = hp_pq v[J] + 1/2 sum_rs (pq|rs) D[rs][J]
__global__ void ci_y_kernel(int n, int64_t dim, const double2* __restrict__ hp, const double2* __restrict__ eri,
                            const double2* __restrict__ v, const double2* __restrict__ D, double2* __restrict__ Y) {
    const int nn = n * n;
    const int64_t total = int64_t(nn) * dim;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < total; o += int64_t(gridDim.x) * blockDim.x) {
        const int pq = int(o / dim);
        const int64_t J = o - int64_t(pq) * dim;
        double2 acc = cmul(hp[pq], v[J]);
        for (int rs = 0; rs < nn; ++rs) {
            const double2 e = eri[pq * nn + rs];
            const double2 d = D[rs * dim + J];
            acc.x += 0.5 * (e.x * d.x - e.y * d.y);
            acc.y += 0.5 * (e.x * d.y + e.y * d.x);
        }
        Y[o] = acc;
    }
}

// RDMs: gamma_pq = C^H D[pq]; Gamma_pqrs = D[qp]^H D[rs] - delta_qr gamma_ps (thread per output).
__global__ void ci_rdm_kernel(int n, int64_t dim, const double2* __restrict__ C, const double2* __restrict__ D,
                              double2* __restrict__ g1, double2* __restrict__ g2) {
    const int nn = n * n;
    const int total = nn + nn * nn;
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < total; o += gridDim.x * blockDim.x) {
        double sx = 0.0, sy = 0.0;
        if (o < nn) {
            for (int64_t I = 0; I < dim; ++I) {
                const double2 t = cconjmul(C[I], D[o * dim + I]);
                sx += t.x;
                sy += t.y;
            }
            g1[o] = make_double2(sx, sy);
        } else {
            const int x = o - nn;
            const int pq = x / nn, rs = x - pq * nn;
            const int p = pq / n, q = pq - p * n;
            const int qp = q * n + p;
            for (int64_t I = 0; I < dim; ++I) {
                const double2 t = cconjmul(D[qp * dim + I], D[rs * dim + I]);
                sx += t.x;
                sy += t.y;
            }
            g2[x] = make_double2(sx, sy);   // delta_qr gamma_ps subtracted in the small kernel
        }
    }
}

// Taylor term: t_next = c_k (sigma - shift t), acc += t_next  (c_k = -i dt / k;
// imaginary time: c_k = -dt / k)
__global__ void ci_taylor_kernel(int64_t dim, const double2* __restrict__ sigma, const double2* __restrict__ t,
                                 const double* __restrict__ shift, double ck, int imag, double2* __restrict__ tn,
                                 double2* __restrict__ acc) {
    const double s = *shift;
    for (int64_t I = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; I < dim; I += int64_t(gridDim.x) * blockDim.x) {
        const double2 u = make_double2(sigma[I].x - s * t[I].x, sigma[I].y - s * t[I].y);
        const double2 r = imag ? make_double2(-ck * u.x, -ck * u.y)    // -ck u
                               : make_double2(ck * u.y, -ck * u.x);    // -i ck u
        tn[I] = r;
        acc[I].x += r.x;
        acc[I].y += r.y;
    }
}

// C = exp(-i dt shift) acc
__global__ void ci_phase_kernel(int64_t dim, const double2* __restrict__ acc, const double* __restrict__ shift,
                                double dt, double2* __restrict__ C) {
    double sn, cs;
    sincos(dt * *shift, &sn, &cs);
    for (int64_t I = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; I < dim; I += int64_t(gridDim.x) * blockDim.x) {
        const double2 v = acc[I];
        C[I] = make_double2(cs * v.x + sn * v.y, cs * v.y - sn * v.x);
    }
}

// C = acc / ||acc|| (one block; the imaginary-time CI step)
__global__ void ci_normalize_kernel(int64_t dim, const double2* __restrict__ acc, double2* __restrict__ C) {
    __shared__ double sa[256];
    __shared__ double s_scale;
    double a = 0.0;
    for (int64_t I = threadIdx.x; I < dim; I += blockDim.x) a += acc[I].x * acc[I].x + acc[I].y * acc[I].y;
    sa[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0;
        for (int i = 0; i < blockDim.x; ++i) x += sa[i];
        s_scale = x > 0.0 ? 1.0 / sqrt(x) : 0.0;
    }
    __syncthreads();
    const double f = s_scale;
    for (int64_t I = threadIdx.x; I < dim; I += blockDim.x) C[I] = make_double2(f * acc[I].x, f * acc[I].y);
}

// phi[k][p] = sum_q src[k][q] T[q][p] (row-major [N][n], T [n][n]; Loewdin)
__global__ void orbital_transform_kernel(int64_t N, int n, const double2* __restrict__ src,
                                         const double2* __restrict__ T, double2* __restrict__ phi) {
    __shared__ double2 sT[64];
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) sT[i] = T[i];
    __syncthreads();
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < N * n; o += int64_t(gridDim.x) * blockDim.x) {
        const int64_t k = o / n;
        const int p = int(o - k * n);
        double x = 0.0, y = 0.0;
        for (int q = 0; q < n; ++q) {
            const double2 a = src[k * n + q], b = sT[q * n + p];
            x += a.x * b.x - a.y * b.y;
            y += a.x * b.y + a.y * b.x;
        }
        phi[o] = make_double2(x, y);
    }
}

// S^-1/2 of a Hermitian positive-definite n x n matrix (row-major, n <= 8) on
// the host: cyclic Jacobi rotations on the real symmetric embedding
// [[Re S, -Im S], [Im S, Re S]], f(R) = Q f(Lambda) Q^T, read back as
// Re = f(R)[0:n, 0:n], Im = f(R)[n:2n, 0:n].  Returns false if S is not
// positive definite.
static bool inverse_sqrt_hermitian(int n, const double2* S, double2* T) {
    const int m = 2 * n;
    double R[16][16], Q[16][16];
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) Q[i][j] = i == j ? 1.0 : 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const double re = 0.5 * (S[i * n + j].x + S[j * n + i].x);
            const double im = 0.5 * (S[i * n + j].y - S[j * n + i].y);
            R[i][j] = re;
            R[i + n][j + n] = re;
            R[i][j + n] = -im;
            R[i + n][j] = im;
        }
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                tot += R[i][j] * R[i][j];
                if (i != j) off += R[i][j] * R[i][j];
            }
        if (off <= 1e-32 * tot) break;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                if (R[p][q] == 0.0) continue;
                const double theta = 0.5 * (R[q][q] - R[p][p]) / R[p][q];
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < m; ++k) {   // columns p, q
                    const double rkp = R[k][p], rkq = R[k][q];
                    R[k][p] = c * rkp - s * rkq;
                    R[k][q] = s * rkp + c * rkq;
                }
                for (int k = 0; k < m; ++k) {   // rows p, q
                    const double rpk = R[p][k], rqk = R[q][k];
                    R[p][k] = c * rpk - s * rqk;
                    R[q][k] = s * rpk + c * rqk;
                }
                for (int k = 0; k < m; ++k) {
                    const double qkp = Q[k][p], qkq = Q[k][q];
                    Q[k][p] = c * qkp - s * qkq;
                    Q[k][q] = s * qkp + c * qkq;
                }
            }
    }
    double f[16];
    for (int i = 0; i < m; ++i) {
        if (!(R[i][i] > 0.0)) return false;
        f[i] = 1.0 / std::sqrt(R[i][i]);
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double re = 0.0, im = 0.0;
            for (int k = 0; k < m; ++k) {
                re += Q[i][k] * f[k] * Q[j][k];
                im += Q[i + n][k] * f[k] * Q[j][k];
            }
            T[i * n + j] = make_double2(re, im);
        }
    return true;
}

// shift = Re(C^H sigma) / (C^H C)   (one block)
__global__ void ci_shift_kernel(int64_t dim, const double2* __restrict__ C, const double2* __restrict__ sigma,
                                double* __restrict__ shift) {
    __shared__ double sa[256], sb[256];
    double a = 0.0, b = 0.0;
    for (int64_t I = threadIdx.x; I < dim; I += blockDim.x) {
        a += C[I].x * sigma[I].x + C[I].y * sigma[I].y;
        b += C[I].x * C[I].x + C[I].y * C[I].y;
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int i = 0; i < blockDim.x; ++i) {
            x += sa[i];
            y += sb[i];
        }
        *shift = x / y;
    }
}

// ------------------------------------------------------ small FP64 block
// One thread: gamma^-1 (Gauss-Jordan, partial pivoting), Gamma' = gamma^-1 Gamma,
// the field-combination matrix M, h'_pq, the energy and cond-type status.
struct SmallOut {
    double2* hp;      // [n*n]  h_pq - 1/2 sum_r (pr|rq)
    double2* M;       // [n*n][n*n]  U_pq = sum_c M[pq][c] Wcol_c
    double* energy;   // [1]
    int* status;      // [1] 0 ok, 1 singular gamma
};

__global__ void small_block_kernel(int n, const double2* __restrict__ h, const double2* __restrict__ eri,
                                   const double2* __restrict__ g1, double2* __restrict__ g2, SmallOut o) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int nn = n * n;
    // Gamma_pqrs -= delta_qr gamma_ps
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q)
            for (int s = 0; s < n; ++s) {
                double2& x = g2[(p * n + q) * nn + q * n + s];
                x.x -= g1[p * n + s].x;
                x.y -= g1[p * n + s].y;
            }
    // energy
    double E = 0.0;
    for (int pq = 0; pq < nn; ++pq) E += h[pq].x * g1[pq].x - h[pq].y * g1[pq].y;
    for (int x = 0; x < nn * nn; ++x) E += 0.5 * (eri[x].x * g2[x].x - eri[x].y * g2[x].y);
    *o.energy = E;
    // h'
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q) {
            double2 a = h[p * n + q];
            for (int r = 0; r < n; ++r) {
                const double2 e = eri[(p * n + r) * nn + r * n + q];
                a.x -= 0.5 * e.x;
                a.y -= 0.5 * e.y;
            }
            o.hp[p * n + q] = a;
        }
    // gamma^-1
    double2 A[8][16];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j)
            A[i][j] = j < n ? g1[i * n + j] : make_double2(j - n == i ? 1.0 : 0.0, 0.0);
    double amax = 0.0;
    for (int i = 0; i < nn; ++i) amax = fmax(amax, hypot(g1[i].x, g1[i].y));
    int singular = 0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        double best = hypot(A[c][c].x, A[c][c].y);
        for (int r = c + 1; r < n; ++r) {
            const double v = hypot(A[r][c].x, A[r][c].y);
            if (v > best) {
                best = v;
                piv = r;
            }
        }
        if (!(best > 1e-14 * amax)) {
            singular = 1;
            break;
        }
        if (piv != c)
            for (int j = 0; j < 2 * n; ++j) {
                const double2 t = A[c][j];
                A[c][j] = A[piv][j];
                A[piv][j] = t;
            }
        const double2 d = A[c][c];
        const double dd = d.x * d.x + d.y * d.y;
        const double2 inv = make_double2(d.x / dd, -d.y / dd);
        for (int j = 0; j < 2 * n; ++j) A[c][j] = cmul(A[c][j], inv);
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double2 f = A[r][c];
            for (int j = 0; j < 2 * n; ++j) {
                const double2 t = cmul(f, A[c][j]);
                A[r][j].x -= t.x;
                A[r][j].y -= t.y;
            }
        }
    }
    *o.status = singular;
    if (singular) return;
    // M[pq][c] from Gamma'_pqrs = sum_o (gamma^-1)_po Gamma_oqrs
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q) {
            auto Gp = [&](int r, int s) {
                double2 acc = make_double2(0.0, 0.0);
                for (int oo = 0; oo < n; ++oo) {
                    const double2 t = cmul(A[p][n + oo], g2[(oo * n + q) * nn + r * n + s]);
                    acc.x += t.x;
                    acc.y += t.y;
                }
                return acc;
            };
            double2* row = o.M + (p * n + q) * nn;
            for (int r = 0; r < n; ++r) row[r] = Gp(r, r);
            int c = n;
            for (int r = 0; r < n; ++r)
                for (int s = r + 1; s < n; ++s) {
                    const double2 a = Gp(r, s), b = Gp(s, r);
                    row[c++] = make_double2(a.x + b.x, a.y + b.y);           // Re column
                    row[c++] = make_double2(-(a.y - b.y), a.x - b.x);        // i (a - b), Im column
                }
        }
}

// <sum_i r_i>_d = sum_pq Re(Z_d[pq] gamma[pq]) for d = x, y, z (one thread; the
// same contraction as the one-body energy, with the position matrices).
__global__ void dipole_kernel(int n, const double2* __restrict__ Z, const double2* __restrict__ g1,
                              double* __restrict__ dip) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int nn = n * n;
    for (int d = 0; d < 3; ++d) {
        double acc = 0.0;
        for (int pq = 0; pq < nn; ++pq) acc += Z[d * nn + pq].x * g1[pq].x - Z[d * nn + pq].y * g1[pq].y;
        dip[d] = acc;
    }
}

// U[k][pq] = sum_c M[pq][c] Wcol[k][c]
__global__ void ufield_kernel(int n, int64_t N, const double2* __restrict__ M, const double* __restrict__ W,
                              double2* __restrict__ U) {
    extern __shared__ double2 s_M[];
    const int nn = n * n;
    for (int i = threadIdx.x; i < nn * nn; i += blockDim.x) s_M[i] = M[i];
    __syncthreads();
    const int64_t total = N * nn;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < total; o += int64_t(gridDim.x) * blockDim.x) {
        const int64_t k = o / nn;
        const int pq = int(o - k * nn);
        double x = 0.0, y = 0.0;
        for (int c = 0; c < nn; ++c) {
            const double w = W[k * nn + c];
            x = fma(s_M[pq * nn + c].x, w, x);
            y = fma(s_M[pq * nn + c].y, w, y);
        }
        U[o] = make_double2(x, y);
    }
}

// Two-electron integrals X[pq][c] = sum_f m_f conj(phi_p) phi_q Wcol_c at all
// support points (masters, then hanging points interpolated through C).
constexpr int kIntTile = 32;
struct IntArgs {
    const double2* phi;
    const double* W;
    int n;
    int64_t N, n_int, nh;
    const double* mf_m;
    const double* mf_h;
    const int32_t* hp;
    const int32_t* hm;
    const double* hw;
};

__global__ void __launch_bounds__(256) integrals_kernel(IntArgs a, double2* __restrict__ partial) {
    extern __shared__ __align__(16) double smem_i[];
    const int n = a.n, nn = n * n;
    double2* s_d = reinterpret_cast<double2*>(smem_i);            // [T][nn] m_f conj(phi_p) phi_q
    double* s_w = reinterpret_cast<double*>(s_d + kIntTile * nn);  // [T][nn]
    double2* s_X = reinterpret_cast<double2*>(s_w + kIntTile * nn); // [nn][nn]
    const int tid = threadIdx.x;
    for (int o = tid; o < nn * nn; o += blockDim.x) s_X[o] = make_double2(0.0, 0.0);
    const int64_t npts = a.N + a.nh;
    const int64_t ntiles = (npts + kIntTile - 1) / kIntTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        // (point, column) work items for the tile
        for (int it = tid; it < kIntTile * nn; it += blockDim.x) {
            const int tp = it / nn, c = it - tp * nn;
            const int64_t f = tile * kIntTile + tp;
            double wv = 0.0;
            double2 dv = make_double2(0.0, 0.0);
            if (f < npts) {
                const int p = c / n, q = c - p * n;
                double2 fp = make_double2(0.0, 0.0), fq = make_double2(0.0, 0.0);
                double mf;
                if (f < a.N) {
                    wv = a.W[f * nn + c];
                    if (f < a.n_int) {
                        fp = a.phi[f * n + p];
                        fq = a.phi[f * n + q];
                    }
                    mf = a.mf_m[f];
                } else {
                    const int64_t h = f - a.N;
                    for (int e = a.hp[h]; e < a.hp[h + 1]; ++e) {
                        const int64_t m = a.hm[e];
                        const double w = a.hw[e];
                        wv = fma(w, a.W[m * nn + c], wv);
                        if (m < a.n_int) {
                            const double2 x = a.phi[m * n + p], y = a.phi[m * n + q];
                            fp.x = fma(w, x.x, fp.x);
                            fp.y = fma(w, x.y, fp.y);
                            fq.x = fma(w, y.x, fq.x);
                            fq.y = fma(w, y.y, fq.y);
                        }
                    }
                    mf = a.mf_h[h];
                }
                dv = cconjmul(fp, fq);
                dv.x *= mf;
                dv.y *= mf;
            }
            s_d[tp * nn + c] = dv;
            s_w[tp * nn + c] = wv;
        }
        __syncthreads();
        for (int o = tid; o < nn * nn; o += blockDim.x) {
            const int pq = o / nn, c = o - pq * nn;
            double2 acc = s_X[o];
            for (int t = 0; t < kIntTile; ++t) {
                const double w = s_w[t * nn + c];
                const double2 d = s_d[t * nn + pq];
                acc.x = fma(d.x, w, acc.x);
                acc.y = fma(d.y, w, acc.y);
            }
            s_X[o] = acc;
        }
    }
    __syncthreads();
    for (int o = tid; o < nn * nn; o += blockDim.x) partial[int64_t(blockIdx.x) * nn * nn + o] = s_X[o];
}

// eri[pq][rs] from X[pq][c] and h_pq from hdot; both written complex.
__global__ void assemble_eri_kernel(int n, const double2* __restrict__ X, double2* __restrict__ eri) {
    const int nn = n * n;
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nn * nn; o += gridDim.x * blockDim.x) {
        const int pq = o / nn, rs = o - pq * nn;
        const int r = rs / n, s = rs - r * n;
        double2 v;
        if (r == s) {
            v = X[pq * nn + r];
        } else {
            const int lo = r < s ? r : s, hi = r < s ? s : r;
            // column index of pair (lo, hi): n + 2 * (#pairs before it)
            const int before = lo * n - lo * (lo + 1) / 2 + (hi - lo - 1);
            const double2 re = X[pq * nn + n + 2 * before], im = X[pq * nn + n + 2 * before + 1];
            v = r < s ? make_double2(re.x - im.y, re.y + im.x) : make_double2(re.x + im.y, re.y - im.x);
        }
        eri[o] = v;
    }
}

static int int_blocks() { return 4 * device_sms(); }   // integral partial rows: 4 blocks per SM
constexpr int kTaylorTerms = 30;

// ------------------------------------------------------------------ solver
}  // namespace afem

struct afem_mctdhf {
    afem_mesh* mesh = nullptr;
    int n = 0, na = 0, nb = 0, krylov_m = 0;
    int precision = AFEM_PREC_FP64;
    double krylov_tol = 0.0;   // 0: one Krylov step per time step (fixed dimension)
    int krylov_adaptive = 0;   // > 0: Sec. 3.2's rule with this many equal Krylov steps per time step
    int imaginary = 0;         // 1: imaginary-time steps (ground-state preparation)
    int gauge = AFEM_GAUGE_LENGTH;
    afem::CiTables ci;
    afem::Workspace ws;
};

namespace afem {

struct StepWork {
    double2 *y, *phi_new, *U, *ipartial, *X, *eri, *h, *g1, *g2, *hp, *M, *cpart;
    double2 *D, *Y, *sigma, *t0, *t1, *acc;
    double2* Z;   // [3][n][n] phi_p^H F[x_d] phi_q
    double *energy, *shift, *dip;
    int* status;
    int* tc_status;   // tensor-core integrals: nonzero if a block gave up waiting
    float2* U32;
    unsigned* counters;
};

static void carve_step(Carver& cv, StepWork& w, int64_t N, int n, int64_t dim, bool mixed) {
    const int nn = n * n;
    w.y = cv.take<double2>(size_t(N) * n);
    w.phi_new = cv.take<double2>(size_t(N) * n);
    w.U = cv.take<double2>(size_t(N) * nn);
    w.ipartial = cv.take<double2>(size_t(int_blocks()) * nn * nn);
    w.X = cv.take<double2>(size_t(nn) * nn);
    w.eri = cv.take<double2>(size_t(nn) * nn);
    w.h = cv.take<double2>(nn);
    w.g1 = cv.take<double2>(nn);
    w.g2 = cv.take<double2>(size_t(nn) * nn);
    w.hp = cv.take<double2>(nn);
    w.M = cv.take<double2>(size_t(nn) * nn);
    w.cpart = cv.take<double2>(size_t(kRedBlocksMax) * 256);
    w.D = cv.take<double2>(size_t(nn) * dim);
    w.Y = cv.take<double2>(size_t(nn) * dim);
    w.sigma = cv.take<double2>(dim);
    w.t0 = cv.take<double2>(dim);
    w.t1 = cv.take<double2>(dim);
    w.acc = cv.take<double2>(dim);
    w.energy = cv.take<double>(1);
    w.shift = cv.take<double>(1);
    w.Z = cv.take<double2>(size_t(3) * nn);
    w.dip = cv.take<double>(3);
    w.status = cv.take<int>(1);
    w.tc_status = cv.take<int>(1);
    w.U32 = mixed ? cv.take<float2>(size_t(N) * nn) : nullptr;
    w.counters = cv.take<unsigned>(4);
}

static void finalize_cpartials(const double2* partial, int nblk, int k, double2* out, cudaStream_t s);

__global__ void csum_blocks_kernel(const double2* __restrict__ partial, int nblk, int k, double2* __restrict__ out) {
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < k; o += gridDim.x * blockDim.x) {
        double x = 0.0, y = 0.0;
        for (int b = 0; b < nblk; ++b) {
            x += partial[int64_t(b) * k + o].x;
            y += partial[int64_t(b) * k + o].y;
        }
        out[o] = make_double2(x, y);
    }
}

static void finalize_cpartials(const double2* partial, int nblk, int k, double2* out, cudaStream_t s) {
    AFEM_LAUNCH((csum_blocks_kernel), (k + 255) / 256, 256, 0, s, partial, nblk, k, out);
}

// eri[pq][rs] = (pq|rs) of orbitals phi with the pair mean fields W: the
// contraction X[pq][c] over all support points (FP64 kernel, or the tensor
// cores in the precision form), the fixed-order sum of the block partials and
// the assembly of the complex W^r_s columns.  partial: [int_blocks()][n^4]
// complex; tc_status: device int, zeroed by the caller.
static int pair_integrals(const afem_mesh* m, const double2* phi, const double* W, int n, bool tensor_cores,
                          double2* partial, double2* X, double2* eri, int* tc_status, cudaStream_t s) {
    const DeviceMesh& D = m->dev;
    const int nn = n * n;
    const int iblk = int_blocks();
    if (tensor_cores) {
        const int rc = integrals_tc(m, phi, W, n, partial, iblk, tc_status, s);
        if (rc) return rc;
    } else {
        IntArgs ia{phi, W, n, D.n_master, D.n_interior, D.n_hanging, D.mf_master, D.mf_hang, D.hang_ptr,
                   D.hang_master, D.hang_w};
        const size_t ismem =
            size_t(kIntTile) * nn * (sizeof(double2) + sizeof(double)) + size_t(nn) * nn * sizeof(double2);
        AFEM_CUDA_TRY(
            allow_dyn_smem(integrals_kernel));
        AFEM_LAUNCH((integrals_kernel), iblk, 256, ismem, s, ia, partial);
    }
    finalize_cpartials(partial, iblk, nn * nn, X, s);
    AFEM_LAUNCH((assemble_eri_kernel), (nn * nn + 255) / 256, 256, 0, s, n, X, eri);
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

int two_electron_integrals(afem_mesh* m, const double2* phi, int n, const double* W, double2* eri, int precision,
                           cudaStream_t s) {
    const int nn = n * n;
    const size_t part_bytes = size_t(int_blocks()) * nn * nn * sizeof(double2);
    const size_t x_bytes = size_t(nn) * nn * sizeof(double2);
    int rc = m->ws_int.reserve(part_bytes + x_bytes + 256);
    if (rc) return rc;
    char* base = static_cast<char*>(m->ws_int.ptr);
    double2* partial = reinterpret_cast<double2*>(base);
    double2* X = reinterpret_cast<double2*>(base + part_bytes);
    int* status = reinterpret_cast<int*>(base + part_bytes + x_bytes);
    AFEM_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    if ((rc = pair_integrals(m, phi, W, n, precision == AFEM_PREC_MIXED, partial, X, eri, status, s))) return rc;
    int st = 0;
    AFEM_CUDA_TRY(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    AFEM_CUDA_TRY(cudaStreamSynchronize(s));
    if (st) return set_error(AFEM_ECUDA, "afem_two_electron_integrals: tensor-core blocks gave up waiting for their MMAs");
    return AFEM_OK;
}

static unsigned ci_grid(int64_t dim) { return grid_for(dim, 128, 8); }

// sigma = H_CI v via D = E v, Y, gather
static int ci_sigma(const CiTables& t, const StepWork& w, const double2* v, double2* sigma, cudaStream_t s) {
    AFEM_LAUNCH((ci_excite_kernel), ci_grid(t.dim), 128, 0, s, t, v, w.D);
    AFEM_LAUNCH((ci_y_kernel), grid_for(int64_t(t.n) * t.n * t.dim, 256, 8), 256, 0, s, t.n, t.dim, w.hp, w.eri, v, w.D, w.Y);
    AFEM_LAUNCH((ci_gather_kernel), ci_grid(t.dim), 128, 0, s, t, w.Y, sigma);
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

int launch_op_apply(afem_mesh* m, int kind, const double* E, const void* x, void* y, int nvec, cudaStream_t s);

int mctdhf_step(afem_mctdhf* S, double2* phi, double2* C, double* W, const double* E, double dt, double cg_rtol,
                int cg_max_it, afem_step_info* info, cudaStream_t s) {
    afem_mesh* m = S->mesh;
    const DeviceMesh& D = m->dev;
    const int n = S->n, nn = n * n;
    const int64_t N = D.n_master, dim = S->ci.dim;
    if (m->ecs_on && (S->imaginary || S->gauge == AFEM_GAUGE_VELOCITY))
        return set_error(AFEM_EINVAL, "afem_mctdhf_step: complex scaling is built for real-time, length-gauge steps");
    StepWork w{};
    Carver measure(nullptr);
    const bool mixed_form = S->precision == AFEM_PREC_MIXED;
    carve_step(measure, w, N, n, dim, mixed_form);
    int rc = S->ws.reserve(measure.size());
    if (rc) return rc;
    Carver cv(S->ws.ptr);
    carve_step(cv, w, N, n, dim, mixed_form);

    // 1. mean fields
    int iters = 0;
    std::vector<double> relres(nn);
    int outer = 0;
    if (mixed_form)
        rc = poisson_batch_mixed(m, phi, n, W, cg_rtol, cg_max_it, 1, 1e-2, &iters, &outer, relres.data(), s);
    else
        rc = poisson_batch(m, phi, n, W, cg_rtol, cg_max_it, 1, &iters, relres.data(), s);
    if (rc && rc != AFEM_ECG_MAXIT) return rc;
    const int cg_rc = rc;
    // 2. integrals: h_pq = phi_p^H M_L (M_L^-1 H1~ phi_q);  (pq|rs)
    if ((rc = launch_op_apply(m, S->gauge == AFEM_GAUGE_VELOCITY ? AFEM_OP_H1_VG : AFEM_OP_H1, E, phi, w.y, n, s)))
        return rc;
    AFEM_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 4 * sizeof(unsigned), s));
    if ((rc = cdot(phi, n, w.y, n, D.ml, D.n_interior, 0, w.cpart, w.h, w.counters, s))) return rc;
    // position matrices Z_d[pq] = phi_p^H F[x_d] phi_q = phi_p^H M_L (M_L^-1 F[x_d] phi_q)
    for (int d = 0; d < 3; ++d) {
        const double e[3] = {d == 0 ? 1.0 : 0.0, d == 1 ? 1.0 : 0.0, d == 2 ? 1.0 : 0.0};
        if ((rc = launch_op_apply(m, AFEM_OP_POS, e, phi, w.y, n, s))) return rc;
        if ((rc = cdot(phi, n, w.y, n, D.ml, D.n_interior, 0, w.cpart, w.Z + d * nn, w.counters, s))) return rc;
    }
    AFEM_CUDA_TRY(cudaMemsetAsync(w.tc_status, 0, sizeof(int), s));
    if ((rc = pair_integrals(m, phi, W, n, mixed_form, w.ipartial, w.X, w.eri, w.tc_status, s))) return rc;
    // RDMs of C(t)
    AFEM_LAUNCH((ci_excite_kernel), ci_grid(dim), 128, 0, s, S->ci, C, w.D);
    AFEM_LAUNCH((ci_rdm_kernel), (nn + nn * nn + 127) / 128, 128, 0, s, n, dim, C, w.D, w.g1, w.g2);
    SmallOut so{w.hp, w.M, w.energy, w.status};
    AFEM_LAUNCH((dipole_kernel), 1, 32, 0, s, n, w.Z, w.g1, w.dip);
    AFEM_LAUNCH((small_block_kernel), 1, 32, 0, s, n, w.h, w.eri, w.g1, w.g2, so);
    AFEM_CUDA_TRY(cudaGetLastError());
    int status = 0;
    double energy = 0.0, dipole[3] = {0.0, 0.0, 0.0};
    AFEM_CUDA_TRY(cudaMemcpyAsync(&status, w.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    int tc_status = 0;
    AFEM_CUDA_TRY(cudaMemcpyAsync(&tc_status, w.tc_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    AFEM_CUDA_TRY(cudaMemcpyAsync(&energy, w.energy, sizeof(double), cudaMemcpyDeviceToHost, s));
    AFEM_CUDA_TRY(cudaMemcpyAsync(dipole, w.dip, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    AFEM_CUDA_TRY(cudaStreamSynchronize(s));
    if (tc_status)
        return set_error(AFEM_ECUDA, "afem_mctdhf_step: tensor-core integrals gave up waiting for their MMAs");
    if (status) return set_error(AFEM_ESINGULAR, "afem_mctdhf_step: one-body density matrix is singular");
    // 3. C(t+dt) = exp(-i dt H_CI) C(t): Taylor series of (H - shift), times exp(-i dt shift)
    if ((rc = ci_sigma(S->ci, w, C, w.sigma, s))) return rc;
    AFEM_LAUNCH((ci_shift_kernel), 1, 256, 0, s, dim, C, w.sigma, w.shift);
    AFEM_CUDA_TRY(cudaMemcpyAsync(w.acc, C, dim * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    AFEM_CUDA_TRY(cudaMemcpyAsync(w.t0, C, dim * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    double2* tk = w.t0;
    double2* tn = w.t1;
    for (int k = 1; k <= kTaylorTerms; ++k) {
        if (k > 1 && (rc = ci_sigma(S->ci, w, tk, w.sigma, s))) return rc;
        AFEM_LAUNCH((ci_taylor_kernel), ci_grid(dim), 128, 0, s, dim, w.sigma, tk, w.shift, dt / k, S->imaginary,
                    tn, w.acc);
        std::swap(tk, tn);
    }
    AFEM_CUDA_TRY(cudaGetLastError());
    // 4. mean-field operator fields and the orbital step
    const size_t usmem = size_t(nn) * nn * sizeof(double2);
    AFEM_CUDA_TRY(allow_dyn_smem(ufield_kernel));
    AFEM_LAUNCH((ufield_kernel), grid_for(N * nn), 256, usmem, s, n, N, w.M, W, w.U);
    AFEM_CUDA_TRY(cudaGetLastError());
    double err = 0.0;
    int m_used = 0, brk = 0;
    const int mixed = S->precision == AFEM_PREC_MIXED;
    float2* U32 = nullptr;
    if (mixed) {
        U32 = w.U32;
        if ((rc = to_c64(w.U, U32, N * nn, s))) return rc;
    }
    int substeps = 1, dim_sum = 0, unmet = 0;
    if (S->krylov_adaptive > 0 && !(S->krylov_tol > 0.0))
        return set_error(AFEM_EINVAL, "afem_mctdhf_step: the adaptive Krylov dimension needs a threshold > 0");
    if ((rc = arnoldi_step(m, E, phi, mixed ? nullptr : w.U, U32, n, S->krylov_m, dt, mixed, S->krylov_tol,
                           w.phi_new, &err, &m_used, &brk, &substeps, s,
                           (S->imaginary ? kArnImaginary : 0) | (S->gauge == AFEM_GAUGE_VELOCITY ? kArnVelocity : 0),
                           S->krylov_adaptive, &dim_sum, &unmet)))
        return rc;
    if (S->imaginary) {
        // commit: phi <- phi_new S^-1/2 (Loewdin, S = phi_new^H M_L phi_new), C <- acc / ||acc||
        AFEM_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 4 * sizeof(unsigned), s));
        if ((rc = cdot(w.phi_new, n, w.phi_new, n, D.ml, D.n_interior, 0, w.cpart, w.h, w.counters, s))) return rc;
        double2 Sh[64], Th[64];
        AFEM_CUDA_TRY(cudaMemcpyAsync(Sh, w.h, size_t(nn) * sizeof(double2), cudaMemcpyDeviceToHost, s));
        AFEM_CUDA_TRY(cudaStreamSynchronize(s));
        if (!inverse_sqrt_hermitian(n, Sh, Th))
            return set_error(AFEM_ESINGULAR, "afem_mctdhf_step: orbital overlap not positive definite (imaginary time)");
        AFEM_CUDA_TRY(cudaMemcpyAsync(w.hp, Th, size_t(nn) * sizeof(double2), cudaMemcpyHostToDevice, s));
        AFEM_LAUNCH((orbital_transform_kernel), grid_for(N * n), 256, 0, s, N, n, w.phi_new, w.hp, phi);
        AFEM_LAUNCH((ci_normalize_kernel), 1, 256, 0, s, dim, w.acc, C);
        AFEM_CUDA_TRY(cudaGetLastError());
        AFEM_CUDA_TRY(cudaStreamSynchronize(s));   // Th is read by the copy before it leaves scope
    } else {
        // commit: phi <- phi_new, C <- exp(-i dt shift) acc
        AFEM_CUDA_TRY(cudaMemcpyAsync(phi, w.phi_new, size_t(N) * n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        AFEM_LAUNCH((ci_phase_kernel), ci_grid(dim), 128, 0, s, dim, w.acc, w.shift, dt, C);
    }
    AFEM_CUDA_TRY(cudaGetLastError());
    AFEM_CUDA_TRY(cudaStreamSynchronize(s));
    if (info) {
        info->energy = energy;
        for (int d = 0; d < 3; ++d) info->dipole[d] = dipole[d];
        info->arnoldi_err = err;
        info->krylov_m_used = m_used;
        info->breakdown = brk;
        info->krylov_substeps = substeps;
        info->krylov_dim_sum = S->krylov_adaptive > 0 ? dim_sum : substeps * m_used;
        info->krylov_unmet = unmet;
        info->cg_iters = iters;
        double mx = 0.0;
        for (double r : relres) mx = std::max(mx, r);
        info->cg_relres_max = mx;
    }
    return cg_rc;
}

int mctdhf_create(afem_mesh* m, int n, int na, int nb, int mk, afem_mctdhf** out) {
    afem_mctdhf* S = new (std::nothrow) afem_mctdhf();
    if (!S) return set_error(AFEM_ENOMEM, "afem_mctdhf_create: host allocation failed");
    S->mesh = m;
    S->n = n;
    S->na = na;
    S->nb = nb;
    S->krylov_m = mk;
    CiTables& t = S->ci;
    t.n = n;
    t.na = na;
    t.nb = nb;
    int rc = build_lists(n, na, t.a_ptr, t.a_pq, t.a_j, t.a_sg, t.nsa);
    if (!rc) rc = build_lists(n, nb, t.b_ptr, t.b_pq, t.b_j, t.b_sg, t.nsb);
    t.dim = t.nsa * t.nsb;
    if (rc) {
        mctdhf_destroy(S);
        return rc;
    }
    *out = S;
    return AFEM_OK;
}

void mctdhf_destroy(afem_mctdhf* S) {
    if (!S) return;
    CiTables& t = S->ci;
    cudaFree(t.a_ptr);
    cudaFree(t.a_pq);
    cudaFree(t.a_j);
    cudaFree(t.a_sg);
    cudaFree(t.b_ptr);
    cudaFree(t.b_pq);
    cudaFree(t.b_j);
    cudaFree(t.b_sg);
    S->ws.release();
    delete S;
}

int64_t mctdhf_ci_dim(const afem_mctdhf* S) { return S->ci.dim; }

afem_mesh* mctdhf_mesh_of(const afem_mctdhf* S) { return S->mesh; }

int mctdhf_orbitals_of(const afem_mctdhf* S) { return S->n; }

void mctdhf_set_precision(afem_mctdhf* S, int precision) { S->precision = precision; }

void mctdhf_set_krylov_tol(afem_mctdhf* S, double tol) { S->krylov_tol = tol; }

void mctdhf_set_krylov_adaptive(afem_mctdhf* S, int steps) { S->krylov_adaptive = steps; }

void mctdhf_set_imaginary(afem_mctdhf* S, int on) { S->imaginary = on ? 1 : 0; }

void mctdhf_set_gauge(afem_mctdhf* S, int gauge) { S->gauge = gauge; }

}  // namespace afem
