// Geometric multigrid preconditioner for the batched Poisson solves of the
// mean fields (Sec. 3.1, Eq. mean-field: the paper solves them by CG with an
// algebraic multigrid preconditioner; this is its geometric counterpart on the
// octree the library already holds).
//
// Levels, fine to coarse: the mesh itself (degree p); the same leaves at
// degree p/2, ..., 1 (p-coarsening); then degree 1 on the octree truncated at
// levels L-1, ..., 0 (h-coarsening: every leaf finer than the cap replaced by
// its ancestor there; the last is the uniform coarse grid).  Every leaf of a
// level has an ancestor-or-self leaf on the next coarser octree, whatever rule
// refined the mesh, and the coarse finite-element space is a
// subspace of the fine one, so the prolongation P is exact interpolation: the
// value of the coarse function at each interior fine master, evaluated in one
// "owner" cell that holds the master as a node (the lowest-index such cell).
// The restriction is R = P^T (the owner's interpolation weights, transposed,
// then the coarse constraints C^T), so the V-cycle is a symmetric operator.
// Smoothing: Chebyshev polynomials in D^-1 A (D the diagonal of the
// constrained stiffness) on [lambda_max / 15, 1.15 lambda_max], degree 3 before
// and after the coarse correction; lambda_max by power iteration at set-up;
// the coarsest level gets a degree-30 Chebyshev polynomial on
// [lambda_max / 400, 1.15 lambda_max].  All levels act on the Dirichlet
// interior (surface rows zero), every column of the batch at once.
//
// Solvers built on it: CG in float64 preconditioned by the float64 V-cycle (the
// FP64 form), and float64 defect correction whose corrections are float32 CG
// iterations preconditioned by the float32 V-cycle (the precision form).
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <unordered_set>
#include <vector>

#include "afem_internal.h"
#include "vec_common.cuh"

namespace afem {

int launch_stiffness32(const afem_mesh* m, const float* x, float* y, int nv, int masked, cudaStream_t s,
                       double* pap_slots);
int poisson_rhs_bc(afem_mesh* m, const double2* phi, int n, double* W, double* b, double* qpart, double* q,
                   cudaStream_t s);
int mom_blocks_count();
constexpr int kPmgMaxP1 = kMaxP1;
constexpr int kPmgPreDegree = 3;      // Chebyshev degree of each smoothing
constexpr int kPmgCoarseDegree = 30;  // Chebyshev degree on the coarsest level
constexpr double kPmgSmoothRange = 15.0;
constexpr double kPmgCoarseRange = 400.0;
constexpr double kPmgLambdaSafety = 1.15;
constexpr int kPmgPowerIters = 40;

struct PmgLevel {
    afem_mesh* mesh = nullptr;   // level 0: the caller's mesh (not owned)
    bool owned = false;
    // transfer from the next coarser level to this one, per cell of this level
    int32_t* coarse_cell = nullptr;   // [ncell] the coarse ancestor-or-self leaf
    float4* xform = nullptr;          // [ncell] (offset x, y, z, scale) in the coarse cell's unit cube
    uint8_t* owner = nullptr;         // [ncell][(p+1)^3] 1: this (cell, node) holds its interior master's value
    double lam_max = 0.0;             // largest eigenvalue of D^-1 A_II
};

}  // namespace afem

struct afem_pmg {
    std::vector<afem::PmgLevel> lv;
    afem::Workspace ws;   // level vectors of the current solve
};

namespace afem {

// ------------------------------------------------------------- set-up (host)
static void free_level(PmgLevel& L) {
    cudaFree(L.coarse_cell);
    cudaFree(L.xform);
    cudaFree(L.owner);
    L.coarse_cell = nullptr;
    L.xform = nullptr;
    L.owner = nullptr;
    if (L.owned && L.mesh) afem_mesh_destroy(L.mesh);
    L.mesh = nullptr;
}

void pmg_free(afem_pmg* g) {
    if (!g) return;
    for (auto& L : g->lv) free_level(L);
    g->ws.release();
    delete g;
}

template <typename T>
static int upload(T*& dst, const std::vector<T>& v) {
    dst = nullptr;
    if (v.empty()) return AFEM_OK;
    cudaError_t e = cudaMalloc(&dst, v.size() * sizeof(T));
    if (e != cudaSuccess) return set_error(AFEM_ENOMEM, "multigrid set-up: cudaMalloc failed");
    AFEM_CUDA_TRY(cudaMemcpy(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return AFEM_OK;
}

// Ancestor map and owner flags of fine level `f` over coarse level `c`.
static int build_transfer(const HostMesh& F, const HostMesh& C, PmgLevel& L) {
    const int64_t nf = int64_t(F.lev.size());
    std::map<std::tuple<int, int, int, int>, int32_t> key;
    for (int32_t c = 0; c < int32_t(C.lev.size()); ++c) key[{C.lev[c], C.ci[c], C.cj[c], C.ck[c]}] = c;
    std::vector<int32_t> cc(nf);
    std::vector<float4> xf(nf);
    for (int64_t f = 0; f < nf; ++f) {
        int l = F.lev[f], i = F.ci[f], j = F.cj[f], k = F.ck[f];
        int found = -1, lc = l;
        for (; lc >= 0; --lc) {
            const int sh = l - lc;
            auto it = key.find({lc, i >> sh, j >> sh, k >> sh});
            if (it != key.end()) {
                found = it->second;
                break;
            }
        }
        if (found < 0) return set_error(AFEM_EMESH, "multigrid set-up: a leaf has no coarse ancestor");
        const int sh = l - lc;
        const float sc = std::ldexp(1.0f, -sh);
        cc[f] = found;
        xf[f] = make_float4(float(i - ((i >> sh) << sh)) * sc, float(j - ((j >> sh) << sh)) * sc,
                            float(k - ((k >> sh) << sh)) * sc, sc);
    }
    const int nn = (F.p + 1) * (F.p + 1) * (F.p + 1);
    std::vector<uint8_t> own(size_t(nf) * nn, 0);
    std::vector<uint8_t> seen(size_t(F.n_master), 0);
    for (int64_t f = 0; f < nf; ++f)
        for (int i = 0; i < nn; ++i) {
            const int32_t idx = F.cell_node[size_t(f) * nn + i];
            if (idx < 0 || idx >= F.n_interior || seen[idx]) continue;
            seen[idx] = 1;
            own[size_t(f) * nn + i] = 1;
        }
    int rc;
    if ((rc = upload(L.coarse_cell, cc))) return rc;
    if ((rc = upload(L.xform, xf))) return rc;
    return upload(L.owner, own);
}

// ------------------------------------------------------------------ kernels
// Lagrange basis of degree pc (1 or 2) on its GLL nodes {0, 1} / {0, 1/2, 1}.
__device__ __forceinline__ float lagrange_c(int pc, int j, float t) {
    if (pc == 1) return j == 0 ? 1.0f - t : t;
    if (j == 0) return 2.0f * (t - 0.5f) * (t - 1.0f);
    if (j == 1) return -4.0f * t * (t - 1.0f);
    return 2.0f * t * (t - 0.5f);
}

struct XferArgs {
    // fine level
    const int32_t* f_node;    // [ncell][(pf+1)^3]
    const int32_t* coarse_cell;
    const float4* xform;
    const uint8_t* owner;
    int pf;
    float xi_f[kPmgMaxP1];
    // coarse level
    const int32_t* c_node;    // [ncell_c][(pc+1)^3]
    const int32_t* c_hp;
    const int32_t* c_hm;
    const double* c_hw;
    int64_t c_ni;             // coarse interior masters
    int pc;
    int k;                    // columns
};

// The (pf+1) x (pc+1) interpolation tables of one fine cell, per direction.
__device__ __forceinline__ void xfer_tables(const XferArgs& a, int64_t f, float (*tab)[kPmgMaxP1][3]) {
    const float4 x = a.xform[f];
    const float off[3] = {x.x, x.y, x.z};
    for (int t = threadIdx.x; t < 3 * (a.pf + 1) * (a.pc + 1); t += blockDim.x) {
        const int d = t / ((a.pf + 1) * (a.pc + 1));
        const int r = t - d * (a.pf + 1) * (a.pc + 1);
        const int i = r / (a.pc + 1), j = r - i * (a.pc + 1);
        tab[d][i][j] = lagrange_c(a.pc, j, off[d] + x.w * a.xi_f[i]);
    }
}

// y_f (+)= P x_c: every interior fine master gets the coarse function's value
// at its position, evaluated in its owner cell.  add: y_f += instead of =.
template <typename T>
__global__ void pmg_prolong_kernel(XferArgs a, const T* __restrict__ xc, T* __restrict__ yf, int add) {
    __shared__ float tab[3][kPmgMaxP1][3];
    __shared__ T s_c[27 * 64];
    const int64_t f = blockIdx.x;
    const int pc1 = a.pc + 1, pf1 = a.pf + 1, k = a.k;
    const int ncn = pc1 * pc1 * pc1, nfn = pf1 * pf1 * pf1;
    const int64_t cc = a.coarse_cell[f];
    xfer_tables(a, f, tab);
    for (int it = threadIdx.x; it < ncn * k; it += blockDim.x) {
        const int j = it / k, l = it - j * k;
        const int idx = a.c_node[cc * ncn + j];
        T v = T(0);
        if (idx >= 0) {
            if (idx < a.c_ni) v = xc[int64_t(idx) * k + l];
        } else {
            const int h = -idx - 1;
            for (int e = a.c_hp[h]; e < a.c_hp[h + 1]; ++e) {
                const int mm = a.c_hm[e];
                if (mm < a.c_ni) v += T(a.c_hw[e]) * xc[int64_t(mm) * k + l];
            }
        }
        s_c[it] = v;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < nfn * k; it += blockDim.x) {
        const int i = it / k, l = it - i * k;
        if (!a.owner[f * nfn + i]) continue;
        const int ia = i % pf1, ib = (i / pf1) % pf1, ic = i / (pf1 * pf1);
        T v = T(0);
        for (int jc = 0; jc < pc1; ++jc)
            for (int jb = 0; jb < pc1; ++jb) {
                const T wbc = T(tab[1][ib][jb]) * T(tab[2][ic][jc]);
                for (int ja = 0; ja < pc1; ++ja)
                    v += T(tab[0][ia][ja]) * wbc * s_c[(ja + pc1 * (jb + pc1 * jc)) * k + l];
            }
        const int64_t o = int64_t(a.f_node[f * nfn + i]) * k + l;
        yf[o] = add ? yf[o] + v : v;
    }
}

// yc += R rf = P^T rf (yc zeroed by the caller): the owner cell's interior
// fine values times the interpolation weights, summed into the coarse nodes,
// then spread through the coarse constraints to interior coarse masters.
template <typename T>
__global__ void pmg_restrict_kernel(XferArgs a, const T* __restrict__ rf, T* __restrict__ yc) {
    __shared__ float tab[3][kPmgMaxP1][3];
    __shared__ T s_f[125 * 16];
    const int64_t f = blockIdx.x;
    const int pc1 = a.pc + 1, pf1 = a.pf + 1, k = a.k;
    const int ncn = pc1 * pc1 * pc1, nfn = pf1 * pf1 * pf1;
    const int64_t cc = a.coarse_cell[f];
    xfer_tables(a, f, tab);
    // columns in chunks that fit the tile
    const int kc = k < 16 ? k : 16;
    for (int l0 = 0; l0 < k; l0 += kc) {
        const int kk = (k - l0) < kc ? (k - l0) : kc;
        __syncthreads();
        for (int it = threadIdx.x; it < nfn * kk; it += blockDim.x) {
            const int i = it / kk, l = it - i * kk;
            s_f[it] = a.owner[f * nfn + i] ? rf[int64_t(a.f_node[f * nfn + i]) * k + l0 + l] : T(0);
        }
        __syncthreads();
        for (int it = threadIdx.x; it < ncn * kk; it += blockDim.x) {
            const int j = it / kk, l = it - j * kk;
            const int ja = j % pc1, jb = (j / pc1) % pc1, jc = j / (pc1 * pc1);
            T v = T(0);
            for (int i = 0; i < nfn; ++i) {
                const int ia = i % pf1, ib = (i / pf1) % pf1, ic = i / (pf1 * pf1);
                v += T(tab[0][ia][ja]) * T(tab[1][ib][jb]) * T(tab[2][ic][jc]) * s_f[i * kk + l];
            }
            if (v == T(0)) continue;
            const int idx = a.c_node[cc * ncn + j];
            if (idx >= 0) {
                if (idx < a.c_ni) atomicAdd(&yc[int64_t(idx) * k + l0 + l], v);
            } else {
                const int h = -idx - 1;
                for (int e = a.c_hp[h]; e < a.c_hp[h + 1]; ++e) {
                    const int mm = a.c_hm[e];
                    if (mm < a.c_ni) atomicAdd(&yc[int64_t(mm) * k + l0 + l], T(a.c_hw[e]) * v);
                }
            }
        }
    }
}

// One Chebyshev step on the interior rows: res = b - A x (ax = A x, or x = 0
// when ax is null), d = c1 d + c2 D^-1 res, x += d.  first: d = c2 D^-1 res
// (d is not read: on the first step it holds whatever the workspace held).
template <typename T>
__global__ void pmg_cheb_kernel(T* __restrict__ x, T* __restrict__ d, const T* __restrict__ b,
                                const T* __restrict__ ax, const T* __restrict__ dinv, int64_t ni, int k, T c1, T c2,
                                int first) {
    const int64_t n = ni * k;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < n; o += int64_t(gridDim.x) * blockDim.x) {
        const T res = ax ? b[o] - ax[o] : b[o];
        const T dn = (first ? T(0) : c1 * d[o]) + c2 * dinv[o / k] * res;
        d[o] = dn;
        x[o] = ax ? x[o] + dn : dn;
    }
}

// r = b - ax on the interior rows.
template <typename T>
__global__ void pmg_residual_kernel(T* __restrict__ r, const T* __restrict__ b, const T* __restrict__ ax,
                                    int64_t ni, int k) {
    const int64_t n = ni * k;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < n; o += int64_t(gridDim.x) * blockDim.x)
        r[o] = b[o] - ax[o];
}

// out[c] += sum over interior rows of x[row][c] y[row][c] (FP64 accumulation)
template <typename T>
__global__ void pmg_coldot_kernel(const T* __restrict__ x, const T* __restrict__ y, int64_t ni, int k,
                                  double* __restrict__ out) {
    __shared__ double s[256];
    const int R = 256 / k;
    const int t = threadIdx.x;
    double acc = 0.0;
    if (t < R * k) {
        const int c = t % k, r0 = t / k;
        for (int64_t row = blockIdx.x * int64_t(R) + r0; row < ni; row += int64_t(gridDim.x) * R)
            acc += double(x[row * k + c]) * double(y[row * k + c]);
    }
    s[t] = acc;
    __syncthreads();
    if (t < k) {
        double v = 0.0;
        for (int r = 0; r < R; ++r) v += s[t + r * k];
        atomicAdd(&out[t], v);
    }
}

// p = z + beta p with beta = rz / rz_old per column (0 when rz_old = 0);
// first: p = z (p is not read).
template <typename T>
__global__ void pmg_pupdate_kernel(T* __restrict__ p, const T* __restrict__ z, const double* __restrict__ rz,
                                   const double* __restrict__ rz_old, int64_t ni, int k, int first) {
    const int64_t n = ni * k;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < n; o += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(o % k);
        const double ro = rz_old[c];
        if (first || !(ro > 0.0)) {
            p[o] = z[o];
            continue;
        }
        p[o] = z[o] + T(rz[c] / ro) * p[o];
    }
}

// x += alpha p, r -= alpha q with alpha = rz / pq per column (0 when pq <= 0);
// x has type TX (float64 for the FP64 CG, float32 inside the corrections).
template <typename T, typename TX>
__global__ void pmg_xr_kernel(TX* __restrict__ x, T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ q,
                              const double* __restrict__ rz, const double* __restrict__ pq, int64_t ni, int k) {
    const int64_t n = ni * k;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < n; o += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(o % k);
        const double den = pq[c];
        const double al = den > 0.0 ? rz[c] / den : 0.0;
        x[o] += TX(al) * TX(p[o]);
        r[o] -= T(al) * q[o];
    }
}

// W += e on the interior rows (the float32 correction into the float64 solution)
__global__ void pmg_add_f32_kernel(double* __restrict__ W, const float* __restrict__ e, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        W[i] += double(e[i]);
}

// deterministic start vector of the power iteration (interior rows)
__global__ void pmg_seed_kernel(double* __restrict__ x, int64_t ni) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < ni; i += int64_t(gridDim.x) * blockDim.x) {
        uint64_t h = uint64_t(i) * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
        h ^= h >> 31;
        h *= 0xBF58476D1CE4E5B9ull;
        h ^= h >> 29;
        x[i] = 0.5 + double(h >> 11) * (1.0 / 9007199254740992.0);
    }
}

// y = D^-1 y on the interior rows, one column
__global__ void pmg_jacobi_scale_kernel(double* __restrict__ y, const double* __restrict__ dinv, int64_t ni,
                                        double s) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < ni; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = s * dinv[i] * y[i];
}

__global__ void pmg_f64_to_f32_kernel(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = float(x[i]);
}

// r = b - t - ax on the interior rows (FP64 residual of the full system with
// the surface data: t = A g_ext, ax = A_II W_I)
__global__ void pmg_residual64_kernel(double* __restrict__ r, const double* __restrict__ b,
                                      const double* __restrict__ t, const double* __restrict__ ax, int64_t ni,
                                      int k) {
    const int64_t n = ni * k;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < n; o += int64_t(gridDim.x) * blockDim.x)
        r[o] = b[o] - t[o] - ax[o];
}

// --------------------------------------------------------------- host parts
template <typename T>
static int stiff(const afem_mesh* m, const T* x, T* y, int k, cudaStream_t s);
template <>
int stiff<double>(const afem_mesh* m, const double* x, double* y, int k, cudaStream_t s) {
    return launch_stiffness(m, x, y, k, 1, s);
}
template <>
int stiff<float>(const afem_mesh* m, const float* x, float* y, int k, cudaStream_t s) {
    return launch_stiffness32(m, x, y, k, 1, s, nullptr);
}
template <typename T>
static const T* dinv_of(const afem_mesh* m);
template <>
const double* dinv_of<double>(const afem_mesh* m) {
    return m->dev.stiff_dinv;
}
template <>
const float* dinv_of<float>(const afem_mesh* m) {
    return m->dev.stiff_dinv32;
}

static XferArgs xfer_args(const PmgLevel& F, const PmgLevel& C, int k) {
    XferArgs a{};
    const DeviceMesh& fd = F.mesh->dev;
    const DeviceMesh& cd = C.mesh->dev;
    a.f_node = fd.cell_node;
    a.coarse_cell = F.coarse_cell;
    a.xform = F.xform;
    a.owner = F.owner;
    a.pf = fd.p;
    for (int i = 0; i <= fd.p; ++i) a.xi_f[i] = float(F.mesh->basis.xi[i]);
    a.c_node = cd.cell_node;
    a.c_hp = cd.hang_ptr;
    a.c_hm = cd.hang_master;
    a.c_hw = cd.hang_w;
    a.c_ni = cd.n_interior;
    a.pc = cd.p;
    a.k = k;
    return a;
}

// Vectors of one level: x (solution), b (right-hand side), t (A x), d (Chebyshev direction).
template <typename T>
struct LevelVec {
    T *x, *b, *t, *d;
};

// Chebyshev smoothing of A x = b on [lo, hi] (eigenvalues of D^-1 A), `deg`
// steps, from x = 0 (zero_start) or the current x.
template <typename T>
static int chebyshev(const afem_mesh* m, LevelVec<T>& v, int k, double lo, double hi, int deg, bool zero_start,
                     cudaStream_t s) {
    const int64_t ni = m->dev.n_interior;
    if (ni == 0) return AFEM_OK;
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
    const unsigned grid = grid_for(ni * k);
    const T* dinv = dinv_of<T>(m);
    double rho = 1.0 / sigma;
    int rc;
    for (int it = 0; it < deg; ++it) {
        const bool x_zero = zero_start && it == 0;
        if (!x_zero && (rc = stiff<T>(m, v.x, v.t, k, s))) return rc;
        double c1, c2;
        if (it == 0) {
            c1 = 0.0;
            c2 = 1.0 / theta;
        } else {
            const double rho_new = 1.0 / (2.0 * sigma - rho);
            c1 = rho_new * rho;
            c2 = 2.0 * rho_new / delta;
            rho = rho_new;
        }
        AFEM_LAUNCH((pmg_cheb_kernel<T>), grid, 256, 0, s, v.x, v.d, v.b, x_zero ? nullptr : v.t, dinv, ni, k, T(c1),
                    T(c2), it == 0 ? 1 : 0);
    }
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

// z = V(l) b on level l (v[l].b holds b; the result is left in v[l].x).
template <typename T>
static int vcycle(afem_pmg* g, std::vector<LevelVec<T>>& v, int l, int k, cudaStream_t s) {
    PmgLevel& L = g->lv[l];
    const afem_mesh* m = L.mesh;
    const int64_t ni = m->dev.n_interior, N = m->dev.n_master;
    int rc;
    if (l + 1 == int(g->lv.size()))
        return chebyshev<T>(m, v[l], k, L.lam_max * kPmgLambdaSafety / kPmgCoarseRange, L.lam_max * kPmgLambdaSafety,
                            kPmgCoarseDegree, true, s);
    const double hi = L.lam_max * kPmgLambdaSafety, lo = hi / kPmgSmoothRange;
    if ((rc = chebyshev<T>(m, v[l], k, lo, hi, kPmgPreDegree, true, s))) return rc;
    // coarse right-hand side R (b - A x)
    if ((rc = stiff<T>(m, v[l].x, v[l].t, k, s))) return rc;
    AFEM_LAUNCH((pmg_residual_kernel<T>), grid_for(ni * k), 256, 0, s, v[l].t, v[l].b, v[l].t, ni, k);
    PmgLevel& C = g->lv[l + 1];
    AFEM_CUDA_TRY(cudaMemsetAsync(v[l + 1].b, 0, size_t(C.mesh->dev.n_master) * k * sizeof(T), s));
    const XferArgs xa = xfer_args(L, C, k);
    AFEM_LAUNCH((pmg_restrict_kernel<T>), unsigned(m->dev.ncell), 128, 0, s, xa, v[l].t, v[l + 1].b);
    AFEM_CUDA_TRY(cudaGetLastError());
    if ((rc = vcycle<T>(g, v, l + 1, k, s))) return rc;
    AFEM_LAUNCH((pmg_prolong_kernel<T>), unsigned(m->dev.ncell), 128, 0, s, xa, v[l + 1].x, v[l].x, 1);
    AFEM_CUDA_TRY(cudaGetLastError());
    (void)N;
    return chebyshev<T>(m, v[l], k, lo, hi, kPmgPreDegree, false, s);
}

// Largest eigenvalue of D^-1 A_II of a level by power iteration (FP64, one
// column): x_hat = x / ||x||, x <- D^-1 A x_hat, lambda ~ ||x||.
static int estimate_lambda(afem_mesh* m, double* lam, cudaStream_t s) {
    const int64_t N = m->dev.n_master, ni = m->dev.n_interior;
    *lam = 1.0;
    if (ni == 0) return AFEM_OK;
    double *x = nullptr, *y = nullptr, *acc = nullptr;
    cudaError_t e = cudaMalloc(&x, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&y, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&acc, sizeof(double));
    int rc = e == cudaSuccess ? AFEM_OK : set_error(AFEM_ENOMEM, "multigrid set-up: cudaMalloc failed");
    auto norm = [&](const double* v, double* out) -> int {
        AFEM_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(double), s));
        AFEM_LAUNCH((pmg_coldot_kernel<double>), grid_for(ni, 256, 4), 256, 0, s, v, v, ni, 1, acc);
        double h = 0.0;
        AFEM_CUDA_TRY(cudaMemcpyAsync(&h, acc, sizeof(double), cudaMemcpyDeviceToHost, s));
        AFEM_CUDA_TRY(cudaStreamSynchronize(s));
        *out = std::sqrt(h);
        return AFEM_OK;
    };
    double nx = 0.0, est = 0.0;
    if (rc == AFEM_OK) {
        if (cudaMemsetAsync(x, 0, N * sizeof(double), s) != cudaSuccess) rc = set_error(AFEM_ECUDA, "memset");
        else {
            AFEM_LAUNCH((pmg_seed_kernel), grid_for(ni), 256, 0, s, x, ni);
            rc = norm(x, &nx);
        }
    }
    for (int it = 0; rc == AFEM_OK && it < kPmgPowerIters && nx > 0.0 && std::isfinite(nx); ++it) {
        if ((rc = launch_stiffness(m, x, y, 1, 1, s))) break;
        AFEM_LAUNCH((pmg_jacobi_scale_kernel), grid_for(ni), 256, 0, s, y, m->dev.stiff_dinv, ni, 1.0 / nx);
        if ((rc = norm(y, &est))) break;
        std::swap(x, y);
        nx = est;
    }
    if (rc == AFEM_OK && est > 0.0 && std::isfinite(est)) *lam = est;
    cudaFree(x);
    cudaFree(y);
    cudaFree(acc);
    return rc;
}

// Builds the level hierarchy of mesh m (once).
static int pmg_setup(afem_mesh* m, cudaStream_t s) {
    if (m->pmg) return AFEM_OK;
    auto* g = new (std::nothrow) afem_pmg();
    if (!g) return set_error(AFEM_ENOMEM, "multigrid set-up: out of host memory");
    PmgLevel top;
    top.mesh = m;
    g->lv.push_back(top);
    int rc = AFEM_OK;
    // p-coarsening on the same leaves, then degree 1 on the leaves truncated at
    // levels Lf-1, ..., 0 (every leaf finer than the cap replaced by its
    // ancestor at the cap): each level's octree coarsens the previous one
    const HostMesh& F = m->host;
    const int Lf = F.max_level;
    std::vector<int> degrees;
    for (int p = m->desc.degree; p > 1;) {
        p = p >= 4 ? p / 2 : 1;
        degrees.push_back(p);
    }
    auto add_level = [&](int degree, int cap) -> int {
        afem_mesh_desc e = m->desc;
        e.degree = degree;
        std::vector<int32_t> lev, ci, cj, ck;
        std::unordered_set<uint64_t> seen;
        for (size_t q = 0; q < F.lev.size(); ++q) {
            const int sh = F.lev[q] > cap ? F.lev[q] - cap : 0;
            const int32_t l = F.lev[q] - sh, i = F.ci[q] >> sh, j = F.cj[q] >> sh, k = F.ck[q] >> sh;
            const uint64_t key = (uint64_t(l) << 60) | (uint64_t(i) << 40) | (uint64_t(j) << 20) | uint64_t(k);
            if (!seen.insert(key).second) continue;
            lev.push_back(l);
            ci.push_back(i);
            cj.push_back(j);
            ck.push_back(k);
        }
        afem_mesh* lm = nullptr;
        int r = create_mesh_from_cells(e, lev, ci, cj, ck, &lm);
        if (r) return r;
        PmgLevel L;
        L.mesh = lm;
        L.owned = true;
        g->lv.push_back(L);
        return AFEM_OK;
    };
    for (int p : degrees)
        if (rc == AFEM_OK) rc = add_level(p, Lf);
    for (int cap = Lf - 1; rc == AFEM_OK && cap >= 0; --cap) rc = add_level(1, cap);
    for (size_t l = 0; rc == AFEM_OK && l + 1 < g->lv.size(); ++l)
        rc = build_transfer(g->lv[l].mesh->host, g->lv[l + 1].mesh->host, g->lv[l]);
    for (size_t l = 0; rc == AFEM_OK && l < g->lv.size(); ++l) rc = estimate_lambda(g->lv[l].mesh, &g->lv[l].lam_max, s);
    if (rc) {
        pmg_free(g);
        return rc;
    }
    m->pmg = g;
    return AFEM_OK;
}

template <typename T>
static int carve_levels(afem_pmg* g, int k, std::vector<LevelVec<T>>& v, Carver& cv) {
    v.resize(g->lv.size());
    for (size_t l = 0; l < g->lv.size(); ++l) {
        const size_t NK = size_t(g->lv[l].mesh->dev.n_master) * k;
        v[l].x = cv.take<T>(NK);
        v[l].b = cv.take<T>(NK);
        v[l].t = cv.take<T>(NK);
        v[l].d = cv.take<T>(NK);
    }
    return AFEM_OK;
}

}  // namespace afem

namespace afem {

// The batched Poisson solve with the multigrid preconditioner.  mixed = 0:
// CG in float64 with the float64 V-cycle; mixed = 1: float64 defect
// correction, each correction `inner` float32 CG iterations with the float32
// V-cycle.  Stopping test per column: ||b - A_IB g - A_II W_I|| <= rtol ||b - A_IB g||.
int poisson_batch_mg(afem_mesh* m, const double2* phi, int n, double* W, double rtol, int max_it, int warm, int mixed,
                     int* iters_out, int* outer_out, double* relres_out, cudaStream_t s) {
    int rc = pmg_setup(m, s);
    if (rc) return rc;
    afem_pmg* g = m->pmg;
    const DeviceMesh& D = m->dev;
    const int k = n * n;
    const int64_t N = D.n_master, Ni = D.n_interior;
    const size_t NK = size_t(N) * k;
    const int nq = kMultipoleTerms;
    double *b, *t, *r, *z64, *p64, *q64, *qpart, *q, *red;
    float *r32, *e32, *p32, *q32;
    std::vector<LevelVec<double>> v64;
    std::vector<LevelVec<float>> v32;
    const int mb = mom_blocks_count();
    auto carve = [&](Carver& cv) {
        b = cv.take<double>(NK);
        t = cv.take<double>(NK);
        r = cv.take<double>(NK);
        z64 = cv.take<double>(NK);
        p64 = cv.take<double>(mixed ? 0 : NK);
        q64 = cv.take<double>(mixed ? 0 : NK);
        qpart = cv.take<double>(size_t(mb) * nq * k);
        q = cv.take<double>(size_t(nq) * k);
        red = cv.take<double>(size_t(8) * k);
        r32 = cv.take<float>(mixed ? NK : 0);
        e32 = cv.take<float>(mixed ? NK : 0);
        p32 = cv.take<float>(mixed ? NK : 0);
        q32 = cv.take<float>(mixed ? NK : 0);
        if (mixed) carve_levels<float>(g, k, v32, cv);
        else carve_levels<double>(g, k, v64, cv);
    };
    Carver measure(nullptr);
    carve(measure);
    if ((rc = g->ws.reserve(measure.size()))) return rc;
    Carver cv(g->ws.ptr);
    carve(cv);
    double* rz = red;            // r.z
    double* rz_old = red + k;
    double* pq = red + 2 * k;
    double* rr = red + 3 * k;    // r.r
    double* bb = red + 4 * k;    // ||b - A_IB g||^2
    const unsigned gk = grid_for(Ni * k);
    const unsigned gdot = grid_for(Ni, std::max(1, 256 / k), 4);

    if (!warm) AFEM_CUDA_TRY(cudaMemsetAsync(W, 0, NK * sizeof(double), s));
    if ((rc = poisson_rhs_bc(m, phi, n, W, b, qpart, q, s))) return rc;
    // t = A g_ext (the surface data alone): W with its interior rows cleared
    AFEM_CUDA_TRY(cudaMemcpyAsync(z64, W, NK * sizeof(double), cudaMemcpyDeviceToDevice, s));
    AFEM_CUDA_TRY(cudaMemsetAsync(z64, 0, size_t(Ni) * k * sizeof(double), s));
    if ((rc = launch_stiffness(m, z64, t, k, 0, s))) return rc;
    // ||b - A_IB g||^2 per column (r as scratch)
    AFEM_CUDA_TRY(cudaMemsetAsync(z64, 0, NK * sizeof(double), s));
    AFEM_LAUNCH((pmg_residual64_kernel), gk, 256, 0, s, r, b, t, z64, Ni, k);
    AFEM_CUDA_TRY(cudaMemsetAsync(red, 0, size_t(8) * k * sizeof(double), s));
    AFEM_LAUNCH((pmg_coldot_kernel<double>), gdot, 256, 0, s, r, r, Ni, k, bb);
    std::vector<double> hb(k), hr(k);
    AFEM_CUDA_TRY(cudaMemcpyAsync(hb.data(), bb, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    AFEM_CUDA_TRY(cudaStreamSynchronize(s));

    // FP64 residual r of the current W, its squared norms into hr, the columns above rtol into active
    int active = 0;
    auto count_active = [&]() {
        active = 0;
        for (int c = 0; c < k; ++c)
            if (hr[c] > rtol * rtol * hb[c]) ++active;
    };
    auto residual = [&]() -> int {
        int r_;
        if ((r_ = launch_stiffness(m, W, z64, k, 1, s))) return r_;
        AFEM_LAUNCH((pmg_residual64_kernel), gk, 256, 0, s, r, b, t, z64, Ni, k);
        AFEM_CUDA_TRY(cudaMemsetAsync(rr, 0, k * sizeof(double), s));
        AFEM_LAUNCH((pmg_coldot_kernel<double>), gdot, 256, 0, s, r, r, Ni, k, rr);
        AFEM_CUDA_TRY(cudaMemcpyAsync(hr.data(), rr, k * sizeof(double), cudaMemcpyDeviceToHost, s));
        AFEM_CUDA_TRY(cudaStreamSynchronize(s));
        count_active();
        return AFEM_OK;
    };
    int it = 0, outer = 0;
    if ((rc = residual())) return rc;
    const int inner = 6;   // float32 CG iterations per correction
    if (!mixed) {
        // float64 CG with the float64 V-cycle; restarted from the true residual
        // whenever the recursively updated one meets rtol (or after 64 iterations)
        std::vector<LevelVec<double>>& v = v64;
        while (active > 0 && it < max_it) {
            ++outer;
            for (int j = 0; j < 64 && active > 0 && it < max_it; ++j, ++it) {
                AFEM_CUDA_TRY(cudaMemcpyAsync(v[0].b, r, NK * sizeof(double), cudaMemcpyDeviceToDevice, s));
                if ((rc = vcycle<double>(g, v, 0, k, s))) return rc;
                AFEM_CUDA_TRY(cudaMemcpyAsync(rz_old, rz, k * sizeof(double), cudaMemcpyDeviceToDevice, s));
                AFEM_CUDA_TRY(cudaMemsetAsync(rz, 0, k * sizeof(double), s));
                AFEM_LAUNCH((pmg_coldot_kernel<double>), gdot, 256, 0, s, r, v[0].x, Ni, k, rz);
                AFEM_LAUNCH((pmg_pupdate_kernel<double>), gk, 256, 0, s, p64, v[0].x, rz, rz_old, Ni, k,
                            j == 0 ? 1 : 0);
                if ((rc = launch_stiffness(m, p64, q64, k, 1, s))) return rc;
                AFEM_CUDA_TRY(cudaMemsetAsync(pq, 0, k * sizeof(double), s));
                AFEM_LAUNCH((pmg_coldot_kernel<double>), gdot, 256, 0, s, p64, q64, Ni, k, pq);
                AFEM_LAUNCH((pmg_xr_kernel<double, double>), gk, 256, 0, s, W, r, p64, q64, rz, pq, Ni, k);
                AFEM_CUDA_TRY(cudaMemsetAsync(rr, 0, k * sizeof(double), s));
                AFEM_LAUNCH((pmg_coldot_kernel<double>), gdot, 256, 0, s, r, r, Ni, k, rr);
                AFEM_CUDA_TRY(cudaMemcpyAsync(hr.data(), rr, k * sizeof(double), cudaMemcpyDeviceToHost, s));
                AFEM_CUDA_TRY(cudaStreamSynchronize(s));
                count_active();
            }
            if ((rc = residual())) return rc;
        }
    } else {
        std::vector<LevelVec<float>>& v = v32;
        while (active > 0 && it < max_it) {
            // correction: `inner` float32 CG iterations on A_II e = r from e = 0
            AFEM_LAUNCH((pmg_f64_to_f32_kernel), gk, 256, 0, s, r, r32, int64_t(Ni) * k);
            AFEM_CUDA_TRY(cudaMemsetAsync(e32, 0, NK * sizeof(float), s));
            for (int j = 0; j < inner && it < max_it; ++j, ++it) {
                AFEM_CUDA_TRY(cudaMemcpyAsync(v[0].b, r32, size_t(Ni) * k * sizeof(float), cudaMemcpyDeviceToDevice,
                                              s));
                if ((rc = vcycle<float>(g, v, 0, k, s))) return rc;
                AFEM_CUDA_TRY(cudaMemcpyAsync(rz_old, rz, k * sizeof(double), cudaMemcpyDeviceToDevice, s));
                AFEM_CUDA_TRY(cudaMemsetAsync(rz, 0, k * sizeof(double), s));
                AFEM_LAUNCH((pmg_coldot_kernel<float>), gdot, 256, 0, s, r32, v[0].x, Ni, k, rz);
                AFEM_LAUNCH((pmg_pupdate_kernel<float>), gk, 256, 0, s, p32, v[0].x, rz, rz_old, Ni, k, j == 0 ? 1 : 0);
                if ((rc = launch_stiffness32(m, p32, q32, k, 1, s, nullptr))) return rc;
                AFEM_CUDA_TRY(cudaMemsetAsync(pq, 0, k * sizeof(double), s));
                AFEM_LAUNCH((pmg_coldot_kernel<float>), gdot, 256, 0, s, p32, q32, Ni, k, pq);
                AFEM_LAUNCH((pmg_xr_kernel<float, float>), gk, 256, 0, s, e32, r32, p32, q32, rz, pq, Ni, k);
            }
            AFEM_CUDA_TRY(cudaGetLastError());
            // W += e (float64), then the float64 residual decides
            AFEM_LAUNCH((pmg_add_f32_kernel), gk, 256, 0, s, W, e32, int64_t(Ni) * k);
            ++outer;
            if ((rc = residual())) return rc;
        }
    }
    if (iters_out) *iters_out = it;
    if (outer_out) *outer_out = outer;
    bool finite = true;
    for (int c = 0; c < k; ++c) {
        const double rel = hb[c] > 0.0 ? std::sqrt(hr[c] / hb[c]) : 0.0;
        if (!std::isfinite(rel)) finite = false;
        if (relres_out) relres_out[c] = rel;
    }
    if (!finite) return set_error(AFEM_ENAN, "afem_poisson_batch: non-finite residual");
    if (active > 0) return set_error(AFEM_ECG_MAXIT, "afem_poisson_batch: CG reached max_it before rtol");
    return AFEM_OK;
}

}  // namespace afem
