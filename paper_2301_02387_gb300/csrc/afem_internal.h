// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/afem_mctdhf.h"

namespace afem {

constexpr int kMaxDegree = 4;
constexpr int kMaxP1 = kMaxDegree + 1;
// Multipole expansion of the mean fields' surface data: l <= kMultipoleLmax,
// (kMultipoleLmax + 1)^2 real solid-harmonic terms.
constexpr int kMultipoleLmax = 12;
constexpr int kMultipoleTerms = (kMultipoleLmax + 1) * (kMultipoleLmax + 1);

// Record the message for afem_last_error() and return `code`.
int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* what);

// Host-side count of kernel launches made by this library (process-wide).
void note_launch();
int64_t launch_count();

#define AFEM_LAUNCH(kern, grid, block, smem, stream, ...)           \
    do {                                                             \
        ::afem::note_launch();                                       \
        kern<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);    \
    } while (0)

// Lets kernel `func` use the device's opt-in maximum of dynamic shared memory
// (less its static shared memory), once per device and kernel.  The limit is
// only ever raised, to the same value, so launches from several host threads
// cannot lower it below another launch's need.
cudaError_t allow_dyn_smem_fn(const void* func);
template <typename K>
inline cudaError_t allow_dyn_smem(K func) {
    return allow_dyn_smem_fn(reinterpret_cast<const void*>(func));
}

// Kernel-class timing (afem_profile_*): while enabled, a ProfScope brackets
// the launches made in its lifetime with CUDA events on stream s and adds
// `work` (the class's algorithmic flops or bytes) to the class.
bool profile_on();
struct ProfScope {
    int cls;
    cudaStream_t s;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double work;
    ProfScope(int cls_, cudaStream_t s_, double work_);
    ~ProfScope();
};

#define AFEM_CUDA_TRY(call)                                    \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return ::afem::cuda_error(e_, #call); \
    } while (0)

// Grow-only device scratch owned by a mesh.
struct Workspace {
    void* ptr = nullptr;
    size_t bytes = 0;
    int reserve(size_t need) {
        if (need <= bytes) return AFEM_OK;
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&ptr, need);
        if (e != cudaSuccess) return set_error(AFEM_ENOMEM, std::string("workspace cudaMalloc: ") + cudaGetErrorString(e));
        bytes = need;
        return AFEM_OK;
    }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
};

// 1D Gauss-Lobatto-Legendre basis on [0, 1] (Sec. 3.1).
struct Basis1D {
    int p = 0;
    double xi[kMaxP1] = {};          // nodes, ascending
    double w[kMaxP1] = {};           // quadrature weights (sum 1)
    double K[kMaxP1][kMaxP1] = {};   // 1D stiffness sum_q w_q L_i'(xi_q) L_j'(xi_q)
    double S[kMaxP1][kMaxP1] = {};   // skew part of int L_i L_j': (w_i L_j'(xi_i) - w_j L_i'(xi_j)) / 2
};
Basis1D make_basis(int p);
double lagrange_value(const Basis1D& b, int j, double t);

// Host-side mesh tables (built once; the mesh is static during a run).
struct HostMesh {
    int p = 0;
    int max_level = 0;
    double lo = 0, hi = 0, h0 = 0;
    int n_coarse = 0;
    // leaves in Morton order
    std::vector<int32_t> lev, ci, cj, ck;
    std::vector<double> corner;            // [ncell][3]
    std::vector<double> h;                 // [ncell]
    // cell node map: >= 0 master index, < 0 -(hanging index) - 1
    std::vector<int32_t> cell_node;        // [ncell][(p+1)^3]
    int64_t n_master = 0, n_interior = 0, n_hanging = 0;
    std::vector<double> master_xyz;        // [N][3]
    std::vector<double> hang_xyz;          // [nh][3]
    std::vector<int32_t> hang_ptr;         // [nh+1]
    std::vector<int32_t> hang_master;      // [nnz]
    std::vector<double> hang_w;            // [nnz]
    std::vector<double> ml;                // [N] lumped mass C^T m_f
    std::vector<double> v_master, v_hang;  // nuclear potential at masters / hanging points
    std::vector<double> f_master, f_hang;  // [N][3] / [nh][3] nuclear force on an electron, -grad V
    std::vector<double> stiff_diag;        // [N] diagonal of the constrained stiffness A
    std::vector<double> mf_master, mf_hang;  // assembled GLL weight m_f at masters / hanging points
};

int build_host_mesh(const afem_mesh_desc& d, HostMesh& out);
// The same from explicit leaves (level, i, j, k), 2:1-balanced here; the
// description supplies the box, degree and nuclei (its refinement is unused).
int build_host_mesh_cells(const afem_mesh_desc& d, const std::vector<int32_t>& lev, const std::vector<int32_t>& ci,
                          const std::vector<int32_t>& cj, const std::vector<int32_t>& ck, HostMesh& out);
// A device mesh from explicit leaves (see build_host_mesh_cells).
int create_mesh_from_cells(const afem_mesh_desc& d, const std::vector<int32_t>& lev, const std::vector<int32_t>& ci,
                           const std::vector<int32_t>& cj, const std::vector<int32_t>& ck, afem_mesh** out);

// Device-resident mesh.
struct DeviceMesh {
    int p = 0;
    int64_t ncell = 0, n_master = 0, n_interior = 0, n_hanging = 0, nnz = 0;
    int32_t* cell_node = nullptr;   // [ncell][(p+1)^3]
    double4* cell_geom = nullptr;   // (corner x, y, z, h)
    int32_t* hang_ptr = nullptr;
    int32_t* hang_master = nullptr;
    double* hang_w = nullptr;
    double* ml = nullptr;           // [N]
    double* ml_inv = nullptr;       // [N]
    double* v_master = nullptr;     // [N]
    double* v_hang = nullptr;       // [nh]
    double* f_master = nullptr;     // [N][3] -grad V
    double* f_hang = nullptr;       // [nh][3]
    double* stiff_dinv = nullptr;   // [N] 1 / diag(A) on interior masters, 0 on the surface
    double* master_xyz = nullptr;   // [N][3]
    double* hang_xyz = nullptr;     // [nh][3]
    double* mf_master = nullptr;    // [N] assembled GLL weight m_f
    double* mf_hang = nullptr;      // [nh]
    // float copies for the FP32 kernels
    float4* cell_geom32 = nullptr;
    float* hang_w32 = nullptr;
    float* v_master32 = nullptr;
    float* v_hang32 = nullptr;
    float* v_cell32 = nullptr;      // [ncell][(p+1)^3] nuclear potential at every cell node
    float* ml_inv32 = nullptr;      // [N] float copy of ml_inv (FP32 projector)
    float* stiff_dinv32 = nullptr;
};

}  // namespace afem

struct afem_pmg;   // multigrid hierarchy of a mesh (pmg.cu)

struct afem_mesh {
    afem_mesh_desc desc;
    afem::HostMesh host;
    afem::Basis1D basis;
    afem::DeviceMesh dev;
    int device = 0;
    bool host_only = false;
    afem::Workspace ws_poisson;
    afem::Workspace ws_arnoldi;
    afem::Workspace ws_tdse;
    afem::Workspace ws_int;   // afem_two_electron_integrals
    afem::Workspace ws_gblocks;   // frozen per-cell blocks of the G cell pass
    int cell32_variant = 0;   // FP32 four-lane cell pass: 0 node-per-thread, 1 line-ordered
    int gcell_blocks = 1;     // G cell pass on frozen per-cell blocks: 0 off, 1 one cell per block, 2 pipelined (n <= 4)
    int poisson_solver = 0;   // AFEM_POISSON_JACOBI or AFEM_POISSON_MULTIGRID
    afem_pmg* pmg = nullptr;  // built on the first multigrid solve
    // exterior complex scaling of the kinetic energy (afem_mesh_set_ecs)
    int ecs_on = 0;
    double ecs_theta = 0.0;
    double ecs_half_width[3] = {0.0, 0.0, 0.0};
    uint8_t* ecs_flags = nullptr;   // [ncell] bit d: the cell lies outside the inner box along axis d
    double2* ecs_rho = nullptr;     // [N] M_L / M_theta
    float2* ecs_rho32 = nullptr;    // [N] the same in complex64
};

namespace afem {
int upload_mesh(afem_mesh* m);
void free_device_mesh(DeviceMesh& d);
int launch_op_apply(afem_mesh* m, int kind, const double* E, const void* x, void* y, int nvec,
                    cudaStream_t s);
int launch_stiffness(const afem_mesh* m, const double* x, double* y, int nv, int masked, cudaStream_t s);
int poisson_batch(afem_mesh* m, const double2* phi, int n, double* W, double rtol, int max_it, int warm,
                  int* iters_out, double* relres_out, cudaStream_t s);
int poisson_batch_mixed(afem_mesh* m, const double2* phi, int n, double* W, double rtol, int max_it, int warm,
                        double inner_rtol, int* iters_out, int* outer_out, double* relres_out, cudaStream_t s);
int multipole_boundary(afem_mesh* m, const double2* phi, int n, double* W, double* qpart, double* q, int nblk,
                       cudaStream_t s);
int ensure_sh_tables();   // uploads the solid-harmonic constants once per device
void pmg_free(afem_pmg* g);
int mesh_set_ecs(afem_mesh* m, double theta, const double half_width[3]);
void mesh_free_ecs(afem_mesh* m);
int mctdhf_create(afem_mesh* m, int n, int na, int nb, int mk, afem_mctdhf** out);
void mctdhf_destroy(afem_mctdhf* S);
int64_t mctdhf_ci_dim(const afem_mctdhf* S);
afem_mesh* mctdhf_mesh_of(const afem_mctdhf* S);
int mctdhf_orbitals_of(const afem_mctdhf* S);
void mctdhf_set_precision(afem_mctdhf* S, int precision);
void mctdhf_set_krylov_tol(afem_mctdhf* S, double tol);
void mctdhf_set_krylov_adaptive(afem_mctdhf* S, int steps);
void mctdhf_set_imaginary(afem_mctdhf* S, int on);
void mctdhf_set_gauge(afem_mctdhf* S, int gauge);
int mctdhf_step(afem_mctdhf* S, double2* phi, double2* C, double* W, const double* E, double dt, double cg_rtol,
                int cg_max_it, afem_step_info* info, cudaStream_t s);
// Two-electron integral columns X[pq][c] = sum_f m_f conj(phi_p) phi_q Wcol_c over
// all support points on the tensor cores (TF32 hi/lo split, FP64 sums of
// 32-point tiles), n = 1..8: partial [grid][n^2][n^2] complex sums per block
// (integrals_tc.cu); *status (device, zeroed by the caller) becomes nonzero if
// a block gave up waiting for its MMAs.
int integrals_tc(const afem_mesh* m, const double2* phi, const double* W, int n, double2* partial, int grid,
                 int* status, cudaStream_t s);
int two_electron_integrals(afem_mesh* m, const double2* phi, int n, const double* W, double2* eri, int precision,
                           cudaStream_t s);
// The G cell pass on frozen per-cell blocks (cell_f32.cu): applicability,
// block storage, formation once per propagation, and the pass itself.
bool gcell_blocks_apply(const afem_mesh* m, int n, int velocity);
size_t gcell_blocks_bytes(const afem_mesh* m, int n);
int build_gcell_blocks32(const afem_mesh* m, const double* E, const float2* U, const float2* U_hang, int n,
                         float4* B, cudaStream_t s);
int launch_g_cell32_blocks(const afem_mesh* m, const float2* v, const float4* B, float2* z, int n, double* err,
                           float4* vh, cudaStream_t s);
int convert_f64_f32(const double* x, float* y, int64_t n, cudaStream_t s);
int convert_f32_f64(const float* x, double* y, int64_t n, cudaStream_t s);
int tdse_forward(afem_mesh* m, const double* e_dir, const double* E, int K, double dt, int mk, double tol,
                 int precision, int observable, const double2* phi0, double2* phi_end, double* d, double2* ckpt,
                 int every, cudaStream_t s);
int tdse_jvp(afem_mesh* m, const double* e_dir, const double* E, int K, double dt, int mk, double tol,
             int precision, int observable, const double2* phi0, const double* v, double* d, double* dd,
             cudaStream_t s);
int tdse_vjp(afem_mesh* m, const double* e_dir, const double* E, int K, double dt, int mk, double tol,
             int precision, int observable, const double2* ckpt, int every, const double* g, double* grad_E,
             double2* lam0, cudaStream_t s);
}  // namespace afem
