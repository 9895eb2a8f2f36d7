// C ABI entry points (declared in include/afem_mctdhf.h).
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <utility>

#include "afem_internal.h"
#include "arnoldi.cuh"

namespace afem {
const char* last_error_cstr();
static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

cudaError_t allow_dyn_smem_fn(const void* func) {
    static std::mutex mu;
    static std::set<std::pair<int, const void*>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({dev, func})) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - int(fa.sharedSizeBytes));
    if (e == cudaSuccess) done.insert({dev, func});
    return e;
}
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

// Kernel-class timing: event pairs are kept per class until read, events are
// recycled through a pool.  Process-wide, guarded by one mutex.
namespace {
struct ProfClass {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    double ms = 0.0, work = 0.0;
    int64_t launches = 0;
};
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
ProfClass g_prof[AFEM_PROF_COUNT];
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Sums the finished event pairs of a class (waits for them).
int drain(ProfClass& c) {
    for (auto& pr : c.pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(pr.second);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pr.first, pr.second);
        if (e != cudaSuccess) return cuda_error(e, "afem_profile_read");
        c.ms += ms;
        g_event_pool.push_back(pr.first);
        g_event_pool.push_back(pr.second);
    }
    c.pending.clear();
    return AFEM_OK;
}
}  // namespace

bool profile_on() { return g_prof_on.load(std::memory_order_relaxed); }

ProfScope::ProfScope(int cls_, cudaStream_t s_, double work_) : cls(cls_), s(s_), work(work_) {
    if (!profile_on() || cls < 0 || cls >= AFEM_PROF_COUNT) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    e0 = take_event();
    e1 = take_event();
    if (e0 && e1) cudaEventRecord(e0, s);
}

ProfScope::~ProfScope() {
    if (!e0 || !e1) return;
    cudaEventRecord(e1, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfClass& c = g_prof[cls];
    c.pending.emplace_back(e0, e1);
    c.work += work;
    c.launches += 1;
    if (c.pending.size() > 4096) drain(c);   // bound the events held
}
}  // namespace afem

using namespace afem;

namespace afem {
int create_mesh_from_cells(const afem_mesh_desc& d, const std::vector<int32_t>& lev, const std::vector<int32_t>& ci,
                           const std::vector<int32_t>& cj, const std::vector<int32_t>& ck, afem_mesh** out) {
    *out = nullptr;
    afem_mesh* m = new (std::nothrow) afem_mesh();
    if (!m) return set_error(AFEM_ENOMEM, "mesh: host allocation failed");
    m->desc = d;
    int rc = build_host_mesh_cells(d, lev, ci, cj, ck, m->host);
    if (rc == AFEM_OK) {
        m->basis = make_basis(d.degree);
        cudaError_t e = cudaGetDevice(&m->device);
        rc = e == cudaSuccess ? upload_mesh(m) : cuda_error(e, "cudaGetDevice");
    }
    if (rc != AFEM_OK) {
        free_device_mesh(m->dev);
        delete m;
        return rc;
    }
    *out = m;
    return AFEM_OK;
}
}  // namespace afem

extern "C" {

const char* afem_last_error(void) { return last_error_cstr(); }

int afem_kernel_launch_count(int64_t* count) {
    if (!count) return set_error(AFEM_EINVAL, "afem_kernel_launch_count: null argument");
    *count = launch_count();
    return AFEM_OK;
}

int afem_profile_enable(int on) {
    afem::g_prof_on.store(on != 0, std::memory_order_relaxed);
    return AFEM_OK;
}

int afem_profile_read(int cls, double* ms, int64_t* calls, double* work, int reset) {
    if (cls < 0 || cls >= AFEM_PROF_COUNT) return set_error(AFEM_EINVAL, "afem_profile_read: unknown class");
    std::lock_guard<std::mutex> lk(afem::g_prof_mu);
    afem::ProfClass& c = afem::g_prof[cls];
    int rc = afem::drain(c);
    if (rc) return rc;
    if (ms) *ms = c.ms;
    if (calls) *calls = c.launches;
    if (work) *work = c.work;
    if (reset) {
        c.ms = 0.0;
        c.work = 0.0;
        c.launches = 0;
    }
    return AFEM_OK;
}

int afem_mesh_create(const afem_mesh_desc* desc, afem_mesh** out) {
    return afem_mesh_create_ex(desc, 0, out);
}

int afem_mesh_create_ex(const afem_mesh_desc* desc, int flags, afem_mesh** out) {
    if (!desc || !out) return set_error(AFEM_EINVAL, "afem_mesh_create: null argument");
    if (flags & ~AFEM_MESH_HOST_ONLY) return set_error(AFEM_EINVAL, "afem_mesh_create_ex: unknown flags");
    *out = nullptr;
    const afem_mesh_desc& d = *desc;
    if (d.degree < 1 || d.degree > kMaxDegree)
        return set_error(AFEM_EINVAL, "afem_mesh_create: degree must be 1..4");
    if (d.n_coarse < 1 || d.n_coarse > 1024)
        return set_error(AFEM_EINVAL, "afem_mesh_create: n_coarse must be 1..1024");
    if (!(d.hi > d.lo)) return set_error(AFEM_EINVAL, "afem_mesh_create: empty box");
    if (d.n_nuclei < 0 || d.n_nuclei > AFEM_MAX_NUCLEI)
        return set_error(AFEM_EINVAL, "afem_mesh_create: n_nuclei out of range");
    if (!(d.refine_c >= 0.0)) return set_error(AFEM_EINVAL, "afem_mesh_create: refine_c < 0");
    for (int n = 0; n < d.n_nuclei; ++n)
        if (d.nuc_levels[n] < 0 || d.nuc_levels[n] > 12)
            return set_error(AFEM_EINVAL, "afem_mesh_create: nuc_levels must be 0..12");
    if (d.refine_mode != AFEM_REFINE_GEOMETRIC && d.refine_mode != AFEM_REFINE_KELLY)
        return set_error(AFEM_EINVAL, "afem_mesh_create: unknown refine_mode");
    if (d.refine_mode == AFEM_REFINE_KELLY &&
        (d.kelly_max_level < 0 || d.kelly_max_level > 12 || !(d.kelly_threshold > 0.0)))
        return set_error(AFEM_EINVAL, "afem_mesh_create: Kelly refinement needs kelly_max_level 0..12 and a "
                                      "threshold > 0");
    afem_mesh* m = new (std::nothrow) afem_mesh();
    if (!m) return set_error(AFEM_ENOMEM, "afem_mesh_create: host allocation failed");
    m->desc = d;
    m->host_only = (flags & AFEM_MESH_HOST_ONLY) != 0;
    int rc = build_host_mesh(d, m->host);
    if (rc == AFEM_OK) {
        m->basis = make_basis(d.degree);
        if (!m->host_only) {
            cudaError_t e = cudaGetDevice(&m->device);
            rc = e == cudaSuccess ? upload_mesh(m) : cuda_error(e, "cudaGetDevice");
        }
    }
    if (rc != AFEM_OK) {
        free_device_mesh(m->dev);
        delete m;
        return rc;
    }
    *out = m;
    return AFEM_OK;
}


int afem_mesh_destroy(afem_mesh* mesh) {
    if (!mesh) return AFEM_OK;
    if (!mesh->host_only) free_device_mesh(mesh->dev);
    pmg_free(mesh->pmg);
    mesh->pmg = nullptr;
    if (!mesh->host_only) mesh_free_ecs(mesh);
    mesh->ws_poisson.release();
    mesh->ws_arnoldi.release();
    mesh->ws_tdse.release();
    mesh->ws_int.release();
    mesh->ws_gblocks.release();
    delete mesh;
    return AFEM_OK;
}

int afem_mesh_set_option(afem_mesh* m, int option, int value) {
    if (!m) return set_error(AFEM_EINVAL, "afem_mesh_set_option: null mesh");
    if (option == AFEM_OPT_CELL32_VARIANT) {
        if (value < 0 || value > 2)
            return set_error(AFEM_EINVAL, "afem_mesh_set_option: variant must be 0, 1 or 2");
        m->cell32_variant = value;
        return AFEM_OK;
    }
    if (option == AFEM_OPT_GCELL_BLOCKS) {
        if (value < 0 || value > 2)
            return set_error(AFEM_EINVAL, "afem_mesh_set_option: G cell blocks must be 0, 1 or 2");
        m->gcell_blocks = value;
        return AFEM_OK;
    }
    if (option == AFEM_OPT_POISSON_SOLVER) {
        if (value != AFEM_POISSON_JACOBI && value != AFEM_POISSON_MULTIGRID)
            return set_error(AFEM_EINVAL, "afem_mesh_set_option: Poisson solver must be AFEM_POISSON_JACOBI or "
                                          "AFEM_POISSON_MULTIGRID");
        if (m->host_only) return set_error(AFEM_EINVAL, "afem_mesh_set_option: mesh was built host-only");
        m->poisson_solver = value;
        return AFEM_OK;
    }
    return set_error(AFEM_EINVAL, "afem_mesh_set_option: unknown option");
}

int afem_mesh_set_ecs(afem_mesh* m, double theta, const double half_width[3]) {
    if (!m) return set_error(AFEM_EINVAL, "afem_mesh_set_ecs: null mesh");
    if (m->host_only) return set_error(AFEM_EINVAL, "afem_mesh_set_ecs: mesh was built host-only");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != m->device)
        return set_error(AFEM_EINVAL, "afem_mesh_set_ecs: the current device is not the mesh's");
    return mesh_set_ecs(m, theta, half_width);
}

int afem_mesh_get_info(const afem_mesh* m, afem_mesh_info* info) {
    if (!m || !info) return set_error(AFEM_EINVAL, "afem_mesh_get_info: null argument");
    const HostMesh& H = m->host;
    info->n_cells = int64_t(H.lev.size());
    info->n_masters = H.n_master;
    info->n_interior = H.n_interior;
    info->n_hanging = H.n_hanging;
    info->n_constraint_entries = int64_t(H.hang_master.size());
    info->degree = H.p;
    info->max_level = H.max_level;
    double hmin = 1e300, hmax = 0.0;
    for (double h : H.h) {
        hmin = h < hmin ? h : hmin;
        hmax = h > hmax ? h : hmax;
    }
    info->h_min = hmin;
    info->h_max = hmax;
    return AFEM_OK;
}

int afem_mesh_tables(const afem_mesh* m, double* coords, double* lumped_mass, int32_t* cells) {
    if (!m) return set_error(AFEM_EINVAL, "afem_mesh_tables: null mesh");
    const HostMesh& H = m->host;
    if (coords) std::memcpy(coords, H.master_xyz.data(), H.master_xyz.size() * sizeof(double));
    if (lumped_mass) std::memcpy(lumped_mass, H.ml.data(), H.ml.size() * sizeof(double));
    if (cells) {
        for (size_t q = 0; q < H.lev.size(); ++q) {
            cells[4 * q + 0] = H.lev[q];
            cells[4 * q + 1] = H.ci[q];
            cells[4 * q + 2] = H.cj[q];
            cells[4 * q + 3] = H.ck[q];
        }
    }
    return AFEM_OK;
}

int afem_op_apply(afem_mesh* m, int kind, const double* E, const void* x, void* y, int n_vec,
                  void* stream) {
    if (!m || !x || !y) return set_error(AFEM_EINVAL, "afem_op_apply: null argument");
    if (n_vec < 1 || n_vec > 64) return set_error(AFEM_EINVAL, "afem_op_apply: n_vec must be 1..64");
    if (x == y) return set_error(AFEM_EINVAL, "afem_op_apply: x and y must not alias");
    if (m->host_only) return set_error(AFEM_EINVAL, "afem_op_apply: mesh was built host-only");
    return launch_op_apply(m, kind, E, x, y, n_vec, static_cast<cudaStream_t>(stream));
}

int afem_poisson_batch(afem_mesh* m, const void* phi, int n_orb, void* W, double rtol, int max_it,
                       int warm_start, int* iters_out, double* relres_out, void* stream) {
    return afem_poisson_batch_ex(m, phi, n_orb, W, rtol, max_it, warm_start, AFEM_PREC_FP64, iters_out, nullptr,
                                 relres_out, stream);
}

int afem_poisson_batch_ex(afem_mesh* m, const void* phi, int n_orb, void* W, double rtol, int max_it,
                          int warm_start, int precision, int* iters_out, int* outer_out, double* relres_out,
                          void* stream) {
    if (precision != AFEM_PREC_FP64 && precision != AFEM_PREC_MIXED)
        return set_error(AFEM_EINVAL, "afem_poisson_batch_ex: unknown precision");
    if (!m || !phi || !W) return set_error(AFEM_EINVAL, "afem_poisson_batch: null argument");
    if (m->host_only) return set_error(AFEM_EINVAL, "afem_poisson_batch: mesh was built host-only");
    if (n_orb < 1 || n_orb > 8) return set_error(AFEM_EINVAL, "afem_poisson_batch: n_orb must be 1..8");
    if (!(rtol > 0.0) || max_it < 0) return set_error(AFEM_EINVAL, "afem_poisson_batch: bad rtol/max_it");
    if (precision == AFEM_PREC_MIXED)
        return poisson_batch_mixed(m, static_cast<const double2*>(phi), n_orb, static_cast<double*>(W), rtol,
                                   max_it, warm_start, 1e-2, iters_out, outer_out, relres_out,
                                   static_cast<cudaStream_t>(stream));
    if (outer_out) *outer_out = 0;
    return poisson_batch(m, static_cast<const double2*>(phi), n_orb, static_cast<double*>(W), rtol, max_it,
                         warm_start, iters_out, relres_out, static_cast<cudaStream_t>(stream));
}

int afem_two_electron_integrals(afem_mesh* m, const void* phi, int n_orb, const void* W, void* eri, int precision,
                                void* stream) {
    if (precision != AFEM_PREC_FP64 && precision != AFEM_PREC_MIXED)
        return set_error(AFEM_EINVAL, "afem_two_electron_integrals: unknown precision");
    if (!m || !phi || !W || !eri) return set_error(AFEM_EINVAL, "afem_two_electron_integrals: null argument");
    if (m->host_only) return set_error(AFEM_EINVAL, "afem_two_electron_integrals: mesh was built host-only");
    if (n_orb < 1 || n_orb > 8) return set_error(AFEM_EINVAL, "afem_two_electron_integrals: n_orb must be 1..8");
    return two_electron_integrals(m, static_cast<const double2*>(phi), n_orb, static_cast<const double*>(W),
                                  static_cast<double2*>(eri), precision, static_cast<cudaStream_t>(stream));
}

int afem_arnoldi_step(afem_mesh* m, const double* E, const void* phi, const void* U, int n_orb, int krylov_m,
                      double dt, void* phi_out, double* err_est, int* m_used, int* breakdown, void* stream) {
    return afem_arnoldi_step_ex(m, E, phi, U, n_orb, krylov_m, dt, AFEM_PREC_FP64, phi_out, err_est, m_used,
                                breakdown, stream);
}

int afem_arnoldi_step_ex(afem_mesh* m, const double* E, const void* phi, const void* U, int n_orb, int krylov_m,
                         double dt, int precision, void* phi_out, double* err_est, int* m_used, int* breakdown,
                         void* stream) {
    if (precision != AFEM_PREC_FP64 && precision != AFEM_PREC_MIXED)
        return set_error(AFEM_EINVAL, "afem_arnoldi_step_ex: unknown precision");
    if (!m || !phi || !phi_out) return set_error(AFEM_EINVAL, "afem_arnoldi_step: null argument");
    if (m->host_only) return set_error(AFEM_EINVAL, "afem_arnoldi_step: mesh was built host-only");
    if (n_orb < 1 || n_orb > 8) return set_error(AFEM_EINVAL, "afem_arnoldi_step: n_orb must be 1..8");
    if (krylov_m < 1 || krylov_m > kMaxKrylov) return set_error(AFEM_EINVAL, "afem_arnoldi_step: krylov_m must be 1..16");
    if (phi == phi_out) return set_error(AFEM_EINVAL, "afem_arnoldi_step: phi and phi_out must not alias");
    return arnoldi_step(m, E, static_cast<const double2*>(phi), static_cast<const double2*>(U), nullptr, n_orb,
                        krylov_m, dt, precision == AFEM_PREC_MIXED, 0.0, static_cast<double2*>(phi_out), err_est,
                        m_used, breakdown, nullptr, static_cast<cudaStream_t>(stream));
}

int afem_arnoldi_propagate(afem_mesh* m, const double* E, const void* phi, const void* U, int n_orb, int krylov_m,
                           double dt, int precision, double tol, void* phi_out, double* err_est, int* substeps,
                           void* stream) {
    if (precision != AFEM_PREC_FP64 && precision != AFEM_PREC_MIXED)
        return set_error(AFEM_EINVAL, "afem_arnoldi_propagate: unknown precision");
    if (!m || !phi || !phi_out) return set_error(AFEM_EINVAL, "afem_arnoldi_propagate: null argument");
    if (m->host_only) return set_error(AFEM_EINVAL, "afem_arnoldi_propagate: mesh was built host-only");
    if (n_orb < 1 || n_orb > 8) return set_error(AFEM_EINVAL, "afem_arnoldi_propagate: n_orb must be 1..8");
    if (krylov_m < 1 || krylov_m > kMaxKrylov)
        return set_error(AFEM_EINVAL, "afem_arnoldi_propagate: krylov_m must be 1..16");
    if (!(tol > 0.0) || !(dt > 0.0)) return set_error(AFEM_EINVAL, "afem_arnoldi_propagate: tol and dt must be > 0");
    if (phi == phi_out) return set_error(AFEM_EINVAL, "afem_arnoldi_propagate: phi and phi_out must not alias");
    return arnoldi_step(m, E, static_cast<const double2*>(phi), static_cast<const double2*>(U), nullptr, n_orb,
                        krylov_m, dt, precision == AFEM_PREC_MIXED, tol, static_cast<double2*>(phi_out), err_est,
                        nullptr, nullptr, substeps, static_cast<cudaStream_t>(stream));
}

int afem_arnoldi_adaptive(afem_mesh* m, const double* E, const void* phi, const void* U, int n_orb, int m_max,
                          double dt, int steps, int precision, double tol, void* phi_out, double* err_est,
                          int* dim_max, int* dim_sum, int* unmet, void* stream) {
    if (precision != AFEM_PREC_FP64 && precision != AFEM_PREC_MIXED)
        return set_error(AFEM_EINVAL, "afem_arnoldi_adaptive: unknown precision");
    if (!m || !phi || !phi_out) return set_error(AFEM_EINVAL, "afem_arnoldi_adaptive: null argument");
    if (m->host_only) return set_error(AFEM_EINVAL, "afem_arnoldi_adaptive: mesh was built host-only");
    if (n_orb < 1 || n_orb > 8) return set_error(AFEM_EINVAL, "afem_arnoldi_adaptive: n_orb must be 1..8");
    if (m_max < 1 || m_max > kMaxKrylov) return set_error(AFEM_EINVAL, "afem_arnoldi_adaptive: m_max must be 1..16");
    if (steps < 1 || steps > 4096) return set_error(AFEM_EINVAL, "afem_arnoldi_adaptive: steps must be 1..4096");
    if (!(tol > 0.0) || !(dt > 0.0)) return set_error(AFEM_EINVAL, "afem_arnoldi_adaptive: tol and dt must be > 0");
    if (phi == phi_out) return set_error(AFEM_EINVAL, "afem_arnoldi_adaptive: phi and phi_out must not alias");
    return arnoldi_step(m, E, static_cast<const double2*>(phi), static_cast<const double2*>(U), nullptr, n_orb,
                        m_max, dt, precision == AFEM_PREC_MIXED, tol, static_cast<double2*>(phi_out), err_est,
                        dim_max, nullptr, nullptr, static_cast<cudaStream_t>(stream), 0, steps, dim_sum, unmet);
}

int afem_mctdhf_create(afem_mesh* m, int n_orb, int n_alpha, int n_beta, int krylov_m, afem_mctdhf** out) {
    if (!m || !out) return set_error(AFEM_EINVAL, "afem_mctdhf_create: null argument");
    *out = nullptr;
    if (m->host_only) return set_error(AFEM_EINVAL, "afem_mctdhf_create: mesh was built host-only");
    if (n_orb < 1 || n_orb > 8) return set_error(AFEM_EINVAL, "afem_mctdhf_create: n_orb must be 1..8");
    if (n_alpha < 0 || n_beta < 0 || n_alpha > n_orb || n_beta > n_orb || n_alpha + n_beta == 0)
        return set_error(AFEM_EINVAL, "afem_mctdhf_create: bad electron counts");
    if (krylov_m < 1 || krylov_m > kMaxKrylov) return set_error(AFEM_EINVAL, "afem_mctdhf_create: krylov_m must be 1..16");
    return mctdhf_create(m, n_orb, n_alpha, n_beta, krylov_m, out);
}

int afem_mctdhf_destroy(afem_mctdhf* s) {
    mctdhf_destroy(s);
    return AFEM_OK;
}

int afem_mctdhf_set_precision(afem_mctdhf* s, int precision) {
    if (!s) return set_error(AFEM_EINVAL, "afem_mctdhf_set_precision: null argument");
    if (precision != AFEM_PREC_FP64 && precision != AFEM_PREC_MIXED)
        return set_error(AFEM_EINVAL, "afem_mctdhf_set_precision: unknown precision");
    mctdhf_set_precision(s, precision);
    return AFEM_OK;
}

int afem_mctdhf_set_krylov_tol(afem_mctdhf* s, double tol) {
    if (!s) return set_error(AFEM_EINVAL, "afem_mctdhf_set_krylov_tol: null argument");
    if (!(tol >= 0.0)) return set_error(AFEM_EINVAL, "afem_mctdhf_set_krylov_tol: tol must be >= 0");
    mctdhf_set_krylov_tol(s, tol);
    return AFEM_OK;
}

int afem_mctdhf_set_krylov_adaptive(afem_mctdhf* s, int steps) {
    if (!s) return set_error(AFEM_EINVAL, "afem_mctdhf_set_krylov_adaptive: null argument");
    if (steps < 0 || steps > 4096) return set_error(AFEM_EINVAL, "afem_mctdhf_set_krylov_adaptive: steps must be 0..4096");
    mctdhf_set_krylov_adaptive(s, steps);
    return AFEM_OK;
}

int afem_mctdhf_set_imaginary(afem_mctdhf* s, int on) {
    if (!s) return set_error(AFEM_EINVAL, "afem_mctdhf_set_imaginary: null argument");
    if (on != 0 && on != 1) return set_error(AFEM_EINVAL, "afem_mctdhf_set_imaginary: on must be 0 or 1");
    mctdhf_set_imaginary(s, on);
    return AFEM_OK;
}

int afem_mctdhf_set_gauge(afem_mctdhf* s, int gauge) {
    if (!s) return set_error(AFEM_EINVAL, "afem_mctdhf_set_gauge: null argument");
    if (gauge != AFEM_GAUGE_LENGTH && gauge != AFEM_GAUGE_VELOCITY)
        return set_error(AFEM_EINVAL, "afem_mctdhf_set_gauge: gauge must be AFEM_GAUGE_LENGTH or AFEM_GAUGE_VELOCITY");
    mctdhf_set_gauge(s, gauge);
    return AFEM_OK;
}

int afem_mctdhf_ci_dim(const afem_mctdhf* s, int64_t* dim) {
    if (!s || !dim) return set_error(AFEM_EINVAL, "afem_mctdhf_ci_dim: null argument");
    *dim = mctdhf_ci_dim(s);
    return AFEM_OK;
}

int afem_mctdhf_step(afem_mctdhf* s, void* phi, void* C, void* W, const double* E, double dt, double cg_rtol,
                     int cg_max_it, afem_step_info* info, void* stream) {
    if (!s || !phi || !C || !W) return set_error(AFEM_EINVAL, "afem_mctdhf_step: null argument");
    if (!(dt > 0.0) || !(cg_rtol > 0.0) || cg_max_it < 0)
        return set_error(AFEM_EINVAL, "afem_mctdhf_step: bad dt / cg_rtol / cg_max_it");
    return mctdhf_step(s, static_cast<double2*>(phi), static_cast<double2*>(C), static_cast<double*>(W), E, dt,
                       cg_rtol, cg_max_it, info, static_cast<cudaStream_t>(stream));
}

int afem_convert(const void* x, void* y, int64_t n, int direction, void* stream) {
    if (n < 0 || (n > 0 && (!x || !y))) return set_error(AFEM_EINVAL, "afem_convert: bad arguments");
    if (direction == AFEM_CONVERT_F64_F32)
        return convert_f64_f32(static_cast<const double*>(x), static_cast<float*>(y), n,
                               static_cast<cudaStream_t>(stream));
    if (direction == AFEM_CONVERT_F32_F64)
        return convert_f32_f64(static_cast<const float*>(x), static_cast<double*>(y), n,
                               static_cast<cudaStream_t>(stream));
    return set_error(AFEM_EINVAL, "afem_convert: unknown direction");
}

int afem_tdse_forward(afem_mesh* m, const double* e_dir, const double* E, int n_steps, double dt, int krylov_m,
                      double tol, int precision, int observable, const void* phi0, void* phi_end, double* d,
                      void* ckpt, int ckpt_every, void* stream) {
    return tdse_forward(m, e_dir, E, n_steps, dt, krylov_m, tol, precision, observable,
                        static_cast<const double2*>(phi0),
                        static_cast<double2*>(phi_end), d, static_cast<double2*>(ckpt), ckpt_every,
                        static_cast<cudaStream_t>(stream));
}

int afem_tdse_jvp(afem_mesh* m, const double* e_dir, const double* E, int n_steps, double dt, int krylov_m,
                  double tol, int precision, int observable, const void* phi0, const double* v, double* d,
                  double* dd, void* stream) {
    return tdse_jvp(m, e_dir, E, n_steps, dt, krylov_m, tol, precision, observable,
                    static_cast<const double2*>(phi0), v, d, dd, static_cast<cudaStream_t>(stream));
}

int afem_tdse_vjp(afem_mesh* m, const double* e_dir, const double* E, int n_steps, double dt, int krylov_m,
                  double tol, int precision, int observable, const void* ckpt, int ckpt_every, const double* g,
                  double* grad_E, void* lam0, void* stream) {
    return tdse_vjp(m, e_dir, E, n_steps, dt, krylov_m, tol, precision, observable,
                    static_cast<const double2*>(ckpt), ckpt_every, g, grad_E, static_cast<double2*>(lam0),
                    static_cast<cudaStream_t>(stream));
}

}  // extern "C"
