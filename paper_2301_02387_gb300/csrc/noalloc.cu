// Surface data of the pair mean fields with no device allocation
// (afem_poisson_boundary_noalloc; a library service with no counterpart in
// the paper).
//
// Callers that must not allocate device memory once they run cannot use
// afem_poisson_batch, whose workspace grows on first use.  This entry point
// computes the same multipole Dirichlet data from scratch that lives in the
// file-scope array below: every GPU that loads the library holds it until the
// process exits.  Its host address is only a stand-in, so the device address
// is looked up here, once per device, with that device current.
#include <mutex>

#include "afem_internal.h"
#include "vec_common.cuh"

namespace afem {

constexpr int kNoallocLmaxTerms = kMultipoleTerms;   // multipole terms of the surface data
constexpr int kNoallocMaxBlocks = 152;               // moment blocks: one per SM, at most 152
constexpr int kNoallocMaxCols = AFEM_NOALLOC_MAX_ORB * AFEM_NOALLOC_MAX_ORB;
constexpr size_t kNoallocDoubles =
    size_t(kNoallocMaxBlocks) * kNoallocLmaxTerms * kNoallocMaxCols + size_t(kNoallocLmaxTerms) * kNoallocMaxCols;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

static double* g_noalloc_ptr[64] = {nullptr};
static std::mutex g_noalloc_mu;

// Set-up of the current device, which must be the mesh's: the device address
// of the scratch array (looked up once per device) and the solid-harmonic
// constants (uploaded once per device).
static int noalloc_scratch(const afem_mesh* m, double** out) {
    int dev = 0;
    AFEM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(AFEM_EINVAL, "afem_poisson_boundary_noalloc: device index out of range");
    if (dev != m->device)
        return set_error(AFEM_EINVAL, "afem_poisson_boundary_noalloc: the current device is not the mesh's device");
    int rc = ensure_sh_tables();
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return AFEM_OK;
}

}  // namespace afem

using namespace afem;

extern "C" int afem_poisson_boundary_noalloc(afem_mesh* m, const void* phi, int n_orb, void* W, void* stream) {
    if (!m || !phi || !W) return set_error(AFEM_EINVAL, "afem_poisson_boundary_noalloc: null argument");
    if (m->host_only) return set_error(AFEM_EINVAL, "afem_poisson_boundary_noalloc: mesh was built host-only");
    if (n_orb < 1 || n_orb > AFEM_NOALLOC_MAX_ORB)
        return set_error(AFEM_EINVAL, "afem_poisson_boundary_noalloc: n_orb must be 1..4 (static scratch limit)");
    double* scratch = nullptr;
    int rc = noalloc_scratch(m, &scratch);
    if (rc) return rc;
    const int sms = device_sms();
    const int nblk = sms < kNoallocMaxBlocks ? sms : kNoallocMaxBlocks;
    // Both regions are overwritten completely by every call before they are read.
    double* qpart = scratch;
    double* q = scratch + size_t(kNoallocMaxBlocks) * kNoallocLmaxTerms * kNoallocMaxCols;
    return multipole_boundary(m, static_cast<const double2*>(phi), n_orb, static_cast<double*>(W), qpart, q, nblk,
                              static_cast<cudaStream_t>(stream));
}
