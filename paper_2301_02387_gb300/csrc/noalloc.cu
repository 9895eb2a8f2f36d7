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

namespace afem {

constexpr int kNoallocLmaxTerms = 13 * 13;     // (l_max + 1)^2 multipole terms, l_max = 12
constexpr int kNoallocBlocks = 152;            // one moment block per SM
constexpr int kNoallocMaxCols = AFEM_NOALLOC_MAX_ORB * AFEM_NOALLOC_MAX_ORB;
constexpr size_t kNoallocDoubles =
    size_t(kNoallocBlocks) * kNoallocLmaxTerms * kNoallocMaxCols + size_t(kNoallocLmaxTerms) * kNoallocMaxCols;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

static double* g_noalloc_ptr[64] = {nullptr};
static std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device (first call per device looks it up).
static int noalloc_scratch(double** out) {
    int dev = 0;
    AFEM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(AFEM_EINVAL, "afem_poisson_boundary_noalloc: device index out of range");
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
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    // Both regions are overwritten completely by every call before they are read.
    double* qpart = scratch;
    double* q = scratch + size_t(kNoallocBlocks) * kNoallocLmaxTerms * kNoallocMaxCols;
    return multipole_boundary(m, static_cast<const double2*>(phi), n_orb, static_cast<double*>(W), qpart, q,
                              kNoallocBlocks, static_cast<cudaStream_t>(stream));
}
