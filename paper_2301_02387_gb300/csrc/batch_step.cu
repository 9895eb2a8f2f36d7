// Batching form at the level of the whole time step: one MCTDHF step (Sec. 2,
// Sec. 3.2: Poisson batch of the pair mean fields, integrals, CI propagation,
// orbital propagation by Arnoldi) of many independent instances of uneven
// size, degree and orbital count per call.
//
// Each instance's step is the single-instance step (its own solver, mesh and
// workspaces), so each computes exactly what afem_mctdhf_step computes for it.
// What is shared is the schedule: the instances are spread over W worker
// streams by longest-processing-time-first on an estimated cost, one host
// thread per stream issues its instances' steps back to back, and the GPU
// overlaps the instances of different streams (the many short launches of the
// small instances' Krylov substeps fill the gaps of the large ones).  W is
// chosen by timing the candidates 1, 2, 4, 8, 16 on the batch's own steps
// (calls 2.. W-candidates + 1; the first call, which allocates workspaces,
// runs on 4 streams); later calls use the fastest.  The caller's stream is
// ordered before and after the batch by events.
#include <algorithm>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include "afem_internal.h"

namespace {
constexpr int kMaxWorkers = 16;
constexpr int kCands[] = {1, 2, 4, 8, 16};
constexpr int kNumCands = 5;
}  // namespace

struct afem_batch_stepper {
    std::vector<afem_mctdhf*> solvers;
    std::vector<double> cost;   // estimated relative cost per instance
    std::vector<const afem_mesh*> mesh;
    int device = 0;
    cudaStream_t streams[kMaxWorkers] = {};
    cudaEvent_t start = nullptr;
    cudaEvent_t done[kMaxWorkers] = {};
    int calls = 0;
    int chosen = 0;                         // worker count in use after tuning (0: still tuning)
    int n_cand = 0;
    int cand_streams[kNumCands] = {};
    double cand_ms[kNumCands] = {};
};

using namespace afem;

namespace {

void destroy_stepper(afem_batch_stepper* b) {
    for (int w = 0; w < kMaxWorkers; ++w) {
        if (b->streams[w]) cudaStreamDestroy(b->streams[w]);
        if (b->done[w]) cudaEventDestroy(b->done[w]);
    }
    if (b->start) cudaEventDestroy(b->start);
    delete b;
}

// Longest processing time first over groups of instances that share a mesh
// (their steps use the mesh's workspaces, so one worker runs them in turn):
// groups by decreasing summed cost, each to the least loaded worker.
std::vector<std::vector<int>> assign(const std::vector<double>& cost, const std::vector<const afem_mesh*>& mesh,
                                     int workers) {
    std::vector<std::vector<int>> groups;
    std::vector<double> gcost;
    for (size_t i = 0; i < cost.size(); ++i) {
        size_t g = 0;
        while (g < groups.size() && mesh[groups[g][0]] != mesh[i]) ++g;
        if (g == groups.size()) {
            groups.emplace_back();
            gcost.push_back(0.0);
        }
        groups[g].push_back(int(i));
        gcost[g] += cost[i];
    }
    std::vector<int> order(groups.size());
    for (size_t g = 0; g < order.size(); ++g) order[g] = int(g);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return gcost[a] > gcost[b]; });
    std::vector<std::vector<int>> out(workers);
    std::vector<double> load(workers, 0.0);
    for (int g : order) {
        const int w = int(std::min_element(load.begin(), load.end()) - load.begin());
        out[w].insert(out[w].end(), groups[g].begin(), groups[g].end());
        load[w] += gcost[g];
    }
    return out;
}

}  // namespace

extern "C" int afem_batch_stepper_create(afem_mctdhf* const* solvers, int count, afem_batch_stepper** out) {
    if (!out) return set_error(AFEM_EINVAL, "afem_batch_stepper_create: null output");
    *out = nullptr;
    if (!solvers || count < 1) return set_error(AFEM_EINVAL, "afem_batch_stepper_create: no instances");
    int dev = 0;
    AFEM_CUDA_TRY(cudaGetDevice(&dev));
    auto* b = new afem_batch_stepper();
    b->device = dev;
    for (int i = 0; i < count; ++i) {
        afem_mctdhf* S = solvers[i];
        if (!S) {
            destroy_stepper(b);
            return set_error(AFEM_EINVAL, "afem_batch_stepper_create: null solver");
        }
        const afem_mesh* m = mctdhf_mesh_of(S);
        if (m->device != dev) {
            destroy_stepper(b);
            return set_error(AFEM_EINVAL, "afem_batch_stepper_create: every instance must live on the current device");
        }
        b->solvers.push_back(S);
        b->mesh.push_back(m);
        // degree-weighted support points times orbitals (the Krylov vectors and
        // the cell passes), plus the n^2 Poisson columns
        const int n = mctdhf_orbitals_of(S);
        const double p1 = m->dev.p + 1.0;
        b->cost.push_back(double(m->dev.n_master) * (n + 0.25 * n * n) * (1.0 + 0.1 * p1));
    }
    for (int w = 0; w < kMaxWorkers; ++w) {
        cudaError_t e = cudaStreamCreateWithFlags(&b->streams[w], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done[w], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            destroy_stepper(b);
            return cuda_error(e, "afem_batch_stepper_create: streams");
        }
    }
    cudaError_t e = cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        destroy_stepper(b);
        return cuda_error(e, "afem_batch_stepper_create: event");
    }
    for (int c = 0; c < kNumCands; ++c)
        if (kCands[c] <= count) b->cand_streams[b->n_cand++] = kCands[c];
    *out = b;
    return AFEM_OK;
}

extern "C" int afem_batch_stepper_destroy(afem_batch_stepper* b) {
    if (b) destroy_stepper(b);
    return AFEM_OK;
}

extern "C" int afem_batch_stepper_step(afem_batch_stepper* b, void* const* phi, void* const* C, void* const* W,
                                       const double* E, double dt, double cg_rtol, int cg_max_it,
                                       afem_step_info* infos, void* stream) {
    if (!b || !phi || !C || !W) return set_error(AFEM_EINVAL, "afem_batch_stepper_step: null argument");
    if (!(dt > 0.0) || !(cg_rtol > 0.0) || cg_max_it < 0)
        return set_error(AFEM_EINVAL, "afem_batch_stepper_step: bad dt / cg_rtol / cg_max_it");
    const int count = int(b->solvers.size());
    for (int i = 0; i < count; ++i)
        if (!phi[i] || !C[i] || !W[i]) return set_error(AFEM_EINVAL, "afem_batch_stepper_step: null instance buffer");
    int dev = 0;
    AFEM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != b->device) return set_error(AFEM_EINVAL, "afem_batch_stepper_step: the current device is not the batch's");
    if (profile_on())
        return set_error(AFEM_EINVAL, "afem_batch_stepper_step: kernel-class timing must be off during batched steps");
    // worker count of this call: the cold first call on 4, then each candidate
    // once, then the fastest
    int workers;
    int cand = -1;
    if (b->chosen > 0) {
        workers = b->chosen;
    } else if (b->calls == 0) {
        workers = std::min(4, count);
    } else {
        cand = b->calls - 1;
        workers = b->cand_streams[cand];
    }
    const auto plan = assign(b->cost, b->mesh, workers);
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    AFEM_CUDA_TRY(cudaEventRecord(b->start, caller));
    for (int w = 0; w < workers; ++w) AFEM_CUDA_TRY(cudaStreamWaitEvent(b->streams[w], b->start, 0));
    std::vector<int> rc(workers, AFEM_OK);
    std::vector<std::string> msg(workers);
    std::vector<afem_step_info> local(count);
    const auto t0 = std::chrono::steady_clock::now();
    auto work = [&](int w) {
        if (cudaSetDevice(b->device) != cudaSuccess) {
            rc[w] = AFEM_ECUDA;
            msg[w] = "afem_batch_stepper_step: cudaSetDevice failed in a worker";
            return;
        }
        for (int i : plan[w]) {
            afem_step_info* inf = infos ? &infos[i] : &local[i];
            const int r = mctdhf_step(b->solvers[i], static_cast<double2*>(phi[i]), static_cast<double2*>(C[i]),
                                      static_cast<double*>(W[i]), E ? E + 3 * i : nullptr, dt, cg_rtol, cg_max_it,
                                      inf, b->streams[w]);
            if (r != AFEM_OK && rc[w] == AFEM_OK) {
                rc[w] = r;
                msg[w] = std::string(afem_last_error()) + " (instance " + std::to_string(i) + ")";
            }
            if (r != AFEM_OK && r != AFEM_ECG_MAXIT) break;
        }
        const cudaError_t e = cudaStreamSynchronize(b->streams[w]);
        if (e != cudaSuccess && rc[w] == AFEM_OK) {
            rc[w] = AFEM_ECUDA;
            msg[w] = std::string("afem_batch_stepper_step: ") + cudaGetErrorString(e);
        }
    };
    std::vector<std::thread> threads;
    threads.reserve(workers > 1 ? workers - 1 : 0);
    for (int w = 1; w < workers; ++w) threads.emplace_back(work, w);
    work(0);
    for (auto& t : threads) t.join();
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (int w = 0; w < workers; ++w) {
        AFEM_CUDA_TRY(cudaEventRecord(b->done[w], b->streams[w]));
        AFEM_CUDA_TRY(cudaStreamWaitEvent(caller, b->done[w], 0));
    }
    ++b->calls;
    // the first error (a hard error before a CG iteration limit)
    int first = AFEM_OK;
    std::string first_msg;
    for (int w = 0; w < workers; ++w) {
        if (rc[w] == AFEM_OK) continue;
        if (first == AFEM_OK || (first == AFEM_ECG_MAXIT && rc[w] != AFEM_ECG_MAXIT)) {
            first = rc[w];
            first_msg = msg[w];
        }
    }
    if (cand >= 0) {
        b->cand_ms[cand] = ms;
        if (cand == b->n_cand - 1) {
            int best = 0;
            for (int c = 1; c < b->n_cand; ++c)
                if (b->cand_ms[c] < b->cand_ms[best]) best = c;
            b->chosen = b->cand_streams[best];
        }
    }
    if (first != AFEM_OK) return set_error(first, first_msg);
    return AFEM_OK;
}

extern "C" int afem_batch_stepper_tuning(const afem_batch_stepper* b, int* streams, int* n_candidates,
                                         int* cand_streams, double* cand_ms) {
    if (!b) return set_error(AFEM_EINVAL, "afem_batch_stepper_tuning: null batch");
    if (streams) *streams = b->chosen;
    if (n_candidates) *n_candidates = b->n_cand;
    for (int c = 0; c < b->n_cand; ++c) {
        if (cand_streams) cand_streams[c] = b->cand_streams[c];
        if (cand_ms) cand_ms[c] = b->cand_ms[c];
    }
    return AFEM_OK;
}
