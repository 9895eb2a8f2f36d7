// Batching form of the hot path: the FP32 cell passes of many independent
// instances (meshes of uneven size and degree, each with its own orbitals or
// pair right-hand sides) in one persistent launch, captured once into a CUDA
// graph and replayed, with the launch shape picked by timing candidates on
// the batch itself.  Each instance computes exactly what afem_op_apply
// computes for it (Sec. 3.1, Eq. discretized_eom); only the scheduling is
// shared.
#include <cstring>
#include <new>
#include <vector>

#include "afem_internal.h"

namespace afem {
size_t batch32_inst_bytes();
int batch32_fill(const afem_mesh* m, int kind, const double* E, const void* x, void* y, int nvec, int64_t cell0,
                 void* out);
size_t batch32_smem(const std::vector<int>& p, const std::vector<int>& L4);
int64_t batch32_items(int p, int L4, int64_t ncell);
int batch32_occupancy(int kind, int block, size_t smem, int* per_sm);
int batch32_launch(int kind, const void* d_inst, int count, int64_t total, int block, unsigned grid, size_t smem,
                   cudaStream_t s);
}  // namespace afem

using namespace afem;

namespace {
constexpr int kParStreams = 16;   // streams available to the per-instance schedule
bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }
}

struct afem_batch {
    std::vector<afem_mesh*> meshes;
    int64_t total_cells = 0;
    int64_t total_items = 0;             // work items of the current signature (small cells grouped)
    int sms = 0;
    size_t rec = 0;                      // bytes of one instance record
    void* d_inst = nullptr;              // device instance table
    void* h_inst = nullptr;              // pinned host staging of each upload
    std::vector<unsigned char> last;     // contents of the last upload
    cudaStream_t cap = nullptr;          // private stream for graph capture
    cudaStream_t par[kParStreams] = {};  // per-instance schedule: instance i runs on par[i % streams]
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kParStreams] = {};
    // arguments of the current apply (the per-instance schedule launches from them)
    std::vector<const void*> cur_x;
    std::vector<void*> cur_y;
    std::vector<int> cur_n;
    std::vector<double> cur_E;
    // launch shape and its graph, valid for one (kind, lanes per instance) signature
    int sig_kind = -1;
    std::vector<int> sig_L4;
    int block = 0, grid = 0, per_sm = 0;
    size_t smem = 0;
    std::vector<double> cand_ms;
    std::vector<int> cand_block, cand_grid;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void drop_graph(afem_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

// The per-instance schedule: each instance's own pass (the kernels of
// afem_op_apply) on one of `streams` streams forked from s and joined back,
// so that independent instances run concurrently.  Captured into the graph
// like the persistent launch (the streams join the capture through the events).
int launch_per_instance(afem_batch* b, int kind, int streams, cudaStream_t s) {
    if (streams < 1 || streams > kParStreams) return set_error(AFEM_EINVAL, "afem_batch: bad stream count");
    AFEM_CUDA_TRY(cudaEventRecord(b->fork, s));
    for (int j = 0; j < streams; ++j) AFEM_CUDA_TRY(cudaStreamWaitEvent(b->par[j], b->fork, 0));
    const int count = int(b->meshes.size());
    for (int i = 0; i < count; ++i) {
        const double* E = b->cur_E.empty() ? nullptr : b->cur_E.data() + 3 * i;
        int rc = launch_op_apply(b->meshes[i], kind, E, b->cur_x[i], b->cur_y[i], b->cur_n[i],
                                 b->par[i % streams]);
        if (rc) return rc;
    }
    for (int j = 0; j < streams; ++j) {
        AFEM_CUDA_TRY(cudaEventRecord(b->join[j], b->par[j]));
        AFEM_CUDA_TRY(cudaStreamWaitEvent(s, b->join[j], 0));
    }
    return AFEM_OK;
}

// One apply with the chosen schedule (block 0: per instance on `grid` streams).
int launch_schedule(afem_batch* b, int kind, int block, unsigned grid, size_t smem, cudaStream_t s) {
    if (block == 0) return launch_per_instance(b, kind, int(grid), s);
    return batch32_launch(kind, b->d_inst, int(b->meshes.size()), b->total_items, block, grid, smem, s);
}

// Times launch shape (block, grid) on the uploaded batch: best of 3 after a warm-up.
int time_shape(afem_batch* b, int kind, int block, unsigned grid, size_t smem, cudaStream_t s, double* ms) {
    cudaEvent_t e0, e1;
    AFEM_CUDA_TRY(cudaEventCreate(&e0));
    AFEM_CUDA_TRY(cudaEventCreate(&e1));
    double best = 1e30;
    int rc = AFEM_OK;
    for (int r = 0; r < 4 && rc == AFEM_OK; ++r) {
        cudaEventRecord(e0, s);
        rc = launch_schedule(b, kind, block, grid, smem, s);
        cudaEventRecord(e1, s);
        if (rc) break;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = cuda_error(e, "afem_batch tuning");
            break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (r > 0 && t < best) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return rc;
}

// Candidate schedules: the persistent launch with grids of 2 or all resident
// blocks per SM at 256 and 128 threads and one block per work item, and the
// per-instance passes on 4, 8 or 16 parallel streams (block 0, grid =
// streams).  The fastest is kept.  persistent = false (an instance whose
// values per node are not whole 16-byte quads: an odd orbital count, real
// columns not a multiple of 4, or unaligned buffers) leaves only the
// per-instance schedule, whose single-instance passes take any count.
int tune(afem_batch* b, int kind, bool persistent, cudaStream_t s) {
    b->cand_ms.clear();
    b->cand_block.clear();
    b->cand_grid.clear();
    double best = 1e30;
    for (int block : {256, 128}) {
        if (!persistent) break;
        int per_sm = 0;
        int rc = batch32_occupancy(kind, block, b->smem, &per_sm);
        if (rc) return rc;
        std::vector<int64_t> grids = {int64_t(b->sms) * per_sm, int64_t(b->sms) * 2};
        if (block == 256) grids.push_back(b->total_items);
        for (int64_t g : grids) {
            if (g > b->total_items) g = b->total_items;
            if (g > 0x7fffffff) g = 0x7fffffff;
            if (g < 1) continue;
            double ms = 0.0;
            if ((rc = time_shape(b, kind, block, unsigned(g), b->smem, s, &ms))) return rc;
            b->cand_ms.push_back(ms);
            b->cand_block.push_back(block);
            b->cand_grid.push_back(int(g));
            if (ms < best) {
                best = ms;
                b->block = block;
                b->grid = int(g);
                b->per_sm = per_sm;
            }
        }
    }
    for (int streams : {4, 8, 16}) {
        double ms = 0.0;
        int rc = time_shape(b, kind, 0, unsigned(streams), 0, s, &ms);
        if (rc) return rc;
        b->cand_ms.push_back(ms);
        b->cand_block.push_back(0);
        b->cand_grid.push_back(streams);
        if (ms < best) {
            best = ms;
            b->block = 0;
            b->grid = streams;
            b->per_sm = 0;
        }
    }
    return AFEM_OK;
}

}  // namespace

extern "C" {

int afem_batch_create(afem_mesh* const* meshes, int count, afem_batch** out) {
    if (!out) return set_error(AFEM_EINVAL, "afem_batch_create: null output");
    *out = nullptr;
    if (!meshes || count < 1 || count > AFEM_BATCH_MAX)
        return set_error(AFEM_EINVAL, "afem_batch_create: 1..256 meshes required");
    for (int i = 0; i < count; ++i)
        if (!meshes[i] || meshes[i]->host_only)
            return set_error(AFEM_EINVAL, "afem_batch_create: every mesh must be uploaded (not host-only)");
    auto* b = new (std::nothrow) afem_batch();
    if (!b) return set_error(AFEM_ENOMEM, "afem_batch_create: out of host memory");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete b;
        return cuda_error(e, "afem_batch_create");
    }
    for (int i = 0; i < count; ++i) {
        if (meshes[i]->device != dev) {
            delete b;
            return set_error(AFEM_EINVAL, "afem_batch_create: meshes must live on the current device");
        }
        b->meshes.push_back(meshes[i]);
        b->total_cells += meshes[i]->dev.ncell;
    }
    b->rec = batch32_inst_bytes();
    e = cudaMalloc(&b->d_inst, b->rec * count);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_inst, b->rec * count);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    for (int j = 0; j < kParStreams && e == cudaSuccess; ++j) {
        e = cudaStreamCreateWithFlags(&b->par[j], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[j], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        afem_batch_destroy(b);
        return cuda_error(e, "afem_batch_create");
    }
    *out = b;
    return AFEM_OK;
}

int afem_batch_destroy(afem_batch* b) {
    if (!b) return AFEM_OK;
    drop_graph(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (int j = 0; j < kParStreams; ++j) {
        if (b->par[j]) cudaStreamDestroy(b->par[j]);
        if (b->join[j]) cudaEventDestroy(b->join[j]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->d_inst) cudaFree(b->d_inst);
    if (b->h_inst) cudaFreeHost(b->h_inst);
    delete b;
    return AFEM_OK;
}

int afem_batch_op_apply(afem_batch* b, int kind, const double* E, void* const* x, void* const* y,
                        const int* n_vec, int flags, void* stream) {
    if (!b || !x || !y || !n_vec) return set_error(AFEM_EINVAL, "afem_batch_op_apply: null argument");
    if (kind != AFEM_OP_H1_C64 && kind != AFEM_OP_STIFF_F32)
        return set_error(AFEM_EINVAL, "afem_batch_op_apply: kind must be AFEM_OP_H1_C64 or AFEM_OP_STIFF_F32");
    if (flags & ~AFEM_BATCH_GRAPH) return set_error(AFEM_EINVAL, "afem_batch_op_apply: unknown flags");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int count = int(b->meshes.size());
    std::vector<int> p(count), L4(count);
    std::vector<unsigned char> staged(b->rec * count);
    bool quads = true;   // every instance's node values are whole 16-byte quads
    for (int i = 0; i < count; ++i) {
        if (!x[i] || !y[i] || n_vec[i] < 1) return set_error(AFEM_EINVAL, "afem_batch_op_apply: bad instance buffer");
        if (x[i] == y[i]) return set_error(AFEM_EINVAL, "afem_batch_op_apply: x and y must differ");
        const int L = kind == AFEM_OP_H1_C64 ? 2 * n_vec[i] : n_vec[i];
        if (L % 4 != 0 || !aligned16(x[i]) || !aligned16(y[i])) quads = false;
    }
    int64_t item0 = 0;   // first work item of each instance (small cells grouped per item)
    for (int i = 0; i < count; ++i) {
        p[i] = b->meshes[i]->dev.p;
        if (!quads) {   // per-instance schedule only; the signature keeps the column counts
            L4[i] = -n_vec[i];
            continue;
        }
        int rc = batch32_fill(b->meshes[i], kind, E ? E + 3 * i : nullptr, x[i], y[i], n_vec[i], item0,
                              staged.data() + b->rec * i);
        if (rc) return rc;
        L4[i] = (kind == AFEM_OP_H1_C64 ? 2 * n_vec[i] : n_vec[i]) / 4;
        item0 += batch32_items(p[i], L4[i], b->meshes[i]->dev.ncell);
    }
    b->total_items = item0;
    b->cur_x.assign(x, x + count);
    b->cur_y.assign(y, y + count);
    b->cur_n.assign(n_vec, n_vec + count);
    if (E) b->cur_E.assign(E, E + 3 * count);
    else b->cur_E.clear();
    // upload the instance table only when it changed; the pinned staging copy is
    // rewritten only after the previous upload has been consumed
    if (staged != b->last) {
        if (b->block == 0) drop_graph(b);   // the per-instance graph holds the buffers and fields
        AFEM_CUDA_TRY(cudaStreamSynchronize(s));
        std::memcpy(b->h_inst, staged.data(), staged.size());
        AFEM_CUDA_TRY(cudaMemcpyAsync(b->d_inst, b->h_inst, staged.size(), cudaMemcpyHostToDevice, s));
        b->last = staged;
    }
    if (kind != b->sig_kind || L4 != b->sig_L4) {   // new signature: re-tune, drop the graph
        drop_graph(b);
        b->sig_kind = kind;
        b->sig_L4 = L4;
        b->smem = quads ? batch32_smem(p, L4) : 0;
        int rc = tune(b, kind, quads, s);
        if (rc) {
            b->sig_kind = -1;
            return rc;
        }
    }
    if (!(flags & AFEM_BATCH_GRAPH)) return launch_schedule(b, kind, b->block, unsigned(b->grid), b->smem, s);
    if (!b->exec) {
        cudaGraph_t g = nullptr;
        AFEM_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        int rc = launch_schedule(b, kind, b->block, unsigned(b->grid), b->smem, b->cap);
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_error(e, "afem_batch_op_apply: graph capture");
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return cuda_error(e, "afem_batch_op_apply: graph instantiation");
        }
    }
    AFEM_CUDA_TRY(cudaGraphLaunch(b->exec, s));
    return AFEM_OK;
}

int afem_batch_get_tuning(const afem_batch* b, afem_batch_tuning* out) {
    if (!b || !out) return set_error(AFEM_EINVAL, "afem_batch_get_tuning: null argument");
    std::memset(out, 0, sizeof(*out));
    out->tuned = b->sig_kind >= 0 ? 1 : 0;
    out->block = b->block;
    out->grid = b->grid;
    out->blocks_per_sm = b->per_sm;
    out->n_candidates = int(b->cand_ms.size());
    for (int i = 0; i < out->n_candidates && i < AFEM_BATCH_MAX_CAND; ++i) {
        out->cand_ms[i] = b->cand_ms[i];
        out->cand_block[i] = b->cand_block[i];
        out->cand_grid[i] = b->cand_grid[i];
    }
    out->total_cells = b->total_cells;
    out->count = int(b->meshes.size());
    return AFEM_OK;
}

}  // extern "C"
