// A captured CUDA graph of one complete time step (four fused stage kernels,
// the filter, and for persistent plans the work-queue ticket reset), replayed
// once per step: one graph launch advances every instance of a batched plan.
#include <cuda_runtime.h>
#include <stdint.h>

#include <new>

#include "labfm_internal.cuh"
#include "nvtx.cuh"

struct labfm_step_graph {
    const labfm_plan* plan = nullptr;
    void* work = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

using namespace labfm;

namespace {
void destroy_graph(labfm_step_graph* g) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}
}  // namespace

extern "C" int labfm_step_graph_create(labfm_step_graph** out, const labfm_plan* plan, void* work,
                                       size_t work_bytes, double dt, const labfm_phys* phys) {
    LABFM_NVTX("labfm_step_graph_create");
    if (!out) return set_error(LABFM_EINVAL, "null graph output");
    *out = nullptr;
    if (!plan || !plan->row_ptr || !work || !phys) return set_error(LABFM_EINVAL, "null pointer argument");
    if (work_bytes < rk_work_bytes(plan))
        return set_error(LABFM_EINVAL, "work buffer smaller than labfm_rk_workspace_bytes");
    if (reinterpret_cast<uintptr_t>(work) % 16 != 0)
        return set_error(LABFM_EINVAL, "work buffer must be 16-byte aligned");
    if (!(dt > 0.0) && !(dt == 0.0 && plan->dt_node))
        return set_error(LABFM_EINVAL, "dt must be positive (or 0 with per-instance dt set)");
    if (fault_alloc()) return injected_alloc_error("labfm_step_graph_create");
    labfm_step_graph* g = new (std::nothrow) labfm_step_graph();
    if (!g) return set_error(LABFM_ENOMEM, "host allocation failed");
    g->plan = plan;
    g->work = work;
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete g;
        return cuda_error(e, "cudaStreamCreateWithFlags");
    }
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc = LABFM_OK;
    if (e != cudaSuccess) {
        rc = cuda_error(e, "cudaStreamBeginCapture");
    } else {
        rc = rk_one_step(plan, work, dt, phys, false, cs);
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g->graph);
        if (rc == LABFM_OK && e2 != cudaSuccess) rc = cuda_error(e2, "cudaStreamEndCapture");
    }
    if (rc == LABFM_OK) {
        e = cudaGraphInstantiate(&g->exec, g->graph, 0);
        if (e != cudaSuccess) rc = cuda_error(e, "cudaGraphInstantiate");
    }
    cudaStreamDestroy(cs);
    if (rc != LABFM_OK) {
        destroy_graph(g);
        return rc;
    }
    *out = g;
    return LABFM_OK;
}

extern "C" int labfm_step_graph_run(labfm_step_graph* g, void* Q, int nsteps, void* stream) {
    LABFM_NVTX("labfm_step_graph_run");
    if (!g || !g->exec) return set_error(LABFM_EINVAL, "null graph");
    if (!Q) return set_error(LABFM_EINVAL, "null state");
    if (nsteps < 0) return set_error(LABFM_EINVAL, "negative nsteps");
    if (nsteps == 0) return LABFM_OK;
    cudaStream_t st = as_stream(stream);
    if (int rc = rk_pack(g->plan, Q, g->work, st)) return rc;
    for (int k = 0; k < nsteps; ++k) LABFM_CUDA_TRY(cudaGraphLaunch(g->exec, st));
    return rk_unpack(g->plan, Q, g->work, st);
}

extern "C" int labfm_step_graph_destroy(labfm_step_graph* g) {
    if (g) destroy_graph(g);
    return LABFM_OK;
}
