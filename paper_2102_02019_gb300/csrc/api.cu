// C ABI entry points that wrap the time-step kernels: error state, plans,
// launch-shape autotuning, right-hand side, filter, RK steps and the time step.
#include <cuda_runtime.h>
#include <stdint.h>

#include <stdlib.h>
#include <string.h>

#include <new>
#include <string>

#include "labfm_internal.cuh"
#include "nvtx.cuh"

namespace labfm {

namespace {
thread_local std::string g_last_error;
}

int set_error(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_error(cudaError_t e, const char* what) {
    const int code = (e == cudaErrorMemoryAllocation) ? LABFM_ENOMEM : LABFM_ECUDA;
    return set_error(code, std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                               cudaGetErrorString(e) + ")");
}

namespace {
const char* fault_spec() {
    const char* f = getenv("LABFM_FAULT");
    return f ? f : "";
}
}  // namespace

bool fault_alloc() { return strcmp(fault_spec(), "alloc") == 0; }

bool fault_capacity() { return strcmp(fault_spec(), "capacity") == 0; }

bool fault_timeout() { return strcmp(fault_spec(), "timeout") == 0; }

int64_t fault_singular_node() {
    const char* f = fault_spec();
    const char* key = "singular_node:";
    const size_t n = strlen(key);
    if (strncmp(f, key, n) != 0 || f[n] == '\0') return -1;
    char* end = nullptr;
    const long long v = strtoll(f + n, &end, 10);
    if (*end != '\0' || v < 0) return -1;
    return int64_t(v);
}

int injected_alloc_error(const char* where) {
    return set_error(LABFM_ENOMEM, std::string(where) + ": injected allocation failure (LABFM_FAULT=alloc)");
}

}  // namespace labfm

using namespace labfm;

namespace {

void free_prof(labfm_plan* p) {
    if (p->prof_ev) {
        for (int k = 0; k < 2 * p->prof_cap; ++k) cudaEventDestroy(p->prof_ev[k]);
        delete[] p->prof_ev;
        delete[] p->prof_kind;
    }
    p->prof_ev = nullptr;
    p->prof_kind = nullptr;
    p->prof_cap = 0;
    p->prof_used = 0;
}

void free_plan_memory(labfm_plan* p) {
    free_prof(p);
    cudaFree(p->row_ptr);
    cudaFree(p->col);
    cudaFree(p->w);
    cudaFree(p->wf);
    cudaFree(p->inv_s);
    cudaFree(p->inst_off);
    cudaFree(p->dt_node);
    cudaFree(p->trow_ptr);
    cudaFree(p->tw);
    cudaFree(p->twf);
    cudaFree(p->rsum);
    cudaFree(p->dev_status);
    cudaFree(p->wall_slot);
    cudaFree(p->wall_n);
    cudaFree(p->bnd_kind);
    cudaFree(p->bnd_target);
    p->wall_slot = nullptr;
    p->wall_n = nullptr;
    p->bnd_kind = nullptr;
    p->bnd_target = nullptr;
    p->n_wall = 0;
    p->dev_status = nullptr;
    p->trow_ptr = nullptr;
    p->tw = p->twf = p->rsum = nullptr;
    delete[] p->inst_off_host;
    delete[] p->range_begin;
    delete[] p->range_group;
    delete[] p->range_pf;
    p->range_begin = nullptr;
    p->range_group = nullptr;
    p->range_pf = nullptr;
    p->n_ranges = 0;
    p->row_ptr = nullptr;
    p->col = nullptr;
    p->w = p->wf = p->inv_s = nullptr;
    p->inst_off = nullptr;
    p->dt_node = nullptr;
    p->inst_off_host = nullptr;
}

int check_plan(const labfm_plan* p) {
    if (!p || !p->row_ptr) return set_error(LABFM_EINVAL, "null or empty plan");
    return LABFM_OK;
}

int create_plan(labfm_plan** out, const PlanInput* in, int n_inst, labfm_dtype dtype, void* stream) {
    if (dtype != LABFM_F32 && dtype != LABFM_F64) return set_error(LABFM_EINVAL, "unknown dtype");
    labfm_plan* p = new (std::nothrow) labfm_plan();
    if (!p) return set_error(LABFM_ENOMEM, "host allocation of the plan failed");
    for (int k = 0; k < n_inst; ++k) {
        p->N += in[k].N;
        p->nnz += in[k].nnz;
    }
    p->dtype = dtype;
    cudaGetDevice(&p->device);
    p->group = 4;
    p->block = 128;
    const int rc = pack_plan(p, in, n_inst, as_stream(stream));
    if (rc != LABFM_OK) {
        free_plan_memory(p);
        delete p;
        return rc;
    }
    *out = p;
    return LABFM_OK;
}

}  // namespace

namespace labfm {

int prof_begin(labfm_plan* p, int kind, cudaStream_t st) {
    if (!p->profiling) return -1;
    if (p->prof_used >= p->prof_cap) {
        ++p->prof_dropped;
        return -1;
    }
    const int idx = p->prof_used++;
    p->prof_kind[idx] = char(kind);
    cudaEventRecord(p->prof_ev[2 * idx], st);
    return idx;
}

bool prof_step_sampled(labfm_plan* p) {
    if (!p->profiling) return false;
    return p->prof_step++ % p->prof_period == 0;
}

void prof_end(labfm_plan* p, int idx, cudaStream_t st) {
    if (idx >= 0) cudaEventRecord(p->prof_ev[2 * idx + 1], st);
}

}  // namespace labfm

extern "C" const char* labfm_last_error(void) { return g_last_error.c_str(); }

extern "C" int labfm_abi_version(void) { return 5; }

extern "C" int labfm_plan_create(labfm_plan** out, int64_t N, int64_t nnz, labfm_dtype dtype,
                                 const int32_t* row_ptr, const int32_t* col, const double* w,
                                 const double* kappa, const double* s, void* stream) {
    LABFM_NVTX("labfm_plan_create");
    if (!out) return set_error(LABFM_EINVAL, "null plan output");
    *out = nullptr;
    if (!row_ptr || !kappa || !s || (nnz > 0 && (!col || !w)))
        return set_error(LABFM_EINVAL, "null pointer argument");
    if (N <= 0 || N >= (int64_t(1) << 31) - 1) return set_error(LABFM_EINVAL, "N out of range");
    if (nnz < 0 || nnz >= (int64_t(1) << 31)) return set_error(LABFM_EINVAL, "nnz out of range");
    if (dtype != LABFM_F32 && dtype != LABFM_F64) return set_error(LABFM_EINVAL, "unknown dtype");
    if (fault_alloc()) return injected_alloc_error("labfm_plan_create");
    if (int rc = validate_csr(row_ptr, col, N, nnz, as_stream(stream))) return rc;
    const PlanInput in{N, nnz, row_ptr, col, w, kappa, s};
    return create_plan(out, &in, 1, dtype, stream);
}

extern "C" int labfm_plan_create_batched(labfm_plan** out, int n_inst, const int64_t* N_inst,
                                         const int64_t* nnz_inst, const int32_t* const* row_ptr,
                                         const int32_t* const* col, const double* const* w,
                                         const double* const* kappa, const double* const* s,
                                         labfm_dtype dtype, void* stream) {
    LABFM_NVTX("labfm_plan_create_batched");
    if (!out) return set_error(LABFM_EINVAL, "null plan output");
    *out = nullptr;
    if (n_inst <= 0) return set_error(LABFM_EINVAL, "need at least one instance");
    if (!N_inst || !nnz_inst || !row_ptr || !col || !w || !kappa || !s)
        return set_error(LABFM_EINVAL, "null pointer argument");
    PlanInput* in = new (std::nothrow) PlanInput[n_inst];
    if (!in) return set_error(LABFM_ENOMEM, "host allocation failed");
    int64_t Ntot = 0, nnztot = 0;
    int rc = LABFM_OK;
    for (int k = 0; k < n_inst && rc == LABFM_OK; ++k) {
        in[k] = PlanInput{N_inst[k], nnz_inst[k], row_ptr[k], col[k], w[k], kappa[k], s[k]};
        if (N_inst[k] <= 0 || nnz_inst[k] < 0 || !row_ptr[k] || !kappa[k] || !s[k] ||
            (nnz_inst[k] > 0 && (!col[k] || !w[k])))
            rc = set_error(LABFM_EINVAL, "bad instance " + std::to_string(k));
        Ntot += N_inst[k];
        nnztot += nnz_inst[k];
    }
    if (rc == LABFM_OK && (Ntot >= (int64_t(1) << 31) - 1 || nnztot >= (int64_t(1) << 31)))
        rc = set_error(LABFM_EINVAL, "combined size out of range");
    if (rc == LABFM_OK && fault_alloc()) rc = injected_alloc_error("labfm_plan_create_batched");
    for (int k = 0; k < n_inst && rc == LABFM_OK; ++k)
        if ((rc = validate_csr(in[k].row_ptr, in[k].col, in[k].N, in[k].nnz, as_stream(stream))))
            rc = set_error(LABFM_EINVAL, "instance " + std::to_string(k) + ": " + labfm_last_error());
    if (rc == LABFM_OK) rc = create_plan(out, in, n_inst, dtype, stream);
    delete[] in;
    return rc;
}

extern "C" int labfm_plan_set_dt(labfm_plan* p, const double* dt_inst, void* stream) {
    if (int rc = check_plan(p)) return rc;
    if (!dt_inst) return set_error(LABFM_EINVAL, "null dt array");
    if (!p->dt_node && fault_alloc()) return injected_alloc_error("labfm_plan_set_dt");
    return set_node_dt(p, dt_inst, as_stream(stream));
}

extern "C" int labfm_stable_dt_instances(const labfm_plan* p, const void* fields, const double* s,
                                         double c, double mu, double* dt_inst_out, void* stream) {
    if (int rc = check_plan(p)) return rc;
    if (!fields || !s || !dt_inst_out) return set_error(LABFM_EINVAL, "null pointer argument");
    if (!(c >= 0.0) || !(mu > 0.0)) return set_error(LABFM_EINVAL, "need c >= 0 and mu > 0");
    return launch_stable_dt_instances(p, fields, s, c, mu, dt_inst_out, as_stream(stream));
}

extern "C" int labfm_plan_set_persistent(labfm_plan* p, int enable) {
    if (int rc = check_plan(p)) return rc;
    p->persistent = enable != 0;
    p->persist_grid = p->persistent ? persistent_grid(p) : 0;
    return LABFM_OK;
}

extern "C" int labfm_plan_set_prefetch(labfm_plan* p, int distance) {
    if (int rc = check_plan(p)) return rc;
    if (distance < 0 || distance > 8) return set_error(LABFM_EINVAL, "prefetch distance must be in [0, 8]");
    p->prefetch = distance;
    return LABFM_OK;
}

extern "C" int labfm_plan_set_programmatic_launch(labfm_plan* p, int enable) {
    if (int rc = check_plan(p)) return rc;
    if (enable != 0 && enable != 1) return set_error(LABFM_EINVAL, "enable must be 0 or 1");
    p->programmatic = enable != 0;
    return LABFM_OK;
}

extern "C" int labfm_plan_set_staging(labfm_plan* p, int stages, void* stream) {
    if (int rc = check_plan(p)) return rc;
    if (stages != 0 && fault_alloc()) return injected_alloc_error("labfm_plan_set_staging");
    return configure_staging(p, stages, as_stream(stream));
}

extern "C" int labfm_plan_set_wait_limit(labfm_plan* p, int64_t limit_ns) {
    if (int rc = check_plan(p)) return rc;
    if (limit_ns < 0 || limit_ns > int64_t(10000000000))
        return set_error(LABFM_EINVAL, "wait limit must be in [0, 10 s]");
    p->wait_ns = uint64_t(limit_ns);
    return LABFM_OK;
}

extern "C" int labfm_plan_set_check_finite(labfm_plan* p, int every) {
    if (int rc = check_plan(p)) return rc;
    if (every < 0) return set_error(LABFM_EINVAL, "every must be >= 0");
    if (every > 0 && !p->dev_status) {
        if (fault_alloc()) return injected_alloc_error("labfm_plan_set_check_finite");
        LABFM_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&p->dev_status), sizeof(int)));
        LABFM_CUDA_TRY(cudaMemset(p->dev_status, 0, sizeof(int)));
    }
    p->check_every = every;
    return LABFM_OK;
}

extern "C" int labfm_plan_device_status(const labfm_plan* p, int* status_out) {
    if (int rc = check_plan(p)) return rc;
    if (!status_out) return set_error(LABFM_EINVAL, "null status output");
    *status_out = LABFM_OK;
    if (fault_timeout()) {  // LABFM_FAULT=timeout: as if a bounded wait had run out
        *status_out = LABFM_ETIMEOUT;
        return LABFM_OK;
    }
    if (!p->dev_status) return LABFM_OK;
    LABFM_CUDA_TRY(cudaMemcpy(status_out, p->dev_status, sizeof(int), cudaMemcpyDeviceToHost));
    LABFM_CUDA_TRY(cudaMemset(p->dev_status, 0, sizeof(int)));
    return LABFM_OK;
}

extern "C" int labfm_plan_destroy(labfm_plan* p) {
    if (!p) return LABFM_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != p->device) cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    free_plan_memory(p);
    if (dev != p->device) cudaSetDevice(dev);
    delete p;
    return LABFM_OK;
}

extern "C" int labfm_plan_get_info(const labfm_plan* p, labfm_plan_info* info) {
    if (int rc = check_plan(p)) return rc;
    if (!info) return set_error(LABFM_EINVAL, "null info output");
    info->N = p->N;
    info->nnz = p->nnz;
    info->nnz_padded = p->nnz_pad;
    info->dtype = p->dtype;
    info->group = p->group;
    info->block = p->block;
    info->n_instances = p->n_inst;
    info->entry_bytes = plan_entry_bytes(p, false);
    info->filter_entry_bytes = plan_entry_bytes(p, true);
    info->device_bytes = p->device_bytes;
    info->prefetch = p->prefetch;
    info->stages = p->stages;
    info->filter_group = p->filter_group ? p->filter_group : p->group;
    info->filter_persistent = p->filter_persistent ? 1 : 0;
    info->programmatic = p->programmatic ? 1 : 0;
    return LABFM_OK;
}

extern "C" int labfm_plan_set_launch(labfm_plan* p, int group, int block) {
    if (int rc = check_plan(p)) return rc;
    if (!launch_shape_supported(group, block))
        return set_error(LABFM_EINVAL, "unsupported launch shape (group " + std::to_string(group) +
                                           ", block " + std::to_string(block) + ")");
    p->group = group;
    p->block = block;
    if (p->persistent) p->persist_grid = persistent_grid(p);
    if (p->filter_persistent) p->filter_grid = filter_persistent_grid(p);
    return LABFM_OK;
}

extern "C" int labfm_plan_set_launch_ranges(labfm_plan* p, int n, const int64_t* begin, const int32_t* group,
                                            const int32_t* prefetch) {
    if (int rc = check_plan(p)) return rc;
    if (n < 0) return set_error(LABFM_EINVAL, "negative number of ranges");
    if (n > 0) {
        if (!begin || !group || !prefetch) return set_error(LABFM_EINVAL, "null pointer argument");
        if (begin[0] != 0 || begin[n] != p->N) return set_error(LABFM_EINVAL, "ranges must cover [0, N)");
        for (int r = 0; r < n; ++r) {
            if (begin[r + 1] < begin[r]) return set_error(LABFM_EINVAL, "range boundaries must not decrease");
            if (!launch_shape_supported(group[r], p->block))
                return set_error(LABFM_EINVAL, "unsupported lanes per node in range " + std::to_string(r));
            if (prefetch[r] < 0 || prefetch[r] > 8) return set_error(LABFM_EINVAL, "prefetch must be in [0, 8]");
        }
    }
    int64_t* nb = n ? new (std::nothrow) int64_t[n + 1] : nullptr;
    int* ng = n ? new (std::nothrow) int[n] : nullptr;
    int* np = n ? new (std::nothrow) int[n] : nullptr;
    if (n && (!nb || !ng || !np)) {
        delete[] nb;
        delete[] ng;
        delete[] np;
        return set_error(LABFM_ENOMEM, "host allocation failed");
    }
    for (int r = 0; r <= n && n; ++r) nb[r] = begin[r];
    for (int r = 0; r < n; ++r) {
        ng[r] = group[r];
        np[r] = p->dtype == LABFM_F32 ? prefetch[r] : 0;
    }
    delete[] p->range_begin;
    delete[] p->range_group;
    delete[] p->range_pf;
    p->range_begin = nb;
    p->range_group = ng;
    p->range_pf = np;
    p->n_ranges = n;
    return LABFM_OK;
}

extern "C" int labfm_plan_set_filter_launch(labfm_plan* p, int group, int persistent) {
    if (int rc = check_plan(p)) return rc;
    if (group != 0 && !launch_shape_supported(group, p->block))
        return set_error(LABFM_EINVAL, "unsupported filter lanes per node " + std::to_string(group));
    p->filter_group = group;
    p->filter_persistent = persistent != 0;
    p->filter_grid = p->filter_persistent ? filter_persistent_grid(p) : 0;
    return LABFM_OK;
}

extern "C" int labfm_plan_autotune(labfm_plan* p, const void* fields, void* scratch_rhs,
                                   const labfm_phys* phys, int reps, int* group_out, int* block_out,
                                   void* stream) {
    LABFM_NVTX("labfm_plan_autotune");
    if (int rc = check_plan(p)) return rc;
    if (!fields || !scratch_rhs || !phys) return set_error(LABFM_EINVAL, "null pointer argument");
    if (reps <= 0) reps = 5;
    cudaStream_t st = as_stream(stream);
    cudaEvent_t e0, e1;
    LABFM_CUDA_TRY(cudaEventCreate(&e0));
    LABFM_CUDA_TRY(cudaEventCreate(&e1));
    // the gather kernels run fixed one-warp blocks; the lanes per node are tuned
    const int groups[] = {2, 4, 8, 16, 32};
    const int blocks[] = {p->block};
    float best = 1e30f;
    int bg = p->group, bb = p->block;
    int rc = LABFM_OK;
    for (int g : groups) {
        for (int b : blocks) {
            if (!launch_shape_supported(g, b)) continue;
            // warm-up launch, then `reps` timed launches
            if ((rc = launch_rhs(p, fields, scratch_rhs, phys, g, b, st))) break;
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps && rc == LABFM_OK; ++r)
                rc = launch_rhs(p, fields, scratch_rhs, phys, g, b, st);
            cudaEventRecord(e1, st);
            if (rc) break;
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                rc = cuda_error(e, "autotune timing");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bg = g;
                bb = b;
            }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    p->group = bg;
    p->block = bb;
    if (p->persistent) p->persist_grid = persistent_grid(p);
    if (p->filter_persistent) p->filter_grid = filter_persistent_grid(p);
    if (group_out) *group_out = bg;
    if (block_out) *block_out = bb;
    return LABFM_OK;
}

extern "C" int labfm_rhs(const labfm_plan* p, const void* fields, void* rhs,
                         const labfm_phys* phys, void* stream) {
    LABFM_NVTX("labfm_rhs");
    if (int rc = check_plan(p)) return rc;
    if (!fields || !rhs || !phys) return set_error(LABFM_EINVAL, "null pointer argument");
    if (fields == rhs) return set_error(LABFM_EINVAL, "rhs must not alias fields");
    return launch_rhs(p, fields, rhs, phys, p->group, p->block, as_stream(stream));
}

extern "C" int labfm_filter(const labfm_plan* p, const void* in, void* out, void* stream) {
    LABFM_NVTX("labfm_filter");
    if (int rc = check_plan(p)) return rc;
    if (!in || !out) return set_error(LABFM_EINVAL, "null pointer argument");
    if (in == out) return set_error(LABFM_EINVAL, "filter output must not alias its input");
    return launch_filter_soa(p, in, out, as_stream(stream));
}

extern "C" size_t labfm_rk_workspace_bytes(const labfm_plan* p) {
    return p ? rk_work_bytes(p) : 0;
}

extern "C" int labfm_rk_step(const labfm_plan* p, void* Q, void* work, size_t work_bytes,
                             double dt, int nsteps, const labfm_phys* phys, void* stream) {
    LABFM_NVTX("labfm_rk_step");
    if (int rc = check_plan(p)) return rc;
    if (!Q || !work || !phys) return set_error(LABFM_EINVAL, "null pointer argument");
    if (nsteps < 0) return set_error(LABFM_EINVAL, "negative nsteps");
    if (work_bytes < rk_work_bytes(p))
        return set_error(LABFM_EINVAL, "work buffer smaller than labfm_rk_workspace_bytes");
    if (reinterpret_cast<uintptr_t>(work) % 16 != 0)
        return set_error(LABFM_EINVAL, "work buffer must be 16-byte aligned");
    if (nsteps > 0 && !(dt > 0.0) && !(dt == 0.0 && p->dt_node))
        return set_error(LABFM_EINVAL, "dt must be positive (or 0 with per-instance dt set)");
    return launch_rk_steps(p, Q, work, dt, nsteps, phys, as_stream(stream));
}

extern "C" int labfm_stable_dt(const labfm_plan* p, const void* fields, const double* s, double c,
                               double mu, double* dt_out, void* stream) {
    LABFM_NVTX("labfm_stable_dt");
    if (int rc = check_plan(p)) return rc;
    if (!fields || !s || !dt_out) return set_error(LABFM_EINVAL, "null pointer argument");
    if (!(c >= 0.0) || !(mu > 0.0)) return set_error(LABFM_EINVAL, "need c >= 0 and mu > 0");
    return launch_stable_dt(p, fields, s, c, mu, dt_out, as_stream(stream));
}

extern "C" int labfm_rk_step_host(const labfm_plan* p, void* Q_host, void* Q_dev, void* work,
                                  size_t work_bytes, double dt, int nsteps,
                                  const labfm_phys* phys, void* stream) {
    LABFM_NVTX("labfm_rk_step_host");
    if (int rc = check_plan(p)) return rc;
    if (!Q_host || !Q_dev) return set_error(LABFM_EINVAL, "null pointer argument");
    const size_t bytes = size_t(3) * size_t(p->N) * (p->dtype == LABFM_F32 ? sizeof(float) : sizeof(double));
    cudaStream_t st = as_stream(stream);
    // Page-locked, mapped host memory: the pack and unpack kernels of the step read
    // and write it directly over the host link, without a staging copy.
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, Q_host) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
        attr.devicePointer && reinterpret_cast<uintptr_t>(attr.devicePointer) % 16 == 0) {
        if (int rc = labfm_rk_step(p, attr.devicePointer, work, work_bytes, dt, nsteps, phys, stream))
            return rc;
        LABFM_CUDA_TRY(cudaStreamSynchronize(st));
        return LABFM_OK;
    }
    cudaGetLastError();  // pageable memory: not an error, take the copy path
    LABFM_CUDA_TRY(cudaMemcpyAsync(Q_dev, Q_host, bytes, cudaMemcpyHostToDevice, st));
    if (int rc = labfm_rk_step(p, Q_dev, work, work_bytes, dt, nsteps, phys, stream)) return rc;
    LABFM_CUDA_TRY(cudaMemcpyAsync(Q_host, Q_dev, bytes, cudaMemcpyDeviceToHost, st));
    LABFM_CUDA_TRY(cudaStreamSynchronize(st));
    return LABFM_OK;
}

extern "C" int labfm_plan_set_profiling(labfm_plan* p, int enable) {
    if (int rc = check_plan(p)) return rc;
    if (enable < 0) return set_error(LABFM_EINVAL, "enable must be >= 0");
    if (enable && !p->prof_ev) {
        const int cap = 8192;
        p->prof_ev = new (std::nothrow) cudaEvent_t[2 * cap];
        p->prof_kind = new (std::nothrow) char[cap];
        if (!p->prof_ev || !p->prof_kind) {
            delete[] p->prof_ev;
            delete[] p->prof_kind;
            p->prof_ev = nullptr;
            p->prof_kind = nullptr;
            return set_error(LABFM_ENOMEM, "host allocation of the event pool failed");
        }
        for (int k = 0; k < 2 * cap; ++k) {
            cudaError_t e = cudaEventCreate(&p->prof_ev[k]);
            if (e != cudaSuccess) {
                for (int j = 0; j < k; ++j) cudaEventDestroy(p->prof_ev[j]);
                delete[] p->prof_ev;
                delete[] p->prof_kind;
                p->prof_ev = nullptr;
                p->prof_kind = nullptr;
                return cuda_error(e, "cudaEventCreate");
            }
        }
        p->prof_cap = cap;
    }
    p->profiling = enable != 0;
    p->prof_period = enable > 0 ? enable : 1;
    p->prof_step = 0;
    p->prof_used = 0;
    p->prof_dropped = 0;
    return LABFM_OK;
}

extern "C" int labfm_plan_read_profile(labfm_plan* p, labfm_profile* out) {
    if (int rc = check_plan(p)) return rc;
    if (!out) return set_error(LABFM_EINVAL, "null profile output");
    *out = labfm_profile{};
    out->dropped = p->prof_dropped;
    if (p->prof_used > 0) {
        LABFM_CUDA_TRY(cudaEventSynchronize(p->prof_ev[2 * (p->prof_used - 1) + 1]));
        for (int k = 0; k < p->prof_used; ++k) {
            float ms = 0.f;
            LABFM_CUDA_TRY(cudaEventElapsedTime(&ms, p->prof_ev[2 * k], p->prof_ev[2 * k + 1]));
            switch (p->prof_kind[k]) {
                case kProfStage:
                case kProfStages4:
                    out->stage_ms += ms;
                    out->stage_launches += p->prof_kind[k] == kProfStages4 ? 4 : 1;
                    break;
                case kProfFilter:
                    out->filter_ms += ms;
                    ++out->filter_launches;
                    break;
                case kProfRecStages4:
                    out->rec_stage_ms += ms;
                    out->rec_stage_launches += 4;
                    break;
                case kProfAdjA:
                    out->adj_a_ms += ms;
                    ++out->adj_a_launches;
                    break;
                case kProfAdjB:
                    out->adj_b_ms += ms;
                    ++out->adj_b_launches;
                    break;
                case kProfAdjFilter:
                    out->adj_filter_ms += ms;
                    ++out->adj_filter_launches;
                    break;
            }
        }
    }
    p->prof_used = 0;
    p->prof_dropped = 0;
    return LABFM_OK;
}
