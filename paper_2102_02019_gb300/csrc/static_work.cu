// labfm_rk_step_noalloc: the RK time step with its state buffers in a
// fixed-size device array that is part of the library image, for callers that
// cannot allocate device memory themselves (see labfm.h).
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "labfm_internal.cuh"
#include "nvtx.cuh"

namespace {

// Scratch for the three packed state buffers of labfm_rk_step.  Every GPU that
// loads the library holds this array until the process exits.
constexpr size_t kStaticWorkBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_static_work[kStaticWorkBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};  // device address of g_static_work, per device

// The device address of g_static_work on the current device.  In host code the
// name g_static_work is only a host-side stand-in, so the address has to be
// looked up once per device with that device current.  The cached address
// belongs to the device's context at the time of the lookup: after the caller
// resets the device (cudaDeviceReset) it is stale, which the header documents.
int static_work_address(void** out) {
    int dev = 0;
    LABFM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return labfm::set_error(LABFM_EINVAL, "device ordinal beyond the static scratch table");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_work);
        if (e != cudaSuccess) return labfm::cuda_error(e, "cudaGetSymbolAddress(static scratch)");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return LABFM_OK;
}

}  // namespace

extern "C" int labfm_rk_step_noalloc(const labfm_plan* p, void* Q, double dt, int nsteps,
                                     const labfm_phys* phys, void* stream) {
    LABFM_NVTX("labfm_rk_step_noalloc");
    if (!p || !p->row_ptr) return labfm::set_error(LABFM_EINVAL, "null or empty plan");
    if (!Q || !phys) return labfm::set_error(LABFM_EINVAL, "null pointer argument");
    if (nsteps < 0) return labfm::set_error(LABFM_EINVAL, "negative nsteps");
    if (nsteps > 0 && !(dt > 0.0) && !(dt == 0.0 && p->dt_node))
        return labfm::set_error(LABFM_EINVAL, "dt must be positive (or 0 with per-instance dt set)");
    const size_t need = labfm::rk_work_bytes(p);
    if (need > kStaticWorkBytes)
        return labfm::set_error(
            LABFM_ECAPACITY,
            "labfm_rk_step_noalloc: N = " + std::to_string(p->N) + " needs " +
                std::to_string(need) + " bytes of scratch but the static array holds " +
                std::to_string(kStaticWorkBytes) + " bytes (use labfm_rk_step with a work buffer)");
    int dev = 0;
    LABFM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != p->device)
        return labfm::set_error(LABFM_EINVAL, "labfm_rk_step_noalloc: the plan lives on device " +
                                                  std::to_string(p->device) + " but device " +
                                                  std::to_string(dev) + " is current");
    void* work = nullptr;
    if (int rc = static_work_address(&work)) return rc;
    return labfm::launch_rk_steps(p, Q, work, dt, nsteps, phys, labfm::as_stream(stream));
}
