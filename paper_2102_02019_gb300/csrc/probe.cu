// Arithmetic-rate probe: the denominator of the FP64-pipe roofline of the FP64
// kernels (weight build, FP64 right-hand side).  Not part of the paper's method.
#include <cuda_runtime.h>
#include <stdint.h>

#include "labfm_internal.cuh"

namespace labfm {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

// Every thread runs kChains independent fused multiply-add chains of kIters
// steps; the result is stored so that the work cannot be removed.
template <typename T>
__global__ void k_fma_rate(T* out, T a, T b) {
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = T(threadIdx.x + c);
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int time_rate(int sms, double* gflops) {
    const int block = 256, grid = sms * 8;
    T* out = nullptr;
    LABFM_CUDA_TRY(cudaMalloc(&out, size_t(grid) * block * sizeof(T)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_rate<T><<<grid, block>>>(out, T(0.999999), T(1e-7));  // warm-up
    cudaEventRecord(e0);
    const int reps = 3;
    for (int r = 0; r < reps; ++r) k_fma_rate<T><<<grid, block>>>(out, T(0.999999), T(1e-7));
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return cuda_error(e, "rate probe");
    const double flops = 2.0 * double(grid) * block * kChains * kIters * reps;
    *gflops = flops / (double(ms) * 1e-3) / 1e9;
    return LABFM_OK;
}

}  // namespace
}  // namespace labfm

using namespace labfm;

extern "C" int labfm_probe_fma_rate(int dtype, double* gflops_out) {
    if (!gflops_out) return set_error(LABFM_EINVAL, "null output");
    int dev = 0, sms = 0;
    LABFM_CUDA_TRY(cudaGetDevice(&dev));
    LABFM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (dtype == LABFM_F64) return time_rate<double>(sms, gflops_out);
    if (dtype == LABFM_F32) return time_rate<float>(sms, gflops_out);
    return set_error(LABFM_EINVAL, "unknown dtype");
}
