// Pointwise maps and the objectives used with the adjoint: conserved variables
// (rho, rho u, rho v) <-> evolved variables (ln rho, u, v) (Section 7 evolves
// the latter), the domain kinetic energy sum_i 1/2 rho_i |u_i|^2 V_i with node
// volume V_i = s_i^2, and the probe-weighted momentum sum_i rho_i (px_i u_i +
// py_i v_i), with their vector-Jacobian products.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "labfm_internal.cuh"

namespace labfm {
namespace {

template <typename T>
__global__ void k_to_primitive(int64_t N, const T* __restrict__ c, T* __restrict__ q) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N;
         i += int64_t(gridDim.x) * blockDim.x) {
        const T rho = c[i];
        q[i] = log(rho);
        q[N + i] = c[N + i] / rho;
        q[2 * N + i] = c[2 * N + i] / rho;
    }
}

// cbar = (d primitive / d conserved)^T qbar
template <typename T>
__global__ void k_conserved_vjp(int64_t N, const T* __restrict__ c, const T* __restrict__ qb,
                                T* __restrict__ cb) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N;
         i += int64_t(gridDim.x) * blockDim.x) {
        const T rho = c[i], mx = c[N + i], my = c[2 * N + i];
        const T ab = qb[i], ub = qb[N + i], vb = qb[2 * N + i];
        const T ir = T(1) / rho;
        cb[i] = ab * ir - (ub * mx + vb * my) * ir * ir;
        cb[N + i] = ub * ir;
        cb[2 * N + i] = vb * ir;
    }
}

// One block, fixed summation order: the same result on every call.
template <typename T>
__global__ void k_kinetic_energy(int64_t N, const T* __restrict__ q, const double* __restrict__ s,
                                 double* __restrict__ out) {
    __shared__ double red[1024];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double rho = exp(double(q[i])), u = double(q[N + i]), v = double(q[2 * N + i]);
        acc += 0.5 * rho * (u * u + v * v) * s[i] * s[i];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

template <typename T>
__global__ void k_kinetic_energy_grad(int64_t N, const T* __restrict__ q, const double* __restrict__ s,
                                      double scale, T* __restrict__ g) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N;
         i += int64_t(gridDim.x) * blockDim.x) {
        const double rho = exp(double(q[i])), u = double(q[N + i]), v = double(q[2 * N + i]);
        const double V = s[i] * s[i] * scale;
        g[i] = T(0.5 * rho * (u * u + v * v) * V);
        g[N + i] = T(rho * u * V);
        g[2 * N + i] = T(rho * v * V);
    }
}

// One block, fixed summation order (as the kinetic energy).
template <typename T>
__global__ void k_probe_momentum(int64_t N, const T* __restrict__ q, const double* __restrict__ px,
                                 const double* __restrict__ py, double* __restrict__ out) {
    __shared__ double red[1024];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double rho = exp(double(q[i]));
        acc += rho * (px[i] * double(q[N + i]) + py[i] * double(q[2 * N + i]));
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

template <typename T>
__global__ void k_probe_momentum_grad(int64_t N, const T* __restrict__ q, const double* __restrict__ px,
                                      const double* __restrict__ py, double scale, T* __restrict__ g) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N;
         i += int64_t(gridDim.x) * blockDim.x) {
        const double rs = exp(double(q[i])) * scale;
        g[i] = T(rs * (px[i] * double(q[N + i]) + py[i] * double(q[2 * N + i])));
        g[N + i] = T(rs * px[i]);
        g[2 * N + i] = T(rs * py[i]);
    }
}

int grid_of(int64_t N) { return int(std::min<int64_t>((N + 255) / 256, 65535)); }

int check_n(int64_t N, int dtype) {
    if (N <= 0) return set_error(LABFM_EINVAL, "N must be positive");
    if (dtype != LABFM_F32 && dtype != LABFM_F64) return set_error(LABFM_EINVAL, "unknown dtype");
    return LABFM_OK;
}

}  // namespace
}  // namespace labfm

using namespace labfm;

extern "C" int labfm_conserved_to_primitive(const void* c, void* q, int64_t N, labfm_dtype dtype,
                                            void* stream) {
    if (int rc = check_n(N, dtype)) return rc;
    if (!c || !q) return set_error(LABFM_EINVAL, "null pointer argument");
    cudaStream_t st = as_stream(stream);
    if (dtype == LABFM_F32)
        k_to_primitive<float><<<grid_of(N), 256, 0, st>>>(N, static_cast<const float*>(c), static_cast<float*>(q));
    else
        k_to_primitive<double><<<grid_of(N), 256, 0, st>>>(N, static_cast<const double*>(c), static_cast<double*>(q));
    LABFM_LAUNCH_CHECK("conversion kernel");
    return LABFM_OK;
}

extern "C" int labfm_conserved_vjp(const void* c, const void* qbar, void* cbar, int64_t N,
                                   labfm_dtype dtype, void* stream) {
    if (int rc = check_n(N, dtype)) return rc;
    if (!c || !qbar || !cbar) return set_error(LABFM_EINVAL, "null pointer argument");
    cudaStream_t st = as_stream(stream);
    if (dtype == LABFM_F32)
        k_conserved_vjp<float><<<grid_of(N), 256, 0, st>>>(N, static_cast<const float*>(c),
                                                           static_cast<const float*>(qbar), static_cast<float*>(cbar));
    else
        k_conserved_vjp<double><<<grid_of(N), 256, 0, st>>>(N, static_cast<const double*>(c),
                                                            static_cast<const double*>(qbar), static_cast<double*>(cbar));
    LABFM_LAUNCH_CHECK("conversion adjoint kernel");
    return LABFM_OK;
}

extern "C" int labfm_kinetic_energy(const void* q, const double* s, int64_t N, labfm_dtype dtype,
                                    double* ke_out, void* stream) {
    if (int rc = check_n(N, dtype)) return rc;
    if (!q || !s || !ke_out) return set_error(LABFM_EINVAL, "null pointer argument");
    cudaStream_t st = as_stream(stream);
    if (dtype == LABFM_F32)
        k_kinetic_energy<float><<<1, 1024, 0, st>>>(N, static_cast<const float*>(q), s, ke_out);
    else
        k_kinetic_energy<double><<<1, 1024, 0, st>>>(N, static_cast<const double*>(q), s, ke_out);
    LABFM_LAUNCH_CHECK("kinetic energy kernel");
    return LABFM_OK;
}

extern "C" int labfm_kinetic_energy_grad(const void* q, const double* s, int64_t N,
                                         labfm_dtype dtype, double scale, void* grad_out,
                                         void* stream) {
    if (int rc = check_n(N, dtype)) return rc;
    if (!q || !s || !grad_out) return set_error(LABFM_EINVAL, "null pointer argument");
    cudaStream_t st = as_stream(stream);
    if (dtype == LABFM_F32)
        k_kinetic_energy_grad<float><<<grid_of(N), 256, 0, st>>>(N, static_cast<const float*>(q), s, scale,
                                                                 static_cast<float*>(grad_out));
    else
        k_kinetic_energy_grad<double><<<grid_of(N), 256, 0, st>>>(N, static_cast<const double*>(q), s, scale,
                                                                  static_cast<double*>(grad_out));
    LABFM_LAUNCH_CHECK("kinetic energy gradient kernel");
    return LABFM_OK;
}

extern "C" int labfm_probe_momentum(const void* q, const double* px, const double* py, int64_t N,
                                    labfm_dtype dtype, double* j_out, void* stream) {
    if (int rc = check_n(N, dtype)) return rc;
    if (!q || !px || !py || !j_out) return set_error(LABFM_EINVAL, "null pointer argument");
    cudaStream_t st = as_stream(stream);
    if (dtype == LABFM_F32)
        k_probe_momentum<float><<<1, 1024, 0, st>>>(N, static_cast<const float*>(q), px, py, j_out);
    else
        k_probe_momentum<double><<<1, 1024, 0, st>>>(N, static_cast<const double*>(q), px, py, j_out);
    LABFM_LAUNCH_CHECK("probe momentum kernel");
    return LABFM_OK;
}

extern "C" int labfm_probe_momentum_grad(const void* q, const double* px, const double* py, int64_t N,
                                         labfm_dtype dtype, double scale, void* grad_out, void* stream) {
    if (int rc = check_n(N, dtype)) return rc;
    if (!q || !px || !py || !grad_out) return set_error(LABFM_EINVAL, "null pointer argument");
    cudaStream_t st = as_stream(stream);
    if (dtype == LABFM_F32)
        k_probe_momentum_grad<float><<<grid_of(N), 256, 0, st>>>(N, static_cast<const float*>(q), px, py,
                                                                 scale, static_cast<float*>(grad_out));
    else
        k_probe_momentum_grad<double><<<grid_of(N), 256, 0, st>>>(N, static_cast<const double*>(q), px, py,
                                                                  scale, static_cast<double*>(grad_out));
    LABFM_LAUNCH_CHECK("probe momentum gradient kernel");
    return LABFM_OK;
}
