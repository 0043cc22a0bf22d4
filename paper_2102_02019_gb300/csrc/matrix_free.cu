// Matrix-free right-hand side of eq. icns (the alternative the paper's
// conclusions point to for Lagrangian node sets, where the weights would change
// every step): instead of streaming the nnz x 5 stored weights, each node keeps
// the polynomial coefficients of its weight functions, which the weight build
// writes with labfm_build_weights_ex.  With W = psi He_a(x/h) He_b(y/h) (eq.
// hermite) the weight of operator d is w^d_ji = psi(|r_ji|/h_i) P^d(x_ji/h_i,
// y_ji/h_i) for a polynomial P^d of degree m, so every neighbour's five RHS
// weights are recomputed by Horner's rule from (m+1)(m+2)/2 coefficients per
// operator, with the same operations, in the same order, as the weight build.
//
// Work per stencil entry: five Horner evaluations of (m+1)(m+2)/2 fused
// multiply-adds each, the offsets, |r| and psi; the FP64 pipe bounds it.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "gather.cuh"
#include "labfm_internal.cuh"
#include "nvtx.cuh"

namespace labfm {
namespace {

// Wendland C2 with support 2h, in the weight build's operation order.
__device__ __forceinline__ double psi_c2(double q) {
    const double t = 1.0 - 0.5 * q;
    const double t2 = t * t;
    return q <= 2.0 ? (t2 * t2) * (1.0 + 2.0 * q) : 0.0;
}

constexpr int kMfWarps = 4;  // nodes per block: one warp per node

// coef: [N][NC][6] (monomial (p, q) major, operator minor, as the weight build
// keeps them); fields and out: 3 x N structure-of-arrays, FP64.
template <int M>
__global__ void __launch_bounds__(32 * kMfWarps)
    k_rhs_matrix_free(const double* __restrict__ xy, const double* __restrict__ h, int64_t N, double Lx,
                      double Ly, int px, int py, const int32_t* __restrict__ row_ptr,
                      const int32_t* __restrict__ col, const double* __restrict__ coef,
                      const double* __restrict__ f, double* __restrict__ out, Phys<double> ph) {
    constexpr int NC = (M + 1) * (M + 2) / 2;
    __shared__ double s_cf[kMfWarps][NC * 6];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = int64_t(blockIdx.x) * kMfWarps + warp;
    if (i >= N) return;  // uniform per warp
    double* cf = s_cf[warp];
    for (int idx = lane; idx < NC * 6; idx += 32) cf[idx] = coef[i * (NC * 6) + idx];
    __syncwarp();
    const double xi = xy[2 * i], yi = xy[2 * i + 1], ih = 1.0 / h[i];
    const double ai = f[i], ui = f[N + i], vi = f[2 * N + i];
    double d[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) d[k] = 0.0;
    const int r0 = row_ptr[i], r1 = row_ptr[i + 1];
    for (int e = r0 + lane; e < r1; e += 32) {
        const int j = col[e];
        const double dx = min_image(__dsub_rn(xy[2 * j], xi), Lx, px != 0);
        const double dy = min_image(__dsub_rn(xy[2 * j + 1], yi), Ly, py != 0);
        const double xh = dx * ih, yh = dy * ih;
        const double psi = psi_c2(sqrt(dx * dx + dy * dy) * ih);
        double wd[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll 1
        for (int p = M; p >= 0; --p) {
            const double* cp = cf + (p * (2 * M + 3 - p) / 2) * 6;  // (p, 0)
            double in[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) in[k] = cp[(M - p) * 6 + k];
#pragma unroll 1
            for (int qq = M - p - 1; qq >= 0; --qq)
#pragma unroll
                for (int k = 0; k < 5; ++k) in[k] = fma(in[k], yh, cp[qq * 6 + k]);
#pragma unroll
            for (int k = 0; k < 5; ++k) wd[k] = fma(wd[k], xh, in[k]);
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) wd[k] *= psi;
        const double da = f[j] - ai, du = f[N + j] - ui, dv = f[2 * N + j] - vi;
        d[0] = fma(wd[0], da, d[0]);
        d[1] = fma(wd[1], da, d[1]);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            d[2 + k] = fma(wd[k], du, d[2 + k]);
            d[7 + k] = fma(wd[k], dv, d[7 + k]);
        }
    }
#pragma unroll
    for (int k = 0; k < 12; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) d[k] += __shfl_xor_sync(0xffffffffu, d[k], off);
    if (lane == 0) {
        double Ra, Ru, Rv;
        pointwise_rhs<double, false>(d, ai, ui, vi, 1.0, ph.c2, ph.mu, ph.gx, ph.gy, Ra, Ru, Rv);
        out[i] = Ra;
        out[N + i] = Ru;
        out[2 * N + i] = Rv;
    }
}

template <int M>
int launch_matrix_free(const double* xy, const double* h, int64_t N, double Lx, double Ly, uint32_t pm,
                       const int32_t* row_ptr, const int32_t* col, const double* coef, const double* f,
                       double* out, const Phys<double>& ph, cudaStream_t st) {
    const int64_t blocks = (N + kMfWarps - 1) / kMfWarps;
    k_rhs_matrix_free<M><<<unsigned(blocks), 32 * kMfWarps, 0, st>>>(
        xy, h, N, Lx, Ly, int(pm & 1u), int((pm >> 1) & 1u), row_ptr, col, coef, f, out, ph);
    LABFM_LAUNCH_CHECK("matrix-free right-hand side kernel");
    return LABFM_OK;
}

}  // namespace
}  // namespace labfm

using namespace labfm;

extern "C" size_t labfm_weight_coefficients_per_node(int m) {
    if (m < 2 || m > 10 || (m & 1)) return 0;
    return size_t(6) * size_t((m + 1) * (m + 2) / 2);
}

extern "C" int labfm_rhs_matrix_free(const double* xy, const double* h, int64_t N, double Lx, double Ly,
                                     uint32_t periodic_mask, const int32_t* row_ptr, const int32_t* col,
                                     int m, const double* coef, const double* fields, double* rhs,
                                     const labfm_phys* phys, void* stream) {
    LABFM_NVTX("labfm_rhs_matrix_free");
    if (!xy || !h || !row_ptr || !coef || !fields || !rhs || !phys)
        return set_error(LABFM_EINVAL, "null pointer argument");
    if (N <= 0 || N >= (int64_t(1) << 31) - 1) return set_error(LABFM_EINVAL, "N out of range");
    if (m < 2 || m > 10 || (m & 1)) return set_error(LABFM_EINVAL, "order m must be even and in [2, 10]");
    if (!(Lx > 0.0) || !(Ly > 0.0)) return set_error(LABFM_EINVAL, "domain size must be positive");
    if (rhs == fields) return set_error(LABFM_EINVAL, "rhs must not alias fields");
    cudaStream_t st = as_stream(stream);
    if (int rc = validate_csr(row_ptr, col, N, -1, st)) return rc;
    const Phys<double> ph{phys->c2, phys->mu, phys->gx, phys->gy};
    switch (m) {
        case 2: return launch_matrix_free<2>(xy, h, N, Lx, Ly, periodic_mask, row_ptr, col, coef, fields, rhs, ph, st);
        case 4: return launch_matrix_free<4>(xy, h, N, Lx, Ly, periodic_mask, row_ptr, col, coef, fields, rhs, ph, st);
        case 6: return launch_matrix_free<6>(xy, h, N, Lx, Ly, periodic_mask, row_ptr, col, coef, fields, rhs, ph, st);
        case 8: return launch_matrix_free<8>(xy, h, N, Lx, Ly, periodic_mask, row_ptr, col, coef, fields, rhs, ph, st);
        default: return launch_matrix_free<10>(xy, h, N, Lx, Ly, periodic_mask, row_ptr, col, coef, fields, rhs, ph, st);
    }
}
