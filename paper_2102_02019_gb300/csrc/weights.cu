// Batched FP64 weight build (Sections 2, 3 and 6 of the paper).
//
// One CTA per node.  The moment matrix M_i = sum_j X~_ji (x) W_ji (eq. disc_form)
// is assembled from weighted moments instead of neighbour by neighbour: every
// entry X~^r_ji W^c_ji is psi_j times a polynomial in (x/h, y/h), because
// W^c = psi He_a(x/h) He_b(y/h) with the probabilists' Hermite polynomials
// He_a(z) = 2^(-a/2) H_a(z / sqrt 2) (eq. hermite).  So
//   M[r][c] = 1/(a_r! b_r!) sum_{k,l} he_{a_c,k} he_{b_c,l} mu_{a_r+k, b_r+l},
//   mu_{p,q} = sum_j psi_j (x_ji/h)^p (y_ji/h)^q,  p + q <= 2m,
// which needs (2m+1)(2m+2)/2 moment sums per neighbour instead of n^2 products
// (153 vs 1936 at m = 8).  M_i, augmented with the six scaled selectors C~^d, is
// then reduced by Gaussian elimination with partial pivoting (the first row
// holding the largest |pivot| wins) and back substitution; finally every thread
// takes neighbours j and forms w^d_ji = W_ji . Psi^d and the filter sum F_0,i.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>

#include "labfm_internal.cuh"

namespace labfm {
namespace {

template <int M>
struct WCfg {
    static constexpr int n = (M * M + 3 * M) / 2;
    // threads per node: 32 / 64 / 96 / 128 / 192 for m = 2 / 4 / 6 / 8 / 10
    static constexpr int NT = M <= 2 ? 32 : (M <= 4 ? 64 : (M <= 6 ? 96 : (M <= 8 ? 128 : 192)));
    static constexpr int LDA = n + 6;                  // augmented row length
    static constexpr int NPOW = 2 * M + 1;                    // powers 0..2M
    static constexpr int NMOM = (2 * M + 1) * (2 * M + 2) / 2;  // moments p + q <= 2M
    static constexpr size_t chunk_bytes = size_t(2) * NT * NPOW * sizeof(double);
    static constexpr size_t lu_bytes(bool resid) {
        return (size_t(n) * LDA + (resid ? size_t(n) * n : 0)) * sizeof(double);
    }
    static constexpr size_t smem(bool resid) {
        return chunk_bytes > lu_bytes(resid) ? chunk_bytes : lu_bytes(resid);
    }
};

// (a, b) exponents of entry q of X (eq. X): degree 1..M, and within a degree
// descending powers of x.  Degree k starts at q = k (k + 1) / 2 - 1.
__device__ __forceinline__ void exps_of(int q, int& a, int& b) {
    int k = 1, start = 0;
    while (q >= start + k + 1) {
        start += k + 1;
        ++k;
    }
    b = q - start;
    a = k - b;
}

// psi(q) = (1 - q/2)^4 (1 + 2 q) on q <= 2 (Wendland C2, support 2h).
__device__ __forceinline__ double wendland_c2(double q) {
    const double t = 1.0 - 0.5 * q;
    const double t2 = t * t;
    return q <= 2.0 ? (t2 * t2) * (1.0 + 2.0 * q) : 0.0;
}

struct NodeGeom {
    double xi, yi, hi, Lx, Ly;
    bool px, py;
};

// Per-neighbour 1D factors: powers (x/h)^a, (y/h)^b and Hermite values
// H_a(x/(h sqrt2)), H_b(y/(h sqrt2)), plus psi.
template <int M>
__device__ __forceinline__ void neighbour_factors(const double* __restrict__ xy, int j,
                                                  const NodeGeom& g, double (&px)[M + 1],
                                                  double (&py)[M + 1], double (&hx)[M + 1],
                                                  double (&hy)[M + 1], double* psi, double* dxo,
                                                  double* dyo) {
    const double dx = min_image(__dsub_rn(xy[2 * j], g.xi), g.Lx, g.px);
    const double dy = min_image(__dsub_rn(xy[2 * j + 1], g.yi), g.Ly, g.py);
    *dxo = dx;
    *dyo = dy;
    const double xh = dx / g.hi;
    const double yh = dy / g.hi;
    *psi = wendland_c2(sqrt(dx * dx + dy * dy) / g.hi);
    const double hs2 = g.hi * 1.4142135623730951;  // h sqrt(2)
    const double zx = dx / hs2;
    const double zy = dy / hs2;
    px[0] = 1.0;
    py[0] = 1.0;
    hx[0] = 1.0;
    hy[0] = 1.0;
    if (M >= 1) {
        hx[1] = 2.0 * zx;
        hy[1] = 2.0 * zy;
    }
#pragma unroll
    for (int a = 1; a <= M; ++a) {
        px[a] = px[a - 1] * xh;
        py[a] = py[a - 1] * yh;
    }
#pragma unroll
    for (int k = 1; k < M; ++k) {
        hx[k + 1] = 2.0 * zx * hx[k] - 2.0 * k * hx[k - 1];
        hy[k + 1] = 2.0 * zy * hy[k] - 2.0 * k * hy[k - 1];
    }
}

// 1/k! and 1/sqrt(2^k) tables in constant memory (indexed at run time).
__constant__ double c_inv_fact[11] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0,
                                      1.0 / 720.0, 1.0 / 5040.0, 1.0 / 40320.0, 1.0 / 362880.0,
                                      1.0 / 3628800.0};
__constant__ double c_inv_sqrt2_pow[21] = {
    1.0, 0.70710678118654752440, 0.5, 0.35355339059327376220, 0.25, 0.17677669529663688110,
    0.125, 0.088388347648318440550, 0.0625, 0.044194173824159220275, 0.03125,
    0.022097086912079610138, 0.015625, 0.011048543456039805069, 0.0078125,
    0.0055242717280199025344, 0.00390625, 0.0027621358640099512672, 0.001953125,
    0.0013810679320049756336, 0.0009765625};

__device__ __forceinline__ double inv_factorial(int k) { return c_inv_fact[k]; }

// 1 / sqrt(2^k)
__device__ __forceinline__ double inv_sqrt2_pow(int k) { return c_inv_sqrt2_pow[k]; }

// Selector entry C~^d_q / h^-deg for op d at monomial (a, b) (Section 2 and,
// for d = 5, the expansion of (d_xx + d_yy)^{M/2} from Section 6).
template <int M>
__device__ __forceinline__ double selector_coef(int d, int a, int b) {
    switch (d) {
        case 0: return (a == 1 && b == 0) ? 1.0 : 0.0;
        case 1: return (a == 0 && b == 1) ? 1.0 : 0.0;
        case 2: return (a == 2 && b == 0) ? 1.0 : 0.0;
        case 3: return (a == 1 && b == 1) ? 1.0 : 0.0;
        case 4: return (a == 0 && b == 2) ? 1.0 : 0.0;
        default: {
            if (a + b != M || (a & 1)) return 0.0;
            // binom(M/2, a/2)
            const int nh = M / 2, k = a / 2;
            double c = 1.0;
            for (int t = 1; t <= k; ++t) c = c * double(nh - k + t) / double(t);
            return c;
        }
    }
}

__device__ __forceinline__ int op_order(int d, int M) { return d < 2 ? 1 : (d < 5 ? 2 : M); }

template <int M, bool RESID>
__global__ void __launch_bounds__(WCfg<M>::NT)
    k_weight_build(const double* __restrict__ xy, const double* __restrict__ h,
                   const double* __restrict__ s, int64_t N, double Lx, double Ly, int px_, int py_,
                   const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t nnz,
                   double* __restrict__ w, double* __restrict__ kappa, double* __restrict__ residual,
                   int32_t* __restrict__ node_status, unsigned long long* __restrict__ n_failed) {
    using C = WCfg<M>;
    constexpr int n = C::n;
    constexpr int NT = C::NT;
    constexpr int LDA = C::LDA;

    extern __shared__ double smem[];
    double* A = smem;              // [n][LDA], aliases the moment buffers after assembly
    double* A0 = smem + n * LDA;   // [n][n] copy of M for the residual
    __shared__ int s_piv;
    __shared__ int s_flags;
    __shared__ double s_red[NT / 32];

    const int64_t i = blockIdx.x;
    if (i >= N) return;
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int warp = t >> 5;
    NodeGeom g{xy[2 * i], xy[2 * i + 1], h[i], Lx, Ly, px_ != 0, py_ != 0};
    const int r0 = row_ptr[i];
    const int r1 = row_ptr[i + 1];
    const int nn = r1 - r0;
    if (t == 0) s_flags = 0;

    if (nn < n) {  // M_i singular: fewer stencil nodes than unknowns
        for (int e = r0 + t; e < r1; e += NT)
            for (int d = 0; d < 6; ++d) w[int64_t(d) * nnz + e] = 0.0;
        if (t == 0) {
            kappa[i] = 0.0;
            if (RESID) residual[i] = INFINITY;
            node_status[i] = LABFM_NODE_FEW_NEIGHBOURS;
            if (n_failed) atomicAdd(n_failed, 1ull);
        }
        return;
    }

    // ---- weighted moments mu_{p,q} = sum_j psi_j xh^p yh^q, p + q <= 2M
    constexpr int NPOW = C::NPOW;
    constexpr int NMOM = C::NMOM;
    constexpr int MPT = (NMOM + NT - 1) / NT;  // moments per thread
    double* XP = smem;              // [NT][NPOW]: psi xh^p
    double* YP = smem + NT * NPOW;  // [NT][NPOW]: yh^q
    __shared__ double s_mu[NMOM];
    __shared__ double s_he[(M + 1) * (M + 1)];  // he[a][k]: coefficient of z^k in He_a
    if (t == 0) {
        for (int k = 0; k < (M + 1) * (M + 1); ++k) s_he[k] = 0.0;
        s_he[0] = 1.0;
        if (M >= 1) s_he[(M + 1) + 1] = 1.0;
        for (int a = 1; a < M; ++a)  // He_{a+1} = z He_a - a He_{a-1}
            for (int k = 0; k <= a + 1; ++k) {
                const double up = k > 0 ? s_he[a * (M + 1) + k - 1] : 0.0;
                s_he[(a + 1) * (M + 1) + k] = up - double(a) * s_he[(a - 1) * (M + 1) + k];
            }
    }
    int mp[MPT], mq[MPT];
    double macc[MPT];
#pragma unroll
    for (int u = 0; u < MPT; ++u) {
        macc[u] = 0.0;
        const int idx = t + u * NT;
        int d = 0;
        while (idx >= (d + 1) * (d + 2) / 2 && d < 2 * M) ++d;
        mp[u] = d - (idx - d * (d + 1) / 2);
        mq[u] = d - mp[u];
    }
    for (int c0 = r0; c0 < r1; c0 += NT) {
        const int cnt = min(NT, r1 - c0);
        if (t < cnt) {
            const int j = col[c0 + t];
            const double dx = min_image(__dsub_rn(xy[2 * j], g.xi), g.Lx, g.px);
            const double dy = min_image(__dsub_rn(xy[2 * j + 1], g.yi), g.Ly, g.py);
            const double xh = dx / g.hi;
            const double yh = dy / g.hi;
            double xp = wendland_c2(sqrt(dx * dx + dy * dy) / g.hi), yp = 1.0;
            double* xr = XP + t * NPOW;
            double* yr = YP + t * NPOW;
#pragma unroll
            for (int p = 0; p < NPOW; ++p) {
                xr[p] = xp;
                yr[p] = yp;
                xp *= xh;
                yp *= yh;
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < MPT; ++u) {
            if (t + u * NT < NMOM) {
                double acc = macc[u];
                for (int k = 0; k < cnt; ++k) acc = fma(XP[k * NPOW + mp[u]], YP[k * NPOW + mq[u]], acc);
                macc[u] = acc;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < MPT; ++u)
        if (t + u * NT < NMOM) s_mu[t + u * NT] = macc[u];
    __syncthreads();

    // ---- M_i from the moments, into the augmented system [M | C~]
    for (int idx = t; idx < n * n; idx += NT) {
        const int r = idx / n, c = idx - r * n;
        int ar, br, ac, bc;
        exps_of(r, ar, br);
        exps_of(c, ac, bc);
        double sum = 0.0;
        for (int k = ac; k >= 0; k -= 2) {
            const double hk = s_he[ac * (M + 1) + k];
            for (int l = bc; l >= 0; l -= 2) {
                const int pp = ar + k, qq = br + l, dd = pp + qq;
                sum = fma(hk * s_he[bc * (M + 1) + l], s_mu[dd * (dd + 1) / 2 + (dd - pp)], sum);
            }
        }
        const double v = sum * (inv_factorial(ar) * inv_factorial(br));
        A[r * LDA + c] = v;
        if (RESID) A0[r * n + c] = v;
    }
    for (int idx = t; idx < n * 6; idx += NT) {
        const int q = idx / 6, d = idx - q * 6;
        int a, b;
        exps_of(q, a, b);
        const double coef = selector_coef<M>(d, a, b);
        A[q * LDA + n + d] = coef != 0.0 ? coef * pow(g.hi, -double(a + b)) : 0.0;
    }
    __syncthreads();

    // ---- Gaussian elimination with partial pivoting on [M | C~]
    for (int k = 0; k < n; ++k) {
        if (warp == 0) {
            double best = -1.0;
            int bidx = n;
            for (int r = k + lane; r < n; r += 32) {
                const double v = fabs(A[r * LDA + k]);
                if (v > best) {
                    best = v;
                    bidx = r;
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
                if (ob > best || (ob == best && oi < bidx)) {
                    best = ob;
                    bidx = oi;
                }
            }
            if (lane == 0) {
                s_piv = bidx;
                if (!(best > 0.0) || !isfinite(best) || bidx >= n) s_flags |= LABFM_NODE_SINGULAR;
            }
        }
        __syncthreads();
        if (s_flags & LABFM_NODE_SINGULAR) break;
        const int p = s_piv;
        if (p != k) {
            for (int c = t; c < LDA; c += NT) {
                const double tmp = A[k * LDA + c];
                A[k * LDA + c] = A[p * LDA + c];
                A[p * LDA + c] = tmp;
            }
            __syncthreads();
        }
        const double piv = A[k * LDA + k];
        for (int r = k + 1 + t; r < n; r += NT) A[r * LDA + k] = A[r * LDA + k] / piv;
        __syncthreads();
        const int rows = n - k - 1;
        const int cols = LDA - k - 1;
        for (int idx = t; idx < rows * cols; idx += NT) {
            const int r = k + 1 + idx / cols;
            const int c = k + 1 + idx % cols;
            A[r * LDA + c] -= A[r * LDA + k] * A[k * LDA + c];
        }
        __syncthreads();
    }

    const bool singular = (s_flags & LABFM_NODE_SINGULAR) != 0;
    // ---- back substitution (warp 0), Psi^d overwrites the C~ columns
    if (!singular && warp == 0) {
        for (int k = n - 1; k >= 0; --k) {
            const double dkk = A[k * LDA + k];
            double psi[6];
#pragma unroll
            for (int d = 0; d < 6; ++d) psi[d] = A[k * LDA + n + d] / dkk;
            __syncwarp();
            for (int r = lane; r < k; r += 32) {
                const double ark = A[r * LDA + k];
#pragma unroll
                for (int d = 0; d < 6; ++d) A[r * LDA + n + d] -= ark * psi[d];
            }
            if (lane == 0) {
#pragma unroll
                for (int d = 0; d < 6; ++d) A[k * LDA + n + d] = psi[d];
            }
            __syncwarp();
        }
    }
    __syncthreads();

    // ---- residual of eq. lsys in nondimensional form: (M Psi^d - C~^d)_q h^l
    if (RESID) {
        double rmax = singular ? INFINITY : 0.0;
        if (!singular) {
            for (int idx = t; idx < n * 6; idx += NT) {
                const int q = idx / 6, d = idx - q * 6;
                double sum = 0.0;
                for (int c = 0; c < n; ++c) sum = fma(A0[q * n + c], A[c * LDA + n + d], sum);
                int a, b;
                exps_of(q, a, b);
                const double coef = selector_coef<M>(d, a, b);
                const double cq = coef != 0.0 ? coef * pow(g.hi, -double(a + b)) : 0.0;
                const double r = fabs(sum - cq) * pow(g.hi, double(op_order(d, M)));
                rmax = (r > rmax || isnan(r)) ? r : rmax;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, off));
        if (lane == 0) s_red[warp] = rmax;
        __syncthreads();
        if (t == 0) {
            double r = s_red[0];
            for (int k = 1; k < NT / 32; ++k) r = fmax(r, s_red[k]);
            residual[i] = r;
        }
        __syncthreads();
    }

    // ---- weights w^d_j = W_j . Psi^d and the filter sum F_0
    const double kx = 3.0 * 3.141592653589793 / (2.0 * s[i]);
    double f0 = 0.0;
    bool bad = false;
    for (int e = r0 + t; e < r1; e += NT) {
        double wd[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        double dx = 0.0, dy = 0.0;
        if (!singular) {
            double pxv[M + 1], pyv[M + 1], hxv[M + 1], hyv[M + 1], psi;
            neighbour_factors<M>(xy, col[e], g, pxv, pyv, hxv, hyv, &psi, &dx, &dy);
            int q = 0;
#pragma unroll
            for (int k = 1; k <= M; ++k) {
#pragma unroll
                for (int a = k; a >= 0; --a, ++q) {
                    const double Wq = psi * hxv[a] * hyv[k - a] * inv_sqrt2_pow(k);
#pragma unroll
                    for (int d = 0; d < 6; ++d) wd[d] = fma(Wq, A[q * LDA + n + d], wd[d]);
                }
            }
        }
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            w[int64_t(d) * nnz + e] = wd[d];
            bad |= !isfinite(wd[d]);
        }
        const double phi = 1.0 - cos(kx * dx) * cos(kx * dy);
        f0 = fma(phi, wd[5], f0);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) f0 += __shfl_xor_sync(0xffffffffu, f0, off);
    const unsigned badw = __ballot_sync(0xffffffffu, bad);
    __syncthreads();
    if (lane == 0) {
        s_red[warp] = f0;
        if (badw) atomicOr(&s_flags, LABFM_NODE_NONFINITE);
    }
    __syncthreads();
    if (t == 0) {
        double F0 = 0.0;
        for (int k = 0; k < NT / 32; ++k) F0 += s_red[k];
        const double kap = singular ? 0.0 : 2.0 / (3.0 * F0);
        int flags = s_flags;
        if (!singular && !isfinite(kap)) flags |= LABFM_NODE_NONFINITE;
        kappa[i] = kap;
        node_status[i] = flags;
        if (flags && n_failed) atomicAdd(n_failed, 1ull);
    }
}

template <int M>
int launch_weights(const double* xy, const double* h, const double* s, int64_t N, double Lx,
                   double Ly, uint32_t pm, const int32_t* row_ptr, const int32_t* col, int64_t nnz,
                   double* w, double* kappa, double* residual, int32_t* status,
                   unsigned long long* n_failed, cudaStream_t st) {
    using C = WCfg<M>;
    const bool resid = residual != nullptr;
    const size_t sm = C::smem(resid);
    if (resid) {
        auto kern = k_weight_build<M, true>;
        LABFM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
        kern<<<unsigned(N), C::NT, sm, st>>>(xy, h, s, N, Lx, Ly, pm & 1u, (pm >> 1) & 1u, row_ptr,
                                             col, nnz, w, kappa, residual, status, n_failed);
    } else {
        auto kern = k_weight_build<M, false>;
        LABFM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
        kern<<<unsigned(N), C::NT, sm, st>>>(xy, h, s, N, Lx, Ly, pm & 1u, (pm >> 1) & 1u, row_ptr,
                                             col, nnz, w, kappa, residual, status, n_failed);
    }
    LABFM_LAUNCH_CHECK("weight build kernel");
    return LABFM_OK;
}

}  // namespace
}  // namespace labfm

using namespace labfm;

extern "C" int labfm_build_weights(const double* xy, const double* h, const double* s, int64_t N,
                                   double Lx, double Ly, uint32_t periodic_mask,
                                   const int32_t* row_ptr, const int32_t* col, int64_t nnz, int m,
                                   double* w, double* kappa, double* residual,
                                   int32_t* node_status, int64_t* n_failed_out, void* stream) {
    if (!xy || !h || !s || !row_ptr || !w || !kappa || !node_status)
        return set_error(LABFM_EINVAL, "null pointer argument");
    if (nnz > 0 && !col) return set_error(LABFM_EINVAL, "null col with nnz > 0");
    if (N <= 0 || N >= (int64_t(1) << 31) - 1) return set_error(LABFM_EINVAL, "N out of range");
    if (nnz < 0 || nnz >= (int64_t(1) << 31)) return set_error(LABFM_EINVAL, "nnz out of range");
    if (m < 2 || m > 10 || (m & 1))
        return set_error(LABFM_EINVAL, "order m must be even and in [2, 10], got " + std::to_string(m));
    if (!(Lx > 0.0) || !(Ly > 0.0)) return set_error(LABFM_EINVAL, "domain size must be positive");
    cudaStream_t st = as_stream(stream);
    unsigned long long* nf = nullptr;
    if (n_failed_out) {
        LABFM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&nf), sizeof(unsigned long long), st));
        LABFM_CUDA_TRY(cudaMemsetAsync(nf, 0, sizeof(unsigned long long), st));
    }
    int rc = LABFM_OK;
    switch (m) {
        case 2: rc = launch_weights<2>(xy, h, s, N, Lx, Ly, periodic_mask, row_ptr, col, nnz, w, kappa, residual, node_status, nf, st); break;
        case 4: rc = launch_weights<4>(xy, h, s, N, Lx, Ly, periodic_mask, row_ptr, col, nnz, w, kappa, residual, node_status, nf, st); break;
        case 6: rc = launch_weights<6>(xy, h, s, N, Lx, Ly, periodic_mask, row_ptr, col, nnz, w, kappa, residual, node_status, nf, st); break;
        case 8: rc = launch_weights<8>(xy, h, s, N, Lx, Ly, periodic_mask, row_ptr, col, nnz, w, kappa, residual, node_status, nf, st); break;
        case 10: rc = launch_weights<10>(xy, h, s, N, Lx, Ly, periodic_mask, row_ptr, col, nnz, w, kappa, residual, node_status, nf, st); break;
    }
    if (n_failed_out) {
        unsigned long long hf = 0;
        if (rc == LABFM_OK) {
            cudaError_t e = cudaMemcpyAsync(&hf, nf, sizeof(hf), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = cuda_error(e, "reading the failed-node count");
        }
        cudaFreeAsync(nf, st);
        if (rc != LABFM_OK) return rc;
        *n_failed_out = int64_t(hf);
        if (hf > 0)
            return set_error(LABFM_ESINGULAR, std::to_string(hf) + " node(s) failed; see node_status");
    }
    return rc;
}
