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

#include <algorithm>
#include <string>

#include "labfm_internal.cuh"
#include "nvtx.cuh"

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
    // neighbours per round of the moment accumulation: the x and y power tables of
    // a round (2 MCH NPOW doubles) share shared memory with the LU matrix, and
    // rounds of 64 keep them no larger than it, so that more CTAs fit on an SM
    static constexpr int MCH = NT < 64 ? NT : 64;
    static constexpr size_t chunk_bytes = size_t(2) * MCH * NPOW * sizeof(double);
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
    double ih;  // 1 / hi
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
    const double xh = dx * g.ih;
    const double yh = dy * g.ih;
    *psi = wendland_c2(sqrt(dx * dx + dy * dy) * g.ih);
    const double ihs2 = g.ih * 0.70710678118654752440;  // 1 / (h sqrt 2)
    const double zx = dx * ihs2;
    const double zy = dy * ihs2;
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

// 1/k! in constant memory (indexed at run time).
__constant__ double c_inv_fact[11] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0,
                                      1.0 / 720.0, 1.0 / 5040.0, 1.0 / 40320.0, 1.0 / 362880.0,
                                      1.0 / 3628800.0};

__device__ __forceinline__ double inv_factorial(int k) { return c_inv_fact[k]; }

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

// ---------------------------------------------------------------- block-level building blocks
// (one CTA of NT threads per node; every function is called by all threads)

// he[a][k]: coefficient of z^k in the probabilists' Hermite polynomial He_a
// (He_0 = 1, He_1 = z, He_{a+1} = z He_a - a He_{a-1}); integers, exact in FP64.
template <int M>
__device__ void build_he(double* s_he) {
    if (threadIdx.x == 0) {
        for (int k = 0; k < (M + 1) * (M + 1); ++k) s_he[k] = 0.0;
        s_he[0] = 1.0;
        if (M >= 1) s_he[(M + 1) + 1] = 1.0;
        for (int a = 1; a < M; ++a)
            for (int k = 0; k <= a + 1; ++k) {
                const double up = k > 0 ? s_he[a * (M + 1) + k - 1] : 0.0;
                s_he[(a + 1) * (M + 1) + k] = up - double(a) * s_he[(a - 1) * (M + 1) + k];
            }
    }
}

// Weighted moments mu_{p,q} = sum_j psi_j (x_ji/h)^p (y_ji/h)^q, p + q <= 2M, over
// the candidate neighbours col[r0 .. r1) with stencil scale g.hi (candidates
// beyond 2h have psi = 0 and add nothing), in rounds of MCH neighbours.  XP, YP:
// 2 MCH (2M+1) doubles of scratch; s_mu: (2M+1)(2M+2)/2 doubles.  Ends with a
// barrier.
template <int M>
__device__ void block_moments(const double* __restrict__ xy, const int32_t* __restrict__ col, int r0,
                              int r1, const NodeGeom& g, double* XP, double* YP, double* s_mu) {
    using C = WCfg<M>;
    constexpr int NT = C::NT, NPOW = C::NPOW, NMOM = C::NMOM, MCH = C::MCH;
    constexpr int MPT = (NMOM + NT - 1) / NT;  // moments per thread
    const int t = threadIdx.x;
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
    for (int c0 = r0; c0 < r1; c0 += MCH) {
        const int cnt = min(MCH, r1 - c0);
        if (t < cnt) {
            const int j = col[c0 + t];
            const double dx = min_image(__dsub_rn(xy[2 * j], g.xi), g.Lx, g.px);
            const double dy = min_image(__dsub_rn(xy[2 * j + 1], g.yi), g.Ly, g.py);
            const double xh = dx * g.ih;
            const double yh = dy * g.ih;
            double xp = wendland_c2(sqrt(dx * dx + dy * dy) * g.ih), yp = 1.0;
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
}

// M_i[r][c] = 1/(a_r! b_r!) sum_{k,l} he_{a_c,k} he_{b_c,l} mu_{a_r+k, b_r+l} into
// A (row stride LDA) and, when A0 is not null, a copy with stride n.  No barrier.
template <int M, int LDA>
__device__ void block_assemble(double* A, double* A0, const double* s_mu, const double* s_he) {
    using C = WCfg<M>;
    constexpr int n = C::n, NT = C::NT;
    // column-major over the threads: the lanes of a warp share the column c, whose
    // Hermite exponents fix the trip counts of the loops below (no divergence)
    for (int idx = threadIdx.x; idx < n * n; idx += NT) {
        const int c = idx / n, r = idx - c * n;
        int ar, br, ac, bc;
        exps_of(r, ar, br);
        exps_of(c, ac, bc);
        double sum = 0.0;
        for (int k = ac; k >= 0; k -= 2) {
            const int pp = ar + k;
            double inner = 0.0;  // sum_l he_{b_c,l} mu_{a_r+k, b_r+l}
            for (int l = bc; l >= 0; l -= 2) {
                const int dd = pp + br + l;
                inner = fma(s_he[bc * (M + 1) + l], s_mu[dd * (dd + 1) / 2 + (dd - pp)], inner);
            }
            sum = fma(s_he[ac * (M + 1) + k], inner, sum);
        }
        const double v = sum * (inv_factorial(ar) * inv_factorial(br));
        A[r * LDA + c] = v;
        if (A0) A0[r * n + c] = v;
    }
}

// Pivot-search key of |v|: for non-negative doubles the IEEE bit patterns order
// like the values, so the search compares 64-bit integers (off the FP64 pipe).
// NaN maps to -1 and is never chosen, as with a floating-point compare.
__device__ __forceinline__ long long abs_key(double v) {
    const long long b = __double_as_longlong(v) & 0x7fffffffffffffffll;
    return b > 0x7ff0000000000000ll ? -1ll : b;
}

// a / d from y = 1/d (correctly rounded) by Markstein's correction (P. Markstein,
// IBM J. Res. Develop. 34 (1990)): q0 = a y is within an ulp of a / d, the
// remainder a - q0 d is exact in one fused multiply-add, and q0 + (a - q0 d) y
// rounds to the correctly rounded quotient, barring underflow and overflow.
// Three FP64 instructions per quotient once y is known.
__device__ __forceinline__ double div_by_recip(double a, double d, double y) {
    const double q0 = a * y;
    return fma(fma(-q0, d, a), y, q0);
}

// Gaussian elimination with partial pivoting (the first row holding the largest
// |pivot| wins) on the augmented system [M | B] (n x LDA, NRHS = LDA - n right-hand
// sides), then back substitution by warp 0: the solutions overwrite B.  Each
// pivot's reciprocal is taken once during the elimination (lane 0 of warp 0, kept
// in s_rdiag[n]); the multipliers a_rk / a_kk are formed from it by Markstein's
// correction (the exact quotients), and the back substitution multiplies by it.
// Returns true (uniformly) if a pivot was zero or not finite.  Starts and ends
// with a barrier.
template <int M, int LDA>
__device__ bool block_lu_solve(double* A, int* s_piv, int* s_flag, double* s_rdiag) {
    using C = WCfg<M>;
    constexpr int n = C::n, NT = C::NT, NRHS = LDA - n;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) *s_flag = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (warp == 0) {
            long long best = -1;
            int bidx = n;
            for (int r = k + lane; r < n; r += 32) {
                const long long v = abs_key(A[r * LDA + k]);
                if (v > best) {
                    best = v;
                    bidx = r;
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const long long ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
                if (ob > best || (ob == best && oi < bidx)) {
                    best = ob;
                    bidx = oi;
                }
            }
            if (lane == 0) {
                *s_piv = bidx;
                // zero, NaN-only or infinite pivot column: singular
                if (best <= 0 || best >= 0x7ff0000000000000ll || bidx >= n) {
                    *s_flag = 1;
                } else {
                    s_rdiag[k] = 1.0 / A[bidx * LDA + k];
                }
            }
        }
        __syncthreads();
        if (*s_flag) break;
        const int p = *s_piv;
        if (p != k) {
            for (int c = t; c < LDA; c += NT) {
                const double tmp = A[k * LDA + c];
                A[k * LDA + c] = A[p * LDA + c];
                A[p * LDA + c] = tmp;
            }
            __syncthreads();
        }
        const double piv = A[k * LDA + k], rp = s_rdiag[k];
        for (int r = k + 1 + t; r < n; r += NT) A[r * LDA + k] = div_by_recip(A[r * LDA + k], piv, rp);
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
    const bool singular = *s_flag != 0;
    static_assert(NRHS <= 32, "one lane per right-hand side");
    if (!singular && warp == 0) {
        for (int k = n - 1; k >= 0; --k) {
            // lane d finishes unknown k of right-hand side d, then the lanes take the
            // (row, right-hand side) pairs of rows 0 .. k-1
            if (lane < NRHS) A[k * LDA + n + lane] *= s_rdiag[k];
            __syncwarp();
            for (int idx = lane; idx < k * NRHS; idx += 32) {
                const int r = idx / NRHS, d = idx - r * NRHS;
                A[r * LDA + n + d] -= A[r * LDA + k] * A[k * LDA + n + d];
            }
            __syncwarp();
        }
    }
    __syncthreads();
    return singular;
}

// Block-wide sum (all threads get the result).  s_red: NT / 32 doubles.
template <int NT>
__device__ double block_sum(double v, double* s_red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    double tot = 0.0;
    for (int k = 0; k < NT / 32; ++k) tot += s_red[k];
    return tot;
}

// ---------------------------------------------------------------- weight build

template <int M, bool RESID>
__global__ void __launch_bounds__(WCfg<M>::NT)
    k_weight_build(const double* __restrict__ xy, const double* __restrict__ h,
                   const double* __restrict__ s, int64_t N, double Lx, double Ly, int px_, int py_,
                   const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t nnz,
                   double* __restrict__ w, double* __restrict__ kappa, double* __restrict__ residual,
                   int32_t* __restrict__ node_status, unsigned long long* __restrict__ n_failed,
                   double* __restrict__ coef) {
    using C = WCfg<M>;
    constexpr int n = C::n;
    constexpr int NT = C::NT;
    constexpr int LDA = C::LDA;
    constexpr int NC = (M + 1) * (M + 2) / 2;
    extern __shared__ double smem[];
    double* A = smem;              // [n][LDA], aliases the moment scratch after assembly
    double* A0 = smem + n * LDA;   // [n][n] copy of M for the residual
    __shared__ double s_mu[C::NMOM];
    __shared__ double s_he[(M + 1) * (M + 1)];
    __shared__ int s_piv;
    __shared__ int s_flag;
    __shared__ int s_nonfinite;
    __shared__ double s_red[NT / 32];
    __shared__ double s_rdiag[n];
    __shared__ double s_hp[2 * M + 1];  // h^k, k = -M..M, at [k + M]

    const int64_t i = blockIdx.x;
    if (i >= N) return;
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int warp = t >> 5;
    NodeGeom g{xy[2 * i], xy[2 * i + 1], h[i], Lx, Ly, px_ != 0, py_ != 0, 1.0 / h[i]};
    const int r0 = row_ptr[i];
    const int r1 = row_ptr[i + 1];
    if (r1 - r0 < n) {  // M_i singular: fewer stencil nodes than unknowns
        if (w)
            for (int e = r0 + t; e < r1; e += NT)
                for (int d = 0; d < 6; ++d) w[int64_t(d) * nnz + e] = 0.0;
        if (coef)
            for (int idx = t; idx < NC * 6; idx += NT) coef[i * (NC * 6) + idx] = 0.0;
        if (t == 0) {
            kappa[i] = 0.0;
            if (RESID) residual[i] = INFINITY;
            node_status[i] = LABFM_NODE_FEW_NEIGHBOURS;
            if (n_failed) atomicAdd(n_failed, 1ull);
        }
        return;
    }
    if (t == 0) s_nonfinite = 0;
    if (t <= 2 * M) s_hp[t] = pow(g.hi, double(t - M));
    build_he<M>(s_he);
    block_moments<M>(xy, col, r0, r1, g, smem, smem + C::MCH * C::NPOW, s_mu);
    block_assemble<M, LDA>(A, RESID ? A0 : nullptr, s_mu, s_he);
    for (int idx = t; idx < n * 6; idx += NT) {  // selectors C~^d
        const int q = idx / 6, d = idx - q * 6;
        int a, b;
        exps_of(q, a, b);
        A[q * LDA + n + d] = selector_coef<M>(d, a, b) * s_hp[M - (a + b)];
    }
    const bool singular = block_lu_solve<M, LDA>(A, &s_piv, &s_flag, s_rdiag);

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
                const double cq = selector_coef<M>(d, a, b) * s_hp[M - (a + b)];
                const double r = fabs(sum - cq) * s_hp[M + op_order(d, M)];
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

    // ---- weights w^d_j = W_j . Psi^d and the filter sum F_0.  With W = psi He_a(x/h)
    // He_b(y/h), W_j . Psi^d = psi_j P^d(x/h, y/h) for the polynomial
    // P^d = sum_{a,b} Psi^d_ab He_a He_b = sum_{p+q<=M} c^d_pq x^p y^q, whose
    // coefficients follow from the Hermite expansions once per node; each
    // neighbour then takes P^d by Horner's rule (x outer, y inner).
    __shared__ double s_cf[NC * 6];
    if (!singular) {
        for (int idx = t; idx < NC * 6; idx += NT) {
            const int pq = idx / 6, d = idx - pq * 6;
            int p = 0;
            while (pq >= (p + 1) * (2 * M + 2 - p) / 2) ++p;
            const int qy = pq - p * (2 * M + 3 - p) / 2;
            double c = 0.0;
            for (int a = p; a <= M; a += 2) {
                const double ha = s_he[a * (M + 1) + p];
                for (int b = qy; a + b <= M; b += 2) {
                    const int k = a + b;
                    if (k == 0) continue;  // X has no constant monomial
                    const int q = k * (k + 1) / 2 - 1 + b;
                    c = fma(ha * s_he[b * (M + 1) + qy], A[q * LDA + n + d], c);
                }
            }
            s_cf[idx] = c;
        }
    }
    __syncthreads();
    if (coef)  // the polynomial coefficients, for the matrix-free right-hand side
        for (int idx = t; idx < NC * 6; idx += NT) coef[i * (NC * 6) + idx] = singular ? 0.0 : s_cf[idx];
    const double kx = 3.0 * 3.141592653589793 / (2.0 * s[i]);
    double f0 = 0.0;
    bool bad = false;
    // Neighbours go one per lane with all six operators.  When the last warp would
    // hold only a few (rem <= 21 of 32), those are split one (neighbour, operator)
    // pair per lane instead: a sixth of the Horner work per lane, fewer idle lanes.
    const int nn = r1 - r0;
    const int rem = nn % 32;
    const bool split = !singular && rem > 0 && rem <= 21;
    const int nmain = split ? nn - rem : nn;
    for (int e = r0 + t; e < r0 + nmain; e += NT) {
        double wd[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        double dx = 0.0, dy = 0.0;
        if (!singular) {
            const int j = col[e];
            dx = min_image(__dsub_rn(xy[2 * j], g.xi), g.Lx, g.px);
            dy = min_image(__dsub_rn(xy[2 * j + 1], g.yi), g.Ly, g.py);
            const double xh = dx * g.ih, yh = dy * g.ih;
            const double psi = wendland_c2(sqrt(dx * dx + dy * dy) * g.ih);
#pragma unroll 1
            for (int p = M; p >= 0; --p) {
                const double* cp = s_cf + (p * (2 * M + 3 - p) / 2) * 6;  // (p, 0)
                double in[6];
#pragma unroll
                for (int d = 0; d < 6; ++d) in[d] = cp[(M - p) * 6 + d];
#pragma unroll 1
                for (int qq = M - p - 1; qq >= 0; --qq)
#pragma unroll
                    for (int d = 0; d < 6; ++d) in[d] = fma(in[d], yh, cp[qq * 6 + d]);
#pragma unroll
                for (int d = 0; d < 6; ++d) wd[d] = fma(wd[d], xh, in[d]);
            }
#pragma unroll
            for (int d = 0; d < 6; ++d) wd[d] *= psi;
        }
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            if (w) w[int64_t(d) * nnz + e] = wd[d];
            bad |= !isfinite(wd[d]);
        }
        const double phi = 1.0 - cos(kx * dx) * cos(kx * dy);
        f0 = fma(phi, wd[5], f0);
    }
    if (split) {
        for (int task = t; task < 6 * rem; task += NT) {
            const int e = r0 + nmain + task / 6;
            const int d = task - (task / 6) * 6;
            const int j = col[e];
            const double dx = min_image(__dsub_rn(xy[2 * j], g.xi), g.Lx, g.px);
            const double dy = min_image(__dsub_rn(xy[2 * j + 1], g.yi), g.Ly, g.py);
            const double xh = dx * g.ih, yh = dy * g.ih;
            const double psi = wendland_c2(sqrt(dx * dx + dy * dy) * g.ih);
            double acc = 0.0;
#pragma unroll 1
            for (int p = M; p >= 0; --p) {
                const double* cp = s_cf + (p * (2 * M + 3 - p) / 2) * 6 + d;  // (p, 0), operator d
                double in = cp[(M - p) * 6];
#pragma unroll 1
                for (int qq = M - p - 1; qq >= 0; --qq) in = fma(in, yh, cp[qq * 6]);
                acc = fma(acc, xh, in);
            }
            const double wv = acc * psi;
            if (w) w[int64_t(d) * nnz + e] = wv;
            bad |= !isfinite(wv);
            if (d == 5) f0 = fma(1.0 - cos(kx * dx) * cos(kx * dy), wv, f0);
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&s_nonfinite, 1);
    const double F0 = block_sum<NT>(f0, s_red);
    if (t == 0) {
        const double kap = singular ? 0.0 : 2.0 / (3.0 * F0);
        int flags = singular ? LABFM_NODE_SINGULAR : 0;
        if (s_nonfinite) flags |= LABFM_NODE_NONFINITE;
        if (!singular && !isfinite(kap)) flags |= LABFM_NODE_NONFINITE;
        kappa[i] = kap;
        node_status[i] = flags;
        if (flags && n_failed) atomicAdd(n_failed, 1ull);
    }
}

// ---------------------------------------------------------------- stencil optimisation (Section 4)

constexpr int kNk = 16;  // wavenumbers of the amplitude test (n_k = 16 in Section 4)

// Sum of 16 values over the 32 lanes of a warp by recursive halving: at each
// level a lane keeps half of its values and adds its partner's copy of that half
// (16 shuffles and adds instead of 80).  Afterwards lane L holds the total of
// value (L >> 1) & 15.
__device__ __forceinline__ double warp_sum16(double (&v)[16], int lane) {
    {
        const bool hi = lane & 16;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const double keep = hi ? v[8 + i] : v[i], send = hi ? v[i] : v[8 + i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
    }
    {
        const bool hi = lane & 8;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const double keep = hi ? v[4 + i] : v[i], send = hi ? v[i] : v[4 + i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
    }
    {
        const bool hi = lane & 4;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const double keep = hi ? v[2 + i] : v[i], send = hi ? v[i] : v[2 + i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
        }
    }
    {
        const bool hi = lane & 2;
        const double keep = hi ? v[1] : v[0], send = hi ? v[0] : v[1];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Amplitude responses of the d/dx, d/dy and Laplacian operators of node i at
// k_n = (pi / s_i) n / kNk, n = 1..kNk (Section 4, step 3).  The three solutions
// (Psi^x, Psi^y, Psi^L in columns n, n + 1, n + 2 of A) are turned into monomial
// coefficients once (as in the weight build), so each lane gets its neighbour's
// three weights by Horner's rule; sin and cos of n k_1 x_ji and n k_1 y_ji for
// n = 1..kNk follow by rotation from one sincos each (every step multiplies by
// e^{i k_1 x}, so the rounding error grows linearly in n).  Each lane accumulates
// its 3 kNk sums over all its neighbours; they are reduced across the warp once.
// s_cf3: (m+1)(m+2)/2 x 3 doubles; s_part: (NT / 32) x 3 kNk doubles.  Returns
// the largest of the 3 kNk responses (the same value in every thread).
template <int M, int LDA>
__device__ double block_amplitude_max(const double* __restrict__ xy, const int32_t* __restrict__ col,
                                      int r0, int r1, const NodeGeom& g, double s_i, const double* A,
                                      const double* s_he, double* s_cf3, double* s_part,
                                      double* s_amax) {
    using C = WCfg<M>;
    constexpr int n = C::n, NT = C::NT, NW = NT / 32;
    constexpr int NP = 3 * kNk;
    constexpr int NC = (M + 1) * (M + 2) / 2;
    static_assert(kNk == 16, "the warp reduction takes 16 values per operator");
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const double kny = 3.141592653589793 / s_i;
    const double k1 = kny / kNk;
    // coefficients c^d_pq of psi^-1 W . Psi^d = sum_pq c^d_pq (x/h)^p (y/h)^q
    for (int idx = t; idx < NC * 3; idx += NT) {
        const int pq = idx / 3, d = idx - pq * 3;
        int p = 0;
        while (pq >= (p + 1) * (2 * M + 2 - p) / 2) ++p;
        const int qy = pq - p * (2 * M + 3 - p) / 2;
        double c = 0.0;
        for (int a = p; a <= M; a += 2) {
            const double ha = s_he[a * (M + 1) + p];
            for (int b = qy; a + b <= M; b += 2) {
                const int k = a + b;
                if (k == 0) continue;
                c = fma(ha * s_he[b * (M + 1) + qy], A[(k * (k + 1) / 2 - 1 + b) * LDA + n + d], c);
            }
        }
        s_cf3[idx] = c;
    }
    __syncthreads();
    double acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = 0.0;
    for (int c0 = r0; c0 < r1; c0 += NT) {
        if (c0 + warp * 32 >= r1) continue;  // warp-uniform: no neighbour for this warp
        const int e = c0 + t;
        double w0 = 0.0, w1 = 0.0, w2 = 0.0, dx = 0.0, dy = 0.0;
        if (e < r1) {
            const int j = col[e];
            dx = min_image(__dsub_rn(xy[2 * j], g.xi), g.Lx, g.px);
            dy = min_image(__dsub_rn(xy[2 * j + 1], g.yi), g.Ly, g.py);
            const double xh = dx * g.ih, yh = dy * g.ih;
            const double psi = wendland_c2(sqrt(dx * dx + dy * dy) * g.ih);
#pragma unroll 1
            for (int p = M; p >= 0; --p) {
                const double* cp = s_cf3 + (p * (2 * M + 3 - p) / 2) * 3;  // (p, 0)
                double i0 = cp[(M - p) * 3], i1 = cp[(M - p) * 3 + 1], i2 = cp[(M - p) * 3 + 2];
#pragma unroll 1
                for (int qq = M - p - 1; qq >= 0; --qq) {
                    i0 = fma(i0, yh, cp[qq * 3]);
                    i1 = fma(i1, yh, cp[qq * 3 + 1]);
                    i2 = fma(i2, yh, cp[qq * 3 + 2]);
                }
                w0 = fma(w0, xh, i0);
                w1 = fma(w1, xh, i1);
                w2 = fma(w2, xh, i2);
            }
            w0 *= psi;
            w1 *= psi;
            w2 *= psi;
        }
        double s1x, c1x, s1y, c1y;
        sincos(k1 * dx, &s1x, &c1x);
        sincos(k1 * dy, &s1y, &c1y);
        double sx = s1x, cx = c1x, sy = s1y, cy = c1y;
#pragma unroll
        for (int k = 0; k < kNk; ++k) {
            acc[k] = fma(sx, w0, acc[k]);
            acc[kNk + k] = fma(sy, w1, acc[kNk + k]);
            acc[2 * kNk + k] = fma(0.5 - 0.5 * cx * cy, w2, acc[2 * kNk + k]);
            const double nsx = fma(sx, c1x, cx * s1x), ncx = fma(cx, c1x, -(sx * s1x));
            const double nsy = fma(sy, c1y, cy * s1y), ncy = fma(cy, c1y, -(sy * s1y));
            sx = nsx;
            cx = ncx;
            sy = nsy;
            cy = ncy;
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = acc[d * kNk + k];
        const double tot = warp_sum16(v, lane);
        if ((lane & 1) == 0) s_part[warp * NP + d * kNk + ((lane >> 1) & 15)] = tot;
    }
    __syncthreads();
    if (warp == 0) {
        double mx = -INFINITY;
        for (int pr = lane; pr < NP; pr += 32) {
            double v = 0.0;
            for (int wp = 0; wp < NW; ++wp) v += s_part[wp * NP + pr];
            const int d = pr / kNk;
            const double kn = kny * double(pr - d * kNk + 1) / kNk;
            mx = fmax(mx, d < 2 ? v / kn : v / (kn * kn));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        if (lane == 0) *s_amax = mx;
    }
    __syncthreads();
    return *s_amax;
}

// Register budget of the stencil-optimisation kernel: resident CTAs per SM as for
// 96 registers a thread (80 at m = 6, 96 at m = 8 after rounding).  Its 48
// per-lane amplitude sums need ~150 unconstrained, which left 4 CTAs of 96 threads
// per SM at m = 6 and the FP64 pipe 72 % busy; the spills of the tighter budget
// stay in L1 and cost less than the occupancy gains (full size: 128 registers
// 2.69 / 1.93 s, 96: 2.57 / 1.80 s for m = 6 / 8).
#ifndef LABFM_SOPT_REGS
#define LABFM_SOPT_REGS 96
#endif
template <int M>
constexpr int stencil_opt_min_blocks() {
    return 65536 / (WCfg<M>::NT * LABFM_SOPT_REGS);
}

template <int M>
__global__ void __launch_bounds__(WCfg<M>::NT, stencil_opt_min_blocks<M>())
    k_stencil_opt(const double* __restrict__ xy, const double* __restrict__ h0,
                  const double* __restrict__ s, int64_t N, double Lx, double Ly, int px_, int py_,
                  const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                  double factor, double amp_max, double resid_coef, int max_iter,
                  double* __restrict__ h_out, int32_t* __restrict__ solves_out,
                  double* __restrict__ alpha_out) {
    using C = WCfg<M>;
    constexpr int n = C::n;
    constexpr int NT = C::NT;
    constexpr int LDA = n + 3;  // [M | C~x C~y C~L]
    extern __shared__ double smem[];
    double* A = smem;
    double* A0 = smem + n * LDA;
    __shared__ double s_mu[C::NMOM];
    __shared__ double s_he[(M + 1) * (M + 1)];
    __shared__ double s_red[NT / 32];
    __shared__ double s_part[(NT / 32) * 3 * kNk];
    __shared__ double s_cf3[(M + 1) * (M + 2) / 2 * 3];
    __shared__ double s_hp[M + 1];
    __shared__ double s_amax;
    __shared__ double s_rdiag[n];
    __shared__ int s_piv;
    __shared__ int s_flag;

    const int64_t i = blockIdx.x;
    if (i >= N) return;
    const int t = threadIdx.x;
    const int r0 = row_ptr[i];
    const int r1 = row_ptr[i + 1];
    const double eps = 2.220446049250313e-16;
    build_he<M>(s_he);
    NodeGeom g{xy[2 * i], xy[2 * i + 1], h0[i], Lx, Ly, px_ != 0, py_ != 0, 1.0 / h0[i]};
    double best = h0[i];
    int solves = 0;
    // alpha_L at the last h that passed and at the h where the loop stopped (NaN
    // where none was computed)
    double alpha_pass = __longlong_as_double(0x7ff8000000000000ll);
    double alpha_stop = alpha_pass;
    for (int it = 0; it < max_iter; ++it) {
        if (t <= M) s_hp[t] = pow(g.hi, -double(t));  // h^-k (read after the next barrier)
        // nodes inside the current radius (the same exact test as the neighbour search)
        const double two_h = 2.0 * g.hi;
        const double rad2 = __dmul_rn(two_h, two_h);
        double cnt = 0.0;
        for (int e = r0 + t; e < r1; e += NT) {
            const int j = col[e];
            const double dx = min_image(__dsub_rn(xy[2 * j], g.xi), g.Lx, g.px);
            const double dy = min_image(__dsub_rn(xy[2 * j + 1], g.yi), g.Ly, g.py);
            cnt += __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= rad2 ? 1.0 : 0.0;
        }
        if (block_sum<NT>(cnt, s_red) < double(n)) break;
        // Section 4 steps 1-2: solve for x, y and L and test the Laplacian residual
        block_moments<M>(xy, col, r0, r1, g, smem, smem + C::MCH * C::NPOW, s_mu);
        block_assemble<M, LDA>(A, A0, s_mu, s_he);
        for (int idx = t; idx < n * 3; idx += NT) {
            const int q = idx / 3, d = idx - q * 3;
            int a, b;
            exps_of(q, a, b);
            double coef;
            if (d < 2) coef = selector_coef<M>(d, a, b);
            else coef = ((a == 2 && b == 0) || (a == 0 && b == 2)) ? 1.0 : 0.0;
            A[q * LDA + n + d] = coef * s_hp[a + b];
        }
        const bool singular = block_lu_solve<M, LDA>(A, &s_piv, &s_flag, s_rdiag);
        ++solves;
        if (singular) break;
        double r2 = 0.0;
        for (int q = t; q < n; q += NT) {
            double sum = 0.0;
            for (int c = 0; c < n; ++c) sum = fma(A0[q * n + c], A[c * LDA + n + 2], sum);
            int a, b;
            exps_of(q, a, b);
            const double cq = ((a == 2 && b == 0) || (a == 0 && b == 2)) ? s_hp[2] : 0.0;
            const double r = (sum - cq) * g.hi * g.hi;
            r2 = fma(r, r, r2);
        }
        const double alpha = sqrt(block_sum<NT>(r2, s_red));
        const double alpha0 = resid_coef * eps * double(n) * double(n) * double(n) * double(n) / (g.hi * M);
        if (!(alpha <= alpha0)) {
            alpha_stop = alpha;
            break;
        }
        // steps 3-4: amplitude response up to Nyquist
        const double amax = block_amplitude_max<M, LDA>(xy, col, r0, r1, g, s[i], A, s_he, s_cf3, s_part, &s_amax);
        if (!(amax <= amp_max)) {
            alpha_stop = alpha;
            break;
        }
        // step 5
        best = g.hi;
        alpha_pass = alpha;
        g.hi = g.hi * factor;
        g.ih = 1.0 / g.hi;
        __syncthreads();
    }
    if (t == 0) {
        h_out[i] = best;
        if (solves_out) solves_out[i] = solves;
        if (alpha_out) {
            alpha_out[2 * i] = alpha_pass;
            alpha_out[2 * i + 1] = alpha_stop;
        }
    }
}

template <int M>
int launch_stencil_opt(const double* xy, const double* h0, const double* s, int64_t N, double Lx,
                       double Ly, uint32_t pm, const int32_t* row_ptr, const int32_t* col,
                       double factor, double amp_max, double resid_coef, int max_iter, double* h_out,
                       int32_t* solves, double* alpha, cudaStream_t st) {
    using C = WCfg<M>;
    const size_t sm = C::smem(true);
    LABFM_CUDA_TRY(cudaFuncSetAttribute(k_stencil_opt<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
    k_stencil_opt<M><<<unsigned(N), C::NT, sm, st>>>(xy, h0, s, N, Lx, Ly, pm & 1u, (pm >> 1) & 1u,
                                                     row_ptr, col, factor, amp_max, resid_coef, max_iter, h_out, solves,
                                                     alpha);
    LABFM_LAUNCH_CHECK("stencil optimisation kernel");
    return LABFM_OK;
}

// ---------------------------------------------------------------- modal response (Section 3)

// Per node, the amplitude responses of d/dx, d/dy and the Laplacian (w^xx + w^yy)
// of built weights at k_n = n pi / (s_i nk), n = 1..nk: out[(i * 3 + d) * nk + n - 1].
__global__ void k_modal_response(const double* __restrict__ xy, const double* __restrict__ s,
                                 int64_t N, double Lx, double Ly, int px_, int py_,
                                 const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                 int64_t nnz, const double* __restrict__ w, int nk,
                                 double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; i < N; i += warps) {
        const int r0 = row_ptr[i], r1 = row_ptr[i + 1];
        const double xi = xy[2 * i], yi = xy[2 * i + 1];
        const double k0 = 3.141592653589793 / (s[i] * nk);
        for (int k = 1; k <= nk; ++k) {
            const double kn = double(k) * k0;
            double ax = 0.0, ay = 0.0, al = 0.0;
            for (int e = r0 + lane; e < r1; e += 32) {
                const int j = col[e];
                const double dx = min_image(__dsub_rn(xy[2 * j], xi), Lx, px_ != 0);
                const double dy = min_image(__dsub_rn(xy[2 * j + 1], yi), Ly, py_ != 0);
                double sx, cx, sy, cy;
                sincos(kn * dx, &sx, &cx);
                sincos(kn * dy, &sy, &cy);
                ax = fma(sx, w[e], ax);
                ay = fma(sy, w[nnz + e], ay);
                al = fma(0.5 - 0.5 * cx * cy, w[2 * nnz + e] + w[4 * nnz + e], al);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, off);
                ay += __shfl_xor_sync(0xffffffffu, ay, off);
                al += __shfl_xor_sync(0xffffffffu, al, off);
            }
            if (lane == 0) {
                out[(i * 3 + 0) * nk + k - 1] = ax / kn;
                out[(i * 3 + 1) * nk + k - 1] = ay / kn;
                out[(i * 3 + 2) * nk + k - 1] = al / (kn * kn);
            }
        }
    }
}

// Injected failure (LABFM_FAULT=singular_node:<i>): node i flagged singular as if
// its LU had met a zero pivot, counted once in the failed-node total.
__global__ void k_flag_singular(int32_t* __restrict__ node_status, int64_t i,
                                unsigned long long* __restrict__ n_failed) {
    const int32_t old = node_status[i];
    node_status[i] = old | LABFM_NODE_SINGULAR;
    if (n_failed && old == 0) atomicAdd(n_failed, 1ull);
}

template <int M>
int launch_weights(const double* xy, const double* h, const double* s, int64_t N, double Lx,
                   double Ly, uint32_t pm, const int32_t* row_ptr, const int32_t* col, int64_t nnz,
                   double* w, double* kappa, double* residual, int32_t* status,
                   unsigned long long* n_failed, double* coef, cudaStream_t st) {
    using C = WCfg<M>;
    const bool resid = residual != nullptr;
    const size_t sm = C::smem(resid);
    if (resid) {
        auto kern = k_weight_build<M, true>;
        LABFM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
        kern<<<unsigned(N), C::NT, sm, st>>>(xy, h, s, N, Lx, Ly, pm & 1u, (pm >> 1) & 1u, row_ptr,
                                             col, nnz, w, kappa, residual, status, n_failed, coef);
    } else {
        auto kern = k_weight_build<M, false>;
        LABFM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
        kern<<<unsigned(N), C::NT, sm, st>>>(xy, h, s, N, Lx, Ly, pm & 1u, (pm >> 1) & 1u, row_ptr,
                                             col, nnz, w, kappa, residual, status, n_failed, coef);
    }
    LABFM_LAUNCH_CHECK("weight build kernel");
    return LABFM_OK;
}

}  // namespace
}  // namespace labfm

using namespace labfm;

extern "C" int labfm_build_weights_ex(const double* xy, const double* h, const double* s, int64_t N,
                                      double Lx, double Ly, uint32_t periodic_mask,
                                      const int32_t* row_ptr, const int32_t* col, int64_t nnz, int m,
                                      double* w, double* kappa, double* residual, int32_t* node_status,
                                      int64_t* n_failed_out, double* coef_out, void* stream) {
    LABFM_NVTX("labfm_build_weights");
    if (!xy || !h || !s || !row_ptr || !kappa || !node_status || (nnz > 0 && !w && !coef_out))
        return set_error(LABFM_EINVAL, "null pointer argument");
    if (nnz > 0 && !col) return set_error(LABFM_EINVAL, "null col with nnz > 0");
    if (N <= 0 || N >= (int64_t(1) << 31) - 1) return set_error(LABFM_EINVAL, "N out of range");
    if (nnz < 0 || nnz >= (int64_t(1) << 31)) return set_error(LABFM_EINVAL, "nnz out of range");
    if (m < 2 || m > 10 || (m & 1))
        return set_error(LABFM_EINVAL, "order m must be even and in [2, 10], got " + std::to_string(m));
    if (!(Lx > 0.0) || !(Ly > 0.0)) return set_error(LABFM_EINVAL, "domain size must be positive");
    if (n_failed_out && fault_alloc()) return injected_alloc_error("labfm_build_weights");
    if (int rc = validate_csr(row_ptr, col, N, nnz, as_stream(stream))) return rc;
    cudaStream_t st = as_stream(stream);
    unsigned long long* nf = nullptr;
    if (n_failed_out) {
        LABFM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&nf), sizeof(unsigned long long), st));
        LABFM_CUDA_TRY(cudaMemsetAsync(nf, 0, sizeof(unsigned long long), st));
    }
    int rc = LABFM_OK;
    switch (m) {
        case 2: rc = launch_weights<2>(xy, h, s, N, Lx, Ly, periodic_mask, row_ptr, col, nnz, w, kappa, residual, node_status, nf, coef_out, st); break;
        case 4: rc = launch_weights<4>(xy, h, s, N, Lx, Ly, periodic_mask, row_ptr, col, nnz, w, kappa, residual, node_status, nf, coef_out, st); break;
        case 6: rc = launch_weights<6>(xy, h, s, N, Lx, Ly, periodic_mask, row_ptr, col, nnz, w, kappa, residual, node_status, nf, coef_out, st); break;
        case 8: rc = launch_weights<8>(xy, h, s, N, Lx, Ly, periodic_mask, row_ptr, col, nnz, w, kappa, residual, node_status, nf, coef_out, st); break;
        case 10: rc = launch_weights<10>(xy, h, s, N, Lx, Ly, periodic_mask, row_ptr, col, nnz, w, kappa, residual, node_status, nf, coef_out, st); break;
    }
    const int64_t fnode = fault_singular_node();
    if (rc == LABFM_OK && fnode >= 0 && fnode < N) {
        k_flag_singular<<<1, 1, 0, st>>>(node_status, fnode, nf);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_error(e, "injected singular node");
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

extern "C" int labfm_build_weights(const double* xy, const double* h, const double* s, int64_t N,
                                   double Lx, double Ly, uint32_t periodic_mask,
                                   const int32_t* row_ptr, const int32_t* col, int64_t nnz, int m,
                                   double* w, double* kappa, double* residual,
                                   int32_t* node_status, int64_t* n_failed_out, void* stream) {
    if (nnz > 0 && !w) return set_error(LABFM_EINVAL, "null pointer argument");
    return labfm_build_weights_ex(xy, h, s, N, Lx, Ly, periodic_mask, row_ptr, col, nnz, m, w, kappa, residual,
                                  node_status, n_failed_out, nullptr, stream);
}

extern "C" int labfm_stencil_optimise(const double* xy, const double* h0, const double* s, int64_t N,
                                      double Lx, double Ly, uint32_t periodic_mask,
                                      const int32_t* row_ptr, const int32_t* col, int m,
                                      double factor, double amp_max, double resid_coef, int max_iter,
                                      double* h_out, int32_t* solves_out, double* alpha_out, void* stream) {
    LABFM_NVTX("labfm_stencil_optimise");
    if (!xy || !h0 || !s || !row_ptr || !col || !h_out)
        return set_error(LABFM_EINVAL, "null pointer argument");
    if (N <= 0 || N >= (int64_t(1) << 31) - 1) return set_error(LABFM_EINVAL, "N out of range");
    if (m < 2 || m > 10 || (m & 1)) return set_error(LABFM_EINVAL, "order m must be even and in [2, 10]");
    if (!(factor > 0.0 && factor < 1.0)) return set_error(LABFM_EINVAL, "factor must be in (0, 1)");
    if (max_iter < 0) return set_error(LABFM_EINVAL, "negative max_iter");
    if (!(resid_coef > 0.0)) return set_error(LABFM_EINVAL, "resid_coef must be positive");
    cudaStream_t st = as_stream(stream);
    if (int rc = validate_csr(row_ptr, col, N, -1, st)) return rc;
    switch (m) {
        case 2: return launch_stencil_opt<2>(xy, h0, s, N, Lx, Ly, periodic_mask, row_ptr, col, factor, amp_max, resid_coef, max_iter, h_out, solves_out, alpha_out, st);
        case 4: return launch_stencil_opt<4>(xy, h0, s, N, Lx, Ly, periodic_mask, row_ptr, col, factor, amp_max, resid_coef, max_iter, h_out, solves_out, alpha_out, st);
        case 6: return launch_stencil_opt<6>(xy, h0, s, N, Lx, Ly, periodic_mask, row_ptr, col, factor, amp_max, resid_coef, max_iter, h_out, solves_out, alpha_out, st);
        case 8: return launch_stencil_opt<8>(xy, h0, s, N, Lx, Ly, periodic_mask, row_ptr, col, factor, amp_max, resid_coef, max_iter, h_out, solves_out, alpha_out, st);
        default: return launch_stencil_opt<10>(xy, h0, s, N, Lx, Ly, periodic_mask, row_ptr, col, factor, amp_max, resid_coef, max_iter, h_out, solves_out, alpha_out, st);
    }
}

extern "C" int labfm_modal_response(const double* xy, const double* s, int64_t N, double Lx,
                                    double Ly, uint32_t periodic_mask, const int32_t* row_ptr,
                                    const int32_t* col, int64_t nnz, const double* w, int nk,
                                    double* out, void* stream) {
    LABFM_NVTX("labfm_modal_response");
    if (!xy || !s || !row_ptr || !out || (nnz > 0 && (!col || !w)))
        return set_error(LABFM_EINVAL, "null pointer argument");
    if (N <= 0 || N >= (int64_t(1) << 31) - 1) return set_error(LABFM_EINVAL, "N out of range");
    if (nk < 1 || nk > 4096) return set_error(LABFM_EINVAL, "nk out of range");
    cudaStream_t st = as_stream(stream);
    if (int rc = validate_csr(row_ptr, col, N, nnz, st)) return rc;
    const int grid = int(std::min<int64_t>((N + 7) / 8, 1 << 20));
    k_modal_response<<<grid, 256, 0, st>>>(xy, s, N, Lx, Ly, periodic_mask & 1u, (periodic_mask >> 1) & 1u,
                                           row_ptr, col, nnz, w, nk, out);
    LABFM_LAUNCH_CHECK("modal response kernel");
    return LABFM_OK;
}
