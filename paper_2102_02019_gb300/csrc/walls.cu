// Operators near walls (Section 7.1, Table "Schemes for derivatives near
// boundaries", and Appendix A) and the walls of a plan.
//
// A wall is described, as in Section 7.1, by its nodes i0 with their inward unit
// normals n, each with the four nodes i1..i4 of its normal column (at q s along
// n).  The operator of the whole domain is one difference-form CSR with the six
// weights of labfm_build_weights per entry, so that the step kernels use it
// unchanged:
//   rows q >= 3 and the interior: LABFM of order m;
//   rows q = 1, 2: d/dx, d/dy from a five-point difference along the normal
//     column (asymmetric at q = 1, central at q = 2) and one-dimensional LABFM of
//     order 4 along the row of the same q (Appendix A), rotated to (x, y); second
//     derivatives and the filter from LABFM of order m_wall;
//   boundary nodes q = 0: d/dx, d/dy from the one-sided five-point difference and
//     1D LABFM; second derivatives from the one-sided second difference along the
//     column, 1D LABFM d2/deta2 along the boundary row, and d2/dxi deta as the
//     one-sided first difference along the column of the rows' 1D LABFM d/deta;
//     no filter (kappa = 0).  A wall holds the velocity at zero there and does not
//     use the second derivatives; an outflow or inflow follows its LODI equations.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "labfm_internal.cuh"
#include "nvtx.cuh"

namespace labfm {
namespace {

constexpr int kColumn = 5;    // nodes of a normal column, q = 0..4
constexpr int kStripRows = 3; // rows with boundary-specific first derivatives
constexpr int kOrder1d = 4;   // order of the one-dimensional LABFM along the rows
constexpr int kMaxRow = 16;   // row neighbours per node handled by the merge
constexpr int kMaxEnt = kColumn + kColumn * kMaxRow;  // strip entries of a boundary node

// Five-point first-derivative weights (units of 1/s) for the rows q = 0, 1, 2 of a
// normal column over its points r = 0..4 (offsets r - q): the derivative at 0 of
// the Lagrange interpolant through the five points,
//   w_r = sum_{k != r} prod_{l != r, k} (0 - o_l) / prod_{l != r} (o_r - o_l).
struct FdTable {
    double w[kStripRows][kColumn];
    double w2[kColumn];  // second derivative at q = 0 (one-sided), units of 1/s^2
};

FdTable fd_first_derivative_table() {
    FdTable t{};
    // second derivative at 0 of the Lagrange interpolant over offsets 0..4:
    //   w2_r = sum_{k != r} sum_{l != r, k} prod_{m != r, k, l} (0 - o_m) / prod_{m != r} (o_r - o_m)
    for (int r = 0; r < kColumn; ++r) {
        double den = 1.0;
        for (int m = 0; m < kColumn; ++m)
            if (m != r) den *= double(r - m);
        double num = 0.0;
        for (int k = 0; k < kColumn; ++k) {
            if (k == r) continue;
            for (int l = 0; l < kColumn; ++l) {
                if (l == r || l == k) continue;
                double p = 1.0;
                for (int m = 0; m < kColumn; ++m)
                    if (m != r && m != k && m != l) p *= -double(m);
                num += p;
            }
        }
        t.w2[r] = num / den;
    }
    for (int q = 0; q < kStripRows; ++q) {
        double o[kColumn];
        for (int r = 0; r < kColumn; ++r) o[r] = double(r - q);
        for (int r = 0; r < kColumn; ++r) {
            double den = 1.0;
            for (int l = 0; l < kColumn; ++l)
                if (l != r) den *= o[r] - o[l];
            double num = 0.0;
            for (int k = 0; k < kColumn; ++k) {
                if (k == r) continue;
                double p = 1.0;
                for (int l = 0; l < kColumn; ++l)
                    if (l != r && l != k) p *= -o[l];
                num += p;
            }
            t.w[q][r] = num / den;
        }
    }
    return t;
}

// Node kinds: -1 for a node in no column, else 5 b + q for row q of wall node b.
__global__ void k_mark_columns(int64_t n_wall, const int32_t* __restrict__ wall_column,
                               const double* __restrict__ wall_normal, int64_t N,
                               int32_t* __restrict__ kind, int* __restrict__ bad) {
    for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n_wall * kColumn;
         k += int64_t(gridDim.x) * blockDim.x) {
        const int32_t node = wall_column[k];
        if (node < 0 || node >= N) {
            atomicOr(bad, 1);
            continue;
        }
        if (atomicExch(kind + node, int32_t(k)) != -1) atomicOr(bad, 2);
        if (k % kColumn == 0) {
            const int64_t b = k / kColumn;
            const double nx = wall_normal[2 * b], ny = wall_normal[2 * b + 1];
            if (!(fabs(nx * nx + ny * ny - 1.0) <= 1e-12)) atomicOr(bad, 4);
        }
    }
}

// Positions and 1D supports of the nodes of row q of every column, compacted by
// wall index, for the row-neighbour search.
__global__ void k_gather_row(int64_t n_wall, int q, const int32_t* __restrict__ wall_column,
                             const double* __restrict__ xy, const double* __restrict__ s, double h1d_over_s,
                             double* __restrict__ xy_q, double* __restrict__ h_q) {
    for (int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; b < n_wall;
         b += int64_t(gridDim.x) * blockDim.x) {
        const int32_t node = wall_column[b * kColumn + q];
        xy_q[2 * b] = xy[2 * node];
        xy_q[2 * b + 1] = xy[2 * node + 1];
        h_q[b] = h1d_over_s * s[node];
    }
}

__device__ __forceinline__ double wendland_c2(double q) {
    if (q >= 2.0) return 0.0;
    const double a = 1.0 - 0.5 * q;
    const double a2 = a * a;
    return a2 * a2 * (1.0 + 2.0 * q);
}

// One-dimensional LABFM of order 4 (Appendix A) for d/deta and d2/deta2 at a node
// from the offsets eta_j of its row neighbours: monomials eta^k / k!, k = 1..4;
// ABFs psi(|eta|/h) H_k(eta / (h sqrt 2)) / sqrt(2^k) with physicists' Hermite H_k;
// M = sum_j X_j (x) W_j; M Psi = [e_1 e_2] (the selectors of d/deta and
// d2/deta2); w_j = W_j . Psi.  w2 may be null.  Returns false for a singular M.
__device__ bool labfm_1d_weights(const double* eta, int n, double h, double* w, double* w2) {
    constexpr int K = kOrder1d;
    double M[K][K + 2];
    for (int a = 0; a < K; ++a)
        for (int c = 0; c < K + 2; ++c) M[a][c] = (a == 0 && c == K) || (a == 1 && c == K + 1) ? 1.0 : 0.0;
    const double inv_sqrt2 = 0.70710678118654752440;
    const double inv_norm[K] = {inv_sqrt2, 0.5, 0.5 * inv_sqrt2, 0.25};  // 1 / sqrt(2^k)
    for (int j = 0; j < n; ++j) {
        const double e = eta[j];
        const double psi = wendland_c2(fabs(e) / h);
        const double z = e / h * inv_sqrt2;
        double H[K + 1];
        H[0] = 1.0;
        H[1] = 2.0 * z;
        for (int k = 1; k < K; ++k) H[k + 1] = 2.0 * z * H[k] - 2.0 * k * H[k - 1];
        double X[K];
        double p = 1.0;
        for (int k = 0; k < K; ++k) {
            p *= e / double(k + 1);  // eta^(k+1) / (k+1)!
            X[k] = p;
        }
        for (int a = 0; a < K; ++a)
            for (int c = 0; c < K; ++c) M[a][c] += X[a] * (psi * H[c + 1] * inv_norm[c]);
    }
    // Gaussian elimination with partial pivoting on [M | e_1]
    for (int c = 0; c < K; ++c) {
        int piv = c;
        for (int r = c + 1; r < K; ++r)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (!(fabs(M[piv][c]) > 0.0)) return false;
        if (piv != c)
            for (int k = 0; k < K + 2; ++k) {
                const double t = M[c][k];
                M[c][k] = M[piv][k];
                M[piv][k] = t;
            }
        for (int r = c + 1; r < K; ++r) {
            const double f = M[r][c] / M[c][c];
            for (int k = c; k < K + 2; ++k) M[r][k] -= f * M[c][k];
        }
    }
    double psi_sol[2][K];
    for (int rhs = 0; rhs < 2; ++rhs)
        for (int c = K - 1; c >= 0; --c) {
            double v = M[c][K + rhs];
            for (int k = c + 1; k < K; ++k) v -= M[c][k] * psi_sol[rhs][k];
            psi_sol[rhs][c] = v / M[c][c];
        }
    for (int j = 0; j < n; ++j) {
        const double e = eta[j];
        const double psi = wendland_c2(fabs(e) / h);
        const double z = e / h * inv_sqrt2;
        double H[K + 1];
        H[0] = 1.0;
        H[1] = 2.0 * z;
        for (int k = 1; k < K; ++k) H[k + 1] = 2.0 * z * H[k] - 2.0 * k * H[k - 1];
        double v = 0.0, v2 = 0.0;
        for (int c = 0; c < K; ++c) {
            const double W = psi * H[c + 1] * inv_norm[c];
            v += W * psi_sol[0][c];
            v2 += W * psi_sol[1][c];
        }
        w[j] = v;
        if (w2) w2[j] = v2;
    }
    return true;
}

struct WallOpArgs {
    const double* xy;
    const double* s;
    int64_t N;
    double Lx, Ly;
    bool px, py;
    const int32_t* kind;
    const int32_t* wall_column;
    const double* wall_normal;
    double h1d_over_s;
    FdTable fd;
    // LABFM stencils and weights (order m, and m_wall for rows 1, 2)
    const int32_t* rpA;
    const int32_t* colA;
    int64_t nnzA;
    const double* wA;
    const double* kA;
    const int32_t* stA;
    const double* wB;
    const double* kB;
    const int32_t* stB;
    // row neighbours (wall indices) of the rows q = 0..4
    const int32_t* rpR[kColumn];
    const int32_t* colR[kColumn];
};

// Per-warp scratch (shared memory) of the strip entries of one node: node and
// its five RHS weights (d/dx, d/dy, d2/dx2, d2/dxdy, d2/dy2).
struct StripScratch {
    int32_t node[kMaxEnt];
    double w[5][kMaxEnt];
    double eta[kMaxRow];
    double w1[kMaxRow];
    double w2[kMaxRow];
};
constexpr int kMergeWarps = 4;  // warps per block of the merge kernel

// 1D LABFM along row r of column b at its node k (support h1d_over_s s_k):
// its row neighbours into S.node[at..], the d/deta (and, if want2, d2/deta2)
// weights into S.w1, S.w2.  Returns the number of neighbours, -1 beyond kMaxRow,
// -2 for a singular system.
__device__ int row_weights(const WallOpArgs& A, int b, int r, bool want2, StripScratch& S, int* nodes) {
    const int32_t k = A.wall_column[int64_t(b) * kColumn + r];
    const double nx = A.wall_normal[2 * b], ny = A.wall_normal[2 * b + 1];
    const double tx = -ny, ty = nx;
    const double xk = A.xy[2 * k], yk = A.xy[2 * k + 1];
    const int e0 = A.rpR[r][b], e1 = A.rpR[r][b + 1];
    const int nr = e1 - e0;
    if (nr > kMaxRow) return -1;
    for (int e = 0; e < nr; ++e) {
        const int bj = A.colR[r][e0 + e];
        const int32_t j = A.wall_column[int64_t(bj) * kColumn + r];
        const double dx = min_image(A.xy[2 * j] - xk, A.Lx, A.px);
        const double dy = min_image(A.xy[2 * j + 1] - yk, A.Ly, A.py);
        S.eta[e] = dx * tx + dy * ty;
        nodes[e] = j;
    }
    if (nr > 0 && !labfm_1d_weights(S.eta, nr, A.h1d_over_s * A.s[k], S.w1, want2 ? S.w2 : nullptr))
        return -2;
    return nr;
}

// The strip entries of node i (row q of wall node b), rotated to (x, y) with
// d/dx = n_x d/dxi - n_y d/deta, d/dy = n_y d/dxi + n_x d/deta:
//   d/dxi: the five-point difference along the column (rows r != q);
//   d/deta: 1D LABFM along the node's row;
//   for a boundary node (q = 0) also d2/dxi2 (the one-sided second difference
//   along the column), d2/deta2 (1D LABFM along row 0) and d2/dxi deta (the
//   one-sided first difference along the column of each row's 1D LABFM d/deta:
//   the row neighbours of column node r with weight w1_r(xi) w^eta_rj, and node r
//   itself with minus their sum).
// Entries are summed per node and sorted; the node itself is left out (the
// difference form).  Returns the number of entries, -1 when a row has more than
// kMaxRow neighbours, -2 for a singular 1D system.
__device__ int strip_entries(const WallOpArgs& A, int64_t i, int b, int q, StripScratch& S) {
    const double nx = A.wall_normal[2 * b], ny = A.wall_normal[2 * b + 1];
    const double si = A.s[i];
    int n = 0;
    auto add = [&](int32_t j, double ax, double ay, double axx, double axy, double ayy) {
        S.node[n] = j;
        S.w[0][n] = ax;
        S.w[1][n] = ay;
        S.w[2][n] = axx;
        S.w[3][n] = axy;
        S.w[4][n] = ayy;
        ++n;
    };
    for (int r = 0; r < kColumn; ++r) {
        if (r == q) continue;
        const double c1 = A.fd.w[q][r] / si;
        const double c2 = q == 0 ? A.fd.w2[r] / (si * si) : 0.0;
        add(A.wall_column[int64_t(b) * kColumn + r], nx * c1, ny * c1, nx * nx * c2, nx * ny * c2, ny * ny * c2);
    }
    {
        const int nr = row_weights(A, b, q, q == 0, S, S.node + n);
        if (nr < 0) return nr;
        for (int e = 0; e < nr; ++e) {
            const double w1 = S.w1[e], w2 = q == 0 ? S.w2[e] : 0.0;
            S.w[0][n + e] = -ny * w1;
            S.w[1][n + e] = nx * w1;
            S.w[2][n + e] = ny * ny * w2;
            S.w[3][n + e] = -nx * ny * w2;
            S.w[4][n + e] = nx * nx * w2;
        }
        n += nr;
    }
    if (q == 0) {
        for (int r = 0; r < kColumn; ++r) {
            const int nr = row_weights(A, b, r, false, S, S.node + n);
            if (nr < 0) return nr;
            const double cm = A.fd.w[0][r] / si;
            double sum = 0.0;
            for (int e = 0; e < nr; ++e) {
                const double m = cm * S.w1[e];
                sum += S.w1[e];
                S.w[0][n + e] = 0.0;
                S.w[1][n + e] = 0.0;
                S.w[2][n + e] = -2.0 * nx * ny * m;
                S.w[3][n + e] = (nx * nx - ny * ny) * m;
                S.w[4][n + e] = 2.0 * nx * ny * m;
            }
            n += nr;
            if (r > 0) {  // the column node's own term (node i's own is left out)
                const double m = -cm * sum;
                add(A.wall_column[int64_t(b) * kColumn + r], 0.0, 0.0, -2.0 * nx * ny * m,
                    (nx * nx - ny * ny) * m, 2.0 * nx * ny * m);
            }
        }
    }
    // insertion sort by node, then sum the entries of one node
    for (int a = 1; a < n; ++a) {
        const int32_t kn = S.node[a];
        double v[5];
        for (int d = 0; d < 5; ++d) v[d] = S.w[d][a];
        int c = a - 1;
        while (c >= 0 && S.node[c] > kn) {
            S.node[c + 1] = S.node[c];
            for (int d = 0; d < 5; ++d) S.w[d][c + 1] = S.w[d][c];
            --c;
        }
        S.node[c + 1] = kn;
        for (int d = 0; d < 5; ++d) S.w[d][c + 1] = v[d];
    }
    int m = 0;
    for (int a = 0; a < n; ++a) {
        if (S.node[a] == int32_t(i)) continue;
        if (m > 0 && S.node[m - 1] == S.node[a]) {
            for (int d = 0; d < 5; ++d) S.w[d][m - 1] += S.w[d][a];
        } else {
            S.node[m] = S.node[a];
            for (int d = 0; d < 5; ++d) S.w[d][m] = S.w[d][a];
            ++m;
        }
    }
    return m;
}

// Warp per node.  FILL = false: the number of entries of each merged row (and the
// node's status bits for a failed strip); FILL = true: columns, the six weights
// (operator-major, stride nnz), kappa and the node status.
template <bool FILL>
__global__ void k_wall_merge(WallOpArgs A, int32_t* __restrict__ cnt, const int32_t* __restrict__ row_ptr,
                             int32_t* __restrict__ col, double* __restrict__ w, int64_t nnz,
                             double* __restrict__ kappa, int32_t* __restrict__ status) {
    __shared__ StripScratch scratch[kMergeWarps];
    const int lane = threadIdx.x & 31;
    StripScratch& S = scratch[threadIdx.x >> 5];
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; i < A.N; i += warps) {
        const int32_t code = A.kind[i];
        const int q = code >= 0 ? code % kColumn : kColumn;
        const int a0 = A.rpA[i], a1 = A.rpA[i + 1];
        if (q >= kStripRows) {  // LABFM of order m
            if (!FILL) {
                if (lane == 0) cnt[i] = a1 - a0;
                continue;
            }
            const int64_t d0 = row_ptr[i];
            for (int e = lane; e < a1 - a0; e += 32) {
                col[d0 + e] = A.colA[a0 + e];
#pragma unroll
                for (int d = 0; d < 6; ++d) w[d * nnz + d0 + e] = A.wA[d * A.nnzA + a0 + e];
            }
            if (lane == 0) {
                kappa[i] = A.kA[i];
                status[i] = A.stA[i];
            }
            continue;
        }
        if (lane != 0) continue;
        const int b = code / kColumn;
        const int ns = strip_entries(A, i, b, q, S);
        const int32_t* node = S.node;
        const bool labfm = q > 0;  // rows 1, 2 keep the LABFM second derivatives and filter
        if (ns < 0) {  // too many row neighbours or a singular 1D system: an empty row
            if (!FILL) {
                cnt[i] = 0;
            } else {
                kappa[i] = 0.0;
                status[i] = LABFM_NODE_SINGULAR;
            }
            continue;
        }
        // merge the strip entries with the LABFM stencil (both sorted by node)
        int64_t dst = FILL ? row_ptr[i] : 0;
        int n = 0, ka = labfm ? a0 : a1, ks = 0;
        while (ka < a1 || ks < ns) {
            const int32_t ja = ka < a1 ? A.colA[ka] : INT32_MAX;
            const int32_t js = ks < ns ? node[ks] : INT32_MAX;
            const int32_t j = ja < js ? ja : js;
            if (FILL) {
                double v[6] = {0, 0, 0, 0, 0, 0};
                if (js == j)
                    for (int d = 0; d < 5; ++d) v[d] = S.w[d][ks];
                if (ja == j)  // rows 1, 2: second derivatives and filter from LABFM of order m_wall
                    for (int d = 2; d < 6; ++d) v[d] += A.wB[d * A.nnzA + ka];
                col[dst + n] = j;
                for (int d = 0; d < 6; ++d) w[d * nnz + dst + n] = v[d];
            }
            if (ja == j) ++ka;
            if (js == j) ++ks;
            ++n;
        }
        if (!FILL) {
            cnt[i] = n;
        } else {
            kappa[i] = labfm ? A.kB[i] : 0.0;
            status[i] = labfm ? A.stB[i] : 0;
        }
    }
}

__global__ void k_count_failed(int64_t N, const int32_t* __restrict__ status, unsigned long long* out) {
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x)
        c += status[i] != 0;
    if (c) atomicAdd(out, c);
}

// Scratch allocations of one call, freed on every return path.
struct Scratch {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit Scratch(cudaStream_t s) : st(s) {}
    template <typename T>
    int get(T** p, size_t count) {
        const cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T), st);
        if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync (wall operator scratch)");
        ptrs.push_back(*p);
        return LABFM_OK;
    }
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
};

int grid_of(int64_t threads) { return int(std::min<int64_t>((threads + 255) / 256, 65535)); }

// CSR of labfm_build_stencils into scratch (query, allocate, fill).
int stencils_into(Scratch& sc, const double* xy, const double* h, int64_t n, double Lx, double Ly, uint32_t mask,
                  int32_t** rp, int32_t** col, int64_t* nnz) {
    int rc;
    if ((rc = sc.get(rp, size_t(n + 1)))) return rc;
    if ((rc = labfm_build_stencils(xy, h, n, Lx, Ly, mask, *rp, nullptr, 0, nnz, sc.st))) return rc;
    if ((rc = sc.get(col, size_t(*nnz)))) return rc;
    return labfm_build_stencils(xy, h, n, Lx, Ly, mask, *rp, *col, std::max<int64_t>(*nnz, 1), nnz, sc.st);
}

}  // namespace

// ---------------------------------------------------------------- walls of a plan

namespace {
template <typename T>
__global__ void k_set_walls(int64_t n_wall, const int32_t* __restrict__ nodes, const double* __restrict__ normal,
                            const int32_t* __restrict__ kind, const double* __restrict__ target, int64_t N,
                            int32_t* __restrict__ slot, T* __restrict__ wn, int32_t* __restrict__ wk,
                            T* __restrict__ wt, int* __restrict__ bad) {
    for (int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; b < n_wall;
         b += int64_t(gridDim.x) * blockDim.x) {
        const int32_t i = nodes[b];
        const double nx = normal[2 * b], ny = normal[2 * b + 1];
        if (i < 0 || i >= N) {
            atomicOr(bad, 1);
            continue;
        }
        if (atomicExch(slot + i, int32_t(b)) != -1) atomicOr(bad, 2);
        if (!(fabs(nx * nx + ny * ny - 1.0) <= 1e-12)) atomicOr(bad, 4);
        wn[2 * b] = T(nx);
        wn[2 * b + 1] = T(ny);
        if (wk) {
            const int32_t k = kind[b];
            if (k != LABFM_WALL && k != LABFM_INFLOW && k != LABFM_OUTFLOW) atomicOr(bad, 8);
            wk[b] = k;
            wt[2 * b] = T(target[2 * b]);
            wt[2 * b + 1] = T(target[2 * b + 1]);
        }
    }
}

void free_boundaries(labfm_plan* p) {
    cudaFree(p->wall_slot);
    cudaFree(p->wall_n);
    cudaFree(p->bnd_kind);
    cudaFree(p->bnd_target);
    p->wall_slot = nullptr;
    p->wall_n = nullptr;
    p->bnd_kind = nullptr;
    p->bnd_target = nullptr;
    p->n_wall = 0;
}
}  // namespace

int set_walls(labfm_plan* p, int64_t n_wall, const int32_t* nodes, const double* normal, const int32_t* kind,
              const double* target, cudaStream_t st) {
    free_boundaries(p);
    if (n_wall == 0) return LABFM_OK;
    const size_t es = p->dtype == LABFM_F32 ? sizeof(float) : sizeof(double);
    LABFM_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&p->wall_slot), size_t(p->N) * sizeof(int32_t)));
    LABFM_CUDA_TRY(cudaMalloc(&p->wall_n, size_t(n_wall) * 2 * es));
    if (kind) {
        LABFM_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&p->bnd_kind), size_t(n_wall) * sizeof(int32_t)));
        LABFM_CUDA_TRY(cudaMalloc(&p->bnd_target, size_t(n_wall) * 2 * es));
    }
    int* bad = nullptr;
    LABFM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&bad), sizeof(int), st));
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->wall_slot, 0xff, size_t(p->N) * sizeof(int32_t), st);
    if (e == cudaSuccess) {
        if (p->dtype == LABFM_F32)
            k_set_walls<float><<<grid_of(n_wall), 256, 0, st>>>(n_wall, nodes, normal, kind, target, p->N,
                                                                  p->wall_slot, static_cast<float*>(p->wall_n),
                                                                  p->bnd_kind, static_cast<float*>(p->bnd_target),
                                                                  bad);
        else
            k_set_walls<double><<<grid_of(n_wall), 256, 0, st>>>(n_wall, nodes, normal, kind, target, p->N,
                                                                   p->wall_slot, static_cast<double*>(p->wall_n),
                                                                   p->bnd_kind, static_cast<double*>(p->bnd_target),
                                                                   bad);
        e = cudaGetLastError();
    }
    int hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(bad, st);
    if (e != cudaSuccess) return cuda_error(e, "setting the boundaries of a plan");
    if (hbad) {
        free_boundaries(p);
        return set_error(LABFM_EINVAL, (hbad & 1) ? "a boundary node is out of range"
                                       : (hbad & 2) ? "a boundary node is listed twice"
                                       : (hbad & 4) ? "a boundary normal is not of unit length"
                                                    : "unknown boundary kind");
    }
    p->n_wall = n_wall;
    p->device_bytes += int64_t(p->N) * 4 + n_wall * 2 * int64_t(es) + (kind ? n_wall * (4 + 2 * int64_t(es)) : 0);
    return LABFM_OK;
}

}  // namespace labfm

using namespace labfm;

extern "C" int labfm_build_wall_operator(const double* xy, const double* h, const double* s, int64_t N,
                                         double Lx, double Ly, uint32_t periodic_mask, int m, int m_wall,
                                         int64_t n_wall, const int32_t* wall_column, const double* wall_normal,
                                         double h1d_over_s, int32_t* row_ptr, int32_t* col,
                                         int64_t col_capacity, int64_t* nnz_out, double* w, double* kappa,
                                         int32_t* node_status, int64_t* n_failed_out, void* stream) {
    LABFM_NVTX("labfm_build_wall_operator");
    if (!xy || !h || !s || !row_ptr || !nnz_out || !wall_column || !wall_normal)
        return set_error(LABFM_EINVAL, "null pointer argument");
    if (N <= 0 || N >= (int64_t(1) << 31) - 1) return set_error(LABFM_EINVAL, "N out of range");
    if (n_wall <= 0 || n_wall * kColumn > N) return set_error(LABFM_EINVAL, "n_wall out of range");
    for (int mm : {m, m_wall})
        if (mm < 2 || mm > 10 || (mm & 1)) return set_error(LABFM_EINVAL, "orders m, m_wall must be even in [2, 10]");
    if (!(h1d_over_s > 0.0) || !isfinite(h1d_over_s)) return set_error(LABFM_EINVAL, "h1d_over_s must be positive");
    if (col_capacity < 0) return set_error(LABFM_EINVAL, "negative col_capacity");
    const bool query = !col && col_capacity == 0;
    if (!query && (!col || !w || !kappa || !node_status))
        return set_error(LABFM_EINVAL, "null output with col_capacity > 0");
    if (fault_alloc()) return injected_alloc_error("labfm_build_wall_operator");
    cudaStream_t st = as_stream(stream);
    Scratch sc(st);
    int rc;
    // 1. node kinds
    int32_t* kind = nullptr;
    int* bad = nullptr;
    if ((rc = sc.get(&kind, size_t(N))) || (rc = sc.get(&bad, 1))) return rc;
    LABFM_CUDA_TRY(cudaMemsetAsync(kind, 0xff, size_t(N) * sizeof(int32_t), st));
    LABFM_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
    k_mark_columns<<<grid_of(n_wall * kColumn), 256, 0, st>>>(n_wall, wall_column, wall_normal, N, kind, bad);
    LABFM_LAUNCH_CHECK("wall column kernel");
    int hbad = 0;
    LABFM_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    LABFM_CUDA_TRY(cudaStreamSynchronize(st));
    if (hbad)
        return set_error(LABFM_EINVAL, (hbad & 1) ? "a wall column node is out of range"
                                       : (hbad & 2) ? "a node appears in two wall columns"
                                                    : "a wall normal is not of unit length");
    // 2. LABFM stencils of every node
    WallOpArgs A{};
    A.xy = xy;
    A.s = s;
    A.N = N;
    A.Lx = Lx;
    A.Ly = Ly;
    A.px = (periodic_mask & 1u) != 0;
    A.py = (periodic_mask & 2u) != 0;
    A.kind = kind;
    A.wall_column = wall_column;
    A.wall_normal = wall_normal;
    A.h1d_over_s = h1d_over_s;
    A.fd = fd_first_derivative_table();
    int32_t *rpA = nullptr, *colA = nullptr;
    if ((rc = stencils_into(sc, xy, h, N, Lx, Ly, periodic_mask, &rpA, &colA, &A.nnzA))) return rc;
    A.rpA = rpA;
    A.colA = colA;
    // 3. row neighbours of the rows q = 0..4 (indices of wall nodes)
    for (int q = 0; q < kColumn; ++q) {
        double *xy_q = nullptr, *h_q = nullptr;
        if ((rc = sc.get(&xy_q, size_t(2 * n_wall))) || (rc = sc.get(&h_q, size_t(n_wall)))) return rc;
        k_gather_row<<<grid_of(n_wall), 256, 0, st>>>(n_wall, q, wall_column, xy, s, h1d_over_s, xy_q, h_q);
        LABFM_LAUNCH_CHECK("wall row gather kernel");
        int32_t *rpR = nullptr, *colR = nullptr;
        int64_t nnzR = 0;
        if ((rc = stencils_into(sc, xy_q, h_q, n_wall, Lx, Ly, periodic_mask, &rpR, &colR, &nnzR))) return rc;
        A.rpR[q] = rpR;
        A.colR[q] = colR;
    }
    // 4. merged row sizes and row pointers
    int32_t* cnt = nullptr;
    int64_t* total = nullptr;
    void* scan_tmp = nullptr;
    const size_t scan_bytes = exclusive_scan_scratch_bytes(N);
    if ((rc = sc.get(&cnt, size_t(N))) || (rc = sc.get(&total, 1)) ||
        (rc = sc.get(reinterpret_cast<char**>(&scan_tmp), scan_bytes)))
        return rc;
    constexpr int kMergeBlock = 32 * kMergeWarps;
    const int gw = int(std::min<int64_t>((N * 32 + kMergeBlock - 1) / kMergeBlock, 1 << 20));
    k_wall_merge<false><<<gw, kMergeBlock, 0, st>>>(A, cnt, nullptr, nullptr, nullptr, 0, nullptr, nullptr);
    LABFM_LAUNCH_CHECK("wall merge count kernel");
    if ((rc = exclusive_scan_i32(cnt, row_ptr, N, total, scan_tmp, scan_bytes, st))) return rc;
    int64_t nnz = 0;
    LABFM_CUDA_TRY(cudaMemcpyAsync(&nnz, total, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LABFM_CUDA_TRY(cudaStreamSynchronize(st));
    *nnz_out = nnz;
    if (nnz >= (int64_t(1) << 31)) return set_error(LABFM_ECAPACITY, "operator has 2^31 or more entries");
    if (query) return LABFM_OK;
    if (col_capacity < nnz)
        return set_error(LABFM_ECAPACITY,
                         "col_capacity " + std::to_string(col_capacity) + " < required " + std::to_string(nnz));
    // 5. LABFM weights of order m and m_wall on the stencils
    double *wA = nullptr, *kA = nullptr;
    int32_t* stA = nullptr;
    if ((rc = sc.get(&wA, size_t(6) * size_t(std::max<int64_t>(A.nnzA, 1)))) || (rc = sc.get(&kA, size_t(N))) ||
        (rc = sc.get(&stA, size_t(N))))
        return rc;
    if ((rc = labfm_build_weights(xy, h, s, N, Lx, Ly, periodic_mask, rpA, colA, A.nnzA, m, wA, kA, nullptr, stA,
                                  nullptr, st)))
        return rc;
    A.wA = wA;
    A.kA = kA;
    A.stA = stA;
    if (m_wall == m) {
        A.wB = wA;
        A.kB = kA;
        A.stB = stA;
    } else {
        double *wB = nullptr, *kB = nullptr;
        int32_t* stB = nullptr;
        if ((rc = sc.get(&wB, size_t(6) * size_t(std::max<int64_t>(A.nnzA, 1)))) || (rc = sc.get(&kB, size_t(N))) ||
            (rc = sc.get(&stB, size_t(N))))
            return rc;
        if ((rc = labfm_build_weights(xy, h, s, N, Lx, Ly, periodic_mask, rpA, colA, A.nnzA, m_wall, wB, kB,
                                      nullptr, stB, nullptr, st)))
            return rc;
        A.wB = wB;
        A.kB = kB;
        A.stB = stB;
    }
    // 6. the merged operator
    k_wall_merge<true><<<gw, kMergeBlock, 0, st>>>(A, nullptr, row_ptr, col, w, nnz, kappa, node_status);
    LABFM_LAUNCH_CHECK("wall merge kernel");
    if (n_failed_out) {
        unsigned long long* nf = nullptr;
        if ((rc = sc.get(&nf, 1))) return rc;
        LABFM_CUDA_TRY(cudaMemsetAsync(nf, 0, sizeof(*nf), st));
        k_count_failed<<<grid_of(N), 256, 0, st>>>(N, node_status, nf);
        LABFM_LAUNCH_CHECK("failed-node count kernel");
        unsigned long long hf = 0;
        LABFM_CUDA_TRY(cudaMemcpyAsync(&hf, nf, sizeof(hf), cudaMemcpyDeviceToHost, st));
        LABFM_CUDA_TRY(cudaStreamSynchronize(st));
        *n_failed_out = int64_t(hf);
        if (hf > 0) return set_error(LABFM_ESINGULAR, std::to_string(hf) + " node(s) failed; see node_status");
    }
    return LABFM_OK;
}

extern "C" int labfm_plan_set_walls(labfm_plan* p, int64_t n_wall, const int32_t* wall_nodes,
                                    const double* wall_normal, void* stream) {
    LABFM_NVTX("labfm_plan_set_walls");
    if (!p || !p->row_ptr) return set_error(LABFM_EINVAL, "null or empty plan");
    if (n_wall < 0 || n_wall > p->N) return set_error(LABFM_EINVAL, "n_wall out of range");
    if (n_wall > 0 && (!wall_nodes || !wall_normal)) return set_error(LABFM_EINVAL, "null pointer argument");
    if (n_wall > 0 && fault_alloc()) return injected_alloc_error("labfm_plan_set_walls");
    return set_walls(p, n_wall, wall_nodes, wall_normal, nullptr, nullptr, as_stream(stream));
}

extern "C" int labfm_plan_set_boundaries(labfm_plan* p, int64_t n, const int32_t* nodes, const double* normal,
                                         const int32_t* kind, const double* target, const labfm_nscbc* params,
                                         void* stream) {
    LABFM_NVTX("labfm_plan_set_boundaries");
    if (!p || !p->row_ptr) return set_error(LABFM_EINVAL, "null or empty plan");
    if (n < 0 || n > p->N) return set_error(LABFM_EINVAL, "number of boundary nodes out of range");
    if (n > 0 && (!nodes || !normal || !kind || !target || !params))
        return set_error(LABFM_EINVAL, "null pointer argument");
    if (n > 0 && (!(params->sigma >= 0.0) || !(params->L > 0.0) || !(params->mach >= 0.0 && params->mach < 1.0) ||
                  !(params->rho0 > 0.0)))
        return set_error(LABFM_EINVAL, "need sigma >= 0, L > 0, 0 <= mach < 1, rho0 > 0");
    if (n > 0 && fault_alloc()) return injected_alloc_error("labfm_plan_set_boundaries");
    if (n > 0) p->nscbc = *params;
    return set_walls(p, n, nodes, normal, kind, target, as_stream(stream));
}
