// Neighbour search (Section 2 of the paper: the stencil of node i is every node
// j != i with |r_ji| <= 2 h_i) on a uniform cell list, plus the exclusive scan
// used to turn per-row counts into CSR row pointers.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "labfm_internal.cuh"
#include "nvtx.cuh"

namespace labfm {

// ---------------------------------------------------------------- scan

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int64_t kScanTile = int64_t(kScanThreads) * kScanItems;

// Inclusive block scan of one int64 per thread; returns the inclusive prefix
// and writes the block total to *total.
__device__ int64_t block_inclusive_scan(int64_t v, int64_t* warp_sums, int64_t* total) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    for (int off = 1; off < 32; off <<= 1) {
        int64_t n = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += n;
    }
    if (lane == 31) warp_sums[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int64_t w = lane < nw ? warp_sums[lane] : 0;
        for (int off = 1; off < 32; off <<= 1) {
            int64_t n = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += n;
        }
        if (lane < nw) warp_sums[lane] = w;
    }
    __syncthreads();
    int64_t incl = v + (warp > 0 ? warp_sums[warp - 1] : 0);
    if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return incl;
}

__global__ void k_scan_reduce(const int32_t* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
    __shared__ int64_t ws[32];
    __shared__ int64_t tot;
    const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
    int64_t local = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t idx = base + k;
        if (idx < n) local += in[idx];
    }
    block_inclusive_scan(local, ws, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One block: exclusive scan of the per-tile sums, carried across chunks.
__global__ void k_scan_sums(int64_t* __restrict__ sums, int64_t nb, int64_t* __restrict__ total) {
    __shared__ int64_t ws[32];
    __shared__ int64_t tot;
    int64_t carry = 0;
    for (int64_t c0 = 0; c0 < nb; c0 += blockDim.x) {
        const int64_t idx = c0 + threadIdx.x;
        const int64_t v = idx < nb ? sums[idx] : 0;
        const int64_t incl = block_inclusive_scan(v, ws, &tot);
        if (idx < nb) sums[idx] = carry + incl - v;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_apply(const int32_t* in, int32_t* out, int64_t n,
                             const int64_t* __restrict__ sums, const int64_t* __restrict__ total) {
    __shared__ int64_t ws[32];
    const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
    int32_t vals[kScanItems];
    int64_t local = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t idx = base + k;
        vals[k] = idx < n ? in[idx] : 0;
        local += vals[k];
    }
    const int64_t incl = block_inclusive_scan(local, ws, nullptr);
    int64_t run = sums[blockIdx.x] + incl - local;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t idx = base + k;
        if (idx < n) out[idx] = int32_t(run);
        run += vals[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = int32_t(*total);
}

}  // namespace

size_t exclusive_scan_scratch_bytes(int64_t n) {
    const int64_t nb = std::max<int64_t>(1, (n + kScanTile - 1) / kScanTile);
    return size_t(nb) * sizeof(int64_t);
}

int exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int64_t* total_dev,
                       void* scratch, size_t scratch_bytes, cudaStream_t st) {
    const int64_t nb = std::max<int64_t>(1, (n + kScanTile - 1) / kScanTile);
    if (scratch_bytes < size_t(nb) * sizeof(int64_t))
        return set_error(LABFM_EINVAL, "scan scratch too small");
    int64_t* sums = static_cast<int64_t*>(scratch);
    k_scan_reduce<<<unsigned(nb), kScanThreads, 0, st>>>(in, n, sums);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(sums, nb, total_dev);
    k_scan_apply<<<unsigned(nb), kScanThreads, 0, st>>>(in, out, n, sums, total_dev);
    LABFM_LAUNCH_CHECK("exclusive scan");
    return LABFM_OK;
}

// ---------------------------------------------------------------- CSR check

namespace {
__global__ void k_check_row_ptr(const int32_t* __restrict__ rp, int64_t N, int64_t nnz, int* flags) {
    const int64_t gt = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    bool bad = false;
    for (int64_t i = gt; i < N; i += int64_t(gridDim.x) * blockDim.x) bad |= rp[i + 1] < rp[i];
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, 4);
    if (gt == 0) {
        if (rp[0] != 0) atomicOr(flags, 1);
        if (nnz >= 0 && int64_t(rp[N]) != nnz) atomicOr(flags, 2);
    }
}

__global__ void k_check_cols(const int32_t* __restrict__ col, int64_t n, int64_t N, int* flags) {
    bool bad = false;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const int32_t c = col[e];
        bad |= c < 0 || int64_t(c) >= N;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, 8);
}
}  // namespace

int validate_csr(const int32_t* row_ptr, const int32_t* col, int64_t N, int64_t nnz, cudaStream_t st) {
    int* f = nullptr;
    LABFM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&f), sizeof(int), st));
    int flags = 0, total = 0;
    cudaError_t e = cudaMemsetAsync(f, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        const int g = int(std::min<int64_t>((N + 255) / 256, 152 * 8));
        k_check_row_ptr<<<g, 256, 0, st>>>(row_ptr, N, nnz, f);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, f, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, row_ptr + N, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && flags == 0 && total > 0) {
        if (!col) {
            flags = 16;
        } else {
            const int g = int(std::min<int64_t>((int64_t(total) + 255) / 256, 152 * 8));
            k_check_cols<<<g, 256, 0, st>>>(col, total, N, f);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, f, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
    }
    cudaFreeAsync(f, st);
    if (e != cudaSuccess) return cuda_error(e, "checking the CSR");
    if (flags & 1) return set_error(LABFM_EINVAL, "row_ptr[0] is not 0");
    if (flags & 2) return set_error(LABFM_EINVAL, "row_ptr[N] differs from nnz");
    if (flags & 4) return set_error(LABFM_EINVAL, "row_ptr decreases");
    if (flags & 16) return set_error(LABFM_EINVAL, "null col for a non-empty CSR");
    if (flags & 8) return set_error(LABFM_EINVAL, "a column index is outside [0, N)");
    return LABFM_OK;
}

// ---------------------------------------------------------------- cell list

namespace {

struct CellGrid {
    double Lx, Ly;
    double csx, csy;  // cell sizes
    int ncx, ncy;
    bool px, py;
};

__device__ __forceinline__ unsigned long long dbl_bits(double v) {
    return static_cast<unsigned long long>(__double_as_longlong(v));
}

// h range and input validation: a periodic axis takes [0, L), a bounded one
// [0, L] (a wall may lie on the edge of the box).  hmin/hmax are kept as the bit
// patterns of positive doubles, which order like the values.
__global__ void k_bounds(const double* __restrict__ xy, const double* __restrict__ h, int64_t N,
                         double Lx, double Ly, bool px, bool py, unsigned long long* hmin,
                         unsigned long long* hmax, int* bad) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N;
         i += int64_t(gridDim.x) * blockDim.x) {
        const double x = xy[2 * i], y = xy[2 * i + 1], hi = h[i];
        const bool ok = isfinite(x) && isfinite(y) && isfinite(hi) && hi > 0.0 && x >= 0.0 &&
                        (px ? x < Lx : x <= Lx) && y >= 0.0 && (py ? y < Ly : y <= Ly);
        if (!ok) {
            atomicOr(bad, 1);
            continue;
        }
        atomicMin(hmin, dbl_bits(hi));
        atomicMax(hmax, dbl_bits(hi));
    }
}

__device__ __forceinline__ int cell_coord(double x, double cs, int nc) {
    int c = int(floor(x / cs));
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_cell_count(const double* __restrict__ xy, int64_t N, CellGrid g,
                             int32_t* __restrict__ cell_of, int32_t* __restrict__ cell_count) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int cx = cell_coord(xy[2 * i], g.csx, g.ncx);
        const int cy = cell_coord(xy[2 * i + 1], g.csy, g.ncy);
        const int c = cy * g.ncx + cx;
        cell_of[i] = c;
        atomicAdd(cell_count + c, 1);
    }
}

__global__ void k_cell_scatter(int64_t N, const int32_t* __restrict__ cell_of,
                               int32_t* __restrict__ cursor, int32_t* __restrict__ cell_nodes) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int slot = atomicAdd(cursor + cell_of[i], 1);
        cell_nodes[slot] = int32_t(i);
    }
}

// Cell index range [lo, hi] covering [x - r, x + r] along one axis; *all is set
// when the range wraps onto itself (then every cell is visited once).
__device__ __forceinline__ void axis_range(double x, double r, double cs, int nc, bool periodic,
                                           int* lo, int* hi) {
    int a = int(floor((x - r) / cs - 1e-9));
    int b = int(floor((x + r) / cs + 1e-9));
    if (periodic) {
        if (b - a + 1 >= nc) {
            a = 0;
            b = nc - 1;
        }
    } else {
        a = a < 0 ? 0 : a;
        b = b >= nc ? nc - 1 : b;
    }
    *lo = a;
    *hi = b;
}

__device__ __forceinline__ int wrap(int c, int nc) {
    c %= nc;
    return c < 0 ? c + nc : c;
}

// Count (FILL = false) or write (FILL = true) the stencil of each node.
template <bool FILL>
__global__ void k_neighbours(const double* __restrict__ xy, const double* __restrict__ h, int64_t N,
                             CellGrid g, const int32_t* __restrict__ cell_start,
                             const int32_t* __restrict__ cell_nodes, int32_t* __restrict__ counts,
                             const int32_t* __restrict__ row_ptr, int32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N;
         i += int64_t(gridDim.x) * blockDim.x) {
        const double xi = xy[2 * i], yi = xy[2 * i + 1];
        const double two_h = 2.0 * h[i];
        const double rad2 = __dmul_rn(two_h, two_h);
        int xlo, xhi, ylo, yhi;
        axis_range(xi, two_h, g.csx, g.ncx, g.px, &xlo, &xhi);
        axis_range(yi, two_h, g.csy, g.ncy, g.py, &ylo, &yhi);
        int32_t cnt = 0;
        int64_t dst = FILL ? row_ptr[i] : 0;
        for (int cy = ylo; cy <= yhi; ++cy) {
            const int wy = g.py ? wrap(cy, g.ncy) : cy;
            for (int cx = xlo; cx <= xhi; ++cx) {
                const int wx = g.px ? wrap(cx, g.ncx) : cx;
                const int c = wy * g.ncx + wx;
                const int k1 = cell_start[c + 1];
                for (int k = cell_start[c]; k < k1; ++k) {
                    const int j = cell_nodes[k];
                    if (j == i) continue;
                    const double dx = min_image(__dsub_rn(xy[2 * j], xi), g.Lx, g.px);
                    const double dy = min_image(__dsub_rn(xy[2 * j + 1], yi), g.Ly, g.py);
                    const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
                    if (d2 <= rad2) {
                        if (FILL) out[dst + cnt] = j;
                        ++cnt;
                    }
                }
            }
        }
        if (!FILL) counts[i] = cnt;
    }
}

// Sort each row by ascending j: warp per row, rank of every entry among its row.
constexpr int kSortCap = 512;
constexpr int kSortWarps = 8;

__global__ void k_sort_rows(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ tmp,
                            int32_t* __restrict__ col, int64_t N) {
    __shared__ int32_t buf[kSortWarps][kSortCap];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    for (int64_t i = blockIdx.x * int64_t(kSortWarps) + warp; i < N;
         i += int64_t(gridDim.x) * kSortWarps) {
        const int r0 = row_ptr[i];
        const int n = row_ptr[i + 1] - r0;
        const int32_t* src = tmp + r0;
        if (n <= kSortCap) {
            for (int e = lane; e < n; e += 32) buf[warp][e] = src[e];
            __syncwarp();
            src = buf[warp];
        }
        for (int e = lane; e < n; e += 32) {
            const int v = src[e];
            int rank = 0;
            for (int k = 0; k < n; ++k) rank += src[k] < v;
            col[r0 + rank] = v;
        }
        __syncwarp();
    }
}

template <typename T>
int scratch_alloc(T** p, size_t count, cudaStream_t st) {
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T), st);
    if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync (neighbour search scratch)");
    return LABFM_OK;
}

struct ScratchList {
    static constexpr int kCap = 16;
    cudaStream_t st;
    void* ptrs[kCap] = {};
    int n = 0;
    explicit ScratchList(cudaStream_t s) : st(s) {}
    void add(void* p) {
        if (n < kCap) ptrs[n++] = p;
    }
    ~ScratchList() {
        for (int k = 0; k < n; ++k)
            if (ptrs[k]) cudaFreeAsync(ptrs[k], st);
    }
};

}  // namespace
}  // namespace labfm

using namespace labfm;

extern "C" int labfm_build_stencils(const double* xy, const double* h, int64_t N, double Lx,
                                    double Ly, uint32_t periodic_mask, int32_t* row_ptr,
                                    int32_t* col, int64_t col_capacity, int64_t* nnz_out,
                                    void* stream) {
    LABFM_NVTX("labfm_build_stencils");
    if (!xy || !h || !row_ptr || !nnz_out) return set_error(LABFM_EINVAL, "null pointer argument");
    if (N <= 0 || N >= (int64_t(1) << 31) - 1) return set_error(LABFM_EINVAL, "N out of range");
    if (!(Lx > 0.0) || !(Ly > 0.0) || !isfinite(Lx) || !isfinite(Ly))
        return set_error(LABFM_EINVAL, "domain size must be positive and finite");
    if (col_capacity < 0) return set_error(LABFM_EINVAL, "negative col_capacity");
    if (fault_alloc()) return injected_alloc_error("labfm_build_stencils");
    if (col && fault_capacity()) {
        *nnz_out = col_capacity + 1;
        return set_error(LABFM_ECAPACITY, "col_capacity " + std::to_string(col_capacity) + " < required " +
                                              std::to_string(col_capacity + 1) +
                                              " (injected: LABFM_FAULT=capacity)");
    }
    cudaStream_t st = as_stream(stream);
    ScratchList scratch(st);

    // 1. h range and validation
    struct Bounds {
        unsigned long long hmin, hmax;
        int bad, pad;
    };
    Bounds* b_dev = nullptr;
    int rc = scratch_alloc(&b_dev, 1, st);
    if (rc) return rc;
    scratch.add(b_dev);
    Bounds init{~0ull, 0ull, 0, 0};
    LABFM_CUDA_TRY(cudaMemcpyAsync(b_dev, &init, sizeof(init), cudaMemcpyHostToDevice, st));
    const int nblk = int(std::min<int64_t>((N + 255) / 256, 65535));
    k_bounds<<<nblk, 256, 0, st>>>(xy, h, N, Lx, Ly, (periodic_mask & 1u) != 0, (periodic_mask & 2u) != 0,
                                   &b_dev->hmin, &b_dev->hmax, &b_dev->bad);
    LABFM_LAUNCH_CHECK("bounds kernel");
    Bounds bh{};
    LABFM_CUDA_TRY(cudaMemcpyAsync(&bh, b_dev, sizeof(bh), cudaMemcpyDeviceToHost, st));
    LABFM_CUDA_TRY(cudaStreamSynchronize(st));
    if (bh.bad)
        return set_error(LABFM_EINVAL,
                         "a node lies outside the box ([0, L) on a periodic axis, [0, L] on a bounded "
                         "one) or has a non-positive or non-finite h");
    double hmin, hmax;
    memcpy(&hmin, &bh.hmin, sizeof(double));
    memcpy(&hmax, &bh.hmax, sizeof(double));

    // 2. cell grid: cells of about h_min, at most ~4 N + 64 of them
    CellGrid g{};
    g.Lx = Lx;
    g.Ly = Ly;
    g.px = (periodic_mask & 1u) != 0;
    g.py = (periodic_mask & 2u) != 0;
    double cs = hmin;
    const double max_cells = 4.0 * double(N) + 64.0;
    if ((Lx / cs) * (Ly / cs) > max_cells) cs = sqrt(Lx * Ly / max_cells);
    g.ncx = std::max(1, int(std::min(Lx / cs, 1.0e9)));
    g.ncy = std::max(1, int(std::min(Ly / cs, 1.0e9)));
    g.csx = Lx / g.ncx;
    g.csy = Ly / g.ncy;
    const int64_t ncells = int64_t(g.ncx) * g.ncy;

    int32_t *cell_of = nullptr, *cell_count = nullptr, *cell_start = nullptr, *cursor = nullptr,
            *cell_nodes = nullptr;
    int64_t* total = nullptr;
    void* scan_tmp = nullptr;
    const size_t scan_bytes =
        std::max(exclusive_scan_scratch_bytes(ncells), exclusive_scan_scratch_bytes(N));
    if ((rc = scratch_alloc(&cell_of, size_t(N), st))) return rc;
    scratch.add(cell_of);
    if ((rc = scratch_alloc(&cell_count, size_t(ncells), st))) return rc;
    scratch.add(cell_count);
    if ((rc = scratch_alloc(&cell_start, size_t(ncells) + 1, st))) return rc;
    scratch.add(cell_start);
    if ((rc = scratch_alloc(&cursor, size_t(ncells), st))) return rc;
    scratch.add(cursor);
    if ((rc = scratch_alloc(&cell_nodes, size_t(N), st))) return rc;
    scratch.add(cell_nodes);
    if ((rc = scratch_alloc(&total, 2, st))) return rc;
    scratch.add(total);
    if ((rc = scratch_alloc(reinterpret_cast<char**>(&scan_tmp), scan_bytes, st))) return rc;
    scratch.add(scan_tmp);

    LABFM_CUDA_TRY(cudaMemsetAsync(cell_count, 0, size_t(ncells) * sizeof(int32_t), st));
    k_cell_count<<<nblk, 256, 0, st>>>(xy, N, g, cell_of, cell_count);
    LABFM_LAUNCH_CHECK("cell count kernel");
    if ((rc = exclusive_scan_i32(cell_count, cell_start, ncells, total, scan_tmp, scan_bytes, st)))
        return rc;
    LABFM_CUDA_TRY(cudaMemcpyAsync(cursor, cell_start, size_t(ncells) * sizeof(int32_t),
                                   cudaMemcpyDeviceToDevice, st));
    k_cell_scatter<<<nblk, 256, 0, st>>>(N, cell_of, cursor, cell_nodes);
    LABFM_LAUNCH_CHECK("cell scatter kernel");

    // 3. count, scan into row_ptr
    const int nblk_n = int(std::min<int64_t>((N + 127) / 128, 1 << 20));
    k_neighbours<false><<<nblk_n, 128, 0, st>>>(xy, h, N, g, cell_start, cell_nodes, row_ptr,
                                                nullptr, nullptr);
    LABFM_LAUNCH_CHECK("neighbour count kernel");
    if ((rc = exclusive_scan_i32(row_ptr, row_ptr, N, total, scan_tmp, scan_bytes, st))) return rc;
    int64_t nnz = 0;
    LABFM_CUDA_TRY(cudaMemcpyAsync(&nnz, total, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LABFM_CUDA_TRY(cudaStreamSynchronize(st));
    *nnz_out = nnz;
    if (nnz >= (int64_t(1) << 31))
        return set_error(LABFM_ECAPACITY, "stencil has 2^31 or more entries (int32 CSR)");
    if (!col && col_capacity == 0) return LABFM_OK;  // size query
    if (!col || col_capacity < nnz)
        return set_error(LABFM_ECAPACITY, "col_capacity " + std::to_string(col_capacity) +
                                              " < required " + std::to_string(nnz));

    // 4. fill unsorted rows into a temporary, then sort each row into col
    int32_t* tmp = nullptr;
    if ((rc = scratch_alloc(&tmp, size_t(nnz), st))) return rc;
    scratch.add(tmp);
    k_neighbours<true><<<nblk_n, 128, 0, st>>>(xy, h, N, g, cell_start, cell_nodes, nullptr,
                                               row_ptr, tmp);
    LABFM_LAUNCH_CHECK("neighbour fill kernel");
    const int nblk_s = int(std::min<int64_t>((N + kSortWarps - 1) / kSortWarps, 1 << 20));
    k_sort_rows<<<nblk_s, 32 * kSortWarps, 0, st>>>(row_ptr, tmp, col, N);
    LABFM_LAUNCH_CHECK("row sort kernel");
    return LABFM_OK;
}
