// Device helpers shared by the time-step kernels (step.cu) and the adjoint
// kernels (adjoint.cu): RK coefficients, packed node state, operator-record
// loads, the fused 12-derivative gather and the pointwise right-hand side.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "labfm_internal.cuh"

namespace labfm {
namespace {

// RK3(2)4[2R+]C (Kennedy, Carpenter & Lewis 2000), the low-storage scheme named
// in Section 7: sub-diagonal a_{k+1,k} and weights b_k.
constexpr double kRkA[3] = {11847461282814.0 / 36547543011857.0,
                            3943225443063.0 / 7078155732230.0,
                            -346793006927.0 / 4029903576067.0};
constexpr double kRkB[4] = {1017324711453.0 / 9774461848756.0,
                            8237718856693.0 / 13685301971492.0,
                            57731312506979.0 / 19404895981398.0,
                            -101169746363290.0 / 37734290219643.0};

// ---------------------------------------------------------------- vector helpers

// Chunks of 4 stencil entries each lane loads before its gathers (1 or 2).
#ifndef LABFM_GATHER_UNROLL
#define LABFM_GATHER_UNROLL 1
#endif
// Cache hint for the operator streams (col and weights, read once per launch):
// 0 = read-only path (ld.global.nc), 1 = evict-first (ld.global.cs),
// 2 = read-only without L1 allocation, so that L1 keeps the gathered fields.
#ifndef LABFM_STREAM_HINT
#define LABFM_STREAM_HINT 1
#endif
constexpr int kUnroll = LABFM_GATHER_UNROLL;

__device__ __forceinline__ float4 ld_na(const float4* p) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}
__device__ __forceinline__ int4 ld_na(const int4* p) {
    int4 v;
    asm("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}
__device__ __forceinline__ double2 ld_na(const double2* p) {
    double2 v;
    asm("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
}

template <typename V>
__device__ __forceinline__ V ld_stream(const V* p) {
#if LABFM_STREAM_HINT == 2
    return ld_na(p);
#elif LABFM_STREAM_HINT == 1
    return __ldcs(p);
#else
    return __ldg(p);
#endif
}

// `o` receives 4 values of an operator stream starting at o + off.
template <int K>
__device__ __forceinline__ void load4(const float* p, float (&o)[K], int off) {
    const float4 t = ld_stream(reinterpret_cast<const float4*>(p));
    o[off] = t.x;
    o[off + 1] = t.y;
    o[off + 2] = t.z;
    o[off + 3] = t.w;
}
template <int K>
__device__ __forceinline__ void load4(const double* p, double (&o)[K], int off) {
    const double2 a = ld_stream(reinterpret_cast<const double2*>(p));
    const double2 b = ld_stream(reinterpret_cast<const double2*>(p) + 1);
    o[off] = a.x;
    o[off + 1] = a.y;
    o[off + 2] = b.x;
    o[off + 3] = b.y;
}
template <int K>
__device__ __forceinline__ void load4i(const int32_t* p, int (&o)[K], int off) {
    const int4 t = ld_stream(reinterpret_cast<const int4*>(p));
    o[off] = t.x;
    o[off + 1] = t.y;
    o[off + 2] = t.z;
    o[off + 3] = t.w;
}

// Operator layout.  0: operator-major streams col[nnz], w[5][nnz], wf[nnz].
// 1: chunk records: for every 4-entry chunk of a row, its four columns and the
//    four weights of each of the five RHS operators in one contiguous record
//    (96 bytes in F32); the filter has its own records (columns, kappa w^hyp).
// 2: interleaved records: kIL consecutive chunks form a block stored
//    component-major (the kIL x 4 columns, then the kIL x 4 weights of each
//    operator), so that lanes taking consecutive chunks read contiguous bytes
//    with every 16-byte load instruction (64 bytes per 4 lanes for kIL = 4, 128
//    bytes per 8 lanes for kIL = 8, the shared-memory bank width of a
//    quarter-warp).
// 3: as 2 with kIL = 4 for F64; for F32 the paired layout below (three 32-byte
//    loads per chunk).
#ifndef LABFM_CHUNK_AOS
#define LABFM_CHUNK_AOS 3
#endif
#ifndef LABFM_CHUNK_IL
#define LABFM_CHUNK_IL 4
#endif
constexpr int kIL = LABFM_CHUNK_IL;

template <typename T>
struct ChunkBytes {
    static constexpr int rhs = 16 + 20 * int(sizeof(T));  // int4 col + 5 x 4 weights
    static constexpr int filt = 16 + 4 * int(sizeof(T));  // int4 col + 4 weights
};

// Byte offsets of the parts of chunk c (entries 4c .. 4c + 3) in the record
// streams: its four columns, the four weights of RHS operator d, its four
// filter columns and filter weights.
template <typename T>
struct Rec {
    static constexpr int64_t W4 = 4 * int64_t(sizeof(T));  // four weights
#if LABFM_CHUNK_AOS >= 2
    static constexpr int64_t BB = int64_t(kIL) * ChunkBytes<T>::rhs;    // bytes per RHS block
    static constexpr int64_t FB = int64_t(kIL) * ChunkBytes<T>::filt;   // bytes per filter block
    __host__ __device__ static int64_t col(int64_t c) { return (c / kIL) * BB + (c % kIL) * 16; }
    __host__ __device__ static int64_t w(int64_t c, int d) {
        return (c / kIL) * BB + kIL * 16 + d * kIL * W4 + (c % kIL) * W4;
    }
    __host__ __device__ static int64_t fcol(int64_t c) { return (c / kIL) * FB + (c % kIL) * 16; }
    __host__ __device__ static int64_t fw(int64_t c) { return (c / kIL) * FB + kIL * 16 + (c % kIL) * W4; }
    static size_t rhs_bytes(int64_t nnz_pad) { return size_t((nnz_pad / 4 + kIL - 1) / kIL) * BB; }
    static size_t filt_bytes(int64_t nnz_pad) { return size_t((nnz_pad / 4 + kIL - 1) / kIL) * FB; }
#else
    __host__ __device__ static int64_t col(int64_t c) { return c * ChunkBytes<T>::rhs; }
    __host__ __device__ static int64_t w(int64_t c, int d) { return c * ChunkBytes<T>::rhs + 16 + d * W4; }
    __host__ __device__ static int64_t fcol(int64_t c) { return c * ChunkBytes<T>::filt; }
    __host__ __device__ static int64_t fw(int64_t c) { return c * ChunkBytes<T>::filt + 16; }
    static size_t rhs_bytes(int64_t nnz_pad) { return size_t(nnz_pad / 4) * ChunkBytes<T>::rhs; }
    static size_t filt_bytes(int64_t nnz_pad) { return size_t(nnz_pad / 4) * ChunkBytes<T>::filt; }
#endif
    // entry-level accessors (entry e of the padded operator)
    __host__ __device__ static int64_t col_e(int64_t e) { return col(e >> 2) + 4 * (e & 3); }
    __host__ __device__ static int64_t w_e(int64_t e, int d) { return w(e >> 2, d) + sizeof(T) * (e & 3); }
    __host__ __device__ static int64_t fcol_e(int64_t e) { return fcol(e >> 2) + 4 * (e & 3); }
    __host__ __device__ static int64_t fw_e(int64_t e) { return fw(e >> 2) + sizeof(T) * (e & 3); }
};

#if LABFM_CHUNK_AOS == 3
static_assert(LABFM_CHUNK_IL == 4, "the paired F32 layout has four chunks per block");
// Paired F32 layout (256-bit loads): a block of four chunks is three 128-byte
// segments; in each, chunk q owns the 32 contiguous bytes at q * 32:
// segment 0 [columns | w^x], segment 1 [w^y | w^xx], segment 2 [w^xy | w^yy].
// A lane reads its chunk with three 32-byte loads and the four lanes of a group
// read whole 128-byte lines.  Filter blocks: [columns | kappa w^hyp] per chunk.
template <>
struct Rec<float> {
    static constexpr int64_t W4 = 16;
    static constexpr int64_t BB = 384;
    static constexpr int64_t FB = 128;
    __host__ __device__ static int64_t col(int64_t c) { return (c >> 2) * BB + (c & 3) * 32; }
    __host__ __device__ static int64_t w(int64_t c, int d) {
        return (c >> 2) * BB + ((d + 1) >> 1) * 128 + (c & 3) * 32 + ((d + 1) & 1) * 16;
    }
    __host__ __device__ static int64_t fcol(int64_t c) { return (c >> 2) * FB + (c & 3) * 32; }
    __host__ __device__ static int64_t fw(int64_t c) { return fcol(c) + 16; }
    static size_t rhs_bytes(int64_t nnz_pad) { return size_t((nnz_pad / 4 + 3) / 4) * BB; }
    static size_t filt_bytes(int64_t nnz_pad) { return size_t((nnz_pad / 4 + 3) / 4) * FB; }
    __host__ __device__ static int64_t col_e(int64_t e) { return col(e >> 2) + 4 * (e & 3); }
    __host__ __device__ static int64_t w_e(int64_t e, int d) { return w(e >> 2, d) + 4 * (e & 3); }
    __host__ __device__ static int64_t fcol_e(int64_t e) { return fcol(e >> 2) + 4 * (e & 3); }
    __host__ __device__ static int64_t fw_e(int64_t e) { return fw(e >> 2) + 4 * (e & 3); }
};

// 32-byte evict-first load of eight floats (32-byte aligned) with an L2
// prefetch-size hint (0: none, 1: 128 bytes, 2: 256 bytes around the access).
// The operator streams are read in order, so the 256-byte fill brings in the
// stream's next line early without a register or an instruction: measured on the
// 262,144-node m = 8 step, stage 115.7 -> 111.1 us and filter 49.0 -> 47.6 us
// (128 bytes: no change).
#ifndef LABFM_LD_PREFETCH
#define LABFM_LD_PREFETCH 2
#endif
#if LABFM_LD_PREFETCH == 2
#define LABFM_LD8 "ld.global.cs.L2::256B.v8.f32"
#elif LABFM_LD_PREFETCH == 1
#define LABFM_LD8 "ld.global.cs.L2::128B.v8.f32"
#else
#define LABFM_LD8 "ld.global.cs.v8.f32"
#endif
__device__ __forceinline__ void ld8(const void* p, float (&v)[8]) {
    asm(LABFM_LD8 " {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(p));
}
#endif

// Slot of padded row entry e (0 <= e < plen, plen a multiple of 4) within its
// row.  With LABFM_ENTRY_PERM, each segment of up to 16 entries (nc chunks) is
// transposed so that chunk q holds entries q, q + nc, q + 2 nc, q + 3 nc: lanes
// that take consecutive chunks then gather consecutive stencil entries (mostly
// neighbouring nodes) with each load instruction.
#ifndef LABFM_ENTRY_PERM
#define LABFM_ENTRY_PERM 1
#endif
__device__ __forceinline__ int entry_slot(int e, int plen) {
#if LABFM_ENTRY_PERM
    const int base = e & ~15;
    const int nc = min(16, plen - base) >> 2;
    const int r = e - base;
    return base + 4 * (r % nc) + r / nc;
#else
    (void)plen;
    return e;
#endif
}

// Node state (ln rho, u, v) packed for one-instruction gathers: float4 for F32
// (w unused), two double2 for F64.
template <typename T> struct Packed;
template <> struct Packed<float> { float4 v; };
template <> struct Packed<double> { double2 au; double2 vp; };

__device__ __forceinline__ void unpack(const Packed<float>* p, int j, float& a, float& u, float& v) {
    const float4 t = __ldg(&p[j].v);
    a = t.x;
    u = t.y;
    v = t.z;
}
__device__ __forceinline__ void unpack(const Packed<double>* p, int j, double& a, double& u, double& v) {
    const double2 t = __ldg(&p[j].au);
    a = t.x;
    u = t.y;
    v = __ldg(&p[j].vp.x);
}
// Plain (coherent) loads for a buffer that the same kernel also writes.
__device__ __forceinline__ void unpack_rw(const Packed<float>* p, int j, float& a, float& u, float& v) {
    const float4 t = p[j].v;
    a = t.x;
    u = t.y;
    v = t.z;
}
__device__ __forceinline__ void unpack_rw(const Packed<double>* p, int j, double& a, double& u, double& v) {
    const double2 t = p[j].au;
    a = t.x;
    u = t.y;
    v = p[j].vp.x;
}
__device__ __forceinline__ void store(Packed<float>* p, int64_t j, float a, float u, float v) {
    p[j].v = make_float4(a, u, v, 0.0f);
}
__device__ __forceinline__ void store(Packed<double>* p, int64_t j, double a, double u, double v) {
    p[j].au = make_double2(a, u);
    p[j].vp = make_double2(v, 0.0);
}

// Field access policies for the gathers: structure-of-arrays (public API) or
// packed (inside labfm_rk_step).
template <typename T>
struct SoA {
    const T* a;
    const T* u;
    const T* v;
    __device__ __forceinline__ void get(int j, T& x, T& y, T& z) const {
        x = __ldg(a + j);
        y = __ldg(u + j);
        z = __ldg(v + j);
    }
};
template <typename T>
struct AoS {
    const Packed<T>* p;
    __device__ __forceinline__ void get(int j, T& x, T& y, T& z) const { unpack(p, j, x, y, z); }
};

// Compensated (Kahan) accumulation used for the F32 second-derivative and
// filter sums; the F64 path adds plainly.
template <typename T, bool KAHAN>
struct Acc {
    T s = T(0), c = T(0);
    __device__ __forceinline__ void add(T x) {
        if (KAHAN) {
            const T y = x - c;
            const T t = s + y;
            c = (t - s) - y;
            s = t;
        } else {
            s += x;
        }
    }
    __device__ __forceinline__ T value() const { return KAHAN ? s - c : s; }
};

template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

template <typename T>
struct PlanView {
    int64_t N;
    int64_t nnz_pad;
    const int32_t* row_ptr;
    const int32_t* col;
    const T* w;   // 5 x nnz_pad
    const T* wf;  // nnz_pad
    const T* inv_s;
    const double* dt_node;  // per-node time step, or null for a uniform dt
    int pf;                 // L2 prefetch distance of the F32 record stream, in iterations (0: off)
    const int32_t* wall_slot;  // per node: boundary slot, -1 in the fluid (null: no boundaries)
    const T* wall_n;           // per slot: inward unit normal (n_x, n_y)
    int64_t n_lo, n_hi;        // nodes [n_lo, n_hi) of this launch (plain stage and filter grids)
    const int32_t* bnd_kind;   // per slot: LABFM_WALL, LABFM_INFLOW, LABFM_OUTFLOW (null: all walls)
    const T* bnd_target;       // per slot: (u_xi,IN, u_eta,IN) of an inflow, p_inf (first) of an outflow
    T sigma, Lb, mach, rho0;   // relaxation coefficient, length, Mach number, reference density
};

// Operator loads of one 4-entry chunk starting at entry e (a multiple of 4).
template <typename T, int K>
__device__ __forceinline__ void load_rhs_chunk(const PlanView<T>& P, int e, int (&cj)[K],
                                               T (&wx)[K], T (&wy)[K], T (&wxx)[K],
                                               T (&wxy)[K], T (&wyy)[K], int off) {
#if LABFM_CHUNK_AOS
    const char* base = reinterpret_cast<const char*>(P.w);
    const int64_t c = e >> 2;
#if LABFM_CHUNK_AOS == 3
    if constexpr (std::is_same<T, float>::value) {
        float a[8], b[8], d[8];
        ld8(base + Rec<float>::col(c), a);
        ld8(base + Rec<float>::w(c, 1), b);
        ld8(base + Rec<float>::w(c, 3), d);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            cj[off + k] = __float_as_int(a[k]);
            wx[off + k] = a[4 + k];
            wy[off + k] = b[k];
            wxx[off + k] = b[4 + k];
            wxy[off + k] = d[k];
            wyy[off + k] = d[4 + k];
        }
        return;
    }
#endif
    load4i(reinterpret_cast<const int32_t*>(base + Rec<T>::col(c)), cj, off);
    load4(reinterpret_cast<const T*>(base + Rec<T>::w(c, 0)), wx, off);
    load4(reinterpret_cast<const T*>(base + Rec<T>::w(c, 1)), wy, off);
    load4(reinterpret_cast<const T*>(base + Rec<T>::w(c, 2)), wxx, off);
    load4(reinterpret_cast<const T*>(base + Rec<T>::w(c, 3)), wxy, off);
    load4(reinterpret_cast<const T*>(base + Rec<T>::w(c, 4)), wyy, off);
#else
    const int64_t nz = P.nnz_pad;
    load4i(P.col + e, cj, off);
    load4(P.w + e, wx, off);
    load4(P.w + nz + e, wy, off);
    load4(P.w + 2 * nz + e, wxx, off);
    load4(P.w + 3 * nz + e, wxy, off);
    load4(P.w + 4 * nz + e, wyy, off);
#endif
}

template <typename T, int K>
__device__ __forceinline__ void load_filt_chunk(const PlanView<T>& P, int e, int (&cj)[K],
                                                T (&wf)[K], int off) {
#if LABFM_CHUNK_AOS
    const char* base = reinterpret_cast<const char*>(P.wf);
    const int64_t c = e >> 2;
#if LABFM_CHUNK_AOS == 3
    if constexpr (std::is_same<T, float>::value) {
        float v[8];
        ld8(base + Rec<float>::fcol(c), v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            cj[off + k] = __float_as_int(v[k]);
            wf[off + k] = v[4 + k];
        }
        return;
    }
#endif
    load4i(reinterpret_cast<const int32_t*>(base + Rec<T>::fcol(c)), cj, off);
    load4(reinterpret_cast<const T*>(base + Rec<T>::fw(c)), wf, off);
#else
    load4i(P.col + e, cj, off);
    load4(P.wf + e, wf, off);
#endif
}

template <typename T>
PlanView<T> view(const labfm_plan* p) {
    return PlanView<T>{p->N,        p->nnz_pad,  p->row_ptr, p->col, static_cast<const T*>(p->w),
                       static_cast<const T*>(p->wf), static_cast<const T*>(p->inv_s), p->dt_node,
                       p->prefetch, p->wall_slot, static_cast<const T*>(p->wall_n), 0, p->N,
                       p->bnd_kind, static_cast<const T*>(p->bnd_target), T(p->nscbc.sigma), T(p->nscbc.L),
                       T(p->nscbc.mach), T(p->nscbc.rho0)};
}

// Chunk loaders for the gathers: from the plan's record stream in global memory,
// or from a copy of a contiguous range of its blocks in shared memory.
// Shortest row (padded entries) whose record stream the stage and filter kernels
// prefetch: m = 8 and 10 stencils (~100-220 entries, 6 or more iterations of a lane
// group) gained 4-8 %.  With plain launches and 128-thread blocks m = 6 stencils
// (~60 entries) lost 2-3 % and m = 4 (~35) neither; with programmatic launches and
// one-warp blocks the m = 6 step gains 5.7 % (512^2 lattice: 310.2 -> 292.6 us with
// a threshold of 48 entries instead of 80), while a threshold of 32 leaves m = 6 as
// at 48 and makes the m = 4 step 1 % slower.
constexpr int kPrefetchMinRow = 48;

// Programmatic dependent launch (sm_90 and later).  The plain-grid stage, filter,
// recording-stage, adjoint pass A and B, filter-transpose, pack and unpack launches
// carry programmatic stream serialization (launch_pdl): such a kernel may start
// while the kernel before it in the stream still runs, once every block of that
// kernel has signalled launch_dependents, and griddepcontrol.wait holds it until
// that kernel has completed and its writes are visible.  Without the launch
// attribute both instructions are no-ops.  LABFM_PDL=0 builds plain launches.
#ifndef LABFM_PDL
#define LABFM_PDL 1
#endif
// Record blocks of its row (16 entries each) a lane group fetches into L2 before
// the wait.  Measured on the 262,144-node m = 8 step (per step, no events):
// 470.8 us with plain launches; with programmatic launches 453.6 / 448.0 / 448.7 /
// 456.7 / 494.2 us for 1 / 2 / 3 / 4 / 6 blocks.
constexpr int kPdlPrefetchBlocks = 2;

__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Start of a plain-grid stage (FILTER = false) or filter (FILTER = true) launch,
// run by every lane (gl: its lane in the group of node i; i < 0: no node): lets
// the next launch of the stream start, fetches into L2 the first record blocks of
// row i (the operator is constant, so this overlaps the previous kernel's last
// blocks), then waits for the previous kernel.  Nothing the previous kernel writes
// is read before the wait.
template <typename T, bool FILTER, int G>
__device__ __forceinline__ void launch_prologue(const PlanView<T>& P, int i, int gl) {
#if LABFM_PDL
    pdl_launch_dependents();
#if LABFM_CHUNK_AOS == 3
    if constexpr (std::is_same<T, float>::value) {
        if (i >= 0) {
            const int e0 = P.row_ptr[i], e1 = P.row_ptr[i + 1];
            if constexpr (FILTER) {
                // one 128-byte filter block per lane
                for (int q = gl; q < kPdlPrefetchBlocks; q += G) {
                    const int ep = e0 + 16 * q;
                    if (ep < e1) {
                        const char* a = reinterpret_cast<const char*>(P.wf) + Rec<float>::fcol(ep >> 2);
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
                    }
                }
            } else if (gl < 3) {
                // lanes 0-2: one 128-byte segment each of every RHS block
#pragma unroll
                for (int q = 0; q < kPdlPrefetchBlocks; ++q) {
                    const int ep = e0 + 16 * q;
                    if (ep < e1) {
                        const char* a = reinterpret_cast<const char*>(P.w) + Rec<float>::col(ep >> 2) + gl * 128;
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
                    }
                }
            }
        }
    }
#endif
    pdl_wait();
#else
    (void)P;
    (void)i;
    (void)gl;
#endif
}

// Launch of a kernel that starts with launch_prologue, with programmatic stream
// serialization (LABFM_PDL and the plan's setting; otherwise a plain launch): the kernel may start while
// the previous kernel of the stream finishes, and waits for it in launch_prologue
// before reading anything that kernel writes.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(const labfm_plan* p, void (*kernel)(KArgs...), int grid, int block, cudaStream_t st,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(unsigned(block));
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = (LABFM_PDL && p->programmatic) ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename T>
struct GlobalChunks {
    static constexpr bool kColAhead = LABFM_CHUNK_AOS >= 2;
#if LABFM_CHUNK_AOS == 3
    static constexpr bool kPaired = std::is_same<T, float>::value;
#else
    static constexpr bool kPaired = false;
#endif
    static constexpr bool kPrefetch = kPaired;
    const PlanView<T>& P;
    // L2 prefetch of segment `seg` of the block holding the chunk of entry e
    __device__ __forceinline__ void prefetch(int e, int seg) const {
        const char* a = reinterpret_cast<const char*>(P.w) + Rec<T>::col(e >> 2) + seg * 128;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
    template <int K>
    __device__ __forceinline__ void load(int e, int (&cj)[K], T (&wx)[K], T (&wy)[K], T (&wxx)[K],
                                         T (&wxy)[K], T (&wyy)[K], int off) const {
        load_rhs_chunk(P, e, cj, wx, wy, wxx, wxy, wyy, off);
    }
#if LABFM_CHUNK_AOS >= 2
    // The part of a chunk loaded one iteration ahead: its columns (and, in the
    // paired layout, w^x, which shares their 32 bytes).
    __device__ __forceinline__ void load_head(int e, int (&cj)[4], T (&wx)[4]) const {
        const char* base = reinterpret_cast<const char*>(P.w) + Rec<T>::col(e >> 2);
        if constexpr (kPaired) {
#if LABFM_CHUNK_AOS == 3
            float v[8];
            ld8(base, v);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                cj[k] = __float_as_int(v[k]);
                wx[k] = v[4 + k];
            }
#endif
        } else {
            load4i(reinterpret_cast<const int32_t*>(base), cj, 0);
        }
    }
    // The rest of the chunk.
    __device__ __forceinline__ void load_tail(int e, T (&wx)[4], T (&wy)[4], T (&wxx)[4], T (&wxy)[4],
                                              T (&wyy)[4]) const {
        const char* base = reinterpret_cast<const char*>(P.w);
        const int64_t c = e >> 2;
        if constexpr (kPaired) {
#if LABFM_CHUNK_AOS == 3
            float v[8], u[8];
            ld8(base + Rec<float>::w(c, 1), v);
            ld8(base + Rec<float>::w(c, 3), u);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                wy[k] = v[k];
                wxx[k] = v[4 + k];
                wxy[k] = u[k];
                wyy[k] = u[4 + k];
            }
#endif
        } else {
            load4(reinterpret_cast<const T*>(base + Rec<T>::w(c, 0)), wx, 0);
            load4(reinterpret_cast<const T*>(base + Rec<T>::w(c, 1)), wy, 0);
            load4(reinterpret_cast<const T*>(base + Rec<T>::w(c, 2)), wxx, 0);
            load4(reinterpret_cast<const T*>(base + Rec<T>::w(c, 3)), wxy, 0);
            load4(reinterpret_cast<const T*>(base + Rec<T>::w(c, 4)), wyy, 0);
        }
    }
#endif
};

// Column indices one chunk ahead (LABFM_COL_AHEAD): a lane loads the columns of
// its next chunk while it gathers and sums the current one, so that the next
// gathers can be issued as soon as that iteration starts.  Measured 3 % faster
// with layout 2 and no faster with the paired layout (whose three 32-byte loads
// per chunk already leave the columns first), so it is off by default.
#ifndef LABFM_COL_AHEAD
#define LABFM_COL_AHEAD 0
#endif

// The 12 derivatives of eq. icns at node i over its padded entries [e0, e1):
// d[0..1] = (a_x, a_y), d[2..6] = (u_x, u_y, u_xx, u_xy, u_yy), d[7..11] = same
// for v, each L^d_i(phi) = sum_j (phi_j - phi_i) w^d_ji.  Every lane of the
// group returns them; an idle group (i < 0, e0 = e1) returns zeros.
template <typename T, int G, bool KAHAN, class F, class Ld>
__device__ __forceinline__ void gather_derivatives_ld(const Ld& ld, const F& fld, int i, int e0,
                                                      int e1, int gl, T ai, T ui, T vi, T (&d)[12]) {
    T ax = 0, ay = 0, ux = 0, uy = 0, vx = 0, vy = 0;
    Acc<T, KAHAN> uxx, uxy, uyy, vxx, vxy, vyy;
#if LABFM_COL_AHEAD
    if constexpr (Ld::kColAhead) {
        int cn[4] = {i, i, i, i};
        T wxn[4] = {T(0), T(0), T(0), T(0)};
        int e = e0 + 4 * gl;
        if (e < e1) ld.load_head(e, cn, wxn);
        for (; e < e1; e += 4 * G) {
            const int cj[4] = {cn[0], cn[1], cn[2], cn[3]};
            T wx[4] = {wxn[0], wxn[1], wxn[2], wxn[3]};
            if (e + 4 * G < e1) ld.load_head(e + 4 * G, cn, wxn);
            T aj[4], uj[4], vj[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) fld.get(cj[k], aj[k], uj[k], vj[k]);
            T wy[4], wxx[4], wxy[4], wyy[4];
            ld.load_tail(e, wx, wy, wxx, wxy, wyy);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const T da = aj[k] - ai, du = uj[k] - ui, dv = vj[k] - vi;
                ax = fma(da, wx[k], ax);
                ay = fma(da, wy[k], ay);
                ux = fma(du, wx[k], ux);
                uy = fma(du, wy[k], uy);
                vx = fma(dv, wx[k], vx);
                vy = fma(dv, wy[k], vy);
                uxx.add(du * wxx[k]);
                uxy.add(du * wxy[k]);
                uyy.add(du * wyy[k]);
                vxx.add(dv * wxx[k]);
                vxy.add(dv * wxy[k]);
                vyy.add(dv * wyy[k]);
            }
        }
    } else
#endif
    // kUnroll 4-entry chunks per iteration (chunks gl, gl + G, ... of this
    // pass): all their operator loads are issued before the gathers
    for (int e = e0 + 4 * gl; e < e1; e += 4 * kUnroll * G) {
        if constexpr (Ld::kPrefetch) {
            // lanes 0-2 of the group fetch into L2 one 128-byte segment each of the
            // block they will read pf iterations later (within the row; rows shorter
            // than kPrefetchMinRow entries, where it was measured slower, skip it)
            const int pf = ld.P.pf;
            if (pf > 0 && e1 - e0 >= kPrefetchMinRow) {
                const int ep = e + 4 * kUnroll * G * pf;
                if (ep < e1 && gl < 3) ld.prefetch(ep, gl);
            }
        }
        int cj[4 * kUnroll];
        T wx[4 * kUnroll], wy[4 * kUnroll], wxx[4 * kUnroll], wxy[4 * kUnroll], wyy[4 * kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int eu = e + 4 * u * G;
            if (u == 0 || eu < e1) {
                ld.load(eu, cj, wx, wy, wxx, wxy, wyy, 4 * u);
            } else {
#pragma unroll
                for (int k = 4 * u; k < 4 * u + 4; ++k) {
                    cj[k] = i;  // the node itself with zero weight adds exactly 0
                    wx[k] = wy[k] = wxx[k] = wxy[k] = wyy[k] = T(0);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 4 * kUnroll; ++k) {
            T aj, uj, vj;
            fld.get(cj[k], aj, uj, vj);
            const T da = aj - ai, du = uj - ui, dv = vj - vi;
            ax = fma(da, wx[k], ax);
            ay = fma(da, wy[k], ay);
            ux = fma(du, wx[k], ux);
            uy = fma(du, wy[k], uy);
            vx = fma(dv, wx[k], vx);
            vy = fma(dv, wy[k], vy);
            uxx.add(du * wxx[k]);
            uxy.add(du * wxy[k]);
            uyy.add(du * wyy[k]);
            vxx.add(dv * wxx[k]);
            vxy.add(dv * wxy[k]);
            vyy.add(dv * wyy[k]);
        }
    }
    d[0] = group_sum<G>(ax);
    d[1] = group_sum<G>(ay);
    d[2] = group_sum<G>(ux);
    d[3] = group_sum<G>(uy);
    d[7] = group_sum<G>(vx);
    d[8] = group_sum<G>(vy);
    if (KAHAN) {
        // the compensations are summed separately and applied once
        d[4] = group_sum<G>(uxx.s) - group_sum<G>(uxx.c);
        d[5] = group_sum<G>(uxy.s) - group_sum<G>(uxy.c);
        d[6] = group_sum<G>(uyy.s) - group_sum<G>(uyy.c);
        d[9] = group_sum<G>(vxx.s) - group_sum<G>(vxx.c);
        d[10] = group_sum<G>(vxy.s) - group_sum<G>(vxy.c);
        d[11] = group_sum<G>(vyy.s) - group_sum<G>(vyy.c);
    } else {
        d[4] = group_sum<G>(uxx.s);
        d[5] = group_sum<G>(uxy.s);
        d[6] = group_sum<G>(uyy.s);
        d[9] = group_sum<G>(vxx.s);
        d[10] = group_sum<G>(vxy.s);
        d[11] = group_sum<G>(vyy.s);
    }
}

template <typename T, int G, bool KAHAN, class F>
__device__ __forceinline__ void gather_derivatives(const PlanView<T>& P, const F& fld, int i,
                                                   int gl, T ai, T ui, T vi, T (&d)[12]) {
    int e0 = 0, e1 = 0;
    if (i >= 0) {
        e0 = P.row_ptr[i];
        e1 = P.row_ptr[i + 1];
    }
    gather_derivatives_ld<T, G, KAHAN>(GlobalChunks<T>{P}, fld, i, e0, e1, gl, ai, ui, vi, d);
}

__device__ __forceinline__ float exp_neg(float a) { return expf(-a); }
__device__ __forceinline__ double exp_neg(double a) { return exp(-a); }

// Pointwise right-hand side of eq. icns from the derivatives.  F32 weights are
// nondimensional (w s^l), so the sums are scaled by s^-1 or s^-2 here.
template <typename T, bool SCALED>
__device__ __forceinline__ void pointwise_rhs(const T (&d)[12], T a, T u, T v, T inv_s, T c2, T mu,
                                              T gx, T gy, T& Ra, T& Ru, T& Rv) {
    const T s1 = SCALED ? inv_s : T(1);
    const T s2 = SCALED ? inv_s * inv_s : T(1);
    const T ax = d[0] * s1, ay = d[1] * s1;
    const T ux = d[2] * s1, uy = d[3] * s1, uxx = d[4] * s2, uxy = d[5] * s2, uyy = d[6] * s2;
    const T vx = d[7] * s1, vy = d[8] * s1, vxx = d[9] * s2, vxy = d[10] * s2, vyy = d[11] * s2;
    const T nu = mu * exp_neg(a);
    const T third = T(1) / T(3);
    const T four_thirds = T(4) / T(3);
    Ra = -(u * ax + v * ay) - (ux + vy);
    Ru = -(u * ux + v * uy) - c2 * ax + nu * (four_thirds * uxx + uyy + third * vxy) + gx;
    Rv = -(u * vx + v * vy) - c2 * ay + nu * (four_thirds * vyy + vxx + third * uxy) + gy;
}

template <typename T>
struct Phys {
    T c2, mu, gx, gy;
};

__device__ __forceinline__ float exp_pos(float a) { return expf(a); }
__device__ __forceinline__ double exp_pos(double a) { return exp(a); }

// Right-hand side at a no-slip wall node (Section 7.1): u = 0 is held (R_u = R_v =
// 0) and ln rho follows eq. lodilnro with u_xi = 0,
//   R_a = -(L4 + L1) / (rho c^2) - d u_eta / d eta,
//   L1 = (u_xi - c)/2 (dp/dxi - rho c du_xi/dxi) (eq. Ldef), dp/dxi = c^2 rho d ln rho/dxi,
//   L4 = L1 + rho c g.n (the incoming wave of the wall; the paper prints a factor
//   2 on rho c g.n, with which eq. lodiu would not hold u_xi at zero: factor 1 is
//   the reading taken),
// with xi along the inward normal n and eta along t = (-n_y, n_x); the derivatives
// are those of the wall rows (one-sided differences along n, 1D LABFM along t).
template <typename T, bool SCALED>
__device__ __forceinline__ void wall_rhs(const T (&d)[12], T a, T inv_s, T c2, T gx, T gy, T nx, T ny,
                                         T& Ra, T& Ru, T& Rv) {
    const T s1 = SCALED ? inv_s : T(1);
    const T ax = d[0] * s1, ay = d[1] * s1;
    const T ux = d[2] * s1, uy = d[3] * s1, vx = d[7] * s1, vy = d[8] * s1;
    const T tx = -ny, ty = nx;
    const T a_xi = ax * nx + ay * ny;
    const T du_xi = nx * (ux * nx + uy * ny) + ny * (vx * nx + vy * ny);
    const T du_eta = tx * (ux * tx + uy * ty) + ty * (vx * tx + vy * ty);
    const T rho = exp_pos(a);
    const T c = sqrt(c2);
    const T dp = c2 * rho * a_xi;
    const T L1 = T(0.5) * (T(0) - c) * (dp - rho * c * du_xi);
    const T L4 = L1 + rho * c * (nx * gx + ny * gy);
    Ra = -(L4 + L1) / (rho * c2) - du_eta;
    Ru = T(0);
    Rv = T(0);
}

// Right-hand side at an outflow or inflow node (Section 7.1): eq. lodi in the
// boundary frame (xi along the inward normal n, eta along t = (-n_y, n_x)) with
// L2 = 0 (isothermal), the outgoing waves from eq. Ldef
//   L1 = (u_xi - c)/2 (dp/dxi - rho c du_xi/dxi), L3 = u_xi du_eta/dxi (outflow),
// and the incoming ones
//   outflow (eq. outflowL): L4 = sigma/(2 L) c (1 - M^2)(p - p_inf) + (1 - M) T4 + V4;
//   inflow: L3 = sigma c / L (u_eta - u_eta,IN) + T3 + V3,
//           L4 = sigma rho0 c^2 (1 - M^2) / L (u_xi - u_xi,IN) + T4 + V4
// (each relaxation drives its own velocity component: the reading taken where the
// printed inflow relaxations are exchanged), with
//   T4 = -1/2 (u_eta dp/deta + p du_eta/deta + rho c u_eta du_xi/deta),
//   V4 = mu c / 2 (4/3 u_xi,xixi + u_xi,etaeta + 1/3 u_eta,xieta),
//   T3 = -(u_eta du_eta/deta + dp/deta / rho),
//   V3 = mu / rho (4/3 u_eta,etaeta + u_eta,xixi + 1/3 u_xi,xieta),
// and the viscous conditions: dtau_etaxi/deta = 0 at an outflow (the viscous force
// of eq. lodiu becomes 4/3 u_xi,xixi - 2/3 u_eta,xieta), dtau_etaeta/deta = 0 at an
// inflow (that of eq. lodiv becomes u_eta,xixi + u_xi,xieta).
template <typename T, bool SCALED>
__device__ __forceinline__ void open_rhs(const T (&d)[12], T a, T u, T v, T inv_s, const Phys<T>& ph, T nx,
                                         T ny, int kind, T t0, T t1, T sigma, T Lb, T mach, T rho0,
                                         T& Ra, T& Ru, T& Rv) {
    const T s1 = SCALED ? inv_s : T(1);
    const T s2 = SCALED ? inv_s * inv_s : T(1);
    const T ax = d[0] * s1, ay = d[1] * s1;
    const T ux = d[2] * s1, uy = d[3] * s1, uxx = d[4] * s2, uxy = d[5] * s2, uyy = d[6] * s2;
    const T vx = d[7] * s1, vy = d[8] * s1, vxx = d[9] * s2, vxy = d[10] * s2, vyy = d[11] * s2;
    const T tx = -ny, ty = nx;
    // first derivatives in the boundary frame
    const T a_xi = nx * ax + ny * ay, a_eta = tx * ax + ty * ay;
    const T u_n = nx * ux + ny * uy, u_t = tx * ux + ty * uy;  // du/dxi, du/deta
    const T v_n = nx * vx + ny * vy, v_t = tx * vx + ty * vy;
    const T u_xi = nx * u + ny * v, u_eta = tx * u + ty * v;
    const T uxi_xi = nx * u_n + ny * v_n, uxi_eta = nx * u_t + ny * v_t;
    const T ueta_xi = tx * u_n + ty * v_n, ueta_eta = tx * u_t + ty * v_t;
    // second derivatives: p . H . r for the Hessians of u and v
    const T u_nn = nx * nx * uxx + 2 * nx * ny * uxy + ny * ny * uyy;
    const T u_tt = tx * tx * uxx + 2 * tx * ty * uxy + ty * ty * uyy;
    const T u_nt = nx * tx * uxx + (nx * ty + ny * tx) * uxy + ny * ty * uyy;
    const T v_nn = nx * nx * vxx + 2 * nx * ny * vxy + ny * ny * vyy;
    const T v_tt = tx * tx * vxx + 2 * tx * ty * vxy + ty * ty * vyy;
    const T v_nt = nx * tx * vxx + (nx * ty + ny * tx) * vxy + ny * ty * vyy;
    const T uxi_xixi = nx * u_nn + ny * v_nn, uxi_etaeta = nx * u_tt + ny * v_tt, uxi_xieta = nx * u_nt + ny * v_nt;
    const T ueta_xixi = tx * u_nn + ty * v_nn, ueta_etaeta = tx * u_tt + ty * v_tt, ueta_xieta = tx * u_nt + ty * v_nt;
    const T c2 = ph.c2, c = sqrt(c2), mu = ph.mu;
    const T rho = exp_pos(a);
    const T p = c2 * rho, p_xi = c2 * rho * a_xi, p_eta = c2 * rho * a_eta;
    const T L1 = T(0.5) * (u_xi - c) * (p_xi - rho * c * uxi_xi);
    const T third = T(1) / T(3), four_thirds = T(4) / T(3), two_thirds = T(2) / T(3);
    const T visc_xi = four_thirds * uxi_xixi + uxi_etaeta + third * ueta_xieta;
    const T visc_eta = four_thirds * ueta_etaeta + ueta_xixi + third * uxi_xieta;
    const T T4 = T(-0.5) * (u_eta * p_eta + p * ueta_eta + rho * c * u_eta * uxi_eta);
    const T V4 = T(0.5) * mu * c * visc_xi;
    T L3, L4, vxi, veta;
    if (kind == LABFM_OUTFLOW) {
        L3 = u_xi * ueta_xi;
        L4 = sigma / (T(2) * Lb) * c * (T(1) - mach * mach) * (p - t0) + (T(1) - mach) * T4 + V4;
        vxi = four_thirds * uxi_xixi - two_thirds * ueta_xieta;
        veta = visc_eta;
    } else {
        const T T3 = -(u_eta * ueta_eta + p_eta / rho);
        const T V3 = mu / rho * visc_eta;
        L3 = sigma * c / Lb * (u_eta - t1) + T3 + V3;
        L4 = sigma * rho0 * c2 * (T(1) - mach * mach) / Lb * (u_xi - t0) + T4 + V4;
        vxi = visc_xi;
        veta = ueta_xixi + uxi_xieta;
    }
    const T g_xi = nx * ph.gx + ny * ph.gy, g_eta = tx * ph.gx + ty * ph.gy;
    Ra = -(L4 + L1) / (rho * c2) - u_eta * a_eta - ueta_eta;
    const T Rxi = -(L4 - L1) / (rho * c) - u_eta * uxi_eta + mu / rho * vxi + g_xi;
    const T Reta = -L3 - u_eta * ueta_eta - p_eta / rho + mu / rho * veta + g_eta;
    Ru = nx * Rxi + tx * Reta;
    Rv = ny * Rxi + ty * Reta;
}

// eq. icns, or the boundary's right-hand side at a boundary node of a plan with
// boundaries (a wall, an outflow or an inflow).
template <typename T, bool SCALED, bool WALL>
__device__ __forceinline__ void node_rhs(const PlanView<T>& P, int i, const T (&d)[12], T a, T u, T v,
                                         T inv_s, const Phys<T>& ph, T& Ra, T& Ru, T& Rv) {
    if (WALL) {
        const int slot = P.wall_slot[i];
        if (slot >= 0) {
            const T nx = P.wall_n[2 * slot], ny = P.wall_n[2 * slot + 1];
            const int kind = P.bnd_kind ? P.bnd_kind[slot] : LABFM_WALL;
            if (kind == LABFM_WALL)
                wall_rhs<T, SCALED>(d, a, inv_s, ph.c2, ph.gx, ph.gy, nx, ny, Ra, Ru, Rv);
            else
                open_rhs<T, SCALED>(d, a, u, v, inv_s, ph, nx, ny, kind, P.bnd_target[2 * slot],
                                    P.bnd_target[2 * slot + 1], P.sigma, P.Lb, P.mach, P.rho0, Ra, Ru, Rv);
            return;
        }
    }
    pointwise_rhs<T, SCALED>(d, a, u, v, inv_s, ph.c2, ph.mu, ph.gx, ph.gy, Ra, Ru, Rv);
}

// The eight combinations of a node's derivatives through which the transpose of
// eq. icns with respect to the node's own state depends on them (physical units):
// a_x, a_y, u_x, u_y, v_x, v_y and the viscous sums 4/3 u_xx + u_yy + 1/3 v_xy,
// 4/3 v_yy + v_xx + 1/3 u_xy.  Kept per stage by the recording time step, so that
// the reverse sweep need not gather the derivatives again.
template <typename T> struct D8;
template <> struct D8<float> { float4 q[2]; };
template <> struct D8<double> { double2 q[4]; };

template <typename T, bool SCALED>
__device__ __forceinline__ void own_coeffs(const T (&d)[12], T inv_s, T (&c)[8]) {
    const T s1 = SCALED ? inv_s : T(1);
    const T s2 = SCALED ? inv_s * inv_s : T(1);
    const T third = T(1) / T(3);
    const T four_thirds = T(4) / T(3);
    c[0] = d[0] * s1;
    c[1] = d[1] * s1;
    c[2] = d[2] * s1;
    c[3] = d[3] * s1;
    c[4] = d[7] * s1;
    c[5] = d[8] * s1;
    c[6] = four_thirds * (d[4] * s2) + d[6] * s2 + third * (d[10] * s2);
    c[7] = four_thirds * (d[11] * s2) + d[9] * s2 + third * (d[5] * s2);
}

__device__ __forceinline__ void d8_store(D8<float>* p, int64_t i, const float (&c)[8]) {
    p[i].q[0] = make_float4(c[0], c[1], c[2], c[3]);
    p[i].q[1] = make_float4(c[4], c[5], c[6], c[7]);
}
__device__ __forceinline__ void d8_store(D8<double>* p, int64_t i, const double (&c)[8]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) p[i].q[k] = make_double2(c[2 * k], c[2 * k + 1]);
}
__device__ __forceinline__ void d8_load(const D8<float>* p, int64_t i, float (&c)[8]) {
    const float4 a = p[i].q[0], b = p[i].q[1];
    c[0] = a.x;
    c[1] = a.y;
    c[2] = a.z;
    c[3] = a.w;
    c[4] = b.x;
    c[5] = b.y;
    c[6] = b.z;
    c[7] = b.w;
}
__device__ __forceinline__ void d8_load(const D8<double>* p, int64_t i, double (&c)[8]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double2 t = p[i].q[k];
        c[2 * k] = t.x;
        c[2 * k + 1] = t.y;
    }
}

}  // namespace
}  // namespace labfm
