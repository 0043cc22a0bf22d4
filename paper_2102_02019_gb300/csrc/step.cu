// Time-step kernels: the fused neighbour-gather right-hand side of the
// isothermal Navier-Stokes equations (Section 7, eq. icns), the RK3(2)4[2R+]C
// stage update fused into it, the hyperviscous filter (Section 6) and the time
// step of eq. dt.  Also the packing of a weight set into a plan.
//
// Layout (per plan): rows padded to multiples of 4 entries.  Every 4-entry
// chunk of a row is one contiguous record holding its four column indices and
// the four weights of each RHS operator (d/dx, d/dy, d2/dx2, d2/dxdy, d2/dy2):
// 96 bytes in F32, read with six 16-byte loads.  The filter has its own records
// (four columns, four kappa_i w^hyp_ji).  A node is served by a group of G
// lanes; lane l of the group takes the chunks l, l + G, l + 2G, ... of the row.
// The 12 partial sums are reduced across the group with xor shuffles.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <new>
#include <string>
#include <type_traits>

#include "bulk.cuh"
#include "gather.cuh"
#include "labfm_internal.cuh"

namespace labfm {
namespace {

// ---------------------------------------------------------------- kernels

// The fused gather kernels (stage, right-hand side) run one-warp blocks, so that
// every warp retires on its own instead of waiting for the slowest warp of a
// larger block (with programmatic launches, per step: m = 8 451.1 -> 445.1 us,
// m = 10 370.4 -> 365.0 us, m = 6 316.5 -> 310.3 us, m = 4 230.7 -> 225.8 us
// against 128-thread blocks; 64-thread blocks in between).  The register budget
// is set in resident threads per SM: a budget for 1024 (64 registers) had been
// faster than the unconstrained allocation while the lanes' own loads were the
// only bytes in flight; with the L2 prefetch of the record stream the natural 72
// registers (896 threads per SM) are faster (m = 8: 111.4 -> 106.7 us, m = 10:
// 599 -> 572 us), so the bound asks for no more than 768.
constexpr int kGatherBlock = 32;
#ifndef LABFM_STAGE_MIN_THREADS
#define LABFM_STAGE_MIN_THREADS 768
#endif
#define LABFM_STAGE_BOUNDS \
    __launch_bounds__(kGatherBlock, (sizeof(T) == 4 ? LABFM_STAGE_MIN_THREADS : 768) / kGatherBlock)

template <typename T, int G, bool KAHAN, bool SCALED, bool WALL = false>
__global__ void LABFM_STAGE_BOUNDS k_rhs_soa(PlanView<T> P, SoA<T> in, T* __restrict__ out, Phys<T> ph) {
    const int64_t gt = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t node = gt / G;
    const int gl = int(gt % G);
    const int i = node < P.N ? int(node) : -1;
    T ai = 0, ui = 0, vi = 0;
    if (i >= 0) in.get(i, ai, ui, vi);
    T d[12];
    gather_derivatives<T, G, KAHAN>(P, in, i, gl, ai, ui, vi, d);
    if (i >= 0 && gl == 0) {
        T Ra, Ru, Rv;
        const T is = SCALED ? P.inv_s[i] : T(1);
        node_rhs<T, SCALED, WALL>(P, i, d, ai, ui, vi, is, ph, Ra, Ru, Rv);
        out[i] = Ra;
        out[P.N + i] = Ru;
        out[2 * P.N + i] = Rv;
    }
}

// The RK stage update at node i from its 12 derivatives: F = R(X_in);
// Q_out = Q_in + dt_i b_k F; X_out = Q_out + dt_i (a - b) F (skipped when X_out
// is null).  Q_in may equal Q_out, and Q_in may equal X_in (first stage, where
// X = Q).  dt_i is the uniform dt or the plan's per-node dt.  Lane 0 of the
// group stores.  WALL: R is the wall's right-hand side at the plan's wall nodes.
template <typename T, bool SCALED, bool WALL = false>
__device__ __forceinline__ void stage_epilogue(const PlanView<T>& P, int i, int gl, const T (&d)[12],
                                               T ai, T ui, T vi, const Packed<T>* X_in,
                                               const Packed<T>* Q_in, Packed<T>* Q_out,
                                               Packed<T>* X_out, double dt, double bk, double ck,
                                               const Phys<T>& ph) {
    if (i >= 0 && gl == 0) {
        T Ra, Ru, Rv;
        const T is = SCALED ? P.inv_s[i] : T(1);
        node_rhs<T, SCALED, WALL>(P, i, d, ai, ui, vi, is, ph, Ra, Ru, Rv);
        const double dti = P.dt_node ? P.dt_node[i] : dt;
        const T cb = T(dti * bk), cx = T(dti * ck);
        T qa, qu, qv;
        if (Q_in == X_in) {
            qa = ai;
            qu = ui;
            qv = vi;
        } else {
            unpack_rw(Q_in, i, qa, qu, qv);
        }
        qa = fma(cb, Ra, qa);
        qu = fma(cb, Ru, qu);
        qv = fma(cb, Rv, qv);
        store(Q_out, i, qa, qu, qv);
        if (X_out) store(X_out, i, fma(cx, Ra, qa), fma(cx, Ru, qu), fma(cx, Rv, qv));
    }
}

// One fused RK stage at node i (i < 0: an idle group that still joins the
// shuffles).
template <typename T, int G, bool KAHAN, bool SCALED, bool WALL = false>
__device__ __forceinline__ void stage_node(const PlanView<T>& P, int i, int gl,
                                           const Packed<T>* X_in, const Packed<T>* Q_in,
                                           Packed<T>* Q_out, Packed<T>* X_out, double dt,
                                           double bk, double ck, const Phys<T>& ph) {
    const AoS<T> fld{X_in};
    T ai = 0, ui = 0, vi = 0;
    if (i >= 0) fld.get(i, ai, ui, vi);
    T d[12];
    gather_derivatives<T, G, KAHAN>(P, fld, i, gl, ai, ui, vi, d);
    stage_epilogue<T, SCALED, WALL>(P, i, gl, d, ai, ui, vi, X_in, Q_in, Q_out, X_out, dt, bk, ck, ph);
}

// Nodes per work-queue tile of the persistent stage kernel, per warp.
constexpr int kTileRows = 4;
#ifndef LABFM_PERSIST_BLOCK_TILES
#define LABFM_PERSIST_BLOCK_TILES 1
#endif

// PERSIST = false: one group of G lanes per node over a full grid.
// PERSIST = true: a grid of (SMs x resident blocks); every warp repeatedly takes
// the next tile of kTileRows * (32 / G) consecutive nodes from an atomic ticket
// (*counter, zeroed before the launch), so that uneven stencils and mixed
// instances balance dynamically across the GPU.

// WALL (plain grid only): plans with walls, whose wall nodes take the wall's
// right-hand side.
#ifndef LABFM_PERSIST_MIN_THREADS
#define LABFM_PERSIST_MIN_THREADS 896
#endif
// The work-queue instantiation keeps 896 resident threads per SM (at most 73
// registers; left to itself it takes 78 and fits 768).
template <typename T, int G, bool KAHAN, bool SCALED, bool PERSIST, bool WALL = false>
__global__ void __launch_bounds__(kGatherBlock, (sizeof(T) == 4 ? (PERSIST ? LABFM_PERSIST_MIN_THREADS
                                                                          : LABFM_STAGE_MIN_THREADS)
                                                                : 768) / kGatherBlock)
    k_stage(PlanView<T> P, const Packed<T>* X_in, const Packed<T>* Q_in,
                        Packed<T>* Q_out, Packed<T>* X_out, double dt, double bk, double ck,
                        Phys<T> ph, int* counter) {
    static_assert(!(PERSIST && WALL), "plans with walls run the plain grid");
    if (!PERSIST) {
        const int64_t gt = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
        const int64_t node = P.n_lo + gt / G;
        const int i = node < P.n_hi ? int(node) : -1;
        launch_prologue<T, false, G>(P, i, int(gt % G));
        stage_node<T, G, KAHAN, SCALED, WALL>(P, i, int(gt % G), X_in, Q_in, Q_out, X_out, dt, bk, ck, ph);
        return;
    }
    constexpr int per_warp = 32 / G;
    const int lane = threadIdx.x & 31;
#if LABFM_PERSIST_BLOCK_TILES
    // the block claims kGatherBlock / G consecutive nodes at a time and its warps
    // take them together, as a block of the plain grid would (neighbouring nodes'
    // gathers share the SM's L1); the counter balances the blocks
    // The next tile is claimed when the current one starts, so the counter's round
    // trip overlaps the work; s_tile[b] holds the tile of the current pass.
    __shared__ int s_tile[2];
    constexpr int tile = kGatherBlock / G;
    const int64_t ntiles = (P.N + tile - 1) / tile;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile[0] = atomicAdd(counter, 1);
    __syncthreads();
    for (int b = 0;; b ^= 1) {
        const int t = s_tile[b];
        if (t >= ntiles) break;
        int next = 0;
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);
        const int64_t node = int64_t(t) * tile + warp * per_warp + lane / G;
        const int i = node < P.N ? int(node) : -1;
        stage_node<T, G, KAHAN, SCALED>(P, i, lane % G, X_in, Q_in, Q_out, X_out, dt, bk, ck, ph);
        if (threadIdx.x == 0) s_tile[b ^ 1] = next;
        __syncthreads();  // the next tile is published; every warp has read s_tile[b]
    }
#else
    constexpr int tile = kTileRows * per_warp;
    const int64_t ntiles = (P.N + tile - 1) / tile;
    while (true) {
        int t = 0;
        if (lane == 0) t = atomicAdd(counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) break;
#pragma unroll 1
        for (int r = 0; r < kTileRows; ++r) {
            const int64_t node = int64_t(t) * tile + r * per_warp + lane / G;
            const int i = node < P.N ? int(node) : -1;
            stage_node<T, G, KAHAN, SCALED>(P, i, lane % G, X_in, Q_in, Q_out, X_out, dt, bk, ck, ph);
        }
    }
#endif
}

// The stage kernel of the recording time step: k_stage (plain grid) that also
// stores the node's eight derivative combinations for the reverse sweep.
template <typename T, int G, bool KAHAN, bool SCALED>
__global__ void LABFM_STAGE_BOUNDS k_stage_rec(PlanView<T> P, const Packed<T>* X_in, const Packed<T>* Q_in,
                                               Packed<T>* Q_out, Packed<T>* X_out, double dt, double bk,
                                               double ck, Phys<T> ph, D8<T>* __restrict__ Dout) {
    const int64_t gt = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t node = gt / G;
    const int gl = int(gt % G);
    const int i = node < P.N ? int(node) : -1;
    launch_prologue<T, false, G>(P, i, gl);
    const AoS<T> fld{X_in};
    T ai = 0, ui = 0, vi = 0;
    if (i >= 0) fld.get(i, ai, ui, vi);
    T d[12];
    gather_derivatives<T, G, KAHAN>(P, fld, i, gl, ai, ui, vi, d);
    stage_epilogue<T, SCALED>(P, i, gl, d, ai, ui, vi, X_in, Q_in, Q_out, X_out, dt, bk, ck, ph);
    if (i >= 0 && gl == 0) {
        T c[8];
        own_coeffs<T, SCALED>(d, SCALED ? P.inv_s[i] : T(1), c);
        d8_store(Dout, i, c);
    }
}

// ---------------------------------------------------------------- staged stage kernel
//
// F32 stage kernel with the operator stream staged through shared memory by the
// bulk-copy (TMA) engine.  The nodes are cut into rounds of kRoundWarps x 32/G
// consecutive nodes, one per group of G lanes.  The interleaved blocks holding a
// round's chunks are one contiguous byte range of the plan, so one
// cp.async.bulk moves a round into a ring slot whose mbarrier counts the bytes.
// CTA b takes rounds b, b + gridDim.x, ... and keeps S rounds in flight, so the
// copy engine, not the registers of the consumer warps, holds the loads in
// flight.  Neighbour fields are gathered from global memory as in k_stage.  A
// wait that runs out (the plan's limit, 1 s by default) sets *status =
// LABFM_ETIMEOUT; the CTA then lets its copies in flight land (waiting at most
// kBulkDrainNs for each) and returns.
constexpr int kBulkBlock = 128;
constexpr int kRoundWarps = kBulkBlock / 32;
constexpr uint64_t kBulkDrainNs = 1000000000ull;

template <int G>
constexpr int round_nodes() {
    return kRoundWarps * (32 / G);
}

struct RoundRange {
    int64_t off;     // byte offset of the round's first block in the RHS record stream
    uint32_t bytes;  // whole blocks, a multiple of 16
};

__device__ __forceinline__ RoundRange round_range(const int32_t* row_ptr, int64_t N, int64_t r, int rn) {
    const int64_t n0 = r * rn;
    const int64_t n1 = n0 + rn < N ? n0 + rn : N;
    const int64_t c0 = row_ptr[n0] >> 2;
    const int64_t c1 = row_ptr[n1] >> 2;
    const int64_t b0 = c0 / kIL;
    const int64_t b1 = (c1 + kIL - 1) / kIL;
    return {b0 * Rec<float>::BB, uint32_t((b1 - b0) * Rec<float>::BB)};
}

// Chunk loads from a ring slot holding the blocks from byte `off` of the stream.
struct SharedChunks {
    static constexpr bool kColAhead = false;
    static constexpr bool kPrefetch = false;
    __device__ __forceinline__ void prefetch(int, int) const {}
    const unsigned char* slot;
    int64_t off;
    template <int K>
    __device__ __forceinline__ void load(int e, int (&cj)[K], float (&wx)[K], float (&wy)[K],
                                         float (&wxx)[K], float (&wxy)[K], float (&wyy)[K],
                                         int o) const {
        const int64_t c = e >> 2;
        const int4 ci = *reinterpret_cast<const int4*>(slot + (Rec<float>::col(c) - off));
        cj[o] = ci.x;
        cj[o + 1] = ci.y;
        cj[o + 2] = ci.z;
        cj[o + 3] = ci.w;
        get4(c, 0, wx, o);
        get4(c, 1, wy, o);
        get4(c, 2, wxx, o);
        get4(c, 3, wxy, o);
        get4(c, 4, wyy, o);
    }
    template <int K>
    __device__ __forceinline__ void get4(int64_t c, int d, float (&w)[K], int o) const {
        const float4 v = *reinterpret_cast<const float4*>(slot + (Rec<float>::w(c, d) - off));
        w[o] = v.x;
        w[o + 1] = v.y;
        w[o + 2] = v.z;
        w[o + 3] = v.w;
    }
};

__device__ __forceinline__ void issue_round(const PlanView<float>& P, int64_t r, int rn,
                                            unsigned char* slot, uint64_t* bar, uint64_t policy) {
    const RoundRange rr = round_range(P.row_ptr, P.N, r, rn);
    mbar_arrive_expect_tx(smem_u32(bar), rr.bytes);
    if (rr.bytes)
        bulk_g2s(smem_u32(slot), reinterpret_cast<const char*>(P.w) + rr.off, rr.bytes, smem_u32(bar),
                 policy);
}

template <int G, int S>
__global__ void __launch_bounds__(kBulkBlock)
    k_stage_bulk(PlanView<float> P, const Packed<float>* X_in, const Packed<float>* Q_in,
                 Packed<float>* Q_out, Packed<float>* X_out, double dt, double bk, double ck,
                 Phys<float> ph, uint32_t slot_bytes, int* status, uint64_t wait_ns) {
    extern __shared__ __align__(128) unsigned char ring[];
    __shared__ __align__(8) uint64_t full[S];
    constexpr int RN = round_nodes<G>();
    const int t = threadIdx.x;
    const int64_t nrounds = (P.N + RN - 1) / RN;
    if (t == 0) {
#pragma unroll
        for (int k = 0; k < S; ++k) mbar_init(smem_u32(&full[k]), 1);
        mbar_fence_init();
    }
    __syncthreads();
    uint64_t policy = 0;
    if (t == 0) {
        policy = l2_evict_first_policy();
        for (int k = 0; k < S; ++k) {
            const int64_t r = blockIdx.x + int64_t(k) * gridDim.x;
            if (r >= nrounds) break;
            issue_round(P, r, RN, ring + size_t(k) * slot_bytes, &full[k], policy);
        }
    }
    const int lane = t & 31;
    const int gl = lane % G;
    const AoS<float> fld{X_in};
    int it = 0;
    for (int64_t r = blockIdx.x; r < nrounds; r += gridDim.x, ++it) {
        const int slot = it % S;
        const bool ok = mbar_wait_bounded(smem_u32(&full[slot]), uint32_t(it / S) & 1u, wait_ns);
        if (__syncthreads_or(!ok)) {
            if (t == 0) {
                atomicExch(status, LABFM_ETIMEOUT);
                for (int k = 0; k < S; ++k) {  // copies still in flight land before exit
                    const int j = it + k;
                    if (blockIdx.x + int64_t(j) * gridDim.x >= nrounds) break;
                    mbar_wait_bounded(smem_u32(&full[j % S]), uint32_t(j / S) & 1u, kBulkDrainNs);
                }
            }
            return;
        }
        const RoundRange rr = round_range(P.row_ptr, P.N, r, RN);
        const SharedChunks ld{ring + size_t(slot) * slot_bytes, rr.off};
        const int64_t node = r * RN + (t >> 5) * (32 / G) + lane / G;
        const int i = node < P.N ? int(node) : -1;
        float ai = 0, ui = 0, vi = 0;
        int e0 = 0, e1 = 0;
        if (i >= 0) {
            fld.get(i, ai, ui, vi);
            e0 = P.row_ptr[i];
            e1 = P.row_ptr[i + 1];
        }
        float d[12];
        gather_derivatives_ld<float, G, true>(ld, fld, i, e0, e1, gl, ai, ui, vi, d);
        stage_epilogue<float, true>(P, i, gl, d, ai, ui, vi, X_in, Q_in, Q_out, X_out, dt, bk, ck, ph);
        __syncthreads();  // the slot is free: every thread has read its chunks
        if (t == 0) {
            const int64_t rn = r + int64_t(S) * gridDim.x;
            if (rn < nrounds) {
                fence_proxy_async_smem();
                issue_round(P, rn, RN, ring + size_t(slot) * slot_bytes, &full[slot], policy);
            }
        }
    }
}

// Bytes of the largest round (whole interleaved blocks) for rn nodes per round.
__global__ void k_max_round_bytes(const int32_t* row_ptr, int64_t N, int rn, unsigned int* out) {
    const int64_t nrounds = (N + rn - 1) / rn;
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < nrounds;
         r += int64_t(gridDim.x) * blockDim.x)
        atomicMax(out, round_range(row_ptr, N, r, rn).bytes);
}

// Filter: out_i = phi_i + sum_j (phi_j - phi_i) (kappa_i w^hyp_ji) for 3 fields.
template <typename T, int G, bool KAHAN, class Fin>
__device__ __forceinline__ void filter_sums(const PlanView<T>& P, const Fin& fld, int i, int gl,
                                            T ai, T ui, T vi, T& sa, T& su, T& sv) {
    Acc<T, KAHAN> aa, uu, vv;
    if (i >= 0) {
        const int e0 = P.row_ptr[i];
        const int e1 = P.row_ptr[i + 1];
        for (int e = e0 + 4 * gl; e < e1; e += 4 * kUnroll * G) {
#if LABFM_CHUNK_AOS == 3
            if constexpr (std::is_same<T, float>::value) {
                // lane 0 of the group fetches into L2 the filter block it will read
                // pf iterations later (within the row)
                if (P.pf > 0 && gl == 0 && e1 - e0 >= kPrefetchMinRow) {
                    const int ep = e + 4 * kUnroll * G * P.pf;
                    if (ep < e1) {
                        const char* a = reinterpret_cast<const char*>(P.wf) + Rec<float>::fcol(ep >> 2);
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
                    }
                }
            }
#endif
            int cj[4 * kUnroll];
            T wf[4 * kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int eu = e + 4 * u * G;
                if (u == 0 || eu < e1) {
                    load_filt_chunk(P, eu, cj, wf, 4 * u);
                } else {
#pragma unroll
                    for (int k = 4 * u; k < 4 * u + 4; ++k) {
                        cj[k] = i;
                        wf[k] = T(0);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 4 * kUnroll; ++k) {
                T aj, uj, vj;
                fld.get(cj[k], aj, uj, vj);
                aa.add((aj - ai) * wf[k]);
                uu.add((uj - ui) * wf[k]);
                vv.add((vj - vi) * wf[k]);
            }
        }
    }
    if (KAHAN) {
        sa = group_sum<G>(aa.s) - group_sum<G>(aa.c);
        su = group_sum<G>(uu.s) - group_sum<G>(uu.c);
        sv = group_sum<G>(vv.s) - group_sum<G>(vv.c);
    } else {
        sa = group_sum<G>(aa.s);
        su = group_sum<G>(uu.s);
        sv = group_sum<G>(vv.s);
    }
}

template <typename T, int G, bool KAHAN>
__global__ void k_filter_soa(PlanView<T> P, SoA<T> in, T* __restrict__ out) {
    const int64_t gt = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t node = gt / G;
    const int gl = int(gt % G);
    const int i = node < P.N ? int(node) : -1;
    T ai = 0, ui = 0, vi = 0;
    if (i >= 0) in.get(i, ai, ui, vi);
    T sa, su, sv;
    filter_sums<T, G, KAHAN>(P, in, i, gl, ai, ui, vi, sa, su, sv);
    if (i >= 0 && gl == 0) {
        out[i] = ai + sa;
        out[P.N + i] = ui + su;
        out[2 * P.N + i] = vi + sv;
    }
}

// PERSIST = false: one group of G lanes per node over a full grid.  PERSIST =
// true: a grid of (SMs x resident blocks) in which warp w takes the 32/G
// consecutive nodes starting at w * 32/G, then strides by all the grid's groups,
// so that no partly filled last wave of blocks idles the GPU at the end.
// soa (or null): the filtered state is also stored there as 3 x N values (the
// caller's state at the end of a time-step call, so that no unpack launch follows).
template <typename T, int G, bool KAHAN, bool PERSIST>
__global__ void k_filter_aos(PlanView<T> P, const Packed<T>* in, Packed<T>* out, T* soa) {
    const int64_t gt = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int gl = int(gt % G);
    const AoS<T> fld{in};
    const int64_t stride = PERSIST ? int64_t(gridDim.x) * blockDim.x / G : P.n_hi;
    // every lane of a warp runs the same iterations (the group sums shuffle
    // across the whole warp); a group past the end runs idle
    const int64_t warp_first = P.n_lo + (gt / 32) * (32 / G);
    if constexpr (!PERSIST) {
        const int64_t node = warp_first + (gt % 32) / G;
        launch_prologue<T, true, G>(P, node < P.n_hi ? int(node) : -1, gl);
    }
    for (int64_t base = warp_first; base < P.n_hi; base += stride) {
        const int64_t node = base + (gt % 32) / G;
        const int i = node < P.n_hi ? int(node) : -1;
        T ai = 0, ui = 0, vi = 0;
        if (i >= 0) fld.get(i, ai, ui, vi);
        T sa, su, sv;
        filter_sums<T, G, KAHAN>(P, fld, i, gl, ai, ui, vi, sa, su, sv);
        if (i >= 0 && gl == 0) {
            store(out, i, ai + sa, ui + su, vi + sv);
            if (soa) {
                soa[i] = ai + sa;
                soa[P.N + i] = ui + su;
                soa[2 * P.N + i] = vi + sv;
            }
        }
        if (!PERSIST) break;
    }
}

template <typename T>
__global__ void k_pack(int64_t N, const T* __restrict__ soa, Packed<T>* __restrict__ out) {
#if LABFM_PDL
    pdl_launch_dependents();
    pdl_wait();
#endif
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N;
         i += int64_t(gridDim.x) * blockDim.x)
        store(out, i, soa[i], soa[N + i], soa[2 * N + i]);
}

template <typename T>
__global__ void k_unpack(int64_t N, const Packed<T>* __restrict__ in, T* __restrict__ soa) {
#if LABFM_PDL
    pdl_launch_dependents();
    pdl_wait();
#endif
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N;
         i += int64_t(gridDim.x) * blockDim.x) {
        T a, u, v;
        unpack(in, int(i), a, u, v);
        soa[i] = a;
        soa[N + i] = u;
        soa[2 * N + i] = v;
    }
}

// eq. dt, reduced with an exact minimum (order independent).
template <typename T>
__global__ void k_dt(int64_t N, const T* __restrict__ f, const double* __restrict__ s, double c,
                     double mu, unsigned long long* __restrict__ out) {
    double best = INFINITY;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N;
         i += int64_t(gridDim.x) * blockDim.x) {
        const double a = double(f[i]), u = double(f[N + i]), v = double(f[2 * N + i]);
        const double si = s[i];
        const double conv = 1.0 * si / (sqrt(u * u + v * v) + c);
        const double visc = 0.4 * si * si * exp(a) / mu;
        best = fmin(best, fmin(conv, visc));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, off));
    if ((threadIdx.x & 31) == 0 && best < INFINITY)
        atomicMin(out, static_cast<unsigned long long>(__double_as_longlong(best)));
}

__global__ void k_set_u64(unsigned long long* p, unsigned long long v) { *p = v; }

// ---------------------------------------------------------------- plan packing

__global__ void k_padded_counts(int64_t N, const int32_t* __restrict__ row_ptr,
                                int32_t* __restrict__ cnt) {  // cnt points at this instance's slice
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int len = row_ptr[i + 1] - row_ptr[i];
        cnt[i] = (len + 3) & ~3;
    }
}

// Warp per row: copy col, scale the RHS weights (F32: w s^l), fold kappa into
// the filter weights, and fill the pad entries (self, weight 0).
template <typename T, bool SCALED>
__global__ void k_pack_rows(int64_t N, int64_t nnz, int64_t nnz_pad, int64_t off,
                            const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const double* __restrict__ w, const double* __restrict__ kappa,
                            const double* __restrict__ s, const int32_t* __restrict__ prow,
                            int32_t* __restrict__ pcol, T* __restrict__ pw, T* __restrict__ pwf,
                            T* __restrict__ inv_s) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t il = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; il < N; il += warps) {
        // il: node within this instance; i: node of the combined plan
        const int64_t i = off + il;
        const int r0 = row_ptr[il], len = row_ptr[il + 1] - r0;
        const int p0 = prow[i], plen = prow[i + 1] - p0;
        const double si = s[il];
        const double sc1 = SCALED ? si : 1.0;
        const double sc2 = SCALED ? si * si : 1.0;
        const double kap = kappa[il];
        for (int e = lane; e < plen; e += 32) {
            const int64_t dst = int64_t(p0) + entry_slot(e, plen);
            int32_t c = int32_t(i);
            T v[5] = {T(0), T(0), T(0), T(0), T(0)};
            T vf = T(0);
            if (e < len) {
                const int64_t src = int64_t(r0) + e;
                c = int32_t(off + col[src]);
                v[0] = T(w[src] * sc1);
                v[1] = T(w[nnz + src] * sc1);
                v[2] = T(w[2 * nnz + src] * sc2);
                v[3] = T(w[3 * nnz + src] * sc2);
                v[4] = T(w[4 * nnz + src] * sc2);
                vf = T(kap * w[5 * nnz + src]);
            }
#if LABFM_CHUNK_AOS
            char* rb = reinterpret_cast<char*>(pw);
            *reinterpret_cast<int32_t*>(rb + Rec<T>::col_e(dst)) = c;
            for (int d = 0; d < 5; ++d) *reinterpret_cast<T*>(rb + Rec<T>::w_e(dst, d)) = v[d];
            char* fb = reinterpret_cast<char*>(pwf);
            *reinterpret_cast<int32_t*>(fb + Rec<T>::fcol_e(dst)) = c;
            *reinterpret_cast<T*>(fb + Rec<T>::fw_e(dst)) = vf;
#else
            pcol[dst] = c;
            for (int d = 0; d < 5; ++d) pw[d * nnz_pad + dst] = v[d];
            pwf[dst] = vf;
#endif
        }
        if (lane == 0 && inv_s) inv_s[i] = T(1.0 / si);
    }
}

int grid_for(int64_t threads, int block) { return int((threads + block - 1) / block); }


// ---------------------------------------------------------------- dispatch

template <typename T, int G>
int rhs_launch_g(const labfm_plan* p, const void* fields, void* rhs, const Phys<T>& ph, int block,
                 cudaStream_t st) {
    const T* f = static_cast<const T*>(fields);
    SoA<T> in{f, f + p->N, f + 2 * p->N};
    (void)block;  // the gather kernels always run kGatherBlock-thread blocks
    const int grid = grid_for(p->N * G, kGatherBlock);
    constexpr bool F = std::is_same<T, float>::value;
    if (p->wall_slot)
        k_rhs_soa<T, G, F, F, true><<<grid, kGatherBlock, 0, st>>>(view<T>(p), in, static_cast<T*>(rhs), ph);
    else
        k_rhs_soa<T, G, F, F><<<grid, kGatherBlock, 0, st>>>(view<T>(p), in, static_cast<T*>(rhs), ph);
    LABFM_LAUNCH_CHECK("rhs kernel");
    return LABFM_OK;
}

template <typename T>
int rhs_launch(const labfm_plan* p, const void* fields, void* rhs, const labfm_phys* php, int group,
               int block, cudaStream_t st) {
    const Phys<T> ph{T(php->c2), T(php->mu), T(php->gx), T(php->gy)};
    switch (group) {
        case 2: return rhs_launch_g<T, 2>(p, fields, rhs, ph, block, st);
        case 4: return rhs_launch_g<T, 4>(p, fields, rhs, ph, block, st);
        case 8: return rhs_launch_g<T, 8>(p, fields, rhs, ph, block, st);
        case 16: return rhs_launch_g<T, 16>(p, fields, rhs, ph, block, st);
        case 32: return rhs_launch_g<T, 32>(p, fields, rhs, ph, block, st);
    }
    return set_error(LABFM_EINVAL, "unsupported group size");
}

template <typename T, int G>
int stage_launch_g(const labfm_plan* p, const Packed<T>* xin, const Packed<T>* qin, Packed<T>* qout,
                   Packed<T>* xout, double dt, double bk, double ck, const Phys<T>& ph,
                   int* counter, cudaStream_t st) {
    const int block = kGatherBlock;
    constexpr bool F = std::is_same<T, float>::value;
    if (p->wall_slot) {
        const int grid = grid_for(p->N * G, block);
        cudaError_t e = launch_pdl(p, k_stage<T, G, F, F, false, true>, grid, block, st, view<T>(p), xin, qin, qout,
                                   xout, dt, bk, ck, ph, counter);
        if (e != cudaSuccess) return cuda_error(e, "rk stage kernel");
    } else if (p->persistent) {
        k_stage<T, G, F, F, true><<<p->persist_grid, block, 0, st>>>(view<T>(p), xin, qin, qout, xout,
                                                                      dt, bk, ck, ph, counter);
    } else {
        const int grid = grid_for(p->N * G, block);
        cudaError_t e = launch_pdl(p, k_stage<T, G, F, F, false>, grid, block, st, view<T>(p), xin, qin, qout, xout,
                                   dt, bk, ck, ph, counter);
        if (e != cudaSuccess) return cuda_error(e, "rk stage kernel");
    }
    LABFM_LAUNCH_CHECK("rk stage kernel");
    return LABFM_OK;
}

// One plain-grid stage launch over the nodes of launch range r of the plan
// (labfm_plan_set_launch_ranges) with that range's lanes per node and prefetch.
template <typename T, int G>
int stage_range_launch_g(const labfm_plan* p, int r, const Packed<T>* xin, const Packed<T>* qin,
                         Packed<T>* qout, Packed<T>* xout, double dt, double bk, double ck, const Phys<T>& ph,
                         cudaStream_t st) {
    constexpr bool F = std::is_same<T, float>::value;
    PlanView<T> v = view<T>(p);
    v.n_lo = p->range_begin[r];
    v.n_hi = p->range_begin[r + 1];
    v.pf = p->range_pf[r];
    if (v.n_hi <= v.n_lo) return LABFM_OK;
    const int grid = grid_for((v.n_hi - v.n_lo) * G, kGatherBlock);
    int* no_counter = nullptr;
    cudaError_t e = p->wall_slot ? launch_pdl(p, k_stage<T, G, F, F, false, true>, grid, kGatherBlock, st, v, xin,
                                              qin, qout, xout, dt, bk, ck, ph, no_counter)
                                 : launch_pdl(p, k_stage<T, G, F, F, false>, grid, kGatherBlock, st, v, xin, qin,
                                              qout, xout, dt, bk, ck, ph, no_counter);
    if (e != cudaSuccess) return cuda_error(e, "rk stage kernel (launch range)");
    LABFM_LAUNCH_CHECK("rk stage kernel (launch range)");
    return LABFM_OK;
}

template <int G, int S>
int stage_bulk_launch(const labfm_plan* p, const Packed<float>* xin, const Packed<float>* qin,
                      Packed<float>* qout, Packed<float>* xout, double dt, double bk, double ck,
                      const Phys<float>& ph, cudaStream_t st) {
    const int gi = G == 32 ? 1 : 0;
    const uint32_t slot = uint32_t(p->stage_slot_bytes[gi]);
    k_stage_bulk<G, S><<<p->stage_grid[gi], kBulkBlock, size_t(S) * slot, st>>>(
        view<float>(p), xin, qin, qout, xout, dt, bk, ck, ph, slot, p->dev_status, p->wait_ns);
    LABFM_LAUNCH_CHECK("staged rk stage kernel");
    return LABFM_OK;
}

template <int G>
int stage_bulk_launch_s(const labfm_plan* p, const Packed<float>* xin, const Packed<float>* qin,
                        Packed<float>* qout, Packed<float>* xout, double dt, double bk, double ck,
                        const Phys<float>& ph, cudaStream_t st) {
    switch (p->stages) {
        case 2: return stage_bulk_launch<G, 2>(p, xin, qin, qout, xout, dt, bk, ck, ph, st);
        case 3: return stage_bulk_launch<G, 3>(p, xin, qin, qout, xout, dt, bk, ck, ph, st);
        case 4: return stage_bulk_launch<G, 4>(p, xin, qin, qout, xout, dt, bk, ck, ph, st);
    }
    return set_error(LABFM_EINVAL, "unsupported number of staging slots");
}

// The staged kernel serves F32 plans with staging on and 16 or 32 lanes per node
// whose largest round fits in shared memory; every other case runs k_stage.
bool staged(const labfm_plan* p) {
    if (p->dtype != LABFM_F32 || p->stages == 0 || p->wall_slot) return false;
    if (p->group != 16 && p->group != 32) return false;
    return p->stage_grid[p->group == 32 ? 1 : 0] > 0;
}

template <typename T>
int stage_launch(const labfm_plan* p, const Packed<T>* xin, const Packed<T>* qin, Packed<T>* qout,
                 Packed<T>* xout, double dt, double bk, double ck, const Phys<T>& ph, int* counter,
                 cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
        if (staged(p)) {
            if (p->group == 32) return stage_bulk_launch_s<32>(p, xin, qin, qout, xout, dt, bk, ck, ph, st);
            return stage_bulk_launch_s<16>(p, xin, qin, qout, xout, dt, bk, ck, ph, st);
        }
    }
    switch (p->group) {
        case 2: return stage_launch_g<T, 2>(p, xin, qin, qout, xout, dt, bk, ck, ph, counter, st);
        case 4: return stage_launch_g<T, 4>(p, xin, qin, qout, xout, dt, bk, ck, ph, counter, st);
        case 8: return stage_launch_g<T, 8>(p, xin, qin, qout, xout, dt, bk, ck, ph, counter, st);
        case 16: return stage_launch_g<T, 16>(p, xin, qin, qout, xout, dt, bk, ck, ph, counter, st);
        case 32: return stage_launch_g<T, 32>(p, xin, qin, qout, xout, dt, bk, ck, ph, counter, st);
    }
    return set_error(LABFM_EINVAL, "unsupported group size");
}

template <typename T, int G>
int filter_aos_g(const labfm_plan* p, const Packed<T>* in, Packed<T>* out, T* soa, cudaStream_t st) {
    constexpr bool F = std::is_same<T, float>::value;
    if (p->filter_persistent && p->filter_grid > 0) {
        k_filter_aos<T, G, F, true><<<p->filter_grid, p->block, 0, st>>>(view<T>(p), in, out, soa);
    } else {
        const int grid = grid_for(p->N * G, p->block);
        cudaError_t e = launch_pdl(p, k_filter_aos<T, G, F, false>, grid, p->block, st, view<T>(p), in, out, soa);
        if (e != cudaSuccess) return cuda_error(e, "filter kernel");
    }
    LABFM_LAUNCH_CHECK("filter kernel");
    return LABFM_OK;
}

// Lanes per node of the filter: its own setting, else the plan's.
int filter_lanes(const labfm_plan* p) { return p->filter_group ? p->filter_group : p->group; }

template <typename T, int G>
int filter_range_launch_g(const labfm_plan* p, int r, const Packed<T>* in, Packed<T>* out, T* soa, cudaStream_t st) {
    PlanView<T> v = view<T>(p);
    v.n_lo = p->range_begin[r];
    v.n_hi = p->range_begin[r + 1];
    v.pf = p->range_pf[r];
    if (v.n_hi <= v.n_lo) return LABFM_OK;
    const int grid = grid_for((v.n_hi - v.n_lo) * G, p->block);
    cudaError_t e = launch_pdl(p, k_filter_aos<T, G, std::is_same<T, float>::value, false>, grid, p->block, st, v, in,
                               out, soa);
    if (e != cudaSuccess) return cuda_error(e, "filter kernel (launch range)");
    LABFM_LAUNCH_CHECK("filter kernel (launch range)");
    return LABFM_OK;
}

// Stage and filter launches over every launch range, each with its own shape.
template <typename T>
int stage_ranges(const labfm_plan* p, const Packed<T>* xin, const Packed<T>* qin, Packed<T>* qout,
                 Packed<T>* xout, double dt, double bk, double ck, const Phys<T>& ph, cudaStream_t st) {
    for (int r = 0; r < p->n_ranges; ++r) {
        int rc = LABFM_EINVAL;
        switch (p->range_group[r]) {
            case 2: rc = stage_range_launch_g<T, 2>(p, r, xin, qin, qout, xout, dt, bk, ck, ph, st); break;
            case 4: rc = stage_range_launch_g<T, 4>(p, r, xin, qin, qout, xout, dt, bk, ck, ph, st); break;
            case 8: rc = stage_range_launch_g<T, 8>(p, r, xin, qin, qout, xout, dt, bk, ck, ph, st); break;
            case 16: rc = stage_range_launch_g<T, 16>(p, r, xin, qin, qout, xout, dt, bk, ck, ph, st); break;
            case 32: rc = stage_range_launch_g<T, 32>(p, r, xin, qin, qout, xout, dt, bk, ck, ph, st); break;
        }
        if (rc) return rc;
    }
    return LABFM_OK;
}

template <typename T>
int filter_ranges(const labfm_plan* p, const Packed<T>* in, Packed<T>* out, cudaStream_t st, T* soa = nullptr) {
    for (int r = 0; r < p->n_ranges; ++r) {
        int rc = LABFM_EINVAL;
        switch (p->range_group[r]) {
            case 2: rc = filter_range_launch_g<T, 2>(p, r, in, out, soa, st); break;
            case 4: rc = filter_range_launch_g<T, 4>(p, r, in, out, soa, st); break;
            case 8: rc = filter_range_launch_g<T, 8>(p, r, in, out, soa, st); break;
            case 16: rc = filter_range_launch_g<T, 16>(p, r, in, out, soa, st); break;
            case 32: rc = filter_range_launch_g<T, 32>(p, r, in, out, soa, st); break;
        }
        if (rc) return rc;
    }
    return LABFM_OK;
}

template <typename T>
int filter_aos(const labfm_plan* p, const Packed<T>* in, Packed<T>* out, cudaStream_t st, T* soa = nullptr) {
    switch (filter_lanes(p)) {
        case 2: return filter_aos_g<T, 2>(p, in, out, soa, st);
        case 4: return filter_aos_g<T, 4>(p, in, out, soa, st);
        case 8: return filter_aos_g<T, 8>(p, in, out, soa, st);
        case 16: return filter_aos_g<T, 16>(p, in, out, soa, st);
        case 32: return filter_aos_g<T, 32>(p, in, out, soa, st);
    }
    return set_error(LABFM_EINVAL, "unsupported group size");
}

template <typename T, int G>
int filter_soa_g(const labfm_plan* p, const void* in, void* out, cudaStream_t st) {
    const T* f = static_cast<const T*>(in);
    SoA<T> src{f, f + p->N, f + 2 * p->N};
    const int grid = grid_for(p->N * G, p->block);
    k_filter_soa<T, G, std::is_same<T, float>::value><<<grid, p->block, 0, st>>>(view<T>(p), src,
                                                                                  static_cast<T*>(out));
    LABFM_LAUNCH_CHECK("filter kernel");
    return LABFM_OK;
}

template <typename T>
int filter_soa(const labfm_plan* p, const void* in, void* out, cudaStream_t st) {
    switch (p->group) {
        case 2: return filter_soa_g<T, 2>(p, in, out, st);
        case 4: return filter_soa_g<T, 4>(p, in, out, st);
        case 8: return filter_soa_g<T, 8>(p, in, out, st);
        case 16: return filter_soa_g<T, 16>(p, in, out, st);
        case 32: return filter_soa_g<T, 32>(p, in, out, st);
    }
    return set_error(LABFM_EINVAL, "unsupported group size");
}

// Work layout: three packed buffers P (solution Q), X, Y of N nodes each, then
// (persistent plans) 64 bytes of work-queue tickets.
//   X <- pack(Q)
//   per step:  stage 1: gather X, Q_i from X, P <- Q, Y <- X-update
//              stage 2: gather Y, P in place, X <- update
//              stage 3: gather X, P in place, Y <- update
//              stage 4: gather Y, P in place
//              filter:  gather P, X <- filtered (the next step's Q = X)
//   Q <- unpack(X)
template <typename T>
int rk_one_step_t(const labfm_plan* p, void* work, double dt, const labfm_phys* php, bool profile,
                  cudaStream_t st, void* soa_out) {
    const Phys<T> ph{T(php->c2), T(php->mu), T(php->gx), T(php->gy)};
    Packed<T>* P = static_cast<Packed<T>*>(work);
    Packed<T>* X = P + p->N;
    Packed<T>* Y = X + p->N;
    int* tickets = reinterpret_cast<int*>(Y + p->N);
    if (p->persistent) LABFM_CUDA_TRY(cudaMemsetAsync(tickets, 0, 4 * sizeof(int), st));
    int rc;
    labfm_plan* pm = const_cast<labfm_plan*>(p);  // only the launch-timing record changes
    const Packed<T>* xin[4] = {X, Y, X, Y};
    const Packed<T>* qin[4] = {X, P, P, P};
    Packed<T>* xout[4] = {Y, X, Y, nullptr};
    const bool timed = profile && prof_step_sampled(pm);
    const int evs = timed ? prof_begin(pm, kProfStages4, st) : -1;  // the four stages as one block
    for (int k = 0; k < 4; ++k) {
        const double bk = kRkB[k];
        const double ck = k < 3 ? kRkA[k] - kRkB[k] : 0.0;
        rc = p->n_ranges ? stage_ranges<T>(p, xin[k], qin[k], P, xout[k], dt, bk, ck, ph, st)
                         : stage_launch<T>(p, xin[k], qin[k], P, xout[k], dt, bk, ck, ph, tickets + k, st);
        if (rc) return rc;
    }
    prof_end(pm, evs, st);
    const int ev = timed ? prof_begin(pm, kProfFilter, st) : -1;
    T* soa = static_cast<T*>(soa_out);
    if ((rc = p->n_ranges ? filter_ranges<T>(p, P, X, st, soa) : filter_aos<T>(p, P, X, st, soa))) return rc;
    prof_end(pm, ev, st);
    return LABFM_OK;
}

}  // namespace

int pack_fields(const labfm_plan* p, const void* soa, void* packed, cudaStream_t st) {
    const int pg = int(std::min<int64_t>((p->N + 255) / 256, 65535));
    if (p->dtype == LABFM_F32)
        k_pack<float><<<pg, 256, 0, st>>>(p->N, static_cast<const float*>(soa),
                                          static_cast<Packed<float>*>(packed));
    else
        k_pack<double><<<pg, 256, 0, st>>>(p->N, static_cast<const double*>(soa),
                                           static_cast<Packed<double>*>(packed));
    LABFM_LAUNCH_CHECK("pack kernel");
    return LABFM_OK;
}

int unpack_fields(const labfm_plan* p, const void* packed, void* soa, cudaStream_t st) {
    const int pg = int(std::min<int64_t>((p->N + 255) / 256, 65535));
    if (p->dtype == LABFM_F32)
        k_unpack<float><<<pg, 256, 0, st>>>(p->N, static_cast<const Packed<float>*>(packed),
                                            static_cast<float*>(soa));
    else
        k_unpack<double><<<pg, 256, 0, st>>>(p->N, static_cast<const Packed<double>*>(packed),
                                             static_cast<double*>(soa));
    LABFM_LAUNCH_CHECK("unpack kernel");
    return LABFM_OK;
}

namespace {
template <typename T, int G>
int stage_rec_launch_g(const labfm_plan* p, const Packed<T>* xin, const Packed<T>* qin, Packed<T>* qout,
                       Packed<T>* xout, double dt, double bk, double ck, const Phys<T>& ph, D8<T>* D,
                       cudaStream_t st) {
    constexpr bool F = std::is_same<T, float>::value;
    const int grid = grid_for(p->N * G, kGatherBlock);
    cudaError_t e = launch_pdl(p, k_stage_rec<T, G, F, F>, grid, kGatherBlock, st, view<T>(p), xin, qin, qout, xout,
                               dt, bk, ck, ph, D);
    if (e != cudaSuccess) return cuda_error(e, "recording rk stage kernel");
    return LABFM_OK;
}

template <typename T>
int stage_rec_launch(const labfm_plan* p, const Packed<T>* xin, const Packed<T>* qin, Packed<T>* qout,
                     Packed<T>* xout, double dt, double bk, double ck, const Phys<T>& ph, D8<T>* D,
                     cudaStream_t st) {
    switch (p->group) {
        case 2: return stage_rec_launch_g<T, 2>(p, xin, qin, qout, xout, dt, bk, ck, ph, D, st);
        case 4: return stage_rec_launch_g<T, 4>(p, xin, qin, qout, xout, dt, bk, ck, ph, D, st);
        case 8: return stage_rec_launch_g<T, 8>(p, xin, qin, qout, xout, dt, bk, ck, ph, D, st);
        case 16: return stage_rec_launch_g<T, 16>(p, xin, qin, qout, xout, dt, bk, ck, ph, D, st);
        case 32: return stage_rec_launch_g<T, 32>(p, xin, qin, qout, xout, dt, bk, ck, ph, D, st);
    }
    return set_error(LABFM_EINVAL, "unsupported group size");
}

// The four stages with the recording kernel: the same arithmetic per node as the
// stage kernels of labfm_rk_step (same lanes per node and summation order).
template <typename T>
int forward_stages_t(const labfm_plan* p, const void* X1v, void* Pv, void* X2v, void* X3v, void* X4v,
                     void* Dv, double dt, const labfm_phys* php, cudaStream_t st) {
    const Phys<T> ph{T(php->c2), T(php->mu), T(php->gx), T(php->gy)};
    const Packed<T>* X1 = static_cast<const Packed<T>*>(X1v);
    Packed<T>* P = static_cast<Packed<T>*>(Pv);
    Packed<T>* X2 = static_cast<Packed<T>*>(X2v);
    Packed<T>* X3 = static_cast<Packed<T>*>(X3v);
    Packed<T>* X4 = static_cast<Packed<T>*>(X4v);
    D8<T>* D = static_cast<D8<T>*>(Dv);
    const int64_t N = p->N;
    labfm_plan* pm = const_cast<labfm_plan*>(p);  // only the launch-timing record changes
    const int ev = prof_begin(pm, kProfRecStages4, st);
    int rc;
    if ((rc = stage_rec_launch<T>(p, X1, X1, P, X2, dt, kRkB[0], kRkA[0] - kRkB[0], ph, D, st))) return rc;
    if ((rc = stage_rec_launch<T>(p, X2, P, P, X3, dt, kRkB[1], kRkA[1] - kRkB[1], ph, D + N, st))) return rc;
    if ((rc = stage_rec_launch<T>(p, X3, P, P, X4, dt, kRkB[2], kRkA[2] - kRkB[2], ph, D + 2 * N, st)))
        return rc;
    if ((rc = stage_rec_launch<T>(p, X4, P, P, nullptr, dt, kRkB[3], 0.0, ph, D + 3 * N, st))) return rc;
    prof_end(pm, ev, st);
    return LABFM_OK;
}

// One step that keeps its stage states: X1 = pack(Q), X2..X4 the inputs of
// stages 2..4, the derivative combinations of all four after them, then the
// filter as labfm_rk_step takes it; Q is replaced by the next state.  P and Y:
// scratch packed states.
template <typename T>
int rk_step_record_t(const labfm_plan* p, void* Q, void* Xv, void* Pv, void* Yv, double dt,
                     const labfm_phys* php, cudaStream_t st) {
    Packed<T>* X = static_cast<Packed<T>*>(Xv);
    Packed<T>* P = static_cast<Packed<T>*>(Pv);
    Packed<T>* Y = static_cast<Packed<T>*>(Yv);
    int rc;
    if ((rc = pack_fields(p, Q, X, st))) return rc;
    if ((rc = forward_stages_t<T>(p, X, P, X + p->N, X + 2 * p->N, X + 3 * p->N, X + 4 * p->N, dt, php,
                                  st)))
        return rc;
    labfm_plan* pm = const_cast<labfm_plan*>(p);
    const int ev = prof_begin(pm, kProfFilter, st);
    if ((rc = filter_aos<T>(p, P, Y, st))) return rc;
    prof_end(pm, ev, st);
    return unpack_fields(p, Y, Q, st);
}
}  // namespace

int rk_step_record(const labfm_plan* p, void* Q, void* X, void* P, void* Y, double dt,
                   const labfm_phys* ph, cudaStream_t st) {
    return p->dtype == LABFM_F32 ? rk_step_record_t<float>(p, Q, X, P, Y, dt, ph, st)
                                 : rk_step_record_t<double>(p, Q, X, P, Y, dt, ph, st);
}

int forward_stages(const labfm_plan* p, const void* X1, void* P, void* X2, void* X3, void* X4, void* D,
                   double dt, const labfm_phys* ph, cudaStream_t st) {
    return p->dtype == LABFM_F32 ? forward_stages_t<float>(p, X1, P, X2, X3, X4, D, dt, ph, st)
                                 : forward_stages_t<double>(p, X1, P, X2, X3, X4, D, dt, ph, st);
}

size_t packed_bytes(const labfm_plan* p) {
    return p->dtype == LABFM_F32 ? sizeof(Packed<float>) : sizeof(Packed<double>);
}

size_t d8_bytes(const labfm_plan* p) {
    return p->dtype == LABFM_F32 ? sizeof(D8<float>) : sizeof(D8<double>);
}

int rk_pack(const labfm_plan* p, const void* Q, void* work, cudaStream_t st) {
    const int pg = int(std::min<int64_t>((p->N + 255) / 256, 65535));
    if (p->dtype == LABFM_F32) {
        Packed<float>* X = static_cast<Packed<float>*>(work) + p->N;
        LABFM_CUDA_TRY(launch_pdl(p, k_pack<float>, pg, 256, st, p->N, static_cast<const float*>(Q), X));
    } else {
        Packed<double>* X = static_cast<Packed<double>*>(work) + p->N;
        LABFM_CUDA_TRY(launch_pdl(p, k_pack<double>, pg, 256, st, p->N, static_cast<const double*>(Q), X));
    }
    return LABFM_OK;
}

int rk_unpack(const labfm_plan* p, void* Q, const void* work, cudaStream_t st) {
    const int pg = int(std::min<int64_t>((p->N + 255) / 256, 65535));
    if (p->dtype == LABFM_F32) {
        const Packed<float>* X = static_cast<const Packed<float>*>(work) + p->N;
        LABFM_CUDA_TRY(launch_pdl(p, k_unpack<float>, pg, 256, st, p->N, X, static_cast<float*>(Q)));
    } else {
        const Packed<double>* X = static_cast<const Packed<double>*>(work) + p->N;
        LABFM_CUDA_TRY(launch_pdl(p, k_unpack<double>, pg, 256, st, p->N, X, static_cast<double*>(Q)));
    }
    return LABFM_OK;
}

int rk_one_step(const labfm_plan* p, void* work, double dt, const labfm_phys* ph, bool profile,
                cudaStream_t st, void* soa_out) {
    return p->dtype == LABFM_F32 ? rk_one_step_t<float>(p, work, dt, ph, profile, st, soa_out)
                                 : rk_one_step_t<double>(p, work, dt, ph, profile, st, soa_out);
}

namespace {
}  // namespace

bool launch_shape_supported(int group, int block) {
    const bool g_ok = group == 2 || group == 4 || group == 8 || group == 16 || group == 32;
    return g_ok && block >= 64 && block <= 1024 && block % 32 == 0 && block % group == 0;
}

int launch_rhs(const labfm_plan* p, const void* fields, void* rhs, const labfm_phys* ph, int group,
               int block, cudaStream_t st) {
    return p->dtype == LABFM_F32 ? rhs_launch<float>(p, fields, rhs, ph, group, block, st)
                                 : rhs_launch<double>(p, fields, rhs, ph, group, block, st);
}

int launch_filter_soa(const labfm_plan* p, const void* in, void* out, cudaStream_t st) {
    return p->dtype == LABFM_F32 ? filter_soa<float>(p, in, out, st)
                                 : filter_soa<double>(p, in, out, st);
}

size_t rk_work_bytes(const labfm_plan* p) {
    const size_t per = p->dtype == LABFM_F32 ? sizeof(Packed<float>) : sizeof(Packed<double>);
    return size_t(3) * size_t(p->N) * per + (p->persistent ? 64 : 0);
}

namespace {
// LABFM_ENONFINITE into the plan's status word (unless a status is already set)
// when any value of the packed state is not finite: one vote per warp, one
// atomic per warp that saw one.
template <typename T>
__global__ void k_check_finite(int64_t N, const Packed<T>* __restrict__ X, int* status) {
    bool bad = false;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N;
         i += int64_t(gridDim.x) * blockDim.x) {
        T a, u, v;
        unpack(X, int(i), a, u, v);
        bad |= !(isfinite(a) && isfinite(u) && isfinite(v));
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicCAS(status, 0, LABFM_ENONFINITE);
}

int check_finite(const labfm_plan* p, const void* work, cudaStream_t st) {
    const int grid = int(std::min<int64_t>((p->N + 255) / 256, 152 * 8));
    if (p->dtype == LABFM_F32)
        k_check_finite<float><<<grid, 256, 0, st>>>(p->N, static_cast<const Packed<float>*>(work) + p->N,
                                                   p->dev_status);
    else
        k_check_finite<double><<<grid, 256, 0, st>>>(p->N, static_cast<const Packed<double>*>(work) + p->N,
                                                    p->dev_status);
    LABFM_LAUNCH_CHECK("state check kernel");
    return LABFM_OK;
}
}  // namespace

int launch_rk_steps(const labfm_plan* p, void* Q, void* work, double dt, int nsteps,
                    const labfm_phys* ph, cudaStream_t st) {
    if (nsteps == 0) return LABFM_OK;
    int rc;
    if ((rc = rk_pack(p, Q, work, st))) return rc;
    const int every = p->dev_status ? p->check_every : 0;
    // the last step's filter also stores the state into Q (no unpack launch)
    for (int step = 0; step < nsteps; ++step) {
        if ((rc = rk_one_step(p, work, dt, ph, true, st, step + 1 == nsteps ? Q : nullptr))) return rc;
        if (every > 0 && ((step + 1) % every == 0 || step + 1 == nsteps))
            if ((rc = check_finite(p, work, st))) return rc;
    }
    return LABFM_OK;
}

int filter_persistent_grid(const labfm_plan* p) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaErrorInvalidValue;
#define LABFM_FOCC(T, G)                                                                            \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                              \
        &per_sm, k_filter_aos<T, G, std::is_same<T, float>::value, true>, p->block, 0)
    const int g = filter_lanes(p);
    if (p->dtype == LABFM_F32) {
        switch (g) {
            case 2: LABFM_FOCC(float, 2); break;
            case 4: LABFM_FOCC(float, 4); break;
            case 8: LABFM_FOCC(float, 8); break;
            case 16: LABFM_FOCC(float, 16); break;
            case 32: LABFM_FOCC(float, 32); break;
        }
    } else {
        switch (g) {
            case 2: LABFM_FOCC(double, 2); break;
            case 4: LABFM_FOCC(double, 4); break;
            case 8: LABFM_FOCC(double, 8); break;
            case 16: LABFM_FOCC(double, 16); break;
            case 32: LABFM_FOCC(double, 32); break;
        }
    }
#undef LABFM_FOCC
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

int persistent_grid(const labfm_plan* p) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaErrorInvalidValue;
#define LABFM_OCC(T, G)                                                                      \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                       \
        &per_sm, k_stage<T, G, std::is_same<T, float>::value, std::is_same<T, float>::value, \
                         true>,                                                             \
        kGatherBlock, 0)
    if (p->dtype == LABFM_F32) {
        switch (p->group) {
            case 2: LABFM_OCC(float, 2); break;
            case 4: LABFM_OCC(float, 4); break;
            case 8: LABFM_OCC(float, 8); break;
            case 16: LABFM_OCC(float, 16); break;
            case 32: LABFM_OCC(float, 32); break;
        }
    } else {
        switch (p->group) {
            case 2: LABFM_OCC(double, 2); break;
            case 4: LABFM_OCC(double, 4); break;
            case 8: LABFM_OCC(double, 8); break;
            case 16: LABFM_OCC(double, 16); break;
            case 32: LABFM_OCC(double, 32); break;
        }
    }
#undef LABFM_OCC
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

int launch_stable_dt(const labfm_plan* p, const void* fields, const double* s, double c, double mu,
                     double* dt_out, cudaStream_t st) {
    unsigned long long* out = reinterpret_cast<unsigned long long*>(dt_out);
    const unsigned long long inf_bits = 0x7ff0000000000000ull;
    k_set_u64<<<1, 1, 0, st>>>(out, inf_bits);
    const int grid = int(std::min<int64_t>((p->N + 255) / 256, 1184));
    if (p->dtype == LABFM_F32)
        k_dt<float><<<grid, 256, 0, st>>>(p->N, static_cast<const float*>(fields), s, c, mu, out);
    else
        k_dt<double><<<grid, 256, 0, st>>>(p->N, static_cast<const double*>(fields), s, c, mu, out);
    LABFM_LAUNCH_CHECK("dt kernel");
    return LABFM_OK;
}

int pack_plan(labfm_plan* p, const PlanInput* in, int n_inst, cudaStream_t st) {
    const int64_t N = p->N;
    // instance node offsets
    p->n_inst = n_inst;
    p->inst_off_host = new (std::nothrow) int64_t[n_inst + 1];
    if (!p->inst_off_host) return set_error(LABFM_ENOMEM, "host allocation failed");
    p->inst_off_host[0] = 0;
    for (int k = 0; k < n_inst; ++k) p->inst_off_host[k + 1] = p->inst_off_host[k] + in[k].N;
    LABFM_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&p->inst_off), size_t(n_inst + 1) * sizeof(int64_t)));
    LABFM_CUDA_TRY(cudaMemcpyAsync(p->inst_off, p->inst_off_host, size_t(n_inst + 1) * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, st));
    p->device_bytes += (n_inst + 1) * sizeof(int64_t);
    // padded row pointers over all instances
    LABFM_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&p->row_ptr), size_t(N + 1) * sizeof(int32_t)));
    p->device_bytes += (N + 1) * sizeof(int32_t);
    int32_t* cnt = nullptr;
    int64_t* total = nullptr;
    void* scan_tmp = nullptr;
    const size_t scan_bytes = exclusive_scan_scratch_bytes(N);
    LABFM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&cnt), size_t(N) * sizeof(int32_t), st));
    LABFM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&total), sizeof(int64_t), st));
    LABFM_CUDA_TRY(cudaMallocAsync(&scan_tmp, scan_bytes, st));
    for (int k = 0; k < n_inst; ++k) {
        const int g = int(std::min<int64_t>((in[k].N + 255) / 256, 65535));
        k_padded_counts<<<g, 256, 0, st>>>(in[k].N, in[k].row_ptr, cnt + p->inst_off_host[k]);
    }
    int rc = exclusive_scan_i32(cnt, p->row_ptr, N, total, scan_tmp, scan_bytes, st);
    int64_t nnz_pad = 0;
    if (rc == LABFM_OK) {
        cudaError_t e = cudaMemcpyAsync(&nnz_pad, total, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_error(e, "reading padded size");
    }
    cudaFreeAsync(cnt, st);
    cudaFreeAsync(total, st);
    cudaFreeAsync(scan_tmp, st);
    if (rc) return rc;
    if (nnz_pad >= (int64_t(1) << 31)) return set_error(LABFM_ECAPACITY, "padded stencil exceeds 2^31 entries");
    p->nnz_pad = nnz_pad;
    // F32 record streams prefetched two iterations ahead (labfm_plan_set_prefetch);
    // the kernels skip rows shorter than kPrefetchMinRow entries
    p->prefetch = p->dtype == LABFM_F32 ? 2 : 0;
    const size_t es = p->dtype == LABFM_F32 ? sizeof(float) : sizeof(double);
    const size_t np = size_t(std::max<int64_t>(nnz_pad, 4));
#if LABFM_CHUNK_AOS
    const size_t rhs_bytes = p->dtype == LABFM_F32 ? Rec<float>::rhs_bytes(np) : Rec<double>::rhs_bytes(np);
    const size_t filt_bytes = p->dtype == LABFM_F32 ? Rec<float>::filt_bytes(np) : Rec<double>::filt_bytes(np);
    LABFM_CUDA_TRY(cudaMalloc(&p->w, rhs_bytes));
    LABFM_CUDA_TRY(cudaMalloc(&p->wf, filt_bytes));
    p->device_bytes += rhs_bytes + filt_bytes;
#else
    LABFM_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&p->col), np * sizeof(int32_t)));
    LABFM_CUDA_TRY(cudaMalloc(&p->w, 5 * np * es));
    LABFM_CUDA_TRY(cudaMalloc(&p->wf, np * es));
    p->device_bytes += np * (sizeof(int32_t) + 6 * es);
#endif
    if (p->dtype == LABFM_F32) {
        LABFM_CUDA_TRY(cudaMalloc(&p->inv_s, size_t(N) * es));
        p->device_bytes += N * es;
    }
    for (int k = 0; k < n_inst; ++k) {
        const PlanInput& I = in[k];
        const int64_t off = p->inst_off_host[k];
        const int gw = int(std::min<int64_t>((I.N * 32 + 255) / 256, 1 << 20));
        if (p->dtype == LABFM_F32)
            k_pack_rows<float, true><<<gw, 256, 0, st>>>(
                I.N, I.nnz, nnz_pad, off, I.row_ptr, I.col, I.w, I.kappa, I.s, p->row_ptr, p->col,
                static_cast<float*>(p->w), static_cast<float*>(p->wf), static_cast<float*>(p->inv_s));
        else
            k_pack_rows<double, false><<<gw, 256, 0, st>>>(
                I.N, I.nnz, nnz_pad, off, I.row_ptr, I.col, I.w, I.kappa, I.s, p->row_ptr, p->col,
                static_cast<double*>(p->w), static_cast<double*>(p->wf), nullptr);
        LABFM_LAUNCH_CHECK("plan pack kernel");
    }
    LABFM_CUDA_TRY(cudaStreamSynchronize(st));
    return LABFM_OK;
}

// ---------------------------------------------------------------- per-instance time steps

namespace {

__global__ void k_fill_dt(int64_t n, double v, double* __restrict__ out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        out[i] = v;
}

__device__ __forceinline__ int instance_of(const int64_t* off, int n_inst, int64_t i) {
    int lo = 0, hi = n_inst - 1;  // largest k with off[k] <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// eq. dt per instance: exact minimum over the instance's nodes.
template <typename T>
__global__ void k_dt_instances(int64_t N, const T* __restrict__ f, const double* __restrict__ s,
                               double c, double mu, const int64_t* __restrict__ off, int n_inst,
                               unsigned long long* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    // warp-uniform loop: nodes of an instance are contiguous, so most warps hold a
    // single instance and need one atomic
    for (int64_t base = blockIdx.x * int64_t(blockDim.x) + (threadIdx.x & ~31); base < N;
         base += stride) {
        const int64_t i = base + lane;
        double dt = INFINITY;
        int inst = -1;
        if (i < N) {
            const double a = double(f[i]), u = double(f[N + i]), v = double(f[2 * N + i]);
            const double si = s[i];
            const double conv = 1.0 * si / (sqrt(u * u + v * v) + c);
            const double visc = 0.4 * si * si * exp(a) / mu;
            dt = fmin(conv, visc);
            inst = instance_of(off, n_inst, i);
        }
        const int inst0 = __shfl_sync(0xffffffffu, inst, 0);
        if (__all_sync(0xffffffffu, inst == inst0 || inst < 0)) {
            double m = dt;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0 && inst0 >= 0)
                atomicMin(out + inst0, static_cast<unsigned long long>(__double_as_longlong(m)));
        } else if (inst >= 0) {
            atomicMin(out + inst, static_cast<unsigned long long>(__double_as_longlong(dt)));
        }
    }
}

__global__ void k_set_u64_n(unsigned long long* p, int n, unsigned long long v) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) p[k] = v;
}

}  // namespace

int set_node_dt(labfm_plan* p, const double* dt_inst_host, cudaStream_t st) {
    if (!p->dt_node) {
        LABFM_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&p->dt_node), size_t(p->N) * sizeof(double)));
        p->device_bytes += p->N * sizeof(double);
    }
    for (int k = 0; k < p->n_inst; ++k) {
        const int64_t a = p->inst_off_host[k], n = p->inst_off_host[k + 1] - a;
        if (!(dt_inst_host[k] > 0.0)) return set_error(LABFM_EINVAL, "instance dt must be positive");
        if (n == 0) continue;
        const int g = int(std::min<int64_t>((n + 255) / 256, 4096));
        k_fill_dt<<<g, 256, 0, st>>>(n, dt_inst_host[k], p->dt_node + a);
    }
    LABFM_LAUNCH_CHECK("dt fill kernel");
    return LABFM_OK;
}

int launch_stable_dt_instances(const labfm_plan* p, const void* fields, const double* s, double c,
                               double mu, double* dt_inst, cudaStream_t st) {
    unsigned long long* out = reinterpret_cast<unsigned long long*>(dt_inst);
    k_set_u64_n<<<(p->n_inst + 255) / 256, 256, 0, st>>>(out, p->n_inst, 0x7ff0000000000000ull);
    const int grid = int(std::min<int64_t>((p->N + 255) / 256, 4096));
    if (p->dtype == LABFM_F32)
        k_dt_instances<float><<<grid, 256, 0, st>>>(p->N, static_cast<const float*>(fields), s, c, mu,
                                                    p->inst_off, p->n_inst, out);
    else
        k_dt_instances<double><<<grid, 256, 0, st>>>(p->N, static_cast<const double*>(fields), s, c,
                                                     mu, p->inst_off, p->n_inst, out);
    LABFM_LAUNCH_CHECK("instance dt kernel");
    return LABFM_OK;
}

}  // namespace labfm

namespace labfm {
namespace {
template <int G, int S>
int staging_shape(labfm_plan* p, int gi, size_t slot, int sms) {
    const size_t smem = size_t(S) * slot;
    p->stage_slot_bytes[gi] = int(slot);
    p->stage_grid[gi] = 0;
    if (smem > size_t(226) * 1024) return LABFM_OK;  // this shape does not fit (static smem too)
    LABFM_CUDA_TRY(cudaFuncSetAttribute(k_stage_bulk<G, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        int(smem)));
    int per_sm = 0;
    LABFM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stage_bulk<G, S>, kBulkBlock,
                                                                 smem));
    const int64_t nrounds = (p->N + round_nodes<G>() - 1) / round_nodes<G>();
    p->stage_grid[gi] = int(std::min<int64_t>(nrounds, int64_t(per_sm) * sms));
    return LABFM_OK;
}

template <int G>
int staging_shape_s(labfm_plan* p, int gi, size_t slot, int sms) {
    switch (p->stages) {
        case 2: return staging_shape<G, 2>(p, gi, slot, sms);
        case 3: return staging_shape<G, 3>(p, gi, slot, sms);
        default: return staging_shape<G, 4>(p, gi, slot, sms);
    }
}
}  // namespace

int plan_entry_bytes(const labfm_plan* p, bool filter) {
#if LABFM_CHUNK_AOS
    if (p->dtype == LABFM_F32) return int((filter ? Rec<float>::FB : Rec<float>::BB) / (4 * kIL));
    return int((filter ? Rec<double>::FB : Rec<double>::BB) / (4 * kIL));
#else
    const int es = p->dtype == LABFM_F32 ? 4 : 8;
    return filter ? 4 + es : 4 + 5 * es;
#endif
}

int configure_staging(labfm_plan* p, int stages, cudaStream_t st) {
    p->stages = 0;
    p->stage_slot_bytes[0] = p->stage_slot_bytes[1] = 0;
    p->stage_grid[0] = p->stage_grid[1] = 0;
    if (stages == 0) return LABFM_OK;
    if (p->dtype != LABFM_F32) return set_error(LABFM_EINVAL, "staging serves F32 plans only");
    if (stages < 2 || stages > 4) return set_error(LABFM_EINVAL, "stages must be 0 or 2..4");
    if (!p->dev_status) {
        LABFM_CUDA_TRY(cudaMalloc(&p->dev_status, sizeof(int)));
        p->device_bytes += sizeof(int);
    }
    LABFM_CUDA_TRY(cudaMemsetAsync(p->dev_status, 0, sizeof(int), st));
    int dev = 0, sms = 0;
    LABFM_CUDA_TRY(cudaGetDevice(&dev));
    LABFM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    unsigned int* d_max = nullptr;
    LABFM_CUDA_TRY(cudaMallocAsync(&d_max, 2 * sizeof(unsigned int), st));
    cudaError_t e = cudaMemsetAsync(d_max, 0, 2 * sizeof(unsigned int), st);
    const int grid = int(std::min<int64_t>((p->N + 255) / 256 + 1, 4096));
    if (e == cudaSuccess) {
        k_max_round_bytes<<<grid, 256, 0, st>>>(p->row_ptr, p->N, round_nodes<16>(), d_max);
        k_max_round_bytes<<<grid, 256, 0, st>>>(p->row_ptr, p->N, round_nodes<32>(), d_max + 1);
        e = cudaGetLastError();
    }
    unsigned int h_max[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_max, d_max, sizeof(h_max), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(d_max, st);
    if (e != cudaSuccess) return cuda_error(e, "staging: largest round");
    p->stages = stages;
    for (int gi = 0; gi < 2; ++gi) {
        const size_t slot = std::max<size_t>(h_max[gi], 16);
        const int rc = gi ? staging_shape_s<32>(p, gi, slot, sms) : staging_shape_s<16>(p, gi, slot, sms);
        if (rc) {
            p->stages = 0;
            return rc;
        }
    }
    return LABFM_OK;
}

}  // namespace labfm
