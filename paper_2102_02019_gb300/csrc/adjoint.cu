// Discrete adjoint of the time step: vector-Jacobian products of the eq. icns
// right-hand side, of the filter and of one RK3(2)4[2R+]C step.  The paper has
// no adjoint; the products are the exact transposes of the forward kernels.
//
// The transpose of a difference-form operator L(phi)_i = sum_j (phi_j - phi_i) w_ij
// is (L^T g)_k = sum_{i : k in N(i)} w_ik g_i - (sum_j w_kj) g_k.  It is applied as
// a gather over a transposed operator (for node k: the rows i that contain k,
// with their weights w_ik), stored in the same 4-entry record layout as the
// forward operator, plus the forward row sums: no scatter, no atomics.
//
// RHS adjoint at state X with cotangent m (two passes):
//   pass A (node i): forward derivatives d_i, then the derivative adjoints
//     g_i = (dR_i/dd_i)^T m_i (twelve values, carried as eight: see G8; scaled
//     by s_i^-l in F32 to match the nondimensional weights) and the own-value
//     adjoints o_i = (dR_i/dX_i)^T m_i;
//   pass B (node k): Xbar_k = o_k + sum over operators of (L^T g)_k.
// One RK step backwards (low-storage form of the reverse sweep):
//   Lambda = Fil^T lambda;  Fbar_4 = dt b_4 Lambda
//   for k = 4..1: Xbar_k = J_R(X_k)^T Fbar_k; Lambda += Xbar_k;
//                 Fbar_{k-1} = dt (b_{k-1} Lambda + (a_{k,k-1} - b_{k-1}) Xbar_k)
//   result: Lambda (the cotangent of the state at the start of the step).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <type_traits>

#include "gather.cuh"
#include "labfm_internal.cuh"
#include "nvtx.cuh"

#if !LABFM_CHUNK_AOS
#error "the transposed-operator build reads the chunk-record layout"
#endif

namespace labfm {
namespace {

// The twelve derivative adjoints of one node in eight values, packed for two
// 16-byte gathers (F32):
//   [g_ax, g_ay, g_ux, g_uy] [g_vx, g_vy, A, B].
// The second derivatives enter eq. icns only through
// nu (4/3 u_xx + u_yy + 1/3 v_xy) in R_u and nu (4/3 v_yy + v_xx + 1/3 u_xy) in
// R_v, so their six adjoints are fixed multiples of A = nu m_u and B = nu m_v:
//   g_uxx = 4/3 A, g_uyy = A, g_vxy = 1/3 A, g_vxx = B, g_vyy = 4/3 B, g_uxy = 1/3 B.
// The transposed records carry the matching operator combinations (see
// k_write_transposed), so that pass B gathers 32 bytes per stencil entry, not 48.
template <typename T> struct G8;
template <> struct G8<float> { float4 q[2]; };
template <> struct G8<double> { double2 q[4]; };

__device__ __forceinline__ void g8_store(G8<float>* p, int64_t i, const float (&g)[8]) {
    p[i].q[0] = make_float4(g[0], g[1], g[2], g[3]);
    p[i].q[1] = make_float4(g[4], g[5], g[6], g[7]);
}
__device__ __forceinline__ void g8_store(G8<double>* p, int64_t i, const double (&g)[8]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) p[i].q[k] = make_double2(g[2 * k], g[2 * k + 1]);
}
__device__ __forceinline__ void g8_load(const G8<float>* p, int i, float (&g)[8]) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float4 t = __ldg(&p[i].q[k]);
        g[4 * k] = t.x;
        g[4 * k + 1] = t.y;
        g[4 * k + 2] = t.z;
        g[4 * k + 3] = t.w;
    }
}
__device__ __forceinline__ void g8_load(const G8<double>* p, int i, double (&g)[8]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double2 t = __ldg(&p[i].q[k]);
        g[2 * k] = t.x;
        g[2 * k + 1] = t.y;
    }
}

// Slots of G8.
constexpr int kGax = 0, kGay = 1, kGux = 2, kGuy = 3, kGvx = 4, kGvy = 5, kGA = 6, kGB = 7;

// LABFM_ADJ_PREFETCH: pass B takes the forward plan's L2 prefetch of the record
// stream (two iterations ahead, rows of kPrefetchMinRow entries or more).
#ifndef LABFM_ADJ_PREFETCH
#define LABFM_ADJ_PREFETCH 1
#endif

template <typename T>
PlanView<T> tview(const labfm_plan* p) {
    return PlanView<T>{p->N, p->tnnz_pad, p->trow_ptr, nullptr, static_cast<const T*>(p->tw),
                       static_cast<const T*>(p->twf), static_cast<const T*>(p->inv_s), p->dt_node,
                       LABFM_ADJ_PREFETCH ? p->prefetch : 0,
                       nullptr, nullptr, 0, p->N, nullptr, nullptr, T(0), T(0), T(0), T(0)};
}

// ---------------------------------------------------------------- pass A

// Pass A at node i from its state (a, u, v), its eight derivative combinations c
// (own_coeffs) and its cotangent M_i: the twelve derivative adjoints g_i and the
// own-value adjoints o_i.
template <typename T, bool SCALED>
__device__ __forceinline__ void node_adjoints_m(const PlanView<T>& P, int i, T a, T u, T v,
                                                const T (&c)[8], T ma, T mu, T mv,
                                                G8<T>* __restrict__ gout, Packed<T>* __restrict__ oout,
                                                const Phys<T>& ph) {
    const T is = SCALED ? P.inv_s[i] : T(1);
    const T s1 = SCALED ? is : T(1), s2 = SCALED ? is * is : T(1);
    const T nu = ph.mu * exp_neg(a);
    T g[8];
    g[kGax] = (-u * ma - ph.c2 * mu) * s1;
    g[kGay] = (-v * ma - ph.c2 * mv) * s1;
    g[kGux] = (-ma - u * mu) * s1;
    g[kGuy] = (-v * mu) * s1;
    g[kGvx] = (-u * mv) * s1;
    g[kGvy] = (-ma - v * mv) * s1;
    g[kGA] = (nu * mu) * s2;
    g[kGB] = (nu * mv) * s2;
    g8_store(gout, i, g);
    // c = (a_x, a_y, u_x, u_y, v_x, v_y, 4/3 u_xx + u_yy + 1/3 v_xy, 4/3 v_yy + v_xx + 1/3 u_xy)
    const T oa = -nu * (c[6] * mu + c[7] * mv);
    const T ou = -(c[0] * ma + c[2] * mu + c[4] * mv);
    const T ov = -(c[1] * ma + c[3] * mu + c[5] * mv);
    store(oout, i, oa, ou, ov);
}

template <typename T, bool SCALED>
__device__ __forceinline__ void node_adjoints(const PlanView<T>& P, int i, T a, T u, T v,
                                              const T (&c)[8], const Packed<T>* M,
                                              G8<T>* __restrict__ gout, Packed<T>* __restrict__ oout,
                                              const Phys<T>& ph) {
    T ma, mu, mv;
    unpack(M, i, ma, mu, mv);
    node_adjoints_m<T, SCALED>(P, i, a, u, v, c, ma, mu, mv, gout, oout, ph);
}

// Pass A of the previous stage, fused into the epilogue of the kernel that forms
// its cotangent (the filter transpose for stage 4, pass B of stage k for stage
// k - 1): at node k, from the stage's recorded state X and combinations D, the
// cotangent just computed in registers, written to g and o.  X == nullptr: none.
template <typename T>
struct FusedA {
    const Packed<T>* X;
    const D8<T>* D;
    G8<T>* g;
    Packed<T>* o;
    Phys<T> ph;
};

template <typename T>
__device__ __forceinline__ void fused_pass_a(const PlanView<T>& P, const FusedA<T>& fa, int k, T ma, T mu,
                                             T mv) {
    constexpr bool SCALED = std::is_same<T, float>::value;
    T a, u, v;
    unpack(fa.X, k, a, u, v);
    T c[8];
    d8_load(fa.D, k, c);
    node_adjoints_m<T, SCALED>(P, k, a, u, v, c, ma, mu, mv, fa.g, fa.o, fa.ph);
}

// Pass A with the derivatives gathered at X (the single right-hand-side adjoint).
template <typename T, int G, bool KAHAN, bool SCALED>
__global__ void k_adj_pointwise(PlanView<T> P, const Packed<T>* X, const Packed<T>* M,
                                G8<T>* __restrict__ gout, Packed<T>* __restrict__ oout, Phys<T> ph) {
    const int64_t gt = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t node = gt / G;
    const int gl = int(gt % G);
    const int i = node < P.N ? int(node) : -1;
    launch_prologue<T, false, G>(P, i, gl);
    const AoS<T> fld{X};
    T a = 0, u = 0, v = 0;
    if (i >= 0) fld.get(i, a, u, v);
    T d[12];
    gather_derivatives<T, G, KAHAN>(P, fld, i, gl, a, u, v, d);
    if (i < 0 || gl != 0) return;
    T c[8];
    own_coeffs<T, SCALED>(d, SCALED ? P.inv_s[i] : T(1), c);
    node_adjoints<T, SCALED>(P, i, a, u, v, c, M, gout, oout, ph);
}

// ---------------------------------------------------------------- pass B

// The transposed records hold, per entry (i -> k), c_0 = w^x_ik, c_1 = w^y_ik,
// c_2 = 4/3 w^xx_ik + w^yy_ik, c_3 = w^xx_ik + 4/3 w^yy_ik, c_4 = 1/3 w^xy_ik
// (in the slots of the forward x, y, xx, xy, yy weights), and rsum the same
// combinations of node k's forward row sums, so that with G8:
//   sum_d w^d_ik g_{u,d,i} = c_0 g_ux + c_1 g_uy + c_2 A + c_4 B,
//   sum_d w^d_ik g_{v,d,i} = c_0 g_vx + c_1 g_vy + c_3 B + c_4 A.
// MODE 0: out = Xbar.  MODE 1 (RK reverse sweep): Lam += Xbar, and when
// Fnext is not null, Fnext = dt_i (bprev Lam + cprev Xbar).
// With fa.X set, pass A of the previous stage follows at each node (fused_pass_a):
// it writes o at the node whose own adjoints this kernel has already read, and a
// G8 buffer other than gin.
template <typename T, int G, int MODE>
__global__ void k_adj_transpose(PlanView<T> PT, const G8<T>* gin, const Packed<T>* oin,
                                const T* __restrict__ rsum, Packed<T>* out, Packed<T>* Lam,
                                Packed<T>* Fnext, double dt, double bprev, double cprev, FusedA<T> fa) {
    const int64_t gt = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t node = gt / G;
    const int gl = int(gt % G);
    const int k = node < PT.N ? int(node) : -1;
    launch_prologue<T, false, G>(PT, k, gl);
    T sa = 0, su = 0, sv = 0;
    if (k >= 0) {
        const int e0 = PT.row_ptr[k];
        const int e1 = PT.row_ptr[k + 1];
        for (int e = e0 + 4 * gl; e < e1; e += 4 * G) {
#if LABFM_CHUNK_AOS == 3
            if constexpr (std::is_same<T, float>::value) {
                // lanes 0-2 of the group fetch into L2 one 128-byte segment each of the
                // record block they will read two iterations later (within the row)
                if (PT.pf > 0 && gl < 3 && e1 - e0 >= kPrefetchMinRow) {
                    const int ep = e + 4 * G * PT.pf;
                    if (ep < e1) {
                        const char* a = reinterpret_cast<const char*>(PT.w) + Rec<float>::col(ep >> 2) + gl * 128;
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
                    }
                }
            }
#endif
            int ci[4];
            T c0[4], c1[4], c2[4], c3[4], c4[4];
            load_rhs_chunk(PT, e, ci, c0, c1, c2, c3, c4, 0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                T g[8];
                g8_load(gin, ci[q], g);
                sa = fma(c0[q], g[kGax], sa);
                sa = fma(c1[q], g[kGay], sa);
                su = fma(c0[q], g[kGux], su);
                su = fma(c1[q], g[kGuy], su);
                su = fma(c2[q], g[kGA], su);
                su = fma(c4[q], g[kGB], su);
                sv = fma(c0[q], g[kGvx], sv);
                sv = fma(c1[q], g[kGvy], sv);
                sv = fma(c3[q], g[kGB], sv);
                sv = fma(c4[q], g[kGA], sv);
            }
        }
    }
    sa = group_sum<G>(sa);
    su = group_sum<G>(su);
    sv = group_sum<G>(sv);
    if (k < 0 || gl != 0) return;
    T g[8];
    g8_load(gin, k, g);
    T r[5];
#pragma unroll
    for (int o = 0; o < 5; ++o) r[o] = rsum[int64_t(o) * PT.N + k];
    T oa, ou, ov;
    unpack(oin, k, oa, ou, ov);
    const T xa = oa + sa - (r[0] * g[kGax] + r[1] * g[kGay]);
    const T xu = ou + su - (r[0] * g[kGux] + r[1] * g[kGuy] + r[2] * g[kGA] + r[4] * g[kGB]);
    const T xv = ov + sv - (r[0] * g[kGvx] + r[1] * g[kGvy] + r[3] * g[kGB] + r[4] * g[kGA]);
    if (MODE == 0) {
        store(out, k, xa, xu, xv);
        return;
    }
    T la, lu, lv;
    unpack_rw(Lam, k, la, lu, lv);
    la += xa;
    lu += xu;
    lv += xv;
    store(Lam, k, la, lu, lv);
    if (Fnext || fa.X) {
        const double h = PT.dt_node ? PT.dt_node[k] : dt;
        const T cb = T(h * bprev), cx = T(h * cprev);
        const T fa_ = cb * la + cx * xa, fu = cb * lu + cx * xu, fv = cb * lv + cx * xv;
        if (Fnext) store(Fnext, k, fa_, fu, fv);
        if (fa.X) fused_pass_a(PT, fa, k, fa_, fu, fv);
    }
}

// ---------------------------------------------------------------- filter adjoint

// Lam_out = lam + L_hyp^T (kappa lam) = lam + sum_i wf_ik lam_i - (sum_j wf_kj) lam_k;
// F_out (if not null) = dt_k b4 Lam_out.
template <typename T, int G>
__global__ void k_filter_adjoint(PlanView<T> PT, const Packed<T>* lam, const T* __restrict__ rsum_f,
                                 Packed<T>* Lam_out, Packed<T>* F_out, double dt, double b4, FusedA<T> fa) {
    const int64_t gt = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t node = gt / G;
    const int gl = int(gt % G);
    const int k = node < PT.N ? int(node) : -1;
    launch_prologue<T, true, G>(PT, k, gl);
    const AoS<T> fld{lam};
    T sa = 0, su = 0, sv = 0;
    if (k >= 0) {
        const int e0 = PT.row_ptr[k];
        const int e1 = PT.row_ptr[k + 1];
        for (int e = e0 + 4 * gl; e < e1; e += 4 * G) {
            int ci[4];
            T wf[4];
            load_filt_chunk(PT, e, ci, wf, 0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                T a, u, v;
                fld.get(ci[q], a, u, v);
                sa = fma(wf[q], a, sa);
                su = fma(wf[q], u, su);
                sv = fma(wf[q], v, sv);
            }
        }
    }
    sa = group_sum<G>(sa);
    su = group_sum<G>(su);
    sv = group_sum<G>(sv);
    if (k < 0 || gl != 0) return;
    T a, u, v;
    fld.get(k, a, u, v);
    const T r = rsum_f[k];
    const T la = a + sa - r * a, lu = u + su - r * u, lv = v + sv - r * v;
    store(Lam_out, k, la, lu, lv);
    if (F_out || fa.X) {
        const double h = PT.dt_node ? PT.dt_node[k] : dt;
        const T cb = T(h * b4);
        if (F_out) store(F_out, k, cb * la, cb * lu, cb * lv);
        if (fa.X) fused_pass_a(PT, fa, k, cb * la, cb * lu, cb * lv);
    }
}

// ---------------------------------------------------------------- transposed operator build

// The combinations of the five RHS weights w (x, y, xx, xy, yy) that pass B
// applies to the G8 adjoints, formed in FP64 and rounded once to T.
template <typename T>
__device__ __forceinline__ void adjoint_combinations(const double (&w)[5], T (&c)[5]) {
    c[0] = T(w[0]);
    c[1] = T(w[1]);
    c[2] = T(4.0 / 3.0 * w[2] + w[4]);
    c[3] = T(w[2] + 4.0 / 3.0 * w[4]);
    c[4] = T(w[3] / 3.0);
}
template <typename T>
__device__ __forceinline__ void adjoint_combinations(const double (&w)[6], T (&c)[5]) {
    const double v[5] = {w[0], w[1], w[2], w[3], w[4]};
    adjoint_combinations(v, c);
}

// Warp per forward row i: count the in-degree of every column k (pads, which
// point at the row itself, are skipped).
template <typename T>
__global__ void k_in_degree(PlanView<T> P, int32_t* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; i < P.N; i += warps) {
        const int e0 = P.row_ptr[i], e1 = P.row_ptr[i + 1];
        for (int e = e0 + lane; e < e1; e += 32) {
            const int k = *reinterpret_cast<const int32_t*>(reinterpret_cast<const char*>(P.w) + Rec<T>::col_e(e));
            if (k != i) atomicAdd(cnt + k, 1);
        }
    }
}

__global__ void k_pad4(int64_t N, const int32_t* __restrict__ cnt, int32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N;
         i += int64_t(gridDim.x) * blockDim.x)
        out[i] = (cnt[i] + 3) & ~3;
}

// Warp per forward row i: append (i, e) to the transposed row of every column.
template <typename T>
__global__ void k_fill_transposed(PlanView<T> P, const int32_t* __restrict__ trow,
                                  int32_t* __restrict__ cursor, int32_t* __restrict__ ti,
                                  int32_t* __restrict__ te) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; i < P.N; i += warps) {
        const int e0 = P.row_ptr[i], e1 = P.row_ptr[i + 1];
        for (int e = e0 + lane; e < e1; e += 32) {
            const int k = *reinterpret_cast<const int32_t*>(reinterpret_cast<const char*>(P.w) + Rec<T>::col_e(e));
            if (k == i) continue;
            const int slot = trow[k] + atomicAdd(cursor + k, 1);
            ti[slot] = int32_t(i);
            te[slot] = e;
        }
    }
}

// Warp per transposed row k: order the entries by source row i (the fill order
// is nondeterministic) and write the records: column i, the combinations of
// the forward weights of entry (i -> k) that pass B applies (k_adj_transpose:
// w^x, w^y, 4/3 w^xx + w^yy, w^xx + 4/3 w^yy, 1/3 w^xy, formed in FP64 and
// rounded once), and the filter weight; pads point at k with weight 0.
template <typename T>
__global__ void k_write_transposed(PlanView<T> P, int64_t N, const int32_t* __restrict__ trow,
                                   const int32_t* __restrict__ cnt, const int32_t* __restrict__ ti,
                                   const int32_t* __restrict__ te, T* __restrict__ tw,
                                   T* __restrict__ twf) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t k = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; k < N; k += warps) {
        const int t0 = trow[k], plen = trow[k + 1] - t0, len = cnt[k];
        for (int q = lane; q < plen; q += 32) {
            int32_t src_i = int32_t(k);
            T v[5] = {T(0), T(0), T(0), T(0), T(0)};
            T vf = T(0);
            int rank = q;
            if (q < len) {
                src_i = ti[t0 + q];
                rank = 0;
                for (int r = 0; r < len; ++r) rank += ti[t0 + r] < src_i;
                const int e = te[t0 + q];
                const char* rb = reinterpret_cast<const char*>(P.w);
                double f[5];
#pragma unroll
                for (int d = 0; d < 5; ++d) f[d] = double(*reinterpret_cast<const T*>(rb + Rec<T>::w_e(e, d)));
                adjoint_combinations(f, v);
                vf = *reinterpret_cast<const T*>(reinterpret_cast<const char*>(P.wf) + Rec<T>::fw_e(e));
            }
            // the same transposition within 16-entry segments as the forward records,
            // so that the lanes of a group gather consecutive entries
            const int64_t dst = int64_t(t0) + entry_slot(rank, plen);
            char* tb = reinterpret_cast<char*>(tw);
            *reinterpret_cast<int32_t*>(tb + Rec<T>::col_e(dst)) = src_i;
#pragma unroll
            for (int d = 0; d < 5; ++d) *reinterpret_cast<T*>(tb + Rec<T>::w_e(dst, d)) = v[d];
            char* tfb = reinterpret_cast<char*>(twf);
            *reinterpret_cast<int32_t*>(tfb + Rec<T>::fcol_e(dst)) = src_i;
            *reinterpret_cast<T*>(tfb + Rec<T>::fw_e(dst)) = vf;
        }
    }
}

// Warp per forward row i: sums of its RHS weights (stored as the combinations
// of adjoint_combinations) and of its filter weights (pads add 0).
template <typename T>
__global__ void k_row_sums(PlanView<T> P, T* __restrict__ rsum) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; i < P.N; i += warps) {
        const int e0 = P.row_ptr[i], e1 = P.row_ptr[i + 1];
        double acc[6] = {0, 0, 0, 0, 0, 0};
        for (int e = e0 + lane; e < e1; e += 32) {
            const char* rb = reinterpret_cast<const char*>(P.w);
#pragma unroll
            for (int d = 0; d < 5; ++d) acc[d] += double(*reinterpret_cast<const T*>(rb + Rec<T>::w_e(e, d)));
            acc[5] += double(*reinterpret_cast<const T*>(reinterpret_cast<const char*>(P.wf) + Rec<T>::fw_e(e)));
        }
#pragma unroll
        for (int d = 0; d < 6; ++d) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[d] += __shfl_xor_sync(0xffffffffu, acc[d], o);
        }
        T comb[5];
        adjoint_combinations(acc, comb);
        if (lane == 0) {
#pragma unroll
            for (int d = 0; d < 5; ++d) rsum[int64_t(d) * P.N + i] = comb[d];
            rsum[int64_t(5) * P.N + i] = T(acc[5]);
        }
    }
}

template <typename T>
int build_transposed(labfm_plan* p, cudaStream_t st) {
    const int64_t N = p->N;
    const PlanView<T> P = view<T>(p);
    int32_t *cnt = nullptr, *pcnt = nullptr, *cursor = nullptr, *ti = nullptr, *te = nullptr;
    int64_t* total = nullptr;
    void* scan_tmp = nullptr;
    const size_t scan_bytes = exclusive_scan_scratch_bytes(N);
    LABFM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&cnt), size_t(N) * 4, st));
    LABFM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&pcnt), size_t(N) * 4, st));
    LABFM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&cursor), size_t(N) * 4, st));
    LABFM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&total), 8, st));
    LABFM_CUDA_TRY(cudaMallocAsync(&scan_tmp, scan_bytes, st));
    LABFM_CUDA_TRY(cudaMemsetAsync(cnt, 0, size_t(N) * 4, st));
    LABFM_CUDA_TRY(cudaMemsetAsync(cursor, 0, size_t(N) * 4, st));
    const int gw = int(std::min<int64_t>((N * 32 + 255) / 256, 1 << 20));
    const int gn = int(std::min<int64_t>((N + 255) / 256, 65535));
    k_in_degree<T><<<gw, 256, 0, st>>>(P, cnt);
    k_pad4<<<gn, 256, 0, st>>>(N, cnt, pcnt);
    LABFM_LAUNCH_CHECK("in-degree kernels");
    LABFM_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&p->trow_ptr), size_t(N + 1) * 4));
    int rc = exclusive_scan_i32(pcnt, p->trow_ptr, N, total, scan_tmp, scan_bytes, st);
    int64_t tpad = 0;
    if (rc == LABFM_OK) {
        cudaError_t e = cudaMemcpyAsync(&tpad, total, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_error(e, "reading transposed size");
    }
    const size_t es = sizeof(T);
    const size_t np = size_t(std::max<int64_t>(tpad, 4));
    if (rc == LABFM_OK) {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&ti), np * 4, st);
        if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&te), np * 4, st);
        if (e == cudaSuccess) e = cudaMalloc(&p->tw, Rec<T>::rhs_bytes(int64_t(np)));
        if (e == cudaSuccess) e = cudaMalloc(&p->twf, Rec<T>::filt_bytes(int64_t(np)));
        if (e == cudaSuccess) e = cudaMalloc(&p->rsum, size_t(6) * N * es);
        if (e != cudaSuccess) rc = cuda_error(e, "transposed operator allocation");
    }
    if (rc == LABFM_OK) {
        p->tnnz_pad = tpad;
        p->device_bytes += (N + 1) * 4 + Rec<T>::rhs_bytes(int64_t(np)) + Rec<T>::filt_bytes(int64_t(np)) + 6 * N * es;
        k_fill_transposed<T><<<gw, 256, 0, st>>>(P, p->trow_ptr, cursor, ti, te);
        k_write_transposed<T><<<gw, 256, 0, st>>>(P, N, p->trow_ptr, cnt, ti, te, static_cast<T*>(p->tw),
                                                  static_cast<T*>(p->twf));
        k_row_sums<T><<<gw, 256, 0, st>>>(P, static_cast<T*>(p->rsum));
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_error(e, "transposed operator kernels");
    }
    cudaFreeAsync(cnt, st);
    cudaFreeAsync(pcnt, st);
    cudaFreeAsync(cursor, st);
    cudaFreeAsync(total, st);
    cudaFreeAsync(scan_tmp, st);
    if (ti) cudaFreeAsync(ti, st);
    if (te) cudaFreeAsync(te, st);
    if (rc == LABFM_OK) {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_error(e, "building the transposed operator");
    }
    return rc;
}

// ---------------------------------------------------------------- launches

template <typename T>
struct AdjWork {
    Packed<T>* X[4];
    Packed<T>* P;
    Packed<T>* Lam;
    Packed<T>* Fb;
    Packed<T>* Ob;
    G8<T>* g;
    D8<T>* D;  // 4 x N: the stages' derivative combinations (recomputing sweep)
    G8<T>* g2;  // the second derivative-adjoint buffer of the reverse sweep
};

template <typename T>
AdjWork<T> split_work(const labfm_plan* p, void* work) {
    AdjWork<T> w;
    Packed<T>* base = static_cast<Packed<T>*>(work);
    for (int k = 0; k < 4; ++k) w.X[k] = base + k * p->N;
    w.P = base + 4 * p->N;
    w.Lam = base + 5 * p->N;
    w.Fb = base + 6 * p->N;
    w.Ob = base + 7 * p->N;
    w.g = reinterpret_cast<G8<T>*>(base + 8 * p->N);
    w.D = reinterpret_cast<D8<T>*>(w.g + p->N);
    w.g2 = reinterpret_cast<G8<T>*>(w.D + 4 * p->N);
    return w;
}

// Passes A and B run one-warp blocks, as the stage kernels do (every warp retires on
// its own): the backward pass of 100 steps 72.09 -> 71.34 ms (64-thread blocks
// 71.96 ms) against the plan's 128-thread blocks, which the filter transpose keeps.
constexpr int kAdjGatherBlock = 32;
template <typename T, int G>
int pass_a_g(const labfm_plan* p, const Packed<T>* X, const Packed<T>* M, G8<T>* g, Packed<T>* o,
             const Phys<T>& ph, cudaStream_t st) {
    constexpr bool F = std::is_same<T, float>::value;
    const int blk = kAdjGatherBlock;
    const int grid = int((p->N * G + blk - 1) / blk);
    cudaError_t e = launch_pdl(p, k_adj_pointwise<T, G, F, F>, grid, blk, st, view<T>(p), X, M, g, o, ph);
    if (e != cudaSuccess) return cuda_error(e, "adjoint pointwise kernel");
    return LABFM_OK;
}

template <typename T, int G>
int pass_b_g(const labfm_plan* p, int mode, const G8<T>* g, const Packed<T>* o, Packed<T>* out,
             Packed<T>* Lam, Packed<T>* Fnext, double dt, double bprev, double cprev, const FusedA<T>& fa,
             cudaStream_t st) {
    const int blk = kAdjGatherBlock;
    const int grid = int((p->N * G + blk - 1) / blk);
    const T* rs = static_cast<const T*>(p->rsum);
    cudaError_t e = mode == 0 ? launch_pdl(p, k_adj_transpose<T, G, 0>, grid, blk, st, tview<T>(p), g, o, rs, out,
                                           Lam, Fnext, dt, bprev, cprev, fa)
                              : launch_pdl(p, k_adj_transpose<T, G, 1>, grid, blk, st, tview<T>(p), g, o, rs, out,
                                           Lam, Fnext, dt, bprev, cprev, fa);
    if (e != cudaSuccess) return cuda_error(e, "adjoint transpose kernel");
    return LABFM_OK;
}

template <typename T, int G>
int filt_adj_g(const labfm_plan* p, const Packed<T>* lam, Packed<T>* Lam, Packed<T>* F, double dt,
               double b4, const FusedA<T>& fa, cudaStream_t st) {
    const int grid = int((p->N * G + p->block - 1) / p->block);
    const T* rsf = static_cast<const T*>(p->rsum) + 5 * p->N;
    cudaError_t e = launch_pdl(p, k_filter_adjoint<T, G>, grid, p->block, st, tview<T>(p), lam, rsf, Lam, F, dt, b4, fa);
    if (e != cudaSuccess) return cuda_error(e, "filter adjoint kernel");
    return LABFM_OK;
}

#define LABFM_G_DISPATCH(call)                                  \
    switch (p->group) {                                         \
        case 2: { constexpr int G = 2; return call; }           \
        case 4: { constexpr int G = 4; return call; }           \
        case 8: { constexpr int G = 8; return call; }           \
        case 16: { constexpr int G = 16; return call; }         \
        case 32: { constexpr int G = 32; return call; }         \
    }                                                           \
    return set_error(LABFM_EINVAL, "unsupported group size")

template <typename T>
int pass_a(const labfm_plan* p, const Packed<T>* X, const Packed<T>* M, G8<T>* g, Packed<T>* o,
           const Phys<T>& ph, cudaStream_t st) {
    LABFM_G_DISPATCH((pass_a_g<T, G>(p, X, M, g, o, ph, st)));
}

template <typename T>
int pass_b(const labfm_plan* p, int mode, const G8<T>* g, const Packed<T>* o, Packed<T>* out,
           Packed<T>* Lam, Packed<T>* Fnext, double dt, double bprev, double cprev, const FusedA<T>& fa,
           cudaStream_t st) {
    LABFM_G_DISPATCH((pass_b_g<T, G>(p, mode, g, o, out, Lam, Fnext, dt, bprev, cprev, fa, st)));
}

template <typename T>
int filt_adj(const labfm_plan* p, const Packed<T>* lam, Packed<T>* Lam, Packed<T>* F, double dt,
             double b4, const FusedA<T>& fa, cudaStream_t st) {
    LABFM_G_DISPATCH((filt_adj_g<T, G>(p, lam, Lam, F, dt, b4, fa, st)));
}

template <typename T>
int rhs_adjoint_t(const labfm_plan* p, const void* fields, const void* lambda, void* grad,
                  const labfm_phys* php, void* work, cudaStream_t st) {
    const Phys<T> ph{T(php->c2), T(php->mu), T(php->gx), T(php->gy)};
    AdjWork<T> w = split_work<T>(p, work);
    int rc;
    if ((rc = pack_fields(p, fields, w.X[0], st))) return rc;
    if ((rc = pack_fields(p, lambda, w.Fb, st))) return rc;
    if ((rc = pass_a<T>(p, w.X[0], w.Fb, w.g, w.Ob, ph, st))) return rc;
    const FusedA<T> none{nullptr, nullptr, nullptr, nullptr, ph};
    if ((rc = pass_b<T>(p, 0, w.g, w.Ob, w.Lam, nullptr, nullptr, 0.0, 0.0, 0.0, none, st))) return rc;
    return unpack_fields(p, w.Lam, grad, st);
}

// The reverse sweep of one step given its stage states X[0..3] (packed) and
// their derivative combinations D (4 x N).
template <typename T>
int adjoint_sweep_t(const labfm_plan* p, const Packed<T>* const (&X)[4], const D8<T>* D, void* lambda,
                    double dt, const Phys<T>& ph, AdjWork<T>& w, cudaStream_t st) {
    int rc;
    labfm_plan* pm = const_cast<labfm_plan*>(p);  // only the launch-timing record changes
    // filter transpose (with pass A of stage 4 fused into it), then the stages
    // backwards, each pass B with pass A of the stage before it fused in; the
    // derivative adjoints alternate between two buffers, since pass B gathers its
    // neighbours' while the fused pass A writes the next stage's
    if ((rc = pack_fields(p, lambda, w.Fb, st))) return rc;
    G8<T>* gbuf[2] = {w.g, w.g2};
    int ev = prof_begin(pm, kProfAdjFilter, st);
    const FusedA<T> a4{X[3], D + 3 * p->N, gbuf[0], w.Ob, ph};
    if ((rc = filt_adj<T>(p, w.Fb, w.Lam, nullptr, dt, kRkB[3], a4, st))) return rc;
    prof_end(pm, ev, st);
    for (int k = 3; k >= 0; --k) {
        const int cur = (3 - k) & 1;
        const double bprev = k > 0 ? kRkB[k - 1] : 0.0;
        const double cprev = k > 0 ? kRkA[k - 1] - kRkB[k - 1] : 0.0;
        const FusedA<T> next = k > 0 ? FusedA<T>{X[k - 1], D + (k - 1) * p->N, gbuf[cur ^ 1], w.Ob, ph}
                                     : FusedA<T>{nullptr, nullptr, nullptr, nullptr, ph};
        ev = prof_begin(pm, kProfAdjB, st);
        if ((rc = pass_b<T>(p, 1, gbuf[cur], w.Ob, nullptr, w.Lam, nullptr, dt, bprev, cprev, next, st)))
            return rc;
        prof_end(pm, ev, st);
    }
    return unpack_fields(p, w.Lam, lambda, st);
}

template <typename T>
int rk_step_adjoint_t(const labfm_plan* p, const void* Q, void* lambda, double dt,
                      const labfm_phys* php, void* work, cudaStream_t st) {
    const Phys<T> ph{T(php->c2), T(php->mu), T(php->gx), T(php->gy)};
    AdjWork<T> w = split_work<T>(p, work);
    int rc;
    // forward recompute of the stage states X1..X4 of this step and of their
    // derivative combinations (the same kernels as labfm_rk_step_record)
    if ((rc = pack_fields(p, Q, w.X[0], st))) return rc;
    if ((rc = forward_stages(p, w.X[0], w.P, w.X[1], w.X[2], w.X[3], w.D, dt, php, st))) return rc;
    const Packed<T>* const X[4] = {w.X[0], w.X[1], w.X[2], w.X[3]};
    return adjoint_sweep_t<T>(p, X, w.D, lambda, dt, ph, w, st);
}

template <typename T>
int rk_step_adjoint_recorded_t(const labfm_plan* p, const void* states, void* lambda, double dt,
                               const labfm_phys* php, void* work, cudaStream_t st) {
    const Phys<T> ph{T(php->c2), T(php->mu), T(php->gx), T(php->gy)};
    AdjWork<T> w = split_work<T>(p, work);
    const Packed<T>* S = static_cast<const Packed<T>*>(states);
    const Packed<T>* const X[4] = {S, S + p->N, S + 2 * p->N, S + 3 * p->N};
    const D8<T>* D = reinterpret_cast<const D8<T>*>(S + 4 * p->N);
    return adjoint_sweep_t<T>(p, X, D, lambda, dt, ph, w, st);
}

template <typename T>
int filter_adjoint_t(const labfm_plan* p, const void* lam_in, void* lam_out, void* work,
                     cudaStream_t st) {
    AdjWork<T> w = split_work<T>(p, work);
    int rc;
    if ((rc = pack_fields(p, lam_in, w.Ob, st))) return rc;
    const FusedA<T> none{nullptr, nullptr, nullptr, nullptr, Phys<T>{}};
    if ((rc = filt_adj<T>(p, w.Ob, w.Lam, nullptr, 0.0, 0.0, none, st))) return rc;
    return unpack_fields(p, w.Lam, lam_out, st);
}

size_t adjoint_work_bytes(const labfm_plan* p) {
    if (p->dtype == LABFM_F32)
        return size_t(p->N) * (8 * sizeof(Packed<float>) + 2 * sizeof(G8<float>) + 4 * sizeof(D8<float>));
    return size_t(p->N) * (8 * sizeof(Packed<double>) + 2 * sizeof(G8<double>) + 4 * sizeof(D8<double>));
}

int check_adjoint(const labfm_plan* p, void* work, size_t work_bytes) {
    if (!p || !p->row_ptr) return set_error(LABFM_EINVAL, "null or empty plan");
    if (p->wall_slot) return set_error(LABFM_EINVAL, "the adjoint of a plan with walls is not implemented");
    if (p->n_ranges) return set_error(LABFM_EINVAL, "the adjoint calls do not take launch ranges");
    if (!p->trow_ptr) return set_error(LABFM_EINVAL, "call labfm_plan_enable_adjoint first");
    if (!work) return set_error(LABFM_EINVAL, "null work buffer");
    if (work_bytes < adjoint_work_bytes(p))
        return set_error(LABFM_EINVAL, "work buffer smaller than labfm_adjoint_workspace_bytes");
    if (reinterpret_cast<uintptr_t>(work) % 16 != 0)
        return set_error(LABFM_EINVAL, "work buffer must be 16-byte aligned");
    return LABFM_OK;
}

}  // namespace
}  // namespace labfm

using namespace labfm;

extern "C" int labfm_plan_enable_adjoint(labfm_plan* p, void* stream) {
    LABFM_NVTX("labfm_plan_enable_adjoint");
    if (!p || !p->row_ptr) return set_error(LABFM_EINVAL, "null or empty plan");
    if (p->trow_ptr) return LABFM_OK;
    if (fault_alloc()) return injected_alloc_error("labfm_plan_enable_adjoint");
    cudaStream_t st = as_stream(stream);
    return p->dtype == LABFM_F32 ? build_transposed<float>(p, st) : build_transposed<double>(p, st);
}

extern "C" size_t labfm_adjoint_workspace_bytes(const labfm_plan* p) {
    return p ? adjoint_work_bytes(p) : 0;
}

extern "C" int labfm_rhs_adjoint(const labfm_plan* p, const void* fields, const void* lambda,
                                 void* grad, const labfm_phys* phys, void* work, size_t work_bytes,
                                 void* stream) {
    LABFM_NVTX("labfm_rhs_adjoint");
    if (int rc = check_adjoint(p, work, work_bytes)) return rc;
    if (!fields || !lambda || !grad || !phys) return set_error(LABFM_EINVAL, "null pointer argument");
    cudaStream_t st = as_stream(stream);
    return p->dtype == LABFM_F32 ? rhs_adjoint_t<float>(p, fields, lambda, grad, phys, work, st)
                                 : rhs_adjoint_t<double>(p, fields, lambda, grad, phys, work, st);
}

extern "C" int labfm_rk_step_adjoint(const labfm_plan* p, const void* Q, void* lambda, double dt,
                                     const labfm_phys* phys, void* work, size_t work_bytes,
                                     void* stream) {
    LABFM_NVTX("labfm_rk_step_adjoint");
    if (int rc = check_adjoint(p, work, work_bytes)) return rc;
    if (!Q || !lambda || !phys) return set_error(LABFM_EINVAL, "null pointer argument");
    if (!(dt > 0.0) && !(dt == 0.0 && p->dt_node))
        return set_error(LABFM_EINVAL, "dt must be positive (or 0 with per-instance dt set)");
    cudaStream_t st = as_stream(stream);
    return p->dtype == LABFM_F32 ? rk_step_adjoint_t<float>(p, Q, lambda, dt, phys, work, st)
                                 : rk_step_adjoint_t<double>(p, Q, lambda, dt, phys, work, st);
}

extern "C" size_t labfm_stage_states_bytes(const labfm_plan* p) {
    if (!p || !p->row_ptr) return 0;
    return size_t(4) * size_t(p->N) * (packed_bytes(p) + d8_bytes(p));
}

extern "C" int labfm_rk_step_record(const labfm_plan* p, void* Q, void* states, size_t states_bytes,
                                    void* work, size_t work_bytes, double dt, const labfm_phys* phys,
                                    void* stream) {
    LABFM_NVTX("labfm_rk_step_record");
    if (!p || !p->row_ptr) return set_error(LABFM_EINVAL, "null or empty plan");
    if (p->wall_slot) return set_error(LABFM_EINVAL, "the recording step of a plan with walls is not implemented");
    if (p->n_ranges) return set_error(LABFM_EINVAL, "the recording step does not take launch ranges");
    if (!Q || !states || !work || !phys) return set_error(LABFM_EINVAL, "null pointer argument");
    if (states_bytes < labfm_stage_states_bytes(p))
        return set_error(LABFM_EINVAL, "states buffer smaller than labfm_stage_states_bytes");
    if (work_bytes < rk_work_bytes(p))
        return set_error(LABFM_EINVAL, "work buffer smaller than labfm_rk_workspace_bytes");
    if ((reinterpret_cast<uintptr_t>(states) | reinterpret_cast<uintptr_t>(work)) % 16 != 0)
        return set_error(LABFM_EINVAL, "states and work buffers must be 16-byte aligned");
    if (!(dt > 0.0) && !(dt == 0.0 && p->dt_node))
        return set_error(LABFM_EINVAL, "dt must be positive (or 0 with per-instance dt set)");
    const size_t ps = p->dtype == LABFM_F32 ? sizeof(Packed<float>) : sizeof(Packed<double>);
    char* wb = static_cast<char*>(work);
    return rk_step_record(p, Q, states, wb, wb + size_t(p->N) * ps, dt, phys, as_stream(stream));
}

extern "C" int labfm_rk_step_adjoint_recorded(const labfm_plan* p, const void* states, void* lambda,
                                              double dt, const labfm_phys* phys, void* work,
                                              size_t work_bytes, void* stream) {
    LABFM_NVTX("labfm_rk_step_adjoint_recorded");
    if (int rc = check_adjoint(p, work, work_bytes)) return rc;
    if (!states || !lambda || !phys) return set_error(LABFM_EINVAL, "null pointer argument");
    if (reinterpret_cast<uintptr_t>(states) % 16 != 0)
        return set_error(LABFM_EINVAL, "states buffer must be 16-byte aligned");
    if (!(dt > 0.0) && !(dt == 0.0 && p->dt_node))
        return set_error(LABFM_EINVAL, "dt must be positive (or 0 with per-instance dt set)");
    cudaStream_t st = as_stream(stream);
    return p->dtype == LABFM_F32 ? rk_step_adjoint_recorded_t<float>(p, states, lambda, dt, phys, work, st)
                                 : rk_step_adjoint_recorded_t<double>(p, states, lambda, dt, phys, work, st);
}

extern "C" int labfm_filter_adjoint(const labfm_plan* p, const void* lam_in, void* lam_out,
                                    void* work, size_t work_bytes, void* stream) {
    LABFM_NVTX("labfm_filter_adjoint");
    if (int rc = check_adjoint(p, work, work_bytes)) return rc;
    if (!lam_in || !lam_out) return set_error(LABFM_EINVAL, "null pointer argument");
    cudaStream_t st = as_stream(stream);
    return p->dtype == LABFM_F32 ? filter_adjoint_t<float>(p, lam_in, lam_out, work, st)
                                 : filter_adjoint_t<double>(p, lam_in, lam_out, work, st);
}
