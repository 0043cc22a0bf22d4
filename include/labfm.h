/*
 * labfm.h -- C ABI of the GB300 (sm_103a) LABFM hot path.
 *
 * LABFM (local anisotropic basis function method) for the isothermal
 * compressible Navier-Stokes equations, after King & Lind, "High-order
 * simulations of isothermal flows using the local anisotropic basis function
 * method (LABFM)".  Section numbers and equation labels below refer to that
 * paper.
 *
 * Conventions for every entry point:
 *  - Pointers named as device buffers are caller-owned CUDA device memory; the
 *    library never frees them.  Host pointers are marked "host".
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    All device work is ordered on that stream; calls return after enqueueing
 *    unless a comment says the call synchronises.
 *  - Return value: LABFM_OK (0) or a labfm_status error code.  No call aborts,
 *    traps or throws.  labfm_last_error() returns a thread-local message for the
 *    most recent failing call on this thread.
 *  - Fault injection (for tests of callers' error handling): the environment
 *    variable LABFM_FAULT, read at each call, makes entry points fail on the
 *    host as they would on a real fault.  "alloc": every call that would
 *    allocate device memory (plan creation, labfm_build_stencils,
 *    labfm_build_weights with n_failed_out, labfm_plan_set_dt's first call,
 *    labfm_plan_set_staging, labfm_plan_enable_adjoint, labfm_step_graph_create)
 *    returns LABFM_ENOMEM before touching the device.  "capacity":
 *    labfm_build_stencils with a col buffer returns LABFM_ECAPACITY with
 *    *nnz_out = col_capacity + 1 before touching the device.
 *    "singular_node:<i>": labfm_build_weights also flags node i
 *    LABFM_NODE_SINGULAR (and counts it as failed).  "timeout":
 *    labfm_plan_device_status reports LABFM_ETIMEOUT as a bounded wait that ran
 *    out would.  Unset or any other value: nothing is injected.
 *  - A caller's CSR (row_ptr N + 1 int32, col nnz int32) is checked before any
 *    kernel indexes with it, by labfm_plan_create(_batched), labfm_build_weights,
 *    labfm_stencil_optimise and labfm_modal_response: row_ptr[0] = 0, row_ptr
 *    non-decreasing, row_ptr[N] = nnz where nnz is given, every column in [0, N).
 *    A malformed one returns LABFM_EINVAL naming the problem; the check reads only
 *    the declared buffers and synchronises the stream.
 *  - Node arrays are indexed 0..N-1.  Fields are structure-of-arrays, "3 x N":
 *    field f of node i at [f * N + i], f = 0 (ln rho), 1 (u), 2 (v).
 *  - Operator order in every weight array (Section 2, selector C^d):
 *    0: d/dx, 1: d/dy, 2: d2/dx2, 3: d2/dxdy, 4: d2/dy2, 5: hyperviscous nabla^m.
 */
#ifndef LABFM_H
#define LABFM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum labfm_status {
    LABFM_OK = 0,
    LABFM_EINVAL = 1,      /* bad argument (null pointer, size, order, alignment) */
    LABFM_ECUDA = 2,       /* a CUDA runtime call or launch failed */
    LABFM_ENOMEM = 3,      /* device allocation failed */
    LABFM_ECAPACITY = 4,   /* output buffer too small (required size reported) */
    LABFM_ESINGULAR = 5,   /* at least one node's moment matrix is singular */
    LABFM_ENONFINITE = 6,  /* a non-finite value was produced */
    LABFM_ETIMEOUT = 7     /* a bounded device-side wait ran out */
} labfm_status;

typedef enum labfm_dtype {
    LABFM_F64 = 0,  /* fields and weights in double precision */
    LABFM_F32 = 1   /* fields in float, weights in float nondimensionalised by s_i^l */
} labfm_dtype;

/* Per-node flags written by labfm_build_weights into node_status. */
#define LABFM_NODE_FEW_NEIGHBOURS 1  /* fewer stencil nodes than unknowns n */
#define LABFM_NODE_SINGULAR 2        /* zero or non-finite pivot in the LU */
#define LABFM_NODE_NONFINITE 4       /* non-finite weight or filter coefficient */

/* Physical constants of the isothermal equations (Section 7, eq. icns):
 * c2 = c^2 (speed of sound squared), mu = dynamic viscosity, (gx, gy) = body force. */
typedef struct labfm_phys {
    double c2;
    double mu;
    double gx;
    double gy;
} labfm_phys;

/* Kinds of boundary node (labfm_plan_set_boundaries, Section 7.1). */
#define LABFM_WALL 0     /* no-slip wall */
#define LABFM_INFLOW 1   /* partially reflecting inflow */
#define LABFM_OUTFLOW 2  /* partially reflecting outflow (eq. outflowL) */

/* Parameters of the inflow and outflow conditions (Section 7.1): the relaxation
 * coefficient sigma (0.278 in the paper), the length L of the relaxation terms
 * (the paper does not give it; the domain's length along the flow), the reference
 * Mach number M and the reference density rho0 of the inflow's L4. */
typedef struct labfm_nscbc {
    double sigma;
    double L;
    double mach;
    double rho0;
} labfm_nscbc;

/* An operator prepared for the time-step kernels (opaque). */
typedef struct labfm_plan labfm_plan;

typedef struct labfm_plan_info {
    int64_t N;          /* nodes */
    int64_t nnz;        /* stencil entries (unpadded) */
    int64_t nnz_padded; /* entries after padding each row to a multiple of 4 */
    int32_t dtype;      /* labfm_dtype */
    int32_t group;      /* lanes per node in the gather kernels */
    int32_t block;      /* threads per block in the gather kernels */
    int32_t n_instances; /* independent instances (1 unless built by labfm_plan_create_batched) */
    int32_t entry_bytes;        /* bytes of the RHS record stream per padded stencil entry */
    int32_t filter_entry_bytes; /* bytes of the filter record stream per padded entry */
    int64_t device_bytes; /* device memory owned by the plan */
    int32_t prefetch;     /* L2 prefetch distance of the F32 record stream (labfm_plan_set_prefetch) */
    int32_t stages;       /* shared-memory staging slots (labfm_plan_set_staging; 0 = off) */
    int32_t filter_group; /* lanes per node of the filter kernel (labfm_plan_set_filter_launch) */
    int32_t filter_persistent; /* 1 if the filter runs a persistent grid-stride grid */
    int32_t programmatic; /* 1 if the kernels use programmatic launches (labfm_plan_set_programmatic_launch) */
} labfm_plan_info;

/* Message for the most recent failing call on this thread ("" if none). */
const char* labfm_last_error(void);

/* ABI version of this header (incremented on incompatible changes). */
int labfm_abi_version(void);

/*
 * Neighbour search (Section 2): the stencil of node i is every node j != i with
 * |r_j - r_i|^2 <= (2 h_i)^2, tested exactly in FP64 (products and sums rounded
 * separately, no fused multiply-add) on the periodic minimum image
 * dx = x_j - x_i; dx -= Lx if dx > Lx/2; dx += Lx if dx < -Lx/2 (same in y).
 *
 *   xy        device, N x 2 doubles (x_i, y_i) row-major; 0 <= x < Lx on a periodic
 *             axis, 0 <= x <= Lx on a bounded one (a wall may lie on the edge), same in y
 *   h         device, N doubles, stencil scale h_i > 0
 *   periodic_mask  bit 0: x periodic, bit 1: y periodic
 *   row_ptr   device, N + 1 int32 (output): row i is col[row_ptr[i] .. row_ptr[i+1])
 *   col       device, col_capacity int32 (output), each row sorted by ascending j;
 *             may be NULL with col_capacity = 0 to query the size
 *   nnz_out   host (output): number of stencil entries
 *
 * Uses a uniform cell list built in stream-ordered scratch memory that the call
 * allocates and frees itself.  Synchronises `stream` once (to read nnz).
 * Errors: EINVAL (bad sizes, node outside the box, N >= 2^31), ECAPACITY
 * (col_capacity < nnz; nnz_out holds the required size, row_ptr is valid),
 * ECAPACITY also if nnz >= 2^31.
 */
int labfm_build_stencils(const double* xy, const double* h, int64_t N, double Lx, double Ly,
                         uint32_t periodic_mask, int32_t* row_ptr, int32_t* col,
                         int64_t col_capacity, int64_t* nnz_out, void* stream);

/*
 * Weight build (Sections 2, 3 and 6), FP64 throughout.  For every node i:
 *   X~_ji = X_ji . H_i  (monomials (x/h)^a (y/h)^b / (a! b!), eq. X and vector H)
 *   W^q_ji = psi(|r_ji|/h_i) H_a(x_ji/(h_i sqrt2)) H_b(y_ji/(h_i sqrt2)) / sqrt(2^(a+b))
 *            (eq. hermite; psi = Wendland C2, (1 - q/2)^4 (1 + 2q) on q <= 2)
 *   M_i = sum_j X~_ji (x) W_ji                              (eq. disc_form;
 *         assembled from the weighted moments sum_j psi (x/h)^p (y/h)^q, p + q <= 2m,
 *         since W = psi He_a(x/h) He_b(y/h) with probabilists' Hermite He_a)
 *   M_i Psi^d = C~^d by LU with partial pivoting           (eq. lsys)
 *   w^d_ji = W_ji . Psi^d                                   (eq. w_abf)
 *   F_0,i = sum_j phi_ji w^hyp_ji, kappa_i = 2 / (3 F_0,i)   (Section 6)
 * for the six operators listed at the top of this file (m even for the filter).
 *
 *   xy, h, s  device, N x 2 / N / N doubles; s_i is the node spacing (Section 2)
 *   row_ptr, col  device CSR from labfm_build_stencils (nnz entries)
 *   m         order of polynomial reproduction, even, 2 <= m <= 10
 *   w         device, 6 x nnz doubles (output), operator-major: w[d * nnz + e]
 *             (may be NULL, like col, when nnz = 0: every stencil is empty)
 *   kappa     device, N doubles (output): filter coefficient kappa_i
 *   residual  device, N doubles (output, may be NULL): max over operators and
 *             monomials of |sum_j X~_ji w_ji h^l - C^d| (nondimensional
 *             reproduction residual, l = derivative order)
 *   node_status device, N int32 (output): OR of LABFM_NODE_* flags, 0 = good
 *   n_failed_out host (output, may be NULL): number of nodes with a nonzero status;
 *             when non-NULL the call synchronises `stream`
 * Errors: EINVAL (sizes, m), ESINGULAR (n_failed_out requested and > 0; the
 * outputs of the good nodes are still valid).
 */
int labfm_build_weights(const double* xy, const double* h, const double* s, int64_t N,
                        double Lx, double Ly, uint32_t periodic_mask,
                        const int32_t* row_ptr, const int32_t* col, int64_t nnz, int m,
                        double* w, double* kappa, double* residual, int32_t* node_status,
                        int64_t* n_failed_out, void* stream);

/*
 * labfm_build_weights that also writes, for the matrix-free right-hand side,
 * every node's weight polynomials: with W = psi He_a(x/h) He_b(y/h),
 * w^d_ji = psi(|r_ji|/h_i) P^d_i(x_ji/h_i, y_ji/h_i) where
 * P^d_i = sum_{p+q<=m} c^d_pq x^p y^q has (m+1)(m+2)/2 coefficients per operator.
 *   coef_out  device, N x labfm_weight_coefficients_per_node(m) doubles (output,
 *             may be NULL), node-major; within a node monomial major (p ascending,
 *             then q = 0..m-p), operator minor: c^d_pq of node i at
 *             coef_out[i * 6 (m+1)(m+2)/2 + 6 idx(p, q) + d], idx(p, q) = p (2m + 3 - p)/2 + q;
 *             zeros for a node whose system is singular or has too few neighbours
 *   w         may be NULL when coef_out is given (the weights are not stored)
 * Other arguments, outputs and errors as labfm_build_weights.
 */
int labfm_build_weights_ex(const double* xy, const double* h, const double* s, int64_t N, double Lx,
                           double Ly, uint32_t periodic_mask, const int32_t* row_ptr, const int32_t* col,
                           int64_t nnz, int m, double* w, double* kappa, double* residual,
                           int32_t* node_status, int64_t* n_failed_out, double* coef_out, void* stream);

/* Doubles of weight-polynomial coefficients per node for order m: 6 (m+1)(m+2)/2
 * (0 for an unsupported m). */
size_t labfm_weight_coefficients_per_node(int m);

/*
 * Matrix-free right-hand side of eq. icns, FP64: as labfm_rhs, but each
 * neighbour's five weights (x, y, xx, xy, yy) are recomputed from the node's
 * weight polynomials (labfm_build_weights_ex) instead of read from a plan:
 * w^d_ji = psi(|r_ji|/h_i) P^d_i(x_ji/h_i, y_ji/h_i) by Horner's rule, the same
 * operations as the weight build.  This trades the 40 bytes of stored FP64
 * weights per stencil entry for about 5 (m+1)(m+2)/2 fused multiply-adds (the
 * alternative the paper's conclusions name for Lagrangian node sets).  One warp
 * per node.
 *   xy, h     device, N x 2 / N doubles (the node set of the weight build)
 *   row_ptr, col  device CSR of the stencils; coef: device, from labfm_build_weights_ex
 *   fields    device, 3 x N doubles (ln rho, u, v); rhs: device, 3 x N doubles
 *             (output, must not alias fields)
 * Errors: EINVAL (sizes, m, aliasing, a malformed CSR).
 */
int labfm_rhs_matrix_free(const double* xy, const double* h, int64_t N, double Lx, double Ly,
                          uint32_t periodic_mask, const int32_t* row_ptr, const int32_t* col, int m,
                          const double* coef, const double* fields, double* rhs, const labfm_phys* phys,
                          void* stream);

/*
 * Stencil optimisation (Section 4), FP64.  For every node i, starting from
 * h = h0_i and the stencil of labfm_build_stencils at h0_i, repeat:
 *   1. stop if fewer than n = (m^2 + 3m)/2 stencil nodes lie within |r_ji| <= 2h;
 *   2. build M_i at h (as labfm_build_weights) and solve for Psi^x, Psi^y and
 *      Psi^L (selector C~^L = C~^xx + C~^yy); stop if M_i is singular;
 *   3. stop if alpha_L = || (M_i Psi^L - C~^L) h^2 ||_2 > alpha_0 =
 *      resid_coef eps n^4 / (h m), eps = 2^-52 (Laplacian residual test; the
 *      paper's resid_coef is 1e-4);
 *   4. stop if the largest amplitude response of d/dx, d/dy or the Laplacian
 *      exceeds amp_max at any of the 16 wavenumbers k_n = (pi/s_i) n/16,
 *      n = 1..16, where A^x = sum_j w^x_ji sin(k x_ji) / k,
 *      A^y = sum_j w^y_ji sin(k y_ji) / k and
 *      A^L = sum_j w^L_ji (1/2 - cos(k x_ji) cos(k y_ji) / 2) / k^2;
 *   5. record h as passing and set h <- factor h.
 * The output is the last h that passed every test (h0_i if none did).  The
 * paper's values are factor = 0.99 and amp_max = 1.01 (a response at most 1 %
 * above the exact one).  alpha_L is a rounding-level quantity, so near alpha_0
 * the outcome of test 3 depends on the order of the floating-point operations:
 * two correct solvers can stop a few factors apart on the same node.
 * resid_coef = +inf switches test 3 off.
 *
 *   xy, h0, s  device, N x 2 / N / N doubles
 *   row_ptr, col device CSR from labfm_build_stencils at h0 (candidates)
 *   m          order, even, 2 <= m <= 10
 *   factor     shrink factor in (0, 1); amp_max: response bound;
 *              resid_coef: > 0 (may be +inf)
 *   max_iter   host, iteration limit per node (>= 0)
 *   h_out      device, N doubles (output)
 *   solves_out device, N int32 (output, may be NULL): systems solved per node
 *   alpha_out  device, N x 2 doubles (output, may be NULL): per node, alpha_L at
 *              the returned h and alpha_L at the h where the iteration stopped
 *              (test 3 or 4 failed there); NaN where none was computed (no h
 *              passed, or the stop came from test 1, a singular M_i or max_iter)
 * One CTA per node; no allocation, no synchronisation.
 * Errors: EINVAL (null pointers, N, m, factor, max_iter).
 */
int labfm_stencil_optimise(const double* xy, const double* h0, const double* s, int64_t N,
                           double Lx, double Ly, uint32_t periodic_mask,
                           const int32_t* row_ptr, const int32_t* col, int m, double factor,
                           double amp_max, double resid_coef, int max_iter, double* h_out,
                           int32_t* solves_out, double* alpha_out, void* stream);

/*
 * Operator of a domain with walls (Section 7.1, Table "Schemes for derivatives
 * near boundaries", and Appendix A), in the format of labfm_build_weights
 * (difference form, six weights per entry, kappa) so that labfm_plan_create
 * takes it unchanged.  A wall is its nodes i0 (wall node b) with their inward
 * unit normals n_b, each with the nodes i1..i4 of its normal column at q s_b
 * along n_b (Section 7.1).  Per node:
 *   - rows q >= 3 and every node in no column: LABFM of order m on the stencil
 *     |r_ji| <= 2 h_i (as labfm_build_stencils and labfm_build_weights);
 *   - rows q = 1, 2: d/dx and d/dy from the five-point difference along the
 *     column (asymmetric at q = 1, central at q = 2) and one-dimensional LABFM
 *     of order 4 along the row (Appendix A: the nodes of the same q of the other
 *     columns within 2 h1d, h1d = h1d_over_s s_i, offsets eta along the tangent
 *     t = (-n_y, n_x)), rotated to (x, y); the second derivatives and the filter
 *     from LABFM of order m_wall on the node's stencil;
 *   - wall nodes q = 0: d/dx and d/dy from the one-sided five-point difference
 *     and 1D LABFM only, no second derivatives, kappa = 0 (the wall is not
 *     filtered; with labfm_plan_set_walls its velocity is held at zero and ln rho
 *     follows the LODI equation of the wall).
 * Rows are sorted by column; the union of a row's LABFM stencil and its column
 * and row nodes.
 *   xy, h, s        device, N x 2 / N / N doubles (bounded axes take [0, L])
 *   m, m_wall       LABFM orders (even, 2..10; the paper uses m = 6, m_wall = 4)
 *   n_wall          number of wall nodes (5 n_wall <= N)
 *   wall_column     device, n_wall x 5 int32: the nodes q = 0..4 of each column
 *   wall_normal     device, n_wall x 2 doubles: inward unit normal of each wall node
 *   h1d_over_s      support of the 1D LABFM (the paper gives none; 1.7 for the
 *                   uniform wall rows)
 *   row_ptr         device, N + 1 int32 (output)
 *   col             device, col_capacity int32 (output), or NULL with
 *                   col_capacity = 0 to query nnz (w, kappa, node_status unused)
 *   w               device, 6 x nnz doubles (output), operator-major w[d * nnz + e]
 *   kappa, node_status  device, N doubles / N int32 (output); a node whose row has
 *                   more than 64 row neighbours or a singular 1D system is flagged
 *                   LABFM_NODE_SINGULAR with an empty row
 *   n_failed_out    host (output, may be NULL; then no ESINGULAR)
 * Allocates and frees stream-ordered scratch; synchronises `stream`.  The row
 * neighbour search is the cell-list search of labfm_build_stencils.
 * Errors: EINVAL (sizes, orders, a column node out of range or in two columns, a
 * normal not of unit length), ECAPACITY (col_capacity < nnz; nnz_out holds the
 * required size), ESINGULAR (n_failed_out requested and > 0).
 */
int labfm_build_wall_operator(const double* xy, const double* h, const double* s, int64_t N,
                              double Lx, double Ly, uint32_t periodic_mask, int m, int m_wall,
                              int64_t n_wall, const int32_t* wall_column, const double* wall_normal,
                              double h1d_over_s, int32_t* row_ptr, int32_t* col, int64_t col_capacity,
                              int64_t* nnz_out, double* w, double* kappa, int32_t* node_status,
                              int64_t* n_failed_out, void* stream);

/*
 * Modal (amplitude) response of built operators (Section 3): per node i and
 * wavenumber k_n = (pi/s_i) n/nk, n = 1..nk,
 *   out[(i * 3 + 0) * nk + n - 1] = sum_j w^x_ji sin(k x_ji) / k
 *   out[(i * 3 + 1) * nk + n - 1] = sum_j w^y_ji sin(k y_ji) / k
 *   out[(i * 3 + 2) * nk + n - 1] = sum_j (w^xx_ji + w^yy_ji)
 *                                   (1/2 - cos(k x_ji) cos(k y_ji) / 2) / k^2
 * (1 for an exact operator on a mode that the node spacing resolves).
 *
 *   xy, s        device, N x 2 / N doubles
 *   row_ptr, col device CSR (nnz entries); w: device, 6 x nnz doubles from
 *                labfm_build_weights (col and w may be NULL when nnz = 0)
 *   nk           wavenumbers per node, 1 <= nk <= 4096
 *   out          device, N x 3 x nk doubles (output)
 * Errors: EINVAL (null pointers, N, nk).
 */
int labfm_modal_response(const double* xy, const double* s, int64_t N, double Lx, double Ly,
                         uint32_t periodic_mask, const int32_t* row_ptr, const int32_t* col,
                         int64_t nnz, const double* w, int nk, double* out, void* stream);

/*
 * Prepare an operator for the time-step kernels: rows padded to a multiple of
 * four entries (pad entries point at the node itself with weight 0, which adds
 * exactly zero in the difference form of eq. general_do); every 4-entry chunk
 * becomes one record of its four columns and the four weights of each of the
 * five RHS operators, in `dtype`, and a second record stream holds the columns
 * with the filter weights kappa_i w^hyp_ji.  For LABFM_F32 the RHS weights are stored nondimensionalised,
 * w^d_ji s_i^l (l = 1 for d/dx, d/dy; 2 for second derivatives), and the kernels
 * multiply the sums by s_i^-l.
 *
 *   w      device, 6 x nnz doubles as written by labfm_build_weights (col and w
 *          may be NULL when nnz = 0; such a plan's steps leave the state unchanged)
 *   kappa  device, N doubles
 *   s      device, N doubles (node spacing)
 * The plan allocates and owns its device memory (cudaMalloc); the input
 * buffers may be freed after the call returns.  Synchronises `stream`.
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
int labfm_plan_create(labfm_plan** plan, int64_t N, int64_t nnz, labfm_dtype dtype,
                      const int32_t* row_ptr, const int32_t* col, const double* w,
                      const double* kappa, const double* s, void* stream);

/*
 * A plan over many independent instances (for example flow problems of
 * different sizes and orders m): the instances' operators are concatenated
 * block-diagonally, node k of instance i becoming node off_i + k with
 * off_i = N_0 + ... + N_{i-1}, so that one launch of each step kernel serves
 * all of them.  Fields and states of a batched plan are 3 x N_total, instance
 * after instance within each field.  Host arrays of n_inst entries:
 *   N_inst, nnz_inst  sizes of each instance
 *   row_ptr, col, w, kappa, s  device pointers of each instance, as for
 *                     labfm_plan_create
 * Synchronises `stream`.  Errors as labfm_plan_create.
 */
int labfm_plan_create_batched(labfm_plan** plan, int n_inst, const int64_t* N_inst,
                              const int64_t* nnz_inst, const int32_t* const* row_ptr,
                              const int32_t* const* col, const double* const* w,
                              const double* const* kappa, const double* const* s,
                              labfm_dtype dtype, void* stream);

/*
 * No-slip walls of a plan (Section 7.1): at the wall nodes the step and
 * right-hand-side kernels hold u = v = 0 (zero right-hand side) and advance
 * ln rho by eq. lodilnro with u_xi = 0, the outgoing wave L1 of eq. Ldef
 * (L2 = 0 for isothermal flow) and the incoming wave L4 = L1 + rho c g.n:
 *   d ln rho/dt = -(L4 + L1) / (rho c^2) - d u_eta / d eta,
 *   L1 = -(c/2) (dp/dxi - rho c du_xi/dxi),  dp/dxi = c^2 rho d ln rho/dxi.
 * The paper prints L4 = L1 + 2 rho c g.n; with eq. lodiu only the factor 1 holds
 * u_xi at zero (a resting hydrostatic column stays at rest), which is taken.  The
 * derivatives are the plan's own (labfm_build_wall_operator gives the wall rows'
 * one-sided differences and 1D LABFM).  Every other node follows eq. icns.
 *   wall_nodes   device, n_wall int32; wall_normal: device, n_wall x 2 doubles
 *                (inward unit normals); n_wall = 0 removes the walls
 * Plans with walls run the plain stage grid (not the persistent or staged
 * kernels); the adjoint and recording calls refuse them.  On a batched plan the
 * nodes are the plan's (instance k's node q is inst_off[k] + q), and launch
 * ranges (labfm_plan_set_launch_ranges) run the same boundary right-hand side.
 * Synchronises `stream`.  Errors: EINVAL (node out of range or listed twice,
 * normal not of unit length), ENOMEM.
 */
int labfm_plan_set_walls(labfm_plan* plan, int64_t n_wall, const int32_t* wall_nodes,
                         const double* wall_normal, void* stream);

/*
 * Boundaries of a plan of any of the three kinds of Section 7.1, each node with
 * its inward unit normal: LABFM_WALL as labfm_plan_set_walls; LABFM_OUTFLOW and
 * LABFM_INFLOW follow eq. lodi in the boundary frame (xi along n, eta along
 * t = (-n_y, n_x)) with L2 = 0, the outgoing waves from eq. Ldef and the incoming
 * ones
 *   outflow (eq. outflowL): L4 = sigma/(2L) c (1 - M^2)(p - p_inf) + (1 - M) T4 + V4,
 *   inflow: L3 = sigma c / L (u_eta - u_eta,IN) + T3 + V3,
 *           L4 = sigma rho0 c^2 (1 - M^2) / L (u_xi - u_xi,IN) + T4 + V4,
 * with the transverse and viscous terms T3, T4, V3, V4 as printed, and the viscous
 * conditions dtau_etaxi/deta = 0 (outflow) and dtau_etaeta/deta = 0 (inflow) taken
 * out of the viscous forces of eq. lodiu and eq. lodiv respectively.  The paper
 * prints the inflow's relaxations on the other components ((u_xi - u_xi,IN) in L3,
 * (u_eta - u_eta,IN) in L4); in eq. lodiu and lodiv L4 drives u_xi and L3 drives
 * u_eta, so each relaxes its own component here.  The boundary nodes' first and
 * second derivatives are the plan's own (labfm_build_wall_operator gives the
 * "FD + 1D-LABFM" schemes of the Table), and they are not filtered (kappa = 0).
 *   nodes   device, n int32;  normal: device, n x 2 doubles (inward unit normals)
 *   kind    device, n int32 (LABFM_WALL, LABFM_INFLOW, LABFM_OUTFLOW)
 *   target  device, n x 2 doubles: an inflow's (u_xi,IN, u_eta,IN); an outflow's
 *           p_inf in the first (the second unused); unused for walls
 *   params  host: sigma, L, M, rho0 (one set per plan)
 * n = 0 removes the boundaries.  As labfm_plan_set_walls otherwise (plain stage
 * grid, no adjoint, the plan's node numbering on batched plans, synchronises `stream`).
 * Errors: EINVAL (node out of range or listed twice, normal not of unit length,
 * unknown kind, sigma < 0, L <= 0, M outside [0, 1), rho0 <= 0), ENOMEM.
 */
int labfm_plan_set_boundaries(labfm_plan* plan, int64_t n, const int32_t* nodes, const double* normal,
                              const int32_t* kind, const double* target, const labfm_nscbc* params,
                              void* stream);

/*
 * Per-instance time steps (host, n_instances values > 0).  Afterwards
 * labfm_rk_step, labfm_rk_step_noalloc and labfm_step_graph_create accept
 * dt = 0, meaning "each instance with its own step" (eq. dt applies per
 * instance: the instances are independent problems).
 */
int labfm_plan_set_dt(labfm_plan* plan, const double* dt_inst, void* stream);

/*
 * eq. dt for every instance of a plan: the exact minimum over the instance's
 * nodes of min(1.0 s_i / (|u_i| + c), 0.4 s_i^2 rho_i / mu).
 *   dt_inst_out  device, n_instances doubles (output)
 */
int labfm_stable_dt_instances(const labfm_plan* plan, const void* fields, const double* s,
                              double c, double mu, double* dt_inst_out, void* stream);

/*
 * Persistent stage kernel on (1) or off (0).  When on, labfm_rk_step launches
 * one stage kernel per stage with a grid of (SMs x resident blocks); each warp
 * takes tiles of consecutive nodes from a work-queue ticket (reset at every
 * step), which balances uneven stencils and mixed instances dynamically.  The
 * workspace grows by 64 bytes for the tickets (query labfm_rk_workspace_bytes
 * after changing this).
 */
int labfm_plan_set_persistent(labfm_plan* plan, int enable);

/*
 * L2 prefetch distance of the F32 stage and filter kernels' operator streams, in
 * loop iterations of a node's lane group (0 = off, at most 8).  When positive,
 * three lanes of each group issue an L2 prefetch of the three 128-byte segments
 * of the record block they will read `distance` iterations later (in the filter,
 * one lane the 128-byte filter block), if it lies within the node's row.
 * Results do not change.  Rows of fewer than 48 padded entries are
 * never prefetched (measured faster for the rows of m = 6, 8 and 10, ~60-220
 * entries; a lower threshold slowed the ~35-entry rows of m = 4).  Plan creation sets 2 for F32 plans and 0 for F64
 * plans (whose kernels do not prefetch).  Host-only call.
 */
int labfm_plan_set_prefetch(labfm_plan* plan, int distance);

/*
 * Programmatic dependent launches (enable = 1, the default) or plain launches
 * (enable = 0) for the plan's plain-grid stage, filter, recording-stage, adjoint,
 * pack and unpack kernels.  With them on, each such kernel is launched with
 * programmatic stream serialization: it may start while the previous kernel of the
 * stream finishes, reads only the plan's constant operator (row pointers, and an L2
 * prefetch of its rows' first record blocks) until griddepcontrol.wait has seen the
 * previous kernel complete, and only then reads or writes the state; results are
 * bit-identical either way.  No counterpart in the paper: a launch-scheduling
 * setting (sm_90 and later).  EINVAL for another value of enable.  Host-only call.
 */
int labfm_plan_set_programmatic_launch(labfm_plan* plan, int enable);

/*
 * Shared-memory staging of the operator stream for the F32 stage kernel
 * (stages = 2, 3 or 4 ring slots per CTA; 0 = off).  With staging on and 16 or
 * 32 lanes per node (labfm_plan_set_launch), labfm_rk_step runs a stage kernel
 * in which the bulk-copy (TMA) engine moves the operator records of whole
 * rounds of consecutive nodes (4 x 32/G nodes per 128-thread CTA) into shared
 * memory ahead of the warps that use them; results are bit-identical to the
 * unstaged kernel with the same lanes per node.  Other lane counts, and F64
 * plans' steps, run the unstaged kernel.  The call measures the largest round
 * (synchronising `stream`) and sizes the grid; a lane count whose largest round
 * does not fit `stages` slots in shared memory keeps the unstaged kernel.  Each
 * wait of the staged kernel on a copy is bounded (1 s by default,
 * labfm_plan_set_wait_limit); one that runs out is reported by
 * labfm_plan_device_status.
 * Errors: EINVAL (F64 plan with stages != 0, stages not in {0, 2, 3, 4}).
 */
int labfm_plan_set_staging(labfm_plan* plan, int stages, void* stream);

/*
 * Limit of every bounded wait of the staged stage kernel on a bulk copy, in
 * nanoseconds (0 .. 10 s; the default is 1 s).  0 makes each wait a single
 * non-blocking test of the copy's barrier, so that waits run out: this exercises
 * the timeout path, which leaves LABFM_ETIMEOUT for labfm_plan_device_status and
 * that step's results invalid.  A CTA whose wait ran out lets its copies in
 * flight land (waiting at most 1 s more for each) before it exits, so the
 * context stays usable.  No counterpart in the paper (failure detection).
 * Host-only call.
 * Errors: EINVAL (limit out of range).
 */
int labfm_plan_set_wait_limit(labfm_plan* plan, int64_t limit_ns);

/*
 * Check of the evolved state for non-finite values during labfm_rk_step (and
 * labfm_rk_step_host, labfm_rk_step_noalloc): after every `every`-th step of a
 * call and after its last step, one pass over the state (12 or 24 bytes per
 * node) sets LABFM_ENONFINITE for labfm_plan_device_status if any value of
 * ln rho, u or v is NaN or infinite.  A diverging run is then caught without
 * copying the state to the host.  every = 0 (the default) turns it off.  Steps
 * replayed from a step graph are not checked.  No counterpart in the paper
 * (failure detection).  Host-only call (the first enabling call allocates the
 * status word, synchronously).
 * Errors: EINVAL (every < 0), ENOMEM.
 */
int labfm_plan_set_check_finite(labfm_plan* plan, int every);

/*
 * Device-side status of the plan's kernels since the last query: LABFM_OK,
 * LABFM_ETIMEOUT when a bounded wait of the staged stage kernel ran out (that
 * step's results are then invalid), or LABFM_ENONFINITE when the state check of
 * labfm_plan_set_check_finite found a non-finite value (the first status set
 * since the last query is kept).  Synchronises the device and clears the status.
 * With LABFM_FAULT=timeout it reports LABFM_ETIMEOUT without touching the device.
 *   status_out  host (output)
 */
int labfm_plan_device_status(const labfm_plan* plan, int* status_out);

/* Free a plan and its device memory (synchronises the device first). NULL is a no-op. */
int labfm_plan_destroy(labfm_plan* plan);

/* Describe a plan (host output). */
int labfm_plan_get_info(const labfm_plan* plan, labfm_plan_info* info);

/*
 * Override the launch shape: `group` lanes per node (2, 4, 8, 16 or 32) in every
 * gather kernel, and `block` threads per block (a multiple of 32 and of group,
 * 64..1024) for the filter and filter-transpose kernels; the fused right-hand-side,
 * stage and adjoint gather kernels always run one-warp (32-thread) blocks.  Defaults: group 4, block 128;
 * labfm_plan_autotune picks the fastest group.
 */
int labfm_plan_set_launch(labfm_plan* plan, int group, int block);

/*
 * Launch shapes per node range (for example the order classes of a batched plan
 * whose instances are grouped by order m): range r covers the nodes
 * [begin[r], begin[r + 1]) and runs its own plain-grid stage and filter launches
 * in labfm_rk_step (and the step graph) with group[r] lanes per node and the L2
 * record prefetch distance prefetch[r] (F32; 0..8).  Results are those of the
 * same lanes per node in one launch.  With ranges set, the persistent, staged
 * and filter settings are not used, and the recording and adjoint calls refuse
 * the plan.  n = 0 removes the ranges.  Host-only; the arrays are copied.
 *   begin  host, n + 1 int64 (begin[0] = 0, begin[n] = N, not decreasing)
 *   group, prefetch  host, n int32
 * Errors: EINVAL (bounds, unsupported lanes per node, prefetch).
 */
int labfm_plan_set_launch_ranges(labfm_plan* plan, int n, const int64_t* begin, const int32_t* group,
                                 const int32_t* prefetch);

/*
 * Launch shape of the filter kernel of labfm_rk_step (and labfm_rk_step_record):
 * `group` lanes per node (2, 4, 8, 16 or 32; 0 = the plan's group of
 * labfm_plan_set_launch), and persistent = 1 for a grid of (SMs x resident
 * blocks) whose warps stride over the nodes, so that no partly filled last wave
 * of blocks leaves the GPU idle (0 = one group per node over a full grid).
 * The filtered state does not depend on `persistent`; with another lane count
 * the filter sums are added in another order (FP rounding only).  Host-only.
 * Errors: EINVAL (unsupported lanes per node).
 */
int labfm_plan_set_filter_launch(labfm_plan* plan, int group, int persistent);

/*
 * Time every supported group size on this plan with CUDA events (the RHS
 * kernel on `fields`, `reps` launches each) and keep the fastest.
 * Writes the chosen pair to *group_out / *block_out (host, may be NULL).
 * Synchronises `stream`.
 */
int labfm_plan_autotune(labfm_plan* plan, const void* fields, void* scratch_rhs,
                        const labfm_phys* phys, int reps, int* group_out, int* block_out,
                        void* stream);

/*
 * Right-hand side of eq. icns in (ln rho, u, v) (Section 7):
 *   R_a = -(u a_x + v a_y) - (u_x + v_y)
 *   R_u = -(u u_x + v u_y) - c^2 a_x + mu e^-a (4/3 u_xx + u_yy + 1/3 v_xy) + g_x
 *   R_v = -(u v_x + v v_y) - c^2 a_y + mu e^-a (4/3 v_yy + v_xx + 1/3 u_xy) + g_y
 * with every derivative L^d_i(phi) = sum_j (phi_j - phi_i) w^d_ji (eq. general_do).
 *   fields  device, 3 x N in the plan's dtype
 *   rhs     device, 3 x N in the plan's dtype (output; must not alias fields)
 *   phys    host
 */
int labfm_rhs(const labfm_plan* plan, const void* fields, void* rhs, const labfm_phys* phys,
              void* stream);

/*
 * Filter (Section 6): phi~_i = phi_i + kappa_i sum_j (phi_j - phi_i) w^hyp_ji for
 * ln rho, u and v, reading only `in` (every node sees its neighbours' unfiltered
 * values).  in/out device, 3 x N in the plan's dtype; out must not alias in.
 */
int labfm_filter(const labfm_plan* plan, const void* in, void* out, void* stream);

/* Bytes of device workspace labfm_rk_step needs for this plan. */
size_t labfm_rk_workspace_bytes(const labfm_plan* plan);

/*
 * `nsteps` complete time steps (Section 7): each is the four stages of the
 * low-storage RK3(2)4[2R+]C scheme with registers (Q, X),
 *   X = Q; for k = 1..4: F = R(X); Q += dt b_k F; X = Q + dt (a_{k+1,k} - b_k) F,
 * fused into one gather kernel per stage (F is never stored), followed by the
 * filter on ln rho, u, v.
 *   Q     device, 3 x N in the plan's dtype: initial state in, final state out
 *   work  device, labfm_rk_workspace_bytes(plan) bytes, 16-byte aligned
 *   dt    time step (see labfm_stable_dt), or 0 to use the per-instance steps set
 *         with labfm_plan_set_dt; nsteps >= 0
 * Capturable in a CUDA graph (no allocation, no synchronisation).
 */
int labfm_rk_step(const labfm_plan* plan, void* Q, void* work, size_t work_bytes, double dt,
                  int nsteps, const labfm_phys* phys, void* stream);

/*
 * Time step of eq. dt: min over nodes of min(1.0 s_i / (|u_i| + c), 0.4 s_i^2 rho_i / mu),
 * rho_i = exp(ln rho_i), computed exactly as a minimum (order independent).
 *   fields  device, 3 x N in the plan's dtype
 *   s       device, N doubles
 *   dt_out  device, one double (output)
 */
int labfm_stable_dt(const labfm_plan* plan, const void* fields, const double* s, double c,
                    double mu, double* dt_out, void* stream);

/*
 * The same as labfm_rk_step for a caller whose state lives in host memory:
 * runs `nsteps` steps on the device with the state taken from and returned to
 * Q_host (3 x N, plan dtype), and synchronises `stream`.  Page-locked (pinned,
 * mapped) host memory is read and written directly by the step's pack and
 * unpack kernels over the host link (Q_dev is not used); other host memory is
 * copied to Q_dev, stepped there and copied back.
 *   Q_host  host, 3 x N
 *   Q_dev   device, 3 x N scratch for the state (used for pageable Q_host)
 */
int labfm_rk_step_host(const labfm_plan* plan, void* Q_host, void* Q_dev, void* work,
                       size_t work_bytes, double dt, int nsteps, const labfm_phys* phys,
                       void* stream);

/*
 * ---- Adjoint (reverse mode).  The paper has no adjoint; these are the exact
 * transposes of the forward operators above (eq. general_do, eq. icns, the RK
 * step of Section 7 and the filter of Section 6), used to differentiate a flow
 * objective with respect to the initial state.
 *
 * Build the transposed operator of a plan: for every node k, the rows i whose
 * stencil contains k with their weights w_ik (same record layout as the forward
 * operator), and the row sums of the forward weights.  Allocates device memory
 * owned by the plan; synchronises `stream`.  Needed by the calls below.
 */
int labfm_plan_enable_adjoint(labfm_plan* plan, void* stream);

/* Bytes of device workspace the adjoint calls need for this plan. */
size_t labfm_adjoint_workspace_bytes(const labfm_plan* plan);

/*
 * grad = (dR/dq)^T lambda: the vector-Jacobian product of the eq. icns
 * right-hand side at state `fields` (3 x N, plan dtype) with cotangent
 * `lambda` (3 x N).  Derivative adjoints are applied through the transposed
 * operator as a gather (no atomics); grad must not alias the inputs.
 */
int labfm_rhs_adjoint(const labfm_plan* plan, const void* fields, const void* lambda, void* grad,
                      const labfm_phys* phys, void* work, size_t work_bytes, void* stream);

/*
 * One time step backwards: lambda <- (dQ_next/dQ)^T lambda for the step
 * Q -> filter(RK3(2)4[2R+]C(Q)) that labfm_rk_step takes from the state Q
 * (3 x N, the state at the start of the step, not modified).  The stage states
 * are recomputed from Q; the reverse sweep is the low-storage transpose of the
 * scheme: Lambda = Fil^T lambda, Fbar_4 = dt b_4 Lambda, then for k = 4..1
 * Xbar_k = J_R(X_k)^T Fbar_k, Lambda += Xbar_k,
 * Fbar_{k-1} = dt (b_{k-1} Lambda + (a_{k,k-1} - b_{k-1}) Xbar_k).
 * dt as for labfm_rk_step.
 */
int labfm_rk_step_adjoint(const labfm_plan* plan, const void* Q, void* lambda, double dt,
                          const labfm_phys* phys, void* work, size_t work_bytes, void* stream);

/*
 * The same reverse step without the recompute, for a caller that keeps the stage
 * states: labfm_rk_step_record advances Q (3 x N, in place) by one step exactly as
 * labfm_rk_step does and stores in `states` the step's four stage states X_1..X_4
 * (the state each of the four RK stages evaluates eq. icns at) and, per stage and
 * node, the eight combinations of the derivatives at X_k that the transpose of
 * eq. icns with respect to the node's own state needs (opaque layout;
 * labfm_stage_states_bytes bytes, 16-byte aligned); labfm_rk_step_adjoint_recorded
 * then applies the reverse sweep of labfm_rk_step_adjoint to lambda with them.
 * The results are identical to labfm_rk_step and labfm_rk_step_adjoint (which
 * recomputes the same records).  A checkpointed rollout that recomputes a segment
 * with labfm_rk_step_record skips the four stage evaluations per step that
 * labfm_rk_step_adjoint repeats; neither reverse sweep gathers derivatives again.
 *   work  (record): labfm_rk_workspace_bytes; (adjoint): labfm_adjoint_workspace_bytes
 */
size_t labfm_stage_states_bytes(const labfm_plan* plan);
int labfm_rk_step_record(const labfm_plan* plan, void* Q, void* states, size_t states_bytes,
                         void* work, size_t work_bytes, double dt, const labfm_phys* phys,
                         void* stream);
int labfm_rk_step_adjoint_recorded(const labfm_plan* plan, const void* states, void* lambda,
                                   double dt, const labfm_phys* phys, void* work,
                                   size_t work_bytes, void* stream);

/* lam_out = Fil^T lam_in = lam + L_hyp^T (kappa lam), per field (3 x N). */
int labfm_filter_adjoint(const labfm_plan* plan, const void* lam_in, void* lam_out, void* work,
                         size_t work_bytes, void* stream);

/*
 * Conserved (rho, rho u, rho v) to evolved (ln rho, u, v) variables, 3 x N in
 * `dtype`, and its vector-Jacobian product cbar = (dq/dc)^T qbar at c.
 */
int labfm_conserved_to_primitive(const void* c, void* q, int64_t N, labfm_dtype dtype,
                                 void* stream);
int labfm_conserved_vjp(const void* c, const void* qbar, void* cbar, int64_t N,
                        labfm_dtype dtype, void* stream);

/*
 * Domain kinetic energy KE = sum_i 1/2 rho_i |u_i|^2 s_i^2 (node volume s_i^2)
 * of a state q = (ln rho, u, v), summed in FP64 in a fixed order by one block
 * (the same result on every call), into one device double; and
 * grad_out = scale * dKE/dq.
 */
int labfm_kinetic_energy(const void* q, const double* s, int64_t N, labfm_dtype dtype,
                         double* ke_out, void* stream);
int labfm_kinetic_energy_grad(const void* q, const double* s, int64_t N, labfm_dtype dtype,
                              double scale, void* grad_out, void* stream);

/*
 * Probe-weighted momentum J = sum_i rho_i (px_i u_i + py_i v_i) of a state
 * q = (ln rho, u, v) (px, py: device, N doubles of probe weights, e.g. a smooth
 * bump around a sensor), summed in FP64 in a fixed order by one block into one
 * device double; and grad_out = scale * dJ/dq (the flow objective alternative to
 * the kinetic energy for the adjoint; the paper itself has no adjoint).
 */
int labfm_probe_momentum(const void* q, const double* px, const double* py, int64_t N,
                         labfm_dtype dtype, double* j_out, void* stream);
int labfm_probe_momentum_grad(const void* q, const double* px, const double* py, int64_t N,
                              labfm_dtype dtype, double scale, void* grad_out, void* stream);

/*
 * One complete time step of labfm_rk_step (four fused stage kernels and the
 * filter, plus the ticket reset of a persistent plan) captured once into a CUDA
 * graph; labfm_step_graph_run packs Q into the workspace, replays the graph
 * `nsteps` times on `stream` (one graph launch per step for every instance of
 * a batched plan) and unpacks the result into Q.  The plan and `work` must
 * outlive the graph; dt as for labfm_rk_step (0 = per-instance steps, whose
 * values may be changed between runs with labfm_plan_set_dt).  The capture
 * uses a private stream; create the graph outside any other capture.
 */
typedef struct labfm_step_graph labfm_step_graph;
int labfm_step_graph_create(labfm_step_graph** graph, const labfm_plan* plan, void* work,
                            size_t work_bytes, double dt, const labfm_phys* phys);
int labfm_step_graph_run(labfm_step_graph* graph, void* Q, int nsteps, void* stream);
int labfm_step_graph_destroy(labfm_step_graph* graph);

/*
 * labfm_rk_step for callers that cannot allocate device memory: the same
 * kernels and the same results, but the three packed state buffers live in a
 * 16 MiB array that is part of the library image (a static __device__ array),
 * so the call allocates nothing and takes no work buffer.  Useful where
 * cudaMalloc is not an option: a host application or plugin that hands the
 * library only the memory it manages itself, or a real-time loop that must not
 * pay for (or synchronise on) an allocation.  The paper has no counterpart; it
 * is an interface convenience.
 *   Limit: labfm_rk_workspace_bytes(plan) must fit in 16 MiB: 3 x N x 16 bytes
 *   (F32) or 3 x N x 32 bytes (F64), plus 64 bytes of work-queue tickets for a
 *   persistent plan, i.e. N <= 349,525 nodes in F32 (349,524 persistent) and
 *   N <= 174,762 in F64; larger plans get LABFM_ECAPACITY with the required
 *   size in labfm_last_error().
 *   The plan must belong to the current device (else LABFM_EINVAL).
 *   The first call on a device looks up the array's device address (once per
 *   device, with that device current); make that first call before any stream
 *   capture.  The address is kept for the life of the process: a caller that
 *   resets a device (cudaDeviceReset) must not call this entry point on that
 *   device afterwards.  Every GPU that loads the library holds the 16 MiB until
 *   exit.
 *   All calls on a device share the array: two calls whose work overlaps on the
 *   GPU (different streams or threads) race and corrupt each other's state.
 *   Nothing in the array needs to start at zero; every buffer is written before
 *   it is read within a call.
 *   Q, dt, nsteps, phys, stream: as for labfm_rk_step.
 */
int labfm_rk_step_noalloc(const labfm_plan* plan, void* Q, double dt, int nsteps,
                          const labfm_phys* phys, void* stream);

/* Device time of the kernels labfm_rk_step enqueues while profiling is enabled,
 * measured with CUDA events recorded on the launching stream: one pair around the
 * four consecutive stage launches of every step (counted as four launches, so
 * stage_ms / stage_launches is the mean launch duration including the short
 * gaps between them) and one pair around every filter launch.  Timing whole
 * blocks keeps the events from stalling the stream between every launch.
 * The adjoint calls are timed the same way: the four recording stage launches of
 * labfm_rk_step_record as one block (its filter launch counts as a filter
 * launch), and in the reverse sweep every pass B (transposed-operator gather)
 * and filter-transpose launch on its own.  The reverse sweep of a step runs each
 * stage's pass A (pointwise derivative adjoints) inside the launch that forms
 * its cotangent (the filter transpose for stage 4, pass B of stage k for stage
 * k - 1), so only labfm_rhs_adjoint launches pass A on its own (untimed). */
typedef struct labfm_profile {
    double stage_ms;         /* summed duration of the fused RHS + RK stage launches */
    int64_t stage_launches;
    double filter_ms;        /* summed duration of the filter launches */
    int64_t filter_launches;
    int64_t dropped;         /* launches not timed because the event pool was full */
    double rec_stage_ms;     /* recording stage launches (labfm_rk_step_record) */
    int64_t rec_stage_launches;
    double adj_a_ms;         /* adjoint pass A launches (none in the reverse sweep: fused) */
    int64_t adj_a_launches;
    double adj_b_ms;         /* adjoint pass B launches */
    int64_t adj_b_launches;
    double adj_filter_ms;    /* filter-transpose launches */
    int64_t adj_filter_launches;
} labfm_profile;

/* Enable (enable >= 1) or disable (0) launch timing on this plan; enabling clears
 * the record.  With enable = k the stage and filter launches of labfm_rk_step are
 * timed on every k-th step only (k = 1: every step), so that the events perturb
 * a long timed run less; the adjoint calls' launches are timed on every call.
 * Errors: EINVAL (enable < 0). */
int labfm_plan_set_profiling(labfm_plan* plan, int enable);

/* Read and clear the launch timings (synchronises on the last recorded event). */
int labfm_plan_read_profile(labfm_plan* plan, labfm_profile* out);

/*
 * Measure the device's fused multiply-add throughput in `dtype` (GFLOP/s,
 * 2 flops per FMA) with a synthetic kernel of independent FMA chains on every
 * SM.  No counterpart in the paper: it supplies the FP64-pipe denominator of
 * the roofline for the FP64 kernels.  Allocates a small device buffer, runs on
 * the legacy default stream and synchronises.
 */
int labfm_probe_fma_rate(int dtype, double* gflops_out);

#ifdef __cplusplus
}
#endif

#endif /* LABFM_H */
