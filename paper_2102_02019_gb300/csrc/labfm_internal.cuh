// Internal declarations shared by the CUDA translation units of liblabfm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "labfm.h"

namespace labfm {

// Record `msg` as this thread's last error and return `code`.
int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* what);

#define LABFM_CUDA_TRY(call)                                      \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return ::labfm::cuda_error(e_, #call); \
    } while (0)

#define LABFM_LAUNCH_CHECK(what)                                  \
    do {                                                          \
        cudaError_t e_ = cudaGetLastError();                      \
        if (e_ != cudaSuccess) return ::labfm::cuda_error(e_, what); \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Host-side fault injection for tests of the error paths (api.cu), read from the
// environment variable LABFM_FAULT at every call that honours it:
//   "alloc"             entry points that allocate device memory return
//                       LABFM_ENOMEM before touching the device;
//   "capacity"          labfm_build_stencils reports a col buffer one entry too
//                       small (LABFM_ECAPACITY) before touching the device;
//   "singular_node:<i>" labfm_build_weights flags node i as singular.
// Nothing is injected when the variable is unset or holds anything else.
bool fault_alloc();
bool fault_capacity();
bool fault_timeout();
int64_t fault_singular_node();  // the node to flag, or -1
int injected_alloc_error(const char* where);

// Periodic minimum image, written out so that the neighbour search and the
// weight build see bit-identical offsets (no contraction, plain IEEE ops).
__device__ __forceinline__ double min_image(double d, double L, bool periodic) {
    if (periodic) {
        if (d > 0.5 * L) {
            d = __dsub_rn(d, L);
        } else if (d < -0.5 * L) {
            d = __dadd_rn(d, L);
        }
    }
    return d;
}

// Exclusive scan of n int32 counts into out[0..n]; out[n] = total.  The total
// is also written (as int64) to *total_dev.  Returns LABFM_ECAPACITY through the
// caller when the host sees total >= 2^31.
int exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int64_t* total_dev,
                       void* scratch, size_t scratch_bytes, cudaStream_t st);
size_t exclusive_scan_scratch_bytes(int64_t n);

// Checks a caller's CSR before any kernel indexes with it: row_ptr[0] == 0,
// row_ptr non-decreasing, row_ptr[N] == nnz (nnz < 0: not given; col then holds
// row_ptr[N] entries), every column in [0, N).  Reads only row_ptr[0..N] and the
// columns the row pointers cover, and those only once the row pointers passed.
// Synchronises st.  EINVAL naming the first problem found.
int validate_csr(const int32_t* row_ptr, const int32_t* col, int64_t N, int64_t nnz, cudaStream_t st);

}  // namespace labfm

// The prepared operator behind labfm_plan (see labfm.h).
struct labfm_plan {
    int64_t N = 0;
    int64_t nnz = 0;
    int64_t nnz_pad = 0;
    labfm_dtype dtype = LABFM_F64;
    int device = 0;
    int group = 8;
    int block = 256;
    int32_t* row_ptr = nullptr;  // N + 1, every entry a multiple of 4
    int32_t* col = nullptr;      // nnz_pad; pad entries point at the row's own node
    void* w = nullptr;           // 5 x nnz_pad RHS weights, operator-major (dtype)
    void* wf = nullptr;          // nnz_pad filter weights kappa_i w^hyp_ji (dtype)
    void* inv_s = nullptr;       // N values 1/s_i (dtype), used by the F32 kernels
    int64_t device_bytes = 0;
    // instances of a batched plan (one instance for labfm_plan_create): node
    // ranges [inst_off[k], inst_off[k+1]) on the host and on the device
    int n_inst = 1;
    int64_t* inst_off_host = nullptr;
    int64_t* inst_off = nullptr;
    double* dt_node = nullptr;   // per-node time step (labfm_plan_set_dt), or null
    bool persistent = false;     // stage kernel takes node tiles from a work queue
    int prefetch = 0;            // L2 prefetch distance of the F32 record stream (labfm_plan_set_prefetch)
    bool programmatic = true;    // programmatic dependent launches (labfm_plan_set_programmatic_launch)
    int persist_grid = 0;
    // filter launch (labfm_plan_set_filter_launch): lanes per node (0 = the plan's
    // group) and a persistent grid-stride grid of filter_grid blocks
    int filter_group = 0;
    bool filter_persistent = false;
    int filter_grid = 0;
    // launch ranges (labfm_plan_set_launch_ranges): nodes [range_begin[r],
    // range_begin[r + 1]) run their own plain stage and filter launches with
    // range_group[r] lanes per node and prefetch range_pf[r] (host arrays)
    int n_ranges = 0;
    int64_t* range_begin = nullptr;
    int* range_group = nullptr;
    int* range_pf = nullptr;
    // F32 stage kernel with the operator staged through shared memory
    // (labfm_plan_set_staging): `stages` ring slots per CTA; for 16 and 32 lanes
    // per node ([0], [1]) the bytes of the largest round and the grid (0 = the
    // shape does not fit in shared memory)
    int stages = 0;
    int stage_slot_bytes[2] = {0, 0};
    int stage_grid[2] = {0, 0};
    int* dev_status = nullptr;   // device word: LABFM_ETIMEOUT after a bounded wait ran out
    uint64_t wait_ns = 1000000000ull;  // limit of each bounded wait (labfm_plan_set_wait_limit)
    int check_every = 0;               // labfm_plan_set_check_finite: steps between state checks
    // transposed operator for the adjoint (labfm_plan_enable_adjoint): for node k
    // the entries (i, w_ik) of every row i whose stencil contains k, in the same
    // record layout as the forward operator, plus row sums of the forward weights
    int32_t* trow_ptr = nullptr;  // N + 1, multiples of 4
    int64_t tnnz_pad = 0;
    void* tw = nullptr;           // transposed RHS records
    void* twf = nullptr;          // transposed filter records
    void* rsum = nullptr;         // 6 x N (dtype): sum_j w~^d_kj for the 5 RHS operators, sum_j wf_kj
    // walls (labfm_plan_set_walls): per node the wall slot (-1 in the fluid) and
    // per slot the inward unit normal (dtype, 2 values)
    int32_t* wall_slot = nullptr;
    void* wall_n = nullptr;
    int64_t n_wall = 0;
    int32_t* bnd_kind = nullptr;   // per slot: LABFM_WALL / INFLOW / OUTFLOW (null: all walls)
    void* bnd_target = nullptr;    // per slot, 2 values (dtype): inflow velocities or outflow p_inf
    labfm_nscbc nscbc = {0.278, 1.0, 0.0, 1.0};
    // launch timing (labfm_plan_set_profiling): event pairs around launches
    bool profiling = false;
    int prof_period = 1;       // time the step launches of every prof_period-th step
    int64_t prof_step = 0;     // steps seen since profiling was enabled
    cudaEvent_t* prof_ev = nullptr;  // 2 * prof_cap events
    char* prof_kind = nullptr;       // labfm::ProfKind of each pair
    int prof_cap = 0;
    int prof_used = 0;
    int64_t prof_dropped = 0;
};

namespace labfm {

struct PlanInput {  // one instance's build outputs, for plan packing
    int64_t N, nnz;
    const int32_t* row_ptr;
    const int32_t* col;
    const double* w;
    const double* kappa;
    const double* s;
};

// Launchers implemented in step.cu.
int launch_rhs(const labfm_plan* p, const void* fields, void* rhs, const labfm_phys* ph,
               int group, int block, cudaStream_t st);
int launch_filter_soa(const labfm_plan* p, const void* in, void* out, cudaStream_t st);
int launch_rk_steps(const labfm_plan* p, void* Q, void* work, double dt, int nsteps,
                    const labfm_phys* ph, cudaStream_t st);
size_t rk_work_bytes(const labfm_plan* p);
int launch_stable_dt(const labfm_plan* p, const void* fields, const double* s, double c,
                     double mu, double* dt_out, cudaStream_t st);
bool launch_shape_supported(int group, int block);

// Launch timing around kernel launches (api.cu); kind 0 = one stage launch,
// 1 = one filter launch, 2 = the four stage launches of a step, 3 = the four
// recording stage launches of labfm_rk_step_record, 4 = one adjoint pass A,
// 5 = one adjoint pass B, 6 = one filter-transpose launch.
// Returns the pair index to close with prof_end, or -1 when not profiling.
enum ProfKind { kProfStage = 0, kProfFilter = 1, kProfStages4 = 2, kProfRecStages4 = 3,
                kProfAdjA = 4, kProfAdjB = 5, kProfAdjFilter = 6 };
int prof_begin(labfm_plan* p, int kind, cudaStream_t st);
// Whether the launches of the step about to be enqueued are timed (every
// prof_period-th step while profiling); counts the step.
bool prof_step_sampled(labfm_plan* p);
void prof_end(labfm_plan* p, int idx, cudaStream_t st);

// Boundaries of a plan (walls.cu): slots, normals, and (kind and target null:
// walls) the kinds and targets; n = 0 removes them.
int set_walls(labfm_plan* p, int64_t n_wall, const int32_t* nodes, const double* normal, const int32_t* kind,
              const double* target, cudaStream_t st);

// Plan packing (step.cu): concatenates the instances block-diagonally.
int pack_plan(labfm_plan* p, const PlanInput* in, int n_inst, cudaStream_t st);

// The pieces of labfm_rk_step (step.cu), also used by the step graphs.
// dt > 0: uniform step; dt == 0: the plan's per-node dt.  `profile` enables the
// launch-timing hooks (off while a graph is being captured).
int rk_pack(const labfm_plan* p, const void* Q, void* work, cudaStream_t st);
int rk_unpack(const labfm_plan* p, void* Q, const void* work, cudaStream_t st);
// soa_out (or null): the step's filter also stores the new state there (3 x N).
int rk_one_step(const labfm_plan* p, void* work, double dt, const labfm_phys* ph, bool profile,
                cudaStream_t st, void* soa_out = nullptr);
int set_node_dt(labfm_plan* p, const double* dt_inst_host, cudaStream_t st);
// Pack / unpack a 3 x N structure-of-arrays state into / out of the packed node
// layout of the step kernels (step.cu).
int pack_fields(const labfm_plan* p, const void* soa, void* packed, cudaStream_t st);
int unpack_fields(const labfm_plan* p, const void* packed, void* soa, cudaStream_t st);
// The four stages of one RK step from the packed state X1, storing the stage
// states X2, X3, X4; P receives the partial solution register (after stage 4, the
// unfiltered next state).  Every stage also stores, at D + (stage - 1) N (D8
// records of the plan's precision), the eight derivative combinations the
// reverse sweep needs (step.cu).
int forward_stages(const labfm_plan* p, const void* X1, void* P, void* X2, void* X3, void* X4,
                   void* D, double dt, const labfm_phys* ph, cudaStream_t st);
// One RK step from Q (3 x N SoA, replaced by the next state) that stores its four
// stage states, packed, in X (4 x N) followed by their derivative combinations
// (4 x N D8 records); P and Y are scratch packed states (step.cu).
int rk_step_record(const labfm_plan* p, void* Q, void* X, void* P, void* Y, double dt,
                   const labfm_phys* ph, cudaStream_t st);
// Bytes of one packed node state and of one D8 record in the plan's precision.
size_t packed_bytes(const labfm_plan* p);
size_t d8_bytes(const labfm_plan* p);
int launch_stable_dt_instances(const labfm_plan* p, const void* fields, const double* s, double c,
                               double mu, double* dt_inst, cudaStream_t st);
int persistent_grid(const labfm_plan* p);
int filter_persistent_grid(const labfm_plan* p);
// Configure the staged F32 stage kernel for `stages` ring slots (0 = off); synchronises.
int configure_staging(labfm_plan* p, int stages, cudaStream_t st);
// Bytes per padded stencil entry of the plan's RHS (filter = false) or filter
// record stream (step.cu).
int plan_entry_bytes(const labfm_plan* p, bool filter);

}  // namespace labfm
