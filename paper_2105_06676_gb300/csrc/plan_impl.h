// The plan object behind the opaque stencil_plan_t handle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "internal.h"

struct AperiodicState;

// Kernel kinds for per-pass timing (stencil_profile_*).
enum PassKind {
    PASS_ROWS_R2C = 0,
    PASS_COLS_FWD = 1,
    PASS_COLS_FUSED = 2,
    PASS_COLS_INV = 3,
    PASS_ROWS_C2R = 4,
    PASS_FUSED_1D = 5,
    PASS_STRIP_R2C = 6,
    PASS_STRIP_COLS = 7,
    PASS_STRIP_C2R = 8,
    PASS_BASE_LOOP = 9,
    PASS_COPY = 10,
    PASS_VTABLE = 11,
    PASS_GATHER = 12,
    PASS_SCATTER = 13,
    PASS_KINDS = 14
};

// Optional CUDA-event bracketing of every kernel launch of a run, on the
// launching stream.
struct Profiler {
    bool enabled = false;
    struct Mark { int kind; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> pool;
    double ms[PASS_KINDS] = {};
    long long launches[PASS_KINDS] = {};
    cudaEvent_t get();
    void begin(int kind, cudaStream_t s);
    void end(cudaStream_t s);
    cudaError_t collect();
    ~Profiler();
};

struct stencil_plan_s {
    int ndim = 0;
    int radius = 0;
    int boundary = 0;
    int precision = 0;
    int64_t dims[3] = {1, 1, 1};
    int64_t n_cells = 0;
    double weights[sfft::kMaxWeights] = {};
    int nweights = 0;
    bool real_symbol = false;
    // toward-reach per face [axis][side] (side 0: the face below index 0): the
    // largest offset towards that face among the nonzero weights; it sets the
    // l-shell regions of the zero-Dirichlet / reflecting solves
    int reach[3][2] = {};
    // implicit stencil Q a_{t+1} = S a_t (weights hold S): Q's weights, also
    // in device memory for the multiplier-table kernel
    bool implicit = false;
    double weights_q[sfft::kMaxWeights] = {};
    double* wq_dev = nullptr;
    // vector-valued fields (stencil_plan_vector): nfields^2 blocks of
    // nweights weights in device memory; H holds every field's half spectrum
    bool vector = false;
    int nfields = 1;
    double* wv_dev = nullptr;
    // per block: |Lambda_ij - Lambda32_ij| <= sum|w_ij| 2^-16 (a generous
    // bound on at most 343 products of three rounded table entries and a
    // rounded weight), for the FP32 underflow screen of the vector multiply
    float vdelta[16] = {};
    // mixed-radix axes (length not a power of two): exp(-2 pi i m / l_a) per
    // such axis at pass precision; such plans run the vector path with one field
    bool mixed = false;
    void* mtw[3] = {nullptr, nullptr, nullptr};
    size_t elem = 0;
    int device = 0;
    // twiddles exp(-2 pi i m / 2^twn_log2) at pass precision
    int twn_log2 = 0;
    void* tw = nullptr;
    // per-axis exp(+2 pi i q / l_a), FP64 and FP32
    double2* E64[3] = {nullptr, nullptr, nullptr};
    float2* E32[3] = {nullptr, nullptr, nullptr};
    // half-spectrum workspace of the whole-grid solve
    void* H = nullptr;
    long long Mp = 0;
    size_t H_bytes = 0;
    // latched device status (bit 0: non-finite output, bit 2: abandoned
    // tensor-core wait)
    int* status = nullptr;
    // device grid owned by stencil_run_host
    void* dev_grid = nullptr;
    // Lambda^T / N over the half spectrum of a periodic 3-D or one-CTA 1-D
    // plan, cached for vt_T once a second consecutive run asks for the same T
    // (implicit plans: every plan shape, built on the first run of each T)
    void* vt = nullptr;
    int* vflags = nullptr;   // FP32 2-D blocked plans: vt in the blocked layout, flag per block
    int64_t vt_T = -1;
    int64_t last_T = -1;
    // zero-Dirichlet schedule and buffers (aperiodic.cu)
    AperiodicState* ap = nullptr;
    int64_t cutoff = 0;  // 0: automatic
    int schedule = 0;    // STENCIL_SCHEDULE_AUTO, _RECURSIVE or _LOOP
    int gemm = -1;       // tensor-core DFT operand mode (kGemm*), -1: CUDA-core FFTs
    Profiler prof;
    bool use_graphs = true;   // replay zero-Dirichlet runs as CUDA graphs
    int pass_variant = -1;    // periodic pass variant (PassVariantScope); -1 default
    size_t dev_bytes = 0;     // device memory this plan holds
};

namespace sfft {
// Records err as the calling thread's last CUDA error (stencil_cuda_error_name).
void note_cuda_error(cudaError_t err);
// Frees a plan none of whose work is still in flight, without a device-wide
// synchronisation (stencil_destroy waits for the whole device).
void plan_free_idle(stencil_plan_s* p);
int ilog2_exact(int64_t v);
void plan_set_weights(stencil_plan_s* p, int radius, const double* w);
// toward-reach per face of (2 radius + 1)^ndim weights into reach[3][2]
void face_reach(const double* w, int ndim, int radius, int reach[3][2]);
int64_t max_axis(int ndim, int precision, int axis);
SymbolParams make_symbol_params(const stencil_plan_s* p, const int64_t* len, int64_t T,
                                const double2* const* E64, const float2* const* E32,
                                const int* perm);
size_t periodic_workspace_bytes(int ndim, const int64_t* dims, int precision);
size_t multiplier_table_bytes(int ndim, const int64_t* dims, int precision);
template <typename R>
cudaError_t batched_solve(stencil_plan_s* p, R* S, const int64_t* len, int items, int64_t T,
                          void* H, long long Mp, const int* orient, const int (*perms)[3],
                          int norient, const void* tw, int twn_log2, const double2* const* E64,
                          const float2* const* E32, int* status, cudaStream_t s,
                          const void* const* vtabs, const void* const* vitems = nullptr,
                          R* Sout = nullptr);
template <typename R>
cudaError_t periodic_solve(stencil_plan_s* p, R* grid, const int64_t* len, int64_t T,
                           void* H, long long Mp, const void* tw, int twn_log2,
                           const double2* const* E64, const float2* const* E32, int* status,
                           cudaStream_t s);
}  // namespace sfft

int aperiodic_run(stencil_plan_s* p, void* grid, int64_t T, cudaStream_t s);
namespace sfft {
// Vector-valued fields (vector.cu): all passes of one run of a vector plan.
cudaError_t vector_run(stencil_plan_s* p, void* grid, int64_t T, cudaStream_t s);
int vector_max_fields();
}  // namespace sfft
// Builds the schedule, buffers and uploaded tables of T ahead of the first run
// (allocates; waits for the uploads); returns a status code.
int aperiodic_prepare(stencil_plan_s* p, int64_t T);
// Measures the schedule candidates for T and keeps the fastest; returns its
// index (times in ms[i] for i < cap) or a negative status.
int aperiodic_autotune(stencil_plan_s* p, const void* grid, int64_t T, cudaStream_t s,
                       double* ms, int cap);
void aperiodic_release(stencil_plan_s* p);
// drop captured graphs (their kernel parameters hold the plan's weights)
void aperiodic_forget_graphs(stencil_plan_s* p);
// Drops the cached per-T schedules (and their graphs and Lambda^T tables).
void aperiodic_forget_schedules(stencil_plan_s* p);
// device bytes held by the zero-Dirichlet machinery of a plan
size_t aperiodic_bytes(const stencil_plan_s* p);
