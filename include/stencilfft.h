/*
 * stencilfft.h -- C ABI of libstencilfft.so, a GB300 (sm_103a) solver that
 * advances a linear, constant-coefficient stencil T time steps in
 * O(N log N) work independent of T ("Fast Stencil Computations using Fast
 * Fourier Transforms", arXiv 2105.06676).
 *
 * Problem (paper Sec. 1, "Problem Specification"; d-D form in the appendix
 * "Supporting d-D Spatial Grids"): a grid a of shape l_1 x ... x l_d
 * (d = 1..3, row-major, last axis contiguous) evolves by
 *
 *     a_{t+1}[i] = sum over m in [-r, r]^d of  w[m] * a_t[i + m]
 *
 * and the library returns a_T. Weights are given over the box [-r, r]^d in
 * row-major order (entry (m_1 + r, ..., m_d + r)); in the paper's circulant
 * notation (Sec. 4) the stored first column of S is s[(-m) mod l] = w[m].
 *
 *   STENCIL_PERIODIC        every index wraps (Sec. 1: the grid is a torus);
 *                           solved by StencilFFT-P (Sec. 4, Eq. final_data:
 *                           a_T = F^-1 Lambda^T F a_0).
 *   STENCIL_ZERO_DIRICHLET  cells outside the grid read 0; solved by
 *                           StencilFFT-A (Sec. 5): the interior from the
 *                           periodic solve, the boundary's region of influence
 *                           from RecursiveBoundary.
 *
 * Precision: STENCIL_FP64 grids are double and every step runs in FP64.
 * STENCIL_FP32 grids are float; the FFT passes run in FP32 while the symbol
 * Lambda and its T-th power are evaluated in FP64 on the GPU and rounded once.
 * STENCIL_FP32_GEMM_* grids are float and run as STENCIL_FP32, except that
 * every 16-point DFT of the transforms along the strided axes (all axes but
 * the last) is a GEMM on the tensor cores (tcgen05, FP32 accumulation) with
 * bf16 or fp16 operands, or with bf16 hi + lo split operands (three products).
 * The single-term variants carry the operand rounding (about 2^-9 for bf16,
 * 2^-12 for fp16 per stage) into the result and are not expected to meet the
 * FP32 path's accuracy; the split variant is. GEMM plans are periodic, d = 2
 * or 3, with every strided axis between 256 and 4096 (else
 * STENCIL_EUNSUPPORTED); an abandoned tensor-core wait makes stencil_status
 * return STENCIL_ETIMEOUT.
 *
 * Supported sizes: every l_k a power of two with l_k >= 2r + 1 and l_k >= 4.
 * Limits per precision are reported by stencil_max_axis().
 *
 * Errors: every call returns 0 (STENCIL_OK) or a negative STENCIL_E* code;
 * stencil_strerror() names it. No call aborts the process. Device-side
 * conditions (non-finite output) are latched in a per-plan status word read
 * by stencil_status().
 *
 * Ownership: the caller owns every grid pointer. The library owns plans and
 * all device workspace, allocated in stencil_plan (and, for zero-Dirichlet
 * plans, on the first stencil_run for a given T) and released by
 * stencil_destroy. A plan may be used from one host thread at a time.
 */
#ifndef STENCILFFT_H
#define STENCILFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stencil_plan_s* stencil_plan_t;

/*
 * Boundary conditions. STENCIL_NEUMANN is the reflecting (zero-flux) boundary:
 * the ghost cell at index -1-k reads cell k and the one at l+k reads cell
 * l-1-k (half-sample mirror, refreshed from the current values every step);
 * the radius must not exceed any axis length. Both aperiodic conditions use
 * RecursiveBoundary (paper Sec. 5): its periodic solves keep only cells the
 * boundary cannot reach, and the condition enters through the base-case loop.
 * The regions are cut per face from the weights (appendix "l-shell Spatial
 * Grid Decomposition"): the largest offset towards a face among the nonzero
 * weights sets how far the boundary reaches through it per step, so a biased
 * or upwind stencil gets narrower regions and a face that no offset looks
 * towards gets none; zero weights at the edge of the (2r+1)^ndim box cost
 * nothing. A symmetric box stencil gets the distance bands of Sec. 5.2.
 */
enum stencil_boundary { STENCIL_PERIODIC = 0, STENCIL_ZERO_DIRICHLET = 1, STENCIL_NEUMANN = 2 };
enum stencil_precision {
    STENCIL_FP64 = 0,
    STENCIL_FP32 = 1,
    STENCIL_FP32_GEMM_BF16 = 2,    /* FP32 grid; strided-axis radix-16 DFTs as bf16 GEMMs */
    STENCIL_FP32_GEMM_FP16 = 3,    /* the same with fp16 operands */
    STENCIL_FP32_GEMM_BF16X3 = 4   /* bf16 hi + lo split operands, three products */
};

enum stencil_status_code {
    STENCIL_OK = 0,
    STENCIL_EINVAL = -1,       /* bad argument: null pointer, ndim, radius, T < 0, size */
    STENCIL_ENOMEM = -2,       /* device or host allocation failed */
    STENCIL_ECUDA = -3,        /* a CUDA runtime call failed */
    STENCIL_ETIMEOUT = -4,     /* a bounded device wait gave up */
    STENCIL_ENONFINITE = -5,   /* the solve produced Inf or NaN */
    STENCIL_EQUEUEFULL = -6,   /* server queue has no free slot */
    STENCIL_EUNSUPPORTED = -7  /* valid request outside this build's size limits */
};

/*
 * Create a plan.
 *   out       receives the plan handle (host pointer, non-null).
 *   ndim      1, 2 or 3.
 *   dims      host array of ndim axis lengths, row-major order.
 *   radius    r >= 0 (paper's sigma for box stencils).
 *   weights   host array of (2r+1)^ndim doubles (copied).
 *   boundary  STENCIL_PERIODIC, STENCIL_ZERO_DIRICHLET or STENCIL_NEUMANN.
 *   precision STENCIL_FP64, STENCIL_FP32 or STENCIL_FP32_GEMM_*.
 * Allocates the FFT workspace and the twiddle and symbol tables on the
 * current CUDA device and builds them there (twiddles by FP64 sincospi,
 * paper Sec. 4 "Step 1").
 */
int stencil_plan(stencil_plan_t* out, int ndim, const int64_t* dims, int radius,
                 const double* weights, int boundary, int precision);

/*
 * Plan an implicit stencil  Q a_{t+1} = S a_t  on a periodic grid (paper
 * Sec. 4.2 "Implicit Stencils", appendix "Supporting Implicit Stencils"): the
 * run advances by the explicit stencil R with symbol
 * Lambda_R = Lambda_Q^+ Lambda_S, where Lambda_Q^+ is 1 / Lambda_Q where
 * Lambda_Q is not zero and 0 where it is (|Lambda_Q| <= 2^-40 sum|q| counts as
 * zero). Where Q is invertible the result satisfies Q a_{t+1} = S a_t.
 *   weights_s, weights_q  host arrays of (2r+1)^ndim doubles each (copied),
 *                         in the layout of stencil_plan's weights:
 *                         (S a)[i] = sum_m weights_s[m] a[i + m], same for Q.
 *   precision             STENCIL_FP64 or STENCIL_FP32.
 * Other arguments as for stencil_plan (the boundary is periodic). Every run
 * multiplies by a table of Lambda_R^T / N built in FP64 on the GPU on the
 * first run of each T (or by stencil_prepare); stencil_run, stencil_run_host,
 * stencil_prepare, stencil_symbol_power (which returns Lambda_R^T), status
 * and destroy apply unchanged. Returns STENCIL_EUNSUPPORTED for other
 * precisions and for 1-D axes whose packed half length is below 16 or above
 * what one CTA holds; stencil_plan_set_weights on the plan returns
 * STENCIL_EUNSUPPORTED.
 */
int stencil_plan_implicit(stencil_plan_t* out, int ndim, const int64_t* dims, int radius,
                          const double* weights_s, const double* weights_q, int precision);

/*
 * Plan m = nfields coupled scalar fields on a periodic grid (paper Sec. 4.2
 * "Vector-Valued Fields", appendix "Supporting Vector Valued Fields"):
 *     a^(i)_{t+1}[x] = sum_j sum_k w_ij[k] a^(j)_t[x + k].
 * Every field takes the forward Multi-FFT; at every wave vector the m x m
 * matrix of symbols is raised to the power T by repeated squaring in FP64 on
 * the GPU (skipped where a bound on its infinity norm shows every entry of the
 * power below half the smallest subnormal of the pass precision), rounded to
 * the pass precision and applied to the m spectra; the inverse Multi-FFT
 * returns every field. This also covers affine stencils (a constant field)
 * and stencils that read several past steps (one field per step).
 *   nfields   1..4.
 *   weights   host array of nfields * nfields * (2r+1)^ndim doubles (copied):
 *             block (i, j), the stencil taking field j into field i, in the
 *             layout of stencil_plan's weights.
 *   precision STENCIL_FP64 or STENCIL_FP32.
 * Other arguments as for stencil_plan (the boundary is periodic). stencil_run
 * then takes a device grid of nfields * prod(dims) elements: field i at
 * offset i * prod(dims). stencil_run_host, stencil_symbol_power and
 * stencil_plan_set_weights return STENCIL_EUNSUPPORTED for vector plans;
 * stencil_prepare is a no-op.
 */
int stencil_plan_vector(stencil_plan_t* out, int ndim, const int64_t* dims, int radius,
                        int nfields, const double* weights, int precision);

/*
 * Advance grid by T >= 0 steps in place (paper Fig. "stencil-fft-algorithm-dD"
 * for periodic plans, Fig. "stencil-fft-algorithm-1D-aperiodic" for
 * zero-Dirichlet plans).
 *   grid    device pointer to prod(dims) elements (double for FP64 plans,
 *           float for FP32 plans), 16-byte aligned.
 *   stream  a cudaStream_t (NULL = legacy default stream).
 * Periodic plans: enqueues work only and allocates nothing; returns before the
 * GPU finishes. Zero-Dirichlet plans: the same once T has been prepared (by
 * stencil_prepare or an earlier run with this T); a first run for a T that
 * was not prepared builds the RecursiveBoundary schedule, which allocates
 * device memory (cudaMalloc, an implicit device synchronisation) and waits for
 * the upload of its tables on the calling thread's per-thread stream. The
 * second run for a (T, grid) pair captures a CUDA graph (host work only) that
 * later runs replay. T == 0 is a no-op.
 */
int stencil_run(stencil_plan_t plan, void* grid, int64_t T, void* stream);

/*
 * Do the per-T set-up of stencil_run ahead of time, so that runs with this T
 * allocate nothing and do not synchronise (paper Sec. 4 "Step 2": the symbol
 * power depends on T only; Sec. 5: the RecursiveBoundary schedule depends on
 * T and the grid shape only).
 *   Zero-Dirichlet plans: builds the schedule, its buffers and its uploaded
 *   tables (allocates; waits for the uploads on the per-thread stream).
 *   Periodic plans that keep a multiplier table (3-D, and 1-D axes of 32 ..
 *   2^15 points FP32 / 2^14 FP64): builds Lambda^T / N for T on `stream`, so
 *   the next run with T uses it; other periodic plans: nothing to do.
 * T == 0 is a no-op. Returns STENCIL_OK, STENCIL_EINVAL (null plan, T < 0),
 * STENCIL_ENOMEM or STENCIL_ECUDA.
 */
int stencil_prepare(stencil_plan_t plan, int64_t T, void* stream);

/*
 * End-to-end variant of stencil_run on host memory; synchronises the stream
 * before returning. host_in and host_out hold prod(dims) elements of the
 * plan's precision and may alias. When both are page-locked host memory the
 * GPU can address (cudaHostGetDevicePointer succeeds; on a Grace-Blackwell
 * node over the coherent chip-to-chip link) and the plan is periodic with
 * d >= 2, the first pass reads host_in in place and the last pass writes
 * host_out in place -- the data crosses the link once each way with no
 * staging copy. Otherwise host_in is copied to a plan-owned device grid, the
 * grid is solved and copied back.
 */
int stencil_run_host(stencil_plan_t plan, const void* host_in, void* host_out,
                     int64_t T, void* stream);

/*
 * Symbol power (paper Sec. 4 "Step 2", repeated squaring of Lambda = F s):
 * writes V[k] = Lambda[k]^T for the half spectrum k_d = 0 .. l_d/2 of the
 * last axis and every k_1..k_{d-1}, as interleaved complex FP64 in row-major
 * order of shape (l_1, ..., l_{d-1}, l_d/2 + 1), to the device buffer out.
 * Lambda[k] = sum_m w[m] exp(+2 pi i sum_j m_j k_j / l_j) (appendix "Proof of
 * Eigenvalue-FFT Relation" with the unnormalised forward DFT of Sec. 4).
 * Same FP64 device arithmetic as the solver's fused spectral multiply, without
 * the 1/N scale and without the underflow shortcut.
 */
int stencil_symbol_power(stencil_plan_t plan, int64_t T, void* out, void* stream);

/*
 * Synchronise stream and report the plan's latched device status:
 * STENCIL_OK, STENCIL_ENONFINITE (Inf/NaN written by a solve since the last
 * call) or STENCIL_ECUDA. Clears the latch.
 */
int stencil_status(stencil_plan_t plan, void* stream);

/*
 * Replace the plan's stencil: radius r (0..3, every axis >= 2r+1) and
 * (2r+1)^ndim weights (host, copied; finite), as in stencil_plan. Runs
 * enqueued afterwards use them; runs already enqueued keep the stencil they
 * were launched with. The plan keeps its tables and workspace; cached graphs,
 * the repeated-T multiplier table and, when the radius changes, the
 * zero-Dirichlet schedules (this waits for the device) are dropped. Serves a
 * caller that solves many stencils of one grid shape (paper Sec. 4: the
 * stencil enters only through the symbol Lambda). Returns STENCIL_OK or
 * STENCIL_EINVAL.
 */
int stencil_plan_set_weights(stencil_plan_t plan, int radius, const double* weights);

/*
 * Base-case cutoff of RecursiveBoundary for zero-Dirichlet plans (paper
 * Fig. "stencil-fft-algorithm-1D-aperiodic", Base Case): subproblems with
 * T < cutoff are advanced by the direct loop. cutoff >= 2, or 0 for the
 * automatic choice (a cutoff fitted to shared memory; with the AUTO schedule
 * below, also the choice between the recursion and the direct loop). The
 * result does not depend on it beyond rounding.
 */
int stencil_plan_set_cutoff(stencil_plan_t plan, int64_t cutoff);

/*
 * Schedule of zero-Dirichlet plans: STENCIL_SCHEDULE_AUTO (RecursiveBoundary,
 * paper Sec. 5, or the direct loop of Sec. 1 "Problem Specification" when a
 * cost estimate of the boundary region says it is cheaper -- a region that
 * covers most of the grid gains nothing from FFTs), STENCIL_SCHEDULE_RECURSIVE
 * (always RecursiveBoundary), STENCIL_SCHEDULE_LOOP (always the temporally
 * blocked direct loop over the whole grid) or STENCIL_SCHEDULE_CLUSTER (the
 * direct loop with the whole grid held in the distributed shared memory of
 * one thread-block cluster, one launch for all T steps; a later
 * stencil_run returns STENCIL_EUNSUPPORTED when the grid does not fit). The
 * result does not depend on it beyond rounding. Changing it or the cutoff drops the plan's cached
 * schedules and graphs (waits for the device). Returns STENCIL_EINVAL for a
 * NULL plan or an unknown mode.
 */
enum stencil_schedule {
    STENCIL_SCHEDULE_AUTO = 0,
    STENCIL_SCHEDULE_RECURSIVE = 1,
    STENCIL_SCHEDULE_LOOP = 2,
    STENCIL_SCHEDULE_CLUSTER = 3
};
int stencil_plan_set_schedule(stencil_plan_t plan, int mode);

/*
 * Measured schedule choice for a zero-Dirichlet plan and one T: runs the
 * candidates -- RecursiveBoundary with the automatic base-case cutoff, with
 * half and with twice that cutoff (when the tiles fit), the whole-grid loop
 * and, when the grid fits one cluster, the cluster-resident loop -- three
 * times each on a scratch copy of grid (device, prod(dims)
 * elements, not modified), times the last run of each with CUDA events on
 * stream, and keeps the fastest for later runs of this T while the plan's
 * schedule is STENCIL_SCHEDULE_AUTO with cutoff 0. Writes the times in ms to
 * ms[i] for the first cap of five fixed slots -- 0 recursive, 1 loop,
 * 2 recursive with half the cutoff, 3 recursive with twice the cutoff,
 * 4 cluster-resident loop; -1 for a slot that does not apply -- and returns
 * the slot of the one kept.
 * Periodic 2-D / 3-D plans (not implicit, vector, mixed-radix or tensor-core
 * plans): times the four pass variants -- 0 the default (FP32 2-D: half
 * spectrum in column blocks, TMA-fed column and C2R passes), 1 row-major half
 * spectrum with the TMA-fed passes, 2 the register kernels only with
 * 1024-thread FP32 column CTAs, 3 the register kernels with 512-thread column
 * CTAs -- four timed runs each after two warm-up runs, keeps the fastest for
 * this plan and for plans of the same shape and precision created later in
 * this process; ms[i] holds variant i's mean time.
 * Synchronises stream. Errors: STENCIL_EINVAL (NULL plan or grid, T < 1,
 * cap < 0, ms NULL with cap > 0), STENCIL_EUNSUPPORTED for the periodic plans
 * named above and 1-D periodic plans, the status of a failing run.
 */
int stencil_plan_autotune(stencil_plan_t plan, const void* grid, int64_t T, void* stream,
                          double* ms, int cap);

/* Set a periodic plan's pass variant (0..3 as listed for stencil_plan_autotune,
 * -1 for the default selection). Variants change kernels and layouts only, not
 * the result beyond rounding. STENCIL_EINVAL for other values,
 * STENCIL_EUNSUPPORTED for aperiodic plans. */
int stencil_plan_set_pass_variant(stencil_plan_t plan, int variant);

/*
 * Per-kernel timing (measurement support, not part of the paper's method).
 * While enabled, every kernel launch of stencil_run on this plan is bracketed
 * by CUDA events recorded on the launching stream. stencil_profile_read
 * waits for those events and returns, per kernel kind k < nkinds, the summed
 * milliseconds ms[k] and the launch count launches[k] since the last read,
 * then resets them. stencil_profile_kind_name gives the static name of kind k
 * (NULL past the last kind).
 */
int stencil_profile_enable(stencil_plan_t plan, int enable);
int stencil_profile_read(stencil_plan_t plan, double* ms, int64_t* launches, int nkinds);
const char* stencil_profile_kind_name(int kind);

/*
 * Host-only view of the zero-Dirichlet schedule (RecursiveBoundary flattened
 * into a sequence of operations, paper Fig.
 * "stencil-fft-algorithm-1D-aperiodic", with its regions over l-shells,
 * appendix "l-shell Spatial Grid Decomposition"), for checking the schedule
 * without a GPU. Writes up to cap int64 values to out (may be NULL) and
 * returns the number needed, or -1 for invalid arguments (radius must be >= 1,
 * T >= 1). Faces are numbered f = 2 a + side (side 0: the face below index 0
 * of axis a, distance g_a + 1; side 1: the face above index l_a - 1, distance
 * l_a - g_a). Records, in execution order:
 *   1, step, T_k, level, n, then per strip: bdims[3], off[3], valid[3],
 *      perm[3], lo[6], hi[6], face_axis, face_side
 *                                      -- periodic solves of the strips (stashed)
 *   2, step                            -- scatter of that step's kept cells
 *   3, T_b, wout[6], n, then per tile: (lo, hi) for each of 3 axes
 *                                      -- base case over output tiles, writing
 *                                         the cells within wout[f] of some face f
 *   4, T_c                             -- T_c steps of the loop on the whole grid
 *   5, T                               -- T single steps of the loop on the whole grid
 *   6, T                               -- T steps of the loop on the whole grid held
 *                                         in one thread-block cluster's shared memory
 *                                         (only where a GPU that can run it is present)
 * With cutoff 0 the schedule is the one the solver runs: RecursiveBoundary, or
 * the plain loop (records 4 / 5 / 6 only) when its estimated cost is lower.
 * Axes beyond ndim are reported with extent 1 and faces beyond 2 ndim with 0.
 * A strip's box axis b is grid axis perm[b]; its box cell q maps to grid cell
 * off + q when q < valid on every axis. A scatter writes the cells farther
 * than lo[f] from every face f that are within hi[f] of the strip's own face
 * (face_axis, face_side), or of some face when face_axis is -1 (a whole-grid
 * solve). stencil_debug_schedule takes the toward-reach of every face to be
 * radius (a (2 radius + 1)^ndim box of nonzero weights);
 * stencil_debug_schedule_reach takes reach[2 a + side] (each in 0..radius, not
 * all 0): the largest offset towards that face among the nonzero weights.
 */
int64_t stencil_debug_schedule(int ndim, const int64_t* dims, int radius, int64_t T,
                               int64_t cutoff, int64_t* out, int64_t cap);
int64_t stencil_debug_schedule_reach(int ndim, const int64_t* dims, int radius, const int* reach,
                                     int64_t T, int64_t cutoff, int64_t* out, int64_t cap);

/*
 * Host-only: the toward-reach a plan derives from its weights, the input of
 * the l-shell regions above. weights: (2 radius + 1)^ndim doubles laid out as
 * for stencil_plan; writes reach[2 a + side] for a < ndim (side 0: the face
 * below index 0, the largest -m_a over the nonzero weights; side 1: the face
 * above the last index, the largest +m_a; 0 where no offset points that way).
 * Returns STENCIL_OK or STENCIL_EINVAL (null pointer, ndim outside 1..3,
 * radius outside 0..3).
 */
int stencil_debug_face_reach(int ndim, int radius, const double* weights, int* reach);

/*
 * Periodic solve that allocates nothing. The paper has no counterpart: this
 * entry point serves callers that cannot allocate device memory when they
 * solve (a latency-critical loop that cannot pay cudaMalloc's implicit device
 * synchronisation, or a program whose allocator has already reserved the
 * device memory). It advances grid (device pointer, 16-byte aligned, prod(dims)
 * elements of the given precision) by T >= 0 steps in place on stream, exactly
 * like stencil_plan + stencil_run with STENCIL_PERIODIC, but takes all scratch
 * (tables, half-spectrum workspace, status word) from one fixed device array of
 * stencil_noalloc_scratch_bytes() bytes (32 MiB) that every GPU loading this
 * library holds until exit. Sizes whose scratch does not fit return
 * STENCIL_EUNSUPPORTED (e.g. a 2-D FP32 grid holds up to 2048 x 2048 cells);
 * bad arguments return STENCIL_EINVAL. Every call looks up the array's address
 * on the current device (after a device reset the array is found again); the
 * first call on a device loads the library's module there and should come
 * before any stream capture. Calls share the array: calls whose work overlaps
 * on the GPU race and must be serialised by the caller. Non-finite output is
 * not reported. Calls no allocating routine.
 */
int stencil_periodic_run_noalloc(int ndim, const int64_t* dims, int radius,
                                 const double* weights, int precision, void* grid,
                                 int64_t T, void* stream);

/* Size in bytes of the fixed scratch array used by stencil_periodic_run_noalloc. */
size_t stencil_noalloc_scratch_bytes(void);

/* ------------------------------------------------------------------------
 * Serving: a persistent request loop with continuous batching (the paper has
 * no serving layer; this is the system around its solver).
 *
 * A server owns a worker thread and max_slots non-blocking CUDA streams on the
 * current device. Requests of any dimension, size, T, boundary, radius and
 * weights are admitted in arrival order whenever a slot is free and the device
 * memory of the plan they need fits hbm_budget_bytes (plans -- twiddles,
 * symbol tables, workspaces -- are pooled by shape and reused; the grids are
 * the caller's and are not counted). Requests admitted while others run
 * overlap on the device. Small periodic requests of one shape are batched
 * into one launch per pass, each with its own Lambda^T table; a request's
 * result is the same alone or batched.
 * ------------------------------------------------------------------------ */
typedef struct stencil_server_s* stencil_server_t;

typedef struct {
    int ndim;            /* 1..3 */
    int64_t dims[3];     /* first ndim entries used */
    int radius;          /* 0..3 */
    const double* weights; /* (2r+1)^ndim, copied at submit */
    int boundary;        /* STENCIL_PERIODIC or STENCIL_ZERO_DIRICHLET */
    int precision;       /* STENCIL_FP64 or STENCIL_FP32 */
    int64_t T;           /* >= 0 */
    void* grid;          /* device, 16-byte aligned, solved in place; the caller keeps it
                            alive and untouched until the ticket completes */
} stencil_request;

/* ------------------------------------------------------------------------
 * Batched small periodic solves of mixed shapes (row C1 of the design: the
 * paper runs independent solves "in parallel", Sec. 5.2, and the Multi-FFT
 * runs one transform per axis with every other index in parallel, Sec. 4).
 * An executor keeps a device work list of request descriptors; one run
 * launches ONE persistent kernel in which every CTA takes the next request
 * from a device counter and performs its whole StencilFFT-P (R2C rows, the
 * strided FFTs, the multiply by Lambda^T / N with the FP64 power, the inverse
 * passes) in shared memory, in place on the request's grid. Requests of one
 * run may differ in dimension, shape, radius, weights and T.
 * ------------------------------------------------------------------------ */
typedef struct stencil_batch_s* stencil_batch_t;

/* Shared memory one request of this shape needs in the executor (bytes), or 0
 * when the executor does not take it: power-of-two axes of 4..8192, rows *
 * (n + 1) <= 8192 half-spectrum values (n = half the last axis), at most
 * 200 KB. precision STENCIL_FP32 or STENCIL_FP64. */
size_t stencil_batch_smem_bytes(int ndim, const int64_t* dims, int precision);

/* Create an executor for up to `capacity` requests per run (1..2^20) of one
 * precision (STENCIL_FP32 or STENCIL_FP64) on the current device: twiddle and
 * symbol tables for axes up to 8192, the device work list, pinned staging.
 * Returns STENCIL_OK, STENCIL_EINVAL, STENCIL_ENOMEM or STENCIL_ECUDA. */
int stencil_batch_create(stencil_batch_t* out, int capacity, int precision);

/* Solve `count` requests (host array; boundary STENCIL_PERIODIC, the
 * executor's precision, stencil_batch_smem_bytes > 0, grids 16-byte aligned
 * device pointers advanced in place) on `stream`. Uploads the work list and the
 * requests' symbol parameters, resets the device counter and launches the
 * persistent kernel; returns before the GPU finishes. A run waits on the host
 * until the previous run's upload has been read; runs of one executor on
 * different streams must not overlap (use one executor per stream).
 * Returns STENCIL_EINVAL / STENCIL_EUNSUPPORTED before any work for a bad
 * request, STENCIL_ECUDA on a launch failure. */
int stencil_batch_run(stencil_batch_t b, int count, const stencil_request* reqs, void* stream);

/* Synchronise `stream` and return STENCIL_ENONFINITE if a result since the last
 * call held a non-finite value (the flag is then cleared), else STENCIL_OK. */
int stencil_batch_status(stencil_batch_t b, void* stream);

/* Wait for the executor's last run (its completion event, no device-wide
 * synchronisation) and free it. */
int stencil_batch_destroy(stencil_batch_t b);

typedef struct {
    uint64_t submitted, completed, failed;
    int max_in_flight;           /* most slots busy at once */
    uint64_t batched_launches;   /* launches that carried stacked small requests */
    uint64_t batched_requests;   /* requests served inside those */
    size_t bytes_in_use, peak_bytes, budget_bytes;
} stencil_server_stats_t;

/* Create a server (max_slots 1..64, queue_capacity >= 1, budget > 0). */
int stencil_server_create(stencil_server_t* out, size_t hbm_budget_bytes, int max_slots,
                          int queue_capacity);
/* Queue a request; returns STENCIL_EQUEUEFULL when queue_capacity requests wait,
 * STENCIL_EINVAL / STENCIL_EUNSUPPORTED for a bad request. Never blocks on the GPU. */
int stencil_server_submit(stencil_server_t s, const stencil_request* r, uint64_t* ticket);
/* *done = 1 once the request finished; then returns its status and sets
 * *latency_s (submit to completion, seconds). */
int stencil_server_poll(stencil_server_t s, uint64_t ticket, int* done, double* latency_s);
/* Block until the request finishes (STENCIL_ETIMEOUT after timeout_s seconds). */
int stencil_server_wait(stencil_server_t s, uint64_t ticket, double timeout_s, double* latency_s);
int stencil_server_stats(stencil_server_t s, stencil_server_stats_t* out);
/* Finish every queued request, then release the server and its plans. */
int stencil_server_destroy(stencil_server_t s);

/* Release a plan and all its device memory (synchronises the device). */
int stencil_destroy(stencil_plan_t plan);

/* Static, human-readable name of a status code. */
const char* stencil_strerror(int code);

/* Name of the CUDA runtime error behind the calling thread's most recent
 * STENCIL_ECUDA or STENCIL_ENOMEM ("cudaSuccess" if there was none): a
 * diagnostic for the caller, static storage. */
const char* stencil_cuda_error_name(void);

/*
 * Largest supported axis length for (ndim, precision, axis). axis 0..ndim-1.
 * Returns 0 for invalid arguments.
 */
int64_t stencil_max_axis(int ndim, int precision, int axis);

/* Bytes of device workspace a plan with these arguments allocates: the half
 * spectrum, plus for periodic plans that keep one the Lambda^T / N table (0 on
 * error). */
size_t stencil_workspace_bytes(int ndim, const int64_t* dims, int radius, int boundary,
                               int precision);

#ifdef __cplusplus
}
#endif

#endif /* STENCILFFT_H */
