// Host side of libstencilfft.so: plans, workspace, and the C ABI declared in
// include/stencilfft.h.
//
// A periodic run is StencilFFT-P (paper Sec. 4, Fig. "stencil-fft-algorithm-dD"):
//   d = 1 : one fused kernel per row (R2C, multiply by V, C2R in shared memory);
//   d = 2 : rows_r2c -> cols_fused(axis 0) -> rows_c2r;
//   d = 3 : rows_r2c -> cols(axis 1, fwd) -> cols_fused(axis 0)
//           -> cols(axis 1, inv) -> rows_c2r.
// A zero-Dirichlet run is StencilFFT-A (Sec. 5), implemented in aperiodic.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <vector>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/stencilfft.h"
#include "internal.h"
#include "plan_impl.h"

using namespace sfft;

// Profiler: events are pooled and only recorded while profiling is enabled.
cudaEvent_t Profiler::get() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
void Profiler::begin(int kind, cudaStream_t s) {
    if (!enabled) return;
    Mark m{kind, get(), get()};
    cudaEventRecord(m.a, s);
    marks.push_back(m);
}
void Profiler::end(cudaStream_t s) {
    if (!enabled || marks.empty()) return;
    cudaEventRecord(marks.back().b, s);
}
cudaError_t Profiler::collect() {
    cudaError_t first = cudaSuccess;
    for (auto& m : marks) {
        cudaError_t err = cudaEventSynchronize(m.b);
        float t = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&t, m.a, m.b);
        if (err == cudaSuccess) {
            ms[m.kind] += t;
            launches[m.kind] += 1;
        } else if (first == cudaSuccess) {
            first = err;
        }
        pool.push_back(m.a);
        pool.push_back(m.b);
    }
    marks.clear();
    return first;
}
Profiler::~Profiler() {
    for (auto& m : marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
}

namespace sfft {

int ilog2_exact(int64_t v) {
    if (v <= 0 || (v & (v - 1))) return -1;
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return l;
}

int64_t max_axis(int ndim, int precision, int axis) {
    if (ndim < 1 || ndim > 3 || axis < 0 || axis >= ndim) return 0;
    const bool f32 = precision == STENCIL_FP32;
    if (ndim == 1) return int64_t(1) << 24;              // longer than 2 x 16 x threads: n1 x n2 passes
    if (axis == ndim - 1) return f32 ? 32768 : 16384;   // real rows: n = L/2 complex in one CTA
    return f32 ? 16384 : 8192;                           // strided complex columns
}

static bool symmetric_weights(const double* w, int ndim, int r) {
    const int W = 2 * r + 1;
    int count = 1;
    for (int a = 0; a < ndim; ++a) count *= W;
    for (int i = 0; i < count; ++i) {
        // index of -m: reverse every digit
        int rest = i, mirror = 0, mul = 1;
        for (int a = 0; a < ndim; ++a) {
            const int digit = rest % W;
            rest /= W;
            mirror += (W - 1 - digit) * mul;
            mul *= W;
        }
        if (w[i] != w[mirror]) return false;
    }
    return true;
}

// Symbol parameters for a periodic solve of a box of shape len[0..ndim-1].
// perm (optional) maps box axis a to grid axis perm[a]: the box then holds a
// transposed region of the grid, and Lambda uses the correspondingly permuted
// weights and the grid axis' tables.
SymbolParams make_symbol_params(const stencil_plan_s* p, const int64_t* len, int64_t T,
                                const double2* const* E64, const float2* const* E32,
                                const int* perm) {
    SymbolParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.ndim = p->ndim;
    sp.r = p->radius;
    sp.T = (long long)T;
    int pm[3] = {0, 1, 2};
    if (perm)
        for (int a = 0; a < p->ndim; ++a) pm[a] = perm[a];
    double N = 1.0;
    for (int a = 0; a < p->ndim; ++a) {
        const int ga = pm[a];
        sp.len[a] = (int)len[a];
        if (ilog2_exact(len[a]) < 0) {
            // mixed-radix axis (whole-grid solves only): indices taken modulo l_a
            sp.tshift[a] = 0;
            sp.tmask[a] = -1;
        } else {
            sp.tshift[a] = ilog2_exact(p->dims[ga]) - ilog2_exact(len[a]);
            sp.tmask[a] = (int)(len[a] - 1);
        }
        N *= (double)len[a];
        sp.E64[a] = E64[ga];
        sp.E32[a] = E32[ga];
    }
    // permuted weights: box offset m' has grid offset m with m[pm[a]] = m'[a]
    const int W = 2 * p->radius + 1;
    double wsum = 0.0;
    for (int i = 0; i < p->nweights; ++i) {
        int rest = i, digits[3] = {0, 0, 0};
        for (int a = p->ndim - 1; a >= 0; --a) {
            digits[a] = rest % W;   // box-axis digit m'_a + r
            rest /= W;
        }
        int gd[3] = {0, 0, 0};
        for (int a = 0; a < p->ndim; ++a) gd[pm[a]] = digits[a];
        int gi = 0;
        for (int a = 0; a < p->ndim; ++a) gi = gi * W + gd[a];
        sp.w[i] = p->weights[gi];
        sp.w32[i] = (float)p->weights[gi];
        wsum += std::fabs(p->weights[gi]);
    }
    sp.scale = 1.0 / N;
    sp.real_symbol = p->real_symbol ? 1 : 0;
    if (p->implicit) {
        // the implicit path is periodic only: boxes are the whole grid (no
        // permutation), so Q's weights keep the plan's order
        double qsum = 0.0;
        for (int i = 0; i < p->nweights; ++i) qsum += std::fabs(p->weights_q[i]);
        sp.wq = p->wq_dev;
        sp.qzero = qsum * std::ldexp(1.0, -40);
    }
    // |Lambda - Lambda_fp32| <= sum|w| * 2^-16: a generous bound on the error of
    // at most 343 products of <= 3 rounded table entries and a rounded weight.
    sp.delta = (float)(wsum * std::ldexp(1.0, -16)) + 1e-30f;
    sp.use_cut = 1;
    sp.cut = p->precision == STENCIL_FP32 ? 154.0f : 1080.0f;
    sp.tau2 = -1.0f;
    if (T > 0) {
        const double tau = std::exp2(-(double)sp.cut / (double)T) - (double)sp.delta;
        if (tau > 0) sp.tau2 = (float)(tau * tau * (1.0 - std::ldexp(1.0, -20)));
    }
    return sp;
}

static cudaError_t alloc_tables(stencil_plan_s* p) {
    cudaError_t err;
    int64_t tmax = 4;
    for (int a = 0; a < p->ndim; ++a)
        if (ilog2_exact(p->dims[a]) >= 0) tmax = std::max(tmax, p->dims[a]);
    p->twn_log2 = ilog2_exact(tmax);
    const size_t celem = p->precision == STENCIL_FP32 ? sizeof(float2) : sizeof(double2);
    err = cudaMalloc(&p->tw, celem << p->twn_log2);
    if (err != cudaSuccess) return err;
    // tables are built on the per-thread stream and awaited there, so creating a
    // plan never waits for work other streams have in flight
    const cudaStream_t ts = cudaStreamPerThread;
    err = p->precision == STENCIL_FP32 ? launch_twiddles<float>(p->tw, p->twn_log2, ts)
                                       : launch_twiddles<double>(p->tw, p->twn_log2, ts);
    if (err != cudaSuccess) return err;
    for (int a = 0; a < p->ndim; ++a) {
        err = cudaMalloc(&p->E64[a], sizeof(double2) * p->dims[a]);
        if (err != cudaSuccess) return err;
        err = cudaMalloc(&p->E32[a], sizeof(float2) * p->dims[a]);
        if (err != cudaSuccess) return err;
        err = launch_axis_table(p->E64[a], p->E32[a], (int)p->dims[a], ts);
        if (err != cudaSuccess) return err;
        if (ilog2_exact(p->dims[a]) < 0) {
            // mixed-radix axis: its own twiddle table exp(-2 pi i m / l_a)
            p->mixed = true;
            err = cudaMalloc(&p->mtw[a], celem * p->dims[a]);
            if (err != cudaSuccess) return err;
            p->dev_bytes += celem * p->dims[a];
            err = p->precision == STENCIL_FP32 ? launch_mixed_table<float>(p->mtw[a], (int)p->dims[a], ts)
                                               : launch_mixed_table<double>(p->mtw[a], (int)p->dims[a], ts);
            if (err != cudaSuccess) return err;
        }
    }
    err = cudaMalloc(&p->status, sizeof(int));
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(p->status, 0, sizeof(int), ts);
    p->dev_bytes += (celem << p->twn_log2) + sizeof(int);
    for (int a = 0; a < p->ndim; ++a) p->dev_bytes += (sizeof(double2) + sizeof(float2)) * p->dims[a];
    return err;
}

// Bytes of the Lambda^T / N table a periodic plan keeps for a repeated T: 3-D
// plans (one half spectrum) and 1-D axes one CTA holds (n + 1 values); 0 for the
// other shapes, which evaluate the multiplier inside their fused pass.
size_t multiplier_table_bytes(int ndim, const int64_t* dims, int precision) {
    const size_t celem = precision == STENCIL_FP32 ? sizeof(float2) : sizeof(double2);
    if (ndim == 3) return periodic_workspace_bytes(ndim, dims, precision);
    if (ndim == 2 && precision == STENCIL_FP32 && blocked_shape(ndim, dims)) {
        // the blocked table (or, for implicit plans, the row-major one)
        const int n_log2 = ilog2_exact(dims[1]) - 1;
        const size_t blk = (size_t)blocked_item_elems(ilog2_exact(dims[0]), n_log2) * celem;
        return std::max(blk, periodic_workspace_bytes(ndim, dims, precision));
    }
    if (ndim == 1) {
        const int64_t n = dims[0] / 2;
        const int64_t cap = 16 * (precision == STENCIL_FP32 ? kMaxThreadsF32 : kMaxThreadsF64);
        if (n >= 16 && n <= cap) return (size_t)(n + 1) * celem;
    }
    return 0;
}

size_t periodic_workspace_bytes(int ndim, const int64_t* dims, int precision) {
    if (ndim == 1) return 0;
    const size_t celem = precision == STENCIL_FP32 ? sizeof(float2) : sizeof(double2);
    const int64_t n = dims[ndim - 1] / 2;
    const int64_t align = precision == STENCIL_FP32 ? 16 : 8;
    const int64_t Mp = (n + 1 + align - 1) / align * align;
    int64_t rows = 1;
    for (int a = 0; a < ndim - 1; ++a) rows *= dims[a];
    return (size_t)rows * (size_t)Mp * celem;
}

// Periodic solve of `grid` (shape len, the plan's weights) in place, with
// workspace H (row stride Mp). Used for the whole-grid solve of periodic
// plans and, in aperiodic.cu, for the interior solve.
#define PROF_LAUNCH(kind, call)          \
    do {                                 \
        p->prof.begin(kind, s);          \
        err = (call);                    \
        p->prof.end(s);                  \
        if (err != cudaSuccess) return err; \
    } while (0)

// Periodic solve of `items` boxes of shape len stacked contiguously in S (in
// place), with their half spectra stacked in H (row stride Mp). Item i is a
// grid region in orientation perms[orient[i]] (box axis a = grid axis
// perms[..][a]); all items share one launch per pass.
template <typename R>
cudaError_t batched_solve(stencil_plan_s* p, R* S, const int64_t* len, int items, int64_t T,
                          void* H, long long Mp, const int* orient, const int (*perms)[3],
                          int norient, const void* tw, int twn_log2, const double2* const* E64,
                          const float2* const* E32, int* status, cudaStream_t s,
                          const void* const* vtabs, const void* const* vitems, R* Sout) {
    const int d = p->ndim;
    if (items < 1 || items > kMaxItems || norient < 1 || norient > kMaxOrient)
        return cudaErrorInvalidValue;
    const PassVariantScope variant(p->pass_variant);
    SymbolSet ss;
    std::memset(&ss, 0, sizeof(ss));
    for (int o = 0; o < norient; ++o)
        ss.p[o] = make_symbol_params(p, len, T, E64, E32, perms ? perms[o] : nullptr);
    for (int i = 0; i < items; ++i) ss.orient[i] = orient ? orient[i] : 0;
    for (int o = 0; o < norient; ++o) ss.vtab[o] = vtabs ? vtabs[o] : nullptr;
    // a blocked-layout table serves only the blocked passes (set below)
    const bool blocked_table = vtabs && vtabs[0] && vtabs[0] == p->vt && p->vflags && !p->implicit;
    if (blocked_table) ss.vtab[0] = nullptr;
    for (int i = 0; i < items; ++i) ss.vtab_item[i] = vitems ? vitems[i] : nullptr;
    const int maxt = sizeof(R) == 4 ? kMaxThreadsF32 : kMaxThreadsF64;
    const int celem = 2 * sizeof(R);
    const int n_log2 = ilog2_exact(len[d - 1]) - 1;
    const int n = 1 << n_log2;
    cudaError_t err;
    if (d == 1) {
        // every item of a 1-D batch has the one orientation
        // n1 x n2 passes when one CTA cannot hold the row, and for a single FP64
        // row of >= 512 points: one CTA would leave every other SM's FP64 units
        // idle (4096-point FP64 heat solve 0.155 ms in one CTA)
        const bool spread = items == 1 && sizeof(R) == 8 && n_log2 >= 9 && !vitems && !p->implicit;
        if (n > 16 * (sizeof(R) == 4 ? kMaxThreadsF32 : kMaxThreadsF64) || spread) {
            // n = n1 x n2 passes; Lambda^T per element
            if (vitems) return cudaErrorInvalidValue;
            const int n2_log2 = std::min(11, (n_log2 + 1) / 2);   // two rows per 256-thread CTA
            PROF_LAUNCH(PASS_FUSED_1D,
                        launch_fused_1d_pairs<R>(S, n_log2 - n2_log2, n2_log2, items, tw, twn_log2,
                                                 ss.p[0], status, s));
            return cudaSuccess;
        }
        RowTables rt;
        for (int i = 0; i < kMaxItems; ++i)
            rt.t[i] = ss.vtab_item[i] ? ss.vtab_item[i] : (i < items ? ss.vtab[0] : nullptr);
        const bool tables = vitems || (vtabs && vtabs[0] && items <= kMaxItems && n >= 16);
        PROF_LAUNCH(PASS_FUSED_1D, launch_fused_1d<R>(S, n_log2, items, tw, twn_log2, ss.p[0],
                                                      status, s, tables ? &rt : nullptr));
        return cudaSuccess;
    }
    const int64_t rows_item = d == 2 ? len[0] : len[0] * len[1];
    const int64_t rows = rows_item * items;
    R* out = Sout ? Sout : S;
    if (d == 2 && sizeof(R) == 4 && p->gemm < 0) {
        // FP32 2-D: half spectra in column blocks (rows_blk.cuh), so the fused
        // column pass moves one contiguous 64 KB block per tile
        const int l0_log2 = ilog2_exact(len[0]);
        if (blocked_ok(S, H, l0_log2, n_log2) && blocked_ok(out, H, l0_log2, n_log2)) {
            ColGeom g;
            g.log2n = l0_log2;
            g.S = 1ll << (13 - l0_log2);   // columns per block: rows are that far apart
            g.outer = items;
            g.os = blocked_item_elems(l0_log2, n_log2);
            g.mid = 1;
            g.ms = 0;
            g.inner_valid = n + 1;
            g.cols_log2 = 13 - l0_log2;
            g.vS = Mp;
            if (blocked_table && items == 1) {
                ss.vtab[0] = vtabs[0];
                ss.vflags = p->vflags;
            }
            PROF_LAUNCH(PASS_ROWS_R2C, launch_rows_blk(-1, S, H, l0_log2, n_log2, (int)rows, tw,
                                                       twn_log2, status, s));
            PROF_LAUNCH(PASS_COLS_FUSED, launch_cols_tma_blk(H, g, tw, twn_log2, ss, status, s));
            PROF_LAUNCH(PASS_ROWS_C2R, launch_rows_blk(+1, H, out, l0_log2, n_log2, (int)rows, tw,
                                                       twn_log2, status, s));
            return cudaSuccess;
        }
    }
    // R2C keeps the register row kernel: its bulk-copy variant measured slower
    // on GB300 (4096^2: 44 -> 48 us; 512^3: 194 -> 228 us)
    PROF_LAUNCH(PASS_ROWS_R2C, launch_rows_r2c<R>(S, H, Mp, n_log2, (int)rows, tw, twn_log2, s));
    if (d == 2) {
        ColGeom g;
        g.log2n = ilog2_exact(len[0]);
        g.S = Mp;
        g.outer = items;
        g.os = len[0] * Mp;
        g.mid = 1;
        g.ms = 0;
        g.inner_valid = n + 1;
        g.cols_log2 = cols_log2_for(g.log2n, celem, maxt);
        if (sizeof(R) == 4 && p->gemm >= 0)
            PROF_LAUNCH(PASS_COLS_FUSED,
                        launch_cols_fused_gemm(H, g, tw, twn_log2, ss, p->gemm, status, s));
        else if (sizeof(R) == 4 && cols_tma_ok(H, g))
            PROF_LAUNCH(PASS_COLS_FUSED, launch_cols_tma(H, g, 0, tw, twn_log2, &ss, status, s));
        else
            PROF_LAUNCH(PASS_COLS_FUSED, launch_cols_fused<R>(H, g, tw, twn_log2, ss, s));
    } else {
        ColGeom g1;
        g1.log2n = ilog2_exact(len[1]);
        g1.S = Mp;
        g1.outer = (int)(len[0] * items);
        g1.os = len[1] * Mp;
        g1.mid = 1;
        g1.ms = 0;
        g1.inner_valid = n + 1;
        g1.cols_log2 = cols_log2_for(g1.log2n, celem, maxt);
        const bool gemm = sizeof(R) == 4 && p->gemm >= 0;
        const bool tma1 = sizeof(R) == 4 && !gemm && cols_tma_ok(H, g1);
        if (gemm)
            PROF_LAUNCH(PASS_COLS_FWD,
                        launch_cols_gemm(H, g1, -1, tw, twn_log2, p->gemm, status, s));
        else if (tma1)
            PROF_LAUNCH(PASS_COLS_FWD,
                        launch_cols_tma(H, g1, -1, tw, twn_log2, nullptr, status, s));
        else
            PROF_LAUNCH(PASS_COLS_FWD, launch_cols<R>(H, g1, -1, tw, twn_log2, s));
        ColGeom g0;
        g0.log2n = ilog2_exact(len[0]);
        g0.S = len[1] * Mp;
        g0.outer = items;
        g0.os = len[0] * len[1] * Mp;
        g0.mid = (int)len[1];
        g0.ms = Mp;
        g0.inner_valid = n + 1;
        g0.cols_log2 = cols_log2_for(g0.log2n, celem, maxt);
        if (gemm) {
            PROF_LAUNCH(PASS_COLS_FUSED,
                        launch_cols_fused_gemm(H, g0, tw, twn_log2, ss, p->gemm, status, s));
            PROF_LAUNCH(PASS_COLS_INV,
                        launch_cols_gemm(H, g1, +1, tw, twn_log2, p->gemm, status, s));
        } else {
            if (sizeof(R) == 4 && cols_tma_ok(H, g0))
                PROF_LAUNCH(PASS_COLS_FUSED,
                            launch_cols_tma(H, g0, 0, tw, twn_log2, &ss, status, s));
            else
                PROF_LAUNCH(PASS_COLS_FUSED, launch_cols_fused<R>(H, g0, tw, twn_log2, ss, s));
            if (tma1)
                PROF_LAUNCH(PASS_COLS_INV,
                            launch_cols_tma(H, g1, +1, tw, twn_log2, nullptr, status, s));
            else
                PROF_LAUNCH(PASS_COLS_INV, launch_cols<R>(H, g1, +1, tw, twn_log2, s));
        }
    }
    // d >= 2 reads S once (R2C) and writes the result once (C2R): Sout may be a
    // different buffer, e.g. host memory the GPU maps over the chip-to-chip link
    // C2R reads H through bulk copies (512^3: 231 -> 189 us; 4096^2: equal)
    if (sizeof(R) == 4 && rows_tma_ok(out, H, Mp, n_log2, (int)rows))
        PROF_LAUNCH(PASS_ROWS_C2R, launch_rows_tma(+1, H, out, Mp, n_log2, (int)rows, tw, twn_log2,
                                                   status, s));
    else
        PROF_LAUNCH(PASS_ROWS_C2R, launch_rows_c2r<R>(H, out, Mp, n_log2, (int)rows, tw, twn_log2,
                                                      status, s));
    return cudaSuccess;
}

template <typename R>
cudaError_t periodic_solve(stencil_plan_s* p, R* grid, const int64_t* len, int64_t T,
                           void* H, long long Mp, const void* tw, int twn_log2,
                           const double2* const* E64, const float2* const* E32, int* status,
                           cudaStream_t s) {
    return batched_solve<R>(p, grid, len, 1, T, H, Mp, nullptr, nullptr, 1, tw, twn_log2, E64, E32,
                            status, s, nullptr, nullptr);
}

#define SFFT_SOLVE_INST(R)                                                                         \
    template cudaError_t periodic_solve<R>(stencil_plan_s*, R*, const int64_t*, int64_t, void*,    \
                                           long long, const void*, int, const double2* const*,     \
                                           const float2* const*, int*, cudaStream_t);              \
    template cudaError_t batched_solve<R>(stencil_plan_s*, R*, const int64_t*, int, int64_t,       \
                                          void*, long long, const int*, const int (*)[3], int,     \
                                          const void*, int, const double2* const*,                 \
                                          const float2* const*, int*, cudaStream_t,                \
                                          const void* const*, const void* const*, R*);
SFFT_SOLVE_INST(float)
SFFT_SOLVE_INST(double)

}  // namespace sfft

namespace sfft {
// The CUDA error behind the calling thread's last STENCIL_ECUDA / ENOMEM.
static thread_local cudaError_t t_last_cuda_error = cudaSuccess;
void note_cuda_error(cudaError_t err) {
    if (err != cudaSuccess) t_last_cuda_error = err;
}
}  // namespace sfft

static int from_cuda(cudaError_t err) {
    if (err == cudaSuccess) return STENCIL_OK;
    note_cuda_error(err);
    if (err == cudaErrorMemoryAllocation) return STENCIL_ENOMEM;
    return STENCIL_ECUDA;
}

extern "C" const char* stencil_cuda_error_name(void) { return cudaGetErrorName(t_last_cuda_error); }

static void free_plan(stencil_plan_s* p) {
    if (!p) return;
    cudaFree(p->tw);
    for (int a = 0; a < 3; ++a) {
        cudaFree(p->E64[a]);
        cudaFree(p->E32[a]);
    }
    cudaFree(p->H);
    cudaFree(p->status);
    cudaFree(p->dev_grid);
    cudaFree(p->vt);
    cudaFree(p->vflags);
    cudaFree(p->wq_dev);
    cudaFree(p->wv_dev);
    for (int a = 0; a < 3; ++a) cudaFree(p->mtw[a]);
    aperiodic_release(p);
    delete p;
}

extern "C" {

const char* stencil_strerror(int code) {
    switch (code) {
        case STENCIL_OK: return "ok";
        case STENCIL_EINVAL: return "invalid argument";
        case STENCIL_ENOMEM: return "out of memory";
        case STENCIL_ECUDA: return "CUDA runtime error";
        case STENCIL_ETIMEOUT: return "bounded device wait timed out";
        case STENCIL_ENONFINITE: return "non-finite value in the result";
        case STENCIL_EQUEUEFULL: return "server queue full";
        case STENCIL_EUNSUPPORTED: return "unsupported size or option";
        default: return "unknown status code";
    }
}

static bool is_gemm(int precision) {
    return precision >= STENCIL_FP32_GEMM_BF16 && precision <= STENCIL_FP32_GEMM_BF16X3;
}
// Arithmetic of the grid and of the CUDA-core passes.
static int base_precision(int precision) { return is_gemm(precision) ? STENCIL_FP32 : precision; }

int64_t stencil_max_axis(int ndim, int precision, int axis) {
    if (precision < STENCIL_FP64 || precision > STENCIL_FP32_GEMM_BF16X3) return 0;
    if (is_gemm(precision)) {
        if (ndim < 2 || ndim > 3 || axis < 0 || axis >= ndim) return 0;
        if (axis < ndim - 1) return 4096;
    }
    return max_axis(ndim, base_precision(precision), axis);
}

static int validate(int ndim, const int64_t* dims, int radius, int boundary, int precision) {
    if (ndim < 1 || ndim > 3 || !dims || radius < 0 || radius > kMaxRadius) return STENCIL_EINVAL;
    if (boundary != STENCIL_PERIODIC && boundary != STENCIL_ZERO_DIRICHLET &&
        boundary != STENCIL_NEUMANN)
        return STENCIL_EINVAL;
    if (precision < STENCIL_FP64 || precision > STENCIL_FP32_GEMM_BF16X3) return STENCIL_EINVAL;
    for (int a = 0; a < ndim; ++a) {
        if (dims[a] < 2 * radius + 1 || dims[a] < 4) return STENCIL_EINVAL;
        if (ilog2_exact(dims[a]) < 0) {
            // mixed-radix axes: periodic FP32 / FP64 plans, prime factors 2, 3, 5,
            // 7, an even last axis (real rows of L are n = L/2 complex values)
            if (boundary != STENCIL_PERIODIC || is_gemm(precision)) return STENCIL_EUNSUPPORTED;
            const bool last = a == ndim - 1;
            if (last && (dims[a] % 2)) return STENCIL_EUNSUPPORTED;
            if (!mixed_length_ok(last ? dims[a] / 2 : dims[a], precision)) return STENCIL_EUNSUPPORTED;
            continue;
        }
        if (dims[a] > max_axis(ndim, base_precision(precision), a)) return STENCIL_EUNSUPPORTED;
    }
    if (is_gemm(precision)) {
        // tensor-core DFTs: periodic, strided axes of 256..4096
        if (boundary != STENCIL_PERIODIC || ndim < 2) return STENCIL_EUNSUPPORTED;
        for (int a = 0; a < ndim - 1; ++a)
            if (!gemm_axis_ok(ilog2_exact(dims[a]))) return STENCIL_EUNSUPPORTED;
    }
    return STENCIL_OK;
}

size_t stencil_workspace_bytes(int ndim, const int64_t* dims, int radius, int boundary,
                               int precision) {
    if (validate(ndim, dims, radius, boundary, precision) != STENCIL_OK) return 0;
    const int bp = base_precision(precision);
    bool mixed = false;
    for (int a = 0; a < ndim; ++a) mixed |= ilog2_exact(dims[a]) < 0;
    if (mixed) {   // the half spectrum only (1-D: one row), no multiplier table
        const int64_t n = dims[ndim - 1] / 2;
        const int64_t align = bp == STENCIL_FP32 ? 16 : 8;
        int64_t rows = 1;
        for (int a = 0; a < ndim - 1; ++a) rows *= dims[a];
        return (size_t)rows * ((n + 1 + align - 1) / align * align) * (bp == STENCIL_FP32 ? 8 : 16);
    }
    size_t bytes = periodic_workspace_bytes(ndim, dims, bp);
    if (boundary == STENCIL_PERIODIC) bytes += multiplier_table_bytes(ndim, dims, bp);
    return bytes;
}

int tuned_variant(const stencil_plan_s* p);

int stencil_plan(stencil_plan_t* out, int ndim, const int64_t* dims, int radius,
                 const double* weights, int boundary, int precision) {
    if (!out || !weights) return STENCIL_EINVAL;
    *out = nullptr;
    int rc = validate(ndim, dims, radius, boundary, precision);
    if (rc != STENCIL_OK) return rc;
    stencil_plan_s* p = new (std::nothrow) stencil_plan_s();
    if (!p) return STENCIL_ENOMEM;
    if (is_gemm(precision)) p->gemm = precision - STENCIL_FP32_GEMM_BF16;   // kGemm* order
    precision = base_precision(precision);
    p->ndim = ndim;
    p->radius = radius;
    p->boundary = boundary;
    p->precision = precision;
    p->nweights = 1;
    for (int a = 0; a < ndim; ++a) {
        p->dims[a] = dims[a];
        p->nweights *= 2 * radius + 1;
    }
    for (int i = 0; i < p->nweights; ++i) {
        if (!std::isfinite(weights[i])) {
            delete p;
            return STENCIL_EINVAL;
        }
        p->weights[i] = weights[i];
    }
    p->real_symbol = symmetric_weights(p->weights, ndim, radius);
    face_reach(p->weights, ndim, radius, p->reach);
    p->elem = precision == STENCIL_FP32 ? sizeof(float) : sizeof(double);
    p->n_cells = 1;
    for (int a = 0; a < ndim; ++a) p->n_cells *= dims[a];
    cudaGetDevice(&p->device);
    cudaError_t err = alloc_tables(p);
    if (err == cudaSuccess) {
        p->H_bytes = periodic_workspace_bytes(ndim, dims, precision);
        const int64_t n = dims[ndim - 1] / 2;
        const int64_t align = precision == STENCIL_FP32 ? 16 : 8;
        p->Mp = (n + 1 + align - 1) / align * align;
        if (p->H_bytes) {
            err = cudaMalloc(&p->H, p->H_bytes);
            if (err == cudaSuccess) err = cudaMemsetAsync(p->H, 0, p->H_bytes, cudaStreamPerThread);
            p->dev_bytes += p->H_bytes;
        }
    }
    // storage for the repeated-T multiplier table (built by a run that repeats
    // the previous T, or by stencil_prepare); without room the passes evaluate
    if (err == cudaSuccess && boundary == STENCIL_PERIODIC) {
        const size_t vbytes = multiplier_table_bytes(ndim, dims, precision);
        if (vbytes) {
            if (cudaMalloc(&p->vt, vbytes) == cudaSuccess) {
                p->dev_bytes += vbytes;
            } else {
                p->vt = nullptr;
                cudaGetLastError();
            }
        }
        if (p->vt && ndim == 2 && precision == STENCIL_FP32 && p->gemm < 0 &&
            blocked_shape(ndim, dims)) {
            const size_t fb = (size_t)(blocked_item_elems(ilog2_exact(dims[0]),
                                                          ilog2_exact(dims[1]) - 1) >> 13) * sizeof(int);
            if (cudaMalloc(&p->vflags, fb) == cudaSuccess) {
                p->dev_bytes += fb;
            } else {
                p->vflags = nullptr;
                cudaGetLastError();
            }
        }
    }
    if (err == cudaSuccess && p->mixed) {
        // a mixed-radix axis: the plan runs the vector path with one field
        // (mixed-radix passes around the multiply of vector.cu)
        if (p->vt) {
            cudaFree(p->vt);
            p->vt = nullptr;
            p->dev_bytes -= multiplier_table_bytes(ndim, dims, precision);
        }
        p->vector = true;
        p->nfields = 1;
        if (!p->H) {   // 1-D: one row of n + 1 values
            p->H_bytes = (size_t)p->Mp * 2 * p->elem;
            err = cudaMalloc(&p->H, p->H_bytes);
            if (err == cudaSuccess) p->dev_bytes += p->H_bytes;
        }
        double wsum = 0.0;
        for (int i = 0; i < p->nweights; ++i) wsum += std::fabs(p->weights[i]);
        p->vdelta[0] = (float)(wsum * std::ldexp(1.0, -16)) + 1e-30f;
        if (err == cudaSuccess) err = cudaMalloc(&p->wv_dev, p->nweights * sizeof(double));
        if (err == cudaSuccess) {
            p->dev_bytes += p->nweights * sizeof(double);
            err = cudaMemcpy(p->wv_dev, p->weights, p->nweights * sizeof(double),
                             cudaMemcpyHostToDevice);
        }
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(cudaStreamPerThread);
    if (err != cudaSuccess) {
        free_plan(p);
        return from_cuda(err);
    }
    if (boundary == STENCIL_PERIODIC) p->pass_variant = tuned_variant(p);
    *out = p;
    return STENCIL_OK;
}

int stencil_plan_implicit(stencil_plan_t* out, int ndim, const int64_t* dims, int radius,
                          const double* weights_s, const double* weights_q, int precision) {
    if (!out || !weights_s || !weights_q) return STENCIL_EINVAL;
    *out = nullptr;
    int rc = validate(ndim, dims, radius, STENCIL_PERIODIC, precision);
    if (rc != STENCIL_OK) return rc;
    if (precision != STENCIL_FP64 && precision != STENCIL_FP32) return STENCIL_EUNSUPPORTED;
    for (int a = 0; a < ndim; ++a)
        if (ilog2_exact(dims[a]) < 0) return STENCIL_EUNSUPPORTED;   // power-of-two axes only
    int nw = 1;
    for (int a = 0; a < ndim; ++a) nw *= 2 * radius + 1;
    for (int i = 0; i < nw; ++i)
        if (!std::isfinite(weights_q[i])) return STENCIL_EINVAL;
    // every pass must read the multiplier table: a 1-D axis longer than one
    // CTA holds (its n1 x n2 passes evaluate in-pass) or shorter than 32 points
    if (multiplier_table_bytes(ndim, dims, precision) == 0 && ndim == 1) return STENCIL_EUNSUPPORTED;
    rc = stencil_plan(out, ndim, dims, radius, weights_s, STENCIL_PERIODIC, precision);
    if (rc != STENCIL_OK) return rc;
    stencil_plan_s* p = *out;
    p->implicit = true;
    for (int i = 0; i < nw; ++i) p->weights_q[i] = weights_q[i];
    p->real_symbol = symmetric_weights(p->weights, ndim, radius) &&
                     symmetric_weights(p->weights_q, ndim, radius);
    cudaError_t err = cudaMalloc(&p->wq_dev, nw * sizeof(double));
    if (err == cudaSuccess) {
        p->dev_bytes += nw * sizeof(double);
        err = cudaMemcpy(p->wq_dev, p->weights_q, nw * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (err == cudaSuccess && !p->vt) {
        // 2-D plans keep no table for explicit stencils: implicit ones need it
        const size_t vbytes = periodic_workspace_bytes(ndim, dims, precision);
        err = cudaMalloc(&p->vt, vbytes);
        if (err == cudaSuccess) p->dev_bytes += vbytes;
        else p->vt = nullptr;
    }
    if (err != cudaSuccess) {
        free_plan(p);
        *out = nullptr;
        return from_cuda(err);
    }
    return STENCIL_OK;
}

int stencil_plan_vector(stencil_plan_t* out, int ndim, const int64_t* dims, int radius,
                        int nfields, const double* weights, int precision) {
    if (!out || !weights) return STENCIL_EINVAL;
    *out = nullptr;
    if (nfields < 1 || nfields > vector_max_fields()) return STENCIL_EINVAL;
    int rc = validate(ndim, dims, radius, STENCIL_PERIODIC, precision);
    if (rc != STENCIL_OK) return rc;
    if (precision != STENCIL_FP64 && precision != STENCIL_FP32) return STENCIL_EUNSUPPORTED;
    int nw = 1;
    for (int a = 0; a < ndim; ++a) nw *= 2 * radius + 1;
    const int total = nfields * nfields * nw;
    for (int i = 0; i < total; ++i)
        if (!std::isfinite(weights[i])) return STENCIL_EINVAL;
    rc = stencil_plan(out, ndim, dims, radius, weights, STENCIL_PERIODIC, precision);
    if (rc != STENCIL_OK) return rc;
    stencil_plan_s* p = *out;
    p->vector = true;
    p->nfields = nfields;
    for (int b = 0; b < nfields * nfields; ++b) {
        double sum = 0.0;
        for (int i = 0; i < nw; ++i) sum += std::fabs(weights[(size_t)b * nw + i]);
        p->vdelta[b] = (float)(sum * std::ldexp(1.0, -16)) + 1e-30f;
    }
    // one half spectrum per field (1-D plans keep none of their own); the
    // scalar multiplier table is never used
    cudaFree(p->H);
    p->dev_bytes -= p->H_bytes;
    p->H = nullptr;
    cudaFree(p->vt);
    p->vt = nullptr;
    int64_t rows = 1;
    for (int a = 0; a < ndim - 1; ++a) rows *= dims[a];
    p->H_bytes = (size_t)nfields * rows * p->Mp * 2 * p->elem;
    if (p->wv_dev) {   // set up by stencil_plan for a mixed-radix grid
        cudaFree(p->wv_dev);
        p->dev_bytes -= p->nweights * sizeof(double);
        p->wv_dev = nullptr;
    }
    cudaError_t err = cudaMalloc(&p->H, p->H_bytes);
    if (err == cudaSuccess) {
        p->dev_bytes += p->H_bytes;
        err = cudaMalloc(&p->wv_dev, total * sizeof(double));
    }
    if (err == cudaSuccess) {
        p->dev_bytes += total * sizeof(double);
        err = cudaMemcpy(p->wv_dev, weights, total * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (err != cudaSuccess) {
        free_plan(p);
        *out = nullptr;
        return from_cuda(err);
    }
    return STENCIL_OK;
}

static cudaError_t periodic_table(stencil_plan_s* p, int64_t T, cudaStream_t s, const void** out);

int stencil_run(stencil_plan_t p, void* grid, int64_t T, void* stream) {
    if (!p || !grid || T < 0) return STENCIL_EINVAL;
    if (reinterpret_cast<uintptr_t>(grid) % 16) return STENCIL_EINVAL;
    if (T == 0) return STENCIL_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (p->boundary != STENCIL_PERIODIC) return aperiodic_run(p, grid, T, s);
    if (p->vector) return from_cuda(vector_run(p, grid, T, s));
    cudaError_t err;
    const void* vtab = nullptr;
    err = periodic_table(p, T, s, &vtab);
    if (err != cudaSuccess) return from_cuda(err);
    if (p->precision == STENCIL_FP32)
        err = batched_solve<float>(p, static_cast<float*>(grid), p->dims, 1, T, p->H, p->Mp,
                                   nullptr, nullptr, 1, p->tw, p->twn_log2, p->E64, p->E32,
                                   p->status, s, vtab ? &vtab : nullptr);
    else
        err = batched_solve<double>(p, static_cast<double*>(grid), p->dims, 1, T, p->H, p->Mp,
                                    nullptr, nullptr, 1, p->tw, p->twn_log2, p->E64, p->E32,
                                    p->status, s, vtab ? &vtab : nullptr);
    return from_cuda(err);
}

// The multiplier table of a periodic 3-D or one-CTA 1-D plan (paper Sec. 4
// "Step 2": the symbol power is computed once per T and reused): a run
// evaluates Lambda^T inside its fused pass, unless the previous run had the
// same T (or stencil_prepare asked for it) -- then the table is built across
// the whole GPU (FP64 powers, stored at pass precision) into storage the plan
// allocated at creation, and kept for T. Measured on GB300: the 3-D fused pass
// gains (512^3 solve 1.75 -> 1.32 ms; its per-column symbol set-up is the
// costly part), and so does a 1-D axis solved by one CTA, which otherwise
// evaluates every FP64 power itself; the 2-D pass loses (the table's extra
// read outweighs the arithmetic it saves), so 2-D evaluates.
static cudaError_t build_table(stencil_plan_s* p, int64_t T, cudaStream_t s) {
    const SymbolParams sp = make_symbol_params(p, p->dims, T, p->E64, p->E32, nullptr);
    cudaError_t err;
    if (p->vflags && !p->implicit)   // FP32 2-D: blocked layout, one flag per column block
        err = launch_vtable_blk(p->vt, p->vflags, sp, ilog2_exact(p->dims[0]),
                                ilog2_exact(p->dims[1]) - 1, s);
    else
        err = p->precision == STENCIL_FP32 ? launch_vtable<float>(p->vt, sp, p->Mp, s)
                                           : launch_vtable<double>(p->vt, sp, p->Mp, s);
    if (err == cudaSuccess) p->vt_T = T;
    return err;
}

static cudaError_t periodic_table(stencil_plan_s* p, int64_t T, cudaStream_t s, const void** out) {
    *out = nullptr;
    if (!p->vt) return cudaSuccess;   // shape without a table, or no room for it
    if (p->vt_T == T) {
        *out = p->vt;
        return cudaSuccess;
    }
    const bool repeat = p->last_T == T;
    p->last_T = T;
    if (!repeat && !p->implicit) return cudaSuccess;   // implicit plans always read the table
    cudaError_t err = build_table(p, T, s);
    if (err != cudaSuccess) return err;
    *out = p->vt;
    return cudaSuccess;
}

// Device addresses of two host buffers that the GPU can access in place
// (page-locked, mapped: on a Grace-Blackwell node the GPU reads and writes them
// over the coherent chip-to-chip link), or false.
static bool mapped_host(const void* a, const void* b, void** da, void** db) {
    if (cudaHostGetDevicePointer(da, const_cast<void*>(a), 0) != cudaSuccess ||
        cudaHostGetDevicePointer(db, const_cast<void*>(b), 0) != cudaSuccess) {
        cudaGetLastError();   // a pageable buffer: clear the error, take the copy path
        return false;
    }
    return reinterpret_cast<uintptr_t>(*da) % 16 == 0 && reinterpret_cast<uintptr_t>(*db) % 16 == 0;
}

int stencil_run_host(stencil_plan_t p, const void* host_in, void* host_out, int64_t T,
                     void* stream) {
    if (!p || !host_in || !host_out || T < 0) return STENCIL_EINVAL;
    if (p->vector) return STENCIL_EUNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)p->n_cells * p->elem;
    cudaError_t err;
    void* din = nullptr;
    void* dout = nullptr;
    if (p->boundary == STENCIL_PERIODIC && p->ndim >= 2 && T > 0 &&
        mapped_host(host_in, host_out, &din, &dout)) {
        // the R2C pass reads the input from host memory, the C2R pass writes the
        // result there: no staging copy of either
        const void* vtab = nullptr;
        err = periodic_table(p, T, s, &vtab);
        if (err != cudaSuccess) return from_cuda(err);
        const void* const* vt = vtab ? &vtab : nullptr;
        if (p->precision == STENCIL_FP32)
            err = batched_solve<float>(p, static_cast<float*>(din), p->dims, 1, T, p->H, p->Mp,
                                       nullptr, nullptr, 1, p->tw, p->twn_log2, p->E64, p->E32,
                                       p->status, s, vt, nullptr, static_cast<float*>(dout));
        else
            err = batched_solve<double>(p, static_cast<double*>(din), p->dims, 1, T, p->H, p->Mp,
                                        nullptr, nullptr, 1, p->tw, p->twn_log2, p->E64, p->E32,
                                        p->status, s, vt, nullptr, static_cast<double*>(dout));
        if (err != cudaSuccess) return from_cuda(err);
        return from_cuda(cudaStreamSynchronize(s));
    }
    if (!p->dev_grid) {
        err = cudaMalloc(&p->dev_grid, bytes);
        if (err != cudaSuccess) {
            p->dev_grid = nullptr;
            return from_cuda(err);
        }
        p->dev_bytes += bytes;
    }
    err = cudaMemcpyAsync(p->dev_grid, host_in, bytes, cudaMemcpyHostToDevice, s);
    if (err != cudaSuccess) return from_cuda(err);
    int rc = stencil_run(p, p->dev_grid, T, stream);
    if (rc != STENCIL_OK) return rc;
    err = cudaMemcpyAsync(host_out, p->dev_grid, bytes, cudaMemcpyDeviceToHost, s);
    if (err != cudaSuccess) return from_cuda(err);
    return from_cuda(cudaStreamSynchronize(s));
}

int stencil_prepare(stencil_plan_t p, int64_t T, void* stream) {
    if (!p || T < 0) return STENCIL_EINVAL;
    if (T == 0) return STENCIL_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (p->boundary != STENCIL_PERIODIC) return aperiodic_prepare(p, T);
    if (!p->vt || p->vt_T == T) return STENCIL_OK;
    p->last_T = T;
    return from_cuda(build_table(p, T, s));
}

int stencil_symbol_power(stencil_plan_t p, int64_t T, void* out, void* stream) {
    if (!p || !out || T < 0) return STENCIL_EINVAL;
    if (p->vector && p->nfields > 1) return STENCIL_EUNSUPPORTED;
    const SymbolParams sp = make_symbol_params(p, p->dims, T, p->E64, p->E32, nullptr);
    const int nlast_half = (int)(p->dims[p->ndim - 1] / 2 + 1);
    long long total = nlast_half;
    for (int a = 0; a < p->ndim - 1; ++a) total *= p->dims[a];
    return from_cuda(launch_symbol_table(static_cast<double2*>(out), sp, nlast_half, total,
                                         static_cast<cudaStream_t>(stream)));
}

int stencil_status(stencil_plan_t p, void* stream) {
    if (!p) return STENCIL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return from_cuda(err);
    int flag = 0;
    err = cudaMemcpyAsync(&flag, p->status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return from_cuda(err);
    if (flag) {
        err = cudaMemsetAsync(p->status, 0, sizeof(int), s);
        if (err == cudaSuccess) err = cudaStreamSynchronize(s);
        if (err != cudaSuccess) return from_cuda(err);
        return (flag & 4) ? STENCIL_ETIMEOUT : STENCIL_ENONFINITE;
    }
    return STENCIL_OK;
}

int stencil_destroy(stencil_plan_t p) {
    if (!p) return STENCIL_EINVAL;
    cudaDeviceSynchronize();
    free_plan(p);
    return STENCIL_OK;
}

}  // extern "C"

namespace sfft {
// Frees a plan that has no work in flight (its last use has completed), without
// waiting for the rest of the device.
void plan_free_idle(stencil_plan_s* p) { free_plan(p); }
}  // namespace sfft

extern "C" {

}  // extern "C"

namespace sfft {
// Replace a plan's weights (same radius bound); captured graphs hold the old
// weights in their kernel parameters and are dropped.
// Weight (m_0 + r, .., m_{d-1} + r) (row-major, axis 0 slowest) multiplies
// a_t[i + m]: the face below index 0 of axis a is looked towards by -m_a, the
// face above the last index by +m_a.
void face_reach(const double* w, int ndim, int radius, int reach[3][2]) {
    const int W = 2 * radius + 1;
    int n = 1;
    for (int a = 0; a < ndim; ++a) n *= W;
    for (int a = 0; a < 3; ++a) reach[a][0] = reach[a][1] = 0;
    for (int i = 0; i < n; ++i) {
        if (w[i] == 0.0) continue;
        int rest = i;
        for (int a = ndim - 1; a >= 0; --a) {
            const int m = rest % W - radius;
            rest /= W;
            reach[a][0] = std::max(reach[a][0], -m);
            reach[a][1] = std::max(reach[a][1], m);
        }
    }
}

void plan_set_weights(stencil_plan_s* p, int radius, const double* w) {
    p->radius = radius;
    p->nweights = 1;
    for (int a = 0; a < p->ndim; ++a) p->nweights *= 2 * radius + 1;
    for (int i = 0; i < p->nweights; ++i) p->weights[i] = w[i];
    p->real_symbol = symmetric_weights(p->weights, p->ndim, radius);
    face_reach(p->weights, p->ndim, radius, p->reach);
    p->vt_T = -1;   // the cached multipliers belong to the old weights
    p->last_T = -1;
    aperiodic_forget_graphs(p);
}
}  // namespace sfft

extern "C" int stencil_plan_set_weights(stencil_plan_t p, int radius, const double* weights) {
    if (!p || !weights || radius < 0 || radius > kMaxRadius) return STENCIL_EINVAL;
    if (p->implicit || p->vector) return STENCIL_EUNSUPPORTED;
    int nw = 1;
    for (int a = 0; a < p->ndim; ++a) {
        if (p->dims[a] < 2 * radius + 1) return STENCIL_EINVAL;
        nw *= 2 * radius + 1;
    }
    for (int i = 0; i < nw; ++i)
        if (!std::isfinite(weights[i])) return STENCIL_EINVAL;
    // the schedule depends on sigma and on the reach towards every face
    int reach[3][2];
    face_reach(weights, p->ndim, radius, reach);
    if (radius != p->radius || std::memcmp(reach, p->reach, sizeof(reach)) != 0)
        aperiodic_forget_schedules(p);
    plan_set_weights(p, radius, weights);
    return STENCIL_OK;
}

extern "C" int stencil_debug_face_reach(int ndim, int radius, const double* weights, int* reach) {
    if (!weights || !reach || ndim < 1 || ndim > 3 || radius < 0 || radius > kMaxRadius)
        return STENCIL_EINVAL;
    int r[3][2];
    face_reach(weights, ndim, radius, r);
    for (int a = 0; a < ndim; ++a) {
        reach[2 * a] = r[a][0];
        reach[2 * a + 1] = r[a][1];
    }
    return STENCIL_OK;
}

extern "C" int stencil_plan_set_cutoff(stencil_plan_t p, int64_t cutoff) {
    if (!p || (cutoff != 0 && cutoff < 2)) return STENCIL_EINVAL;
    if (p->cutoff != cutoff) aperiodic_forget_schedules(p);
    p->cutoff = cutoff;
    return STENCIL_OK;
}

// Size classes tuned in this process: (ndim, dims, precision) -> pass variant;
// new periodic plans of a tuned class start with its choice.
static std::mutex g_tuned_mu;
static std::map<std::vector<int64_t>, int> g_tuned;

static std::vector<int64_t> size_class(const stencil_plan_s* p) {
    return {p->ndim, p->dims[0], p->dims[1], p->dims[2], p->precision, p->gemm};
}

int tuned_variant(const stencil_plan_s* p) {
    std::lock_guard<std::mutex> lock(g_tuned_mu);
    auto it = g_tuned.find(size_class(p));
    return it == g_tuned.end() ? -1 : it->second;
}

// Periodic plans: time every pass variant (PassVariantScope) on a scratch copy
// of grid for T and keep the fastest, for this plan and its size class.
static int periodic_autotune(stencil_plan_s* p, const void* grid, int64_t T, cudaStream_t s,
                             double* ms, int cap) {
    if (p->vector || p->implicit || p->ndim < 2 || p->gemm >= 0) return STENCIL_EUNSUPPORTED;
    const size_t bytes = (size_t)p->n_cells * p->elem;
    void* scratch = nullptr;
    cudaError_t err = cudaMalloc(&scratch, bytes);
    if (err != cudaSuccess) return from_cuda(err);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int keep = p->pass_variant;
    int best = -1;
    double best_ms = 0.0;
    int rc = STENCIL_OK;
    for (int v = 0; v < kPassVariants && rc == STENCIL_OK; ++v) {
        p->pass_variant = v;
        double t = 0.0;
        for (int rep = 0; rep < 6 && rc == STENCIL_OK; ++rep) {
            err = cudaMemcpyAsync(scratch, grid, bytes, cudaMemcpyDeviceToDevice, s);
            if (err != cudaSuccess) rc = from_cuda(err);
            if (rc == STENCIL_OK && rep >= 2) cudaEventRecord(e0, s);
            if (rc == STENCIL_OK) rc = stencil_run(p, scratch, T, s);
            if (rc == STENCIL_OK && rep >= 2) {
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) rc = STENCIL_ECUDA;
                float f = 0.f;
                cudaEventElapsedTime(&f, e0, e1);
                t += f / 4.0;
            }
        }
        if (rc != STENCIL_OK) break;
        if (v < cap) ms[v] = t;
        if (best < 0 || t < best_ms) {
            best = v;
            best_ms = t;
        }
    }
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(scratch);
    if (rc != STENCIL_OK) {
        p->pass_variant = keep;
        return rc;
    }
    p->pass_variant = best;
    {
        std::lock_guard<std::mutex> lock(g_tuned_mu);
        g_tuned[size_class(p)] = best;
    }
    return best;
}

extern "C" int stencil_plan_set_pass_variant(stencil_plan_t p, int variant) {
    if (!p || variant < -1 || variant >= kPassVariants) return STENCIL_EINVAL;
    if (p->boundary != STENCIL_PERIODIC) return STENCIL_EUNSUPPORTED;
    p->pass_variant = variant;
    return STENCIL_OK;
}

extern "C" int stencil_plan_autotune(stencil_plan_t p, const void* grid, int64_t T, void* stream,
                                     double* ms, int cap) {
    if (!p || !grid || T < 1 || cap < 0 || (cap > 0 && !ms)) return STENCIL_EINVAL;
    if (p->boundary == STENCIL_PERIODIC)
        return periodic_autotune(p, grid, T, static_cast<cudaStream_t>(stream), ms, cap);
    return aperiodic_autotune(p, grid, T, static_cast<cudaStream_t>(stream), ms, cap);
}

extern "C" int stencil_plan_set_schedule(stencil_plan_t p, int mode) {
    if (!p || mode < STENCIL_SCHEDULE_AUTO || mode > STENCIL_SCHEDULE_CLUSTER) return STENCIL_EINVAL;
    if (p->schedule != mode) aperiodic_forget_schedules(p);
    p->schedule = mode;
    return STENCIL_OK;
}

static const char* kPassNames[PASS_KINDS] = {
    "rows_r2c", "cols_fwd", "cols_fused", "cols_inv", "rows_c2r", "fused_1d",
    "strip_r2c", "strip_cols", "strip_c2r", "base_loop", "copy", "vtable", "gather", "scatter"};

extern "C" int stencil_profile_enable(stencil_plan_t p, int enable) {
    if (!p) return STENCIL_EINVAL;
    p->prof.enabled = enable != 0;
    return STENCIL_OK;
}

extern "C" int stencil_profile_read(stencil_plan_t p, double* ms, int64_t* launches, int nkinds) {
    if (!p || !ms || !launches || nkinds < 0) return STENCIL_EINVAL;
    cudaError_t err = p->prof.collect();
    for (int k = 0; k < nkinds && k < PASS_KINDS; ++k) {
        ms[k] = p->prof.ms[k];
        launches[k] = p->prof.launches[k];
        p->prof.ms[k] = 0.0;
        p->prof.launches[k] = 0;
    }
    for (int k = PASS_KINDS; k < nkinds; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    return from_cuda(err);
}

extern "C" const char* stencil_profile_kind_name(int kind) {
    if (kind < 0 || kind >= PASS_KINDS) return nullptr;
    return kPassNames[kind];
}
