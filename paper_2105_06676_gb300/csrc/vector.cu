// Vector-valued fields on periodic grids (paper Sec. 4.2 "Vector-Valued
// Fields", appendix "Supporting Vector Valued Fields"): m scalar fields with
// a^(i)_{t+1} = sum_j S^(i,j) a^(j)_t. Every field takes the forward
// Multi-FFT (the scalar plan's passes, batched over the fields); at every
// wave vector k the m x m matrix of symbols Lambda(k), Lambda_ij = symbol of
// S^(i,j), is raised to the power T by repeated squaring in FP64 (the
// appendix: "sequential squaring of a matrix of stencils") and applied to the
// m-vector of spectra; the inverse Multi-FFT returns every field.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>

#include "internal.h"
#include "plan_impl.h"
#include "stencilfft.h"

namespace sfft {

namespace {

constexpr int kMaxFields = 4;

// Half-spectrum geometry of one field: rows of n+1 values (row stride Mp),
// rows = l_0 (2-D) or l_0 l_1 (3-D) or 1 (1-D).
struct VecGeom {
    int ndim;
    int len[3];
    int nh;            // n + 1 values per row
    long long Mp;      // row stride
    long long rows;
    long long item;    // values between fields
    int m;
    const double* w;   // m * m blocks of W^ndim weights (device)
    int nw;            // weights per block
    float cut;         // skip when T log2 ||Lambda||_inf < -cut
    float delta[kMaxFields * kMaxFields];   // bound on |Lambda_ij - its FP32 value|
};

// Lambda_ij at k in FP32 from the block's FP64 weights (the underflow screen).
template <int RAD>
__device__ __forceinline__ float2 block_symbol32(const SymbolParams& p, const double* w, int k0,
                                                 int k1, int k2) {
    constexpr int W = 2 * RAD + 1;
    const int k[3] = {k0, k1, k2};
    float2 e[3][W];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int m = -RAD; m <= RAD; ++m)
            e[a][m + RAD] = a < p.ndim ? __ldg(p.E32[a] + axis_index(p, a, m * k[a])) : float2{1.f, 0.f};
    float2 acc{0.f, 0.f};
    const int W1 = p.ndim >= 2 ? W : 1, W2 = p.ndim >= 3 ? W : 1;
    for (int i = 0; i < W; ++i)
        for (int j = 0; j < W1; ++j)
            for (int q = 0; q < W2; ++q) {
                const float wt = (float)__ldg(w + (i * W1 + j) * W2 + q);
                float2 ph = e[0][i];
                if (p.ndim >= 2) ph = cmul(ph, e[1][j]);
                if (p.ndim >= 3) ph = cmul(ph, e[2][q]);
                acc = cadd(acc, cscale(ph, wt));
            }
    return acc;
}

template <int RAD>
__device__ __forceinline__ double2 block_symbol(const SymbolParams& p, const double* w, int k0,
                                                int k1, int k2) {
    ColSymbol64<RAD> cs;
    col_symbol_init64<RAD>(p, w, k1, k2, cs);
    return col_lambda64<RAD>(p, cs, k0);
}

// y = Lambda(k)^T / N x at every wave vector of the half spectra (in place in H).
template <typename R, int M, int RAD>
__global__ void __launch_bounds__(128)
k_vector_mult(typename CxOf<R>::T* __restrict__ H, const __grid_constant__ VecGeom g,
              const __grid_constant__ SymbolParams p) {
    using C = typename CxOf<R>::T;
    const long long total = g.rows * g.nh;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long row = e / g.nh;
        const int last = (int)(e - row * g.nh);
        int k0, k1 = 0, k2 = 0;
        if (g.ndim == 1) {
            k0 = last;
        } else if (g.ndim == 2) {
            k0 = (int)row;
            k1 = last;
        } else {
            k0 = (int)(row / g.len[1]);
            k1 = (int)(row % g.len[1]);
            k2 = last;
        }
        C* h = H + row * g.Mp + last;
        // screen in FP32: every |V_ij| <= ||Lambda||_inf^T / N, and
        // ||Lambda||_inf <= max_i sum_j (|Lambda32_ij| + delta_ij); below half
        // the smallest subnormal of the pass precision V rounds to 0 (margin
        // 2^-18 for the FP32 rounding of the sums)
        if (p.T > 0) {
            float norm = 0.f;
#pragma unroll
            for (int i = 0; i < M; ++i) {
                float rs = 0.f;
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    const float2 l = block_symbol32<RAD>(p, g.w + (i * M + j) * g.nw, k0, k1, k2);
                    rs += sqrtf(l.x * l.x + l.y * l.y) + g.delta[i * M + j];
                }
                norm = fmaxf(norm, rs);
            }
            norm *= 1.0f + 0x1p-18f;
            if (norm < 1.0f && (float)p.T * log2f(norm) < -g.cut) {
#pragma unroll
                for (int i = 0; i < M; ++i) h[i * g.item] = C{(R)0, (R)0};
                continue;
            }
        }
        double2 lam[M][M];
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int j = 0; j < M; ++j)
                lam[i][j] = block_symbol<RAD>(p, g.w + (i * M + j) * g.nw, k0, k1, k2);
        // V = Lambda^T by repeated squaring
        double2 V[M][M], S[M][M], tmp[M][M];
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int j = 0; j < M; ++j) {
                V[i][j] = double2{i == j ? 1.0 : 0.0, 0.0};
                S[i][j] = lam[i][j];
            }
        long long T = p.T;
        while (T > 0) {
            if (T & 1) {
#pragma unroll
                for (int i = 0; i < M; ++i)
#pragma unroll
                    for (int j = 0; j < M; ++j) {
                        double2 acc{0.0, 0.0};
#pragma unroll
                        for (int k = 0; k < M; ++k) acc = cadd_rn(acc, cmul_rn(V[i][k], S[k][j]));
                        tmp[i][j] = acc;
                    }
#pragma unroll
                for (int i = 0; i < M; ++i)
#pragma unroll
                    for (int j = 0; j < M; ++j) V[i][j] = tmp[i][j];
            }
            T >>= 1;
            if (T > 0) {
#pragma unroll
                for (int i = 0; i < M; ++i)
#pragma unroll
                    for (int j = 0; j < M; ++j) {
                        double2 acc{0.0, 0.0};
#pragma unroll
                        for (int k = 0; k < M; ++k) acc = cadd_rn(acc, cmul_rn(S[i][k], S[k][j]));
                        tmp[i][j] = acc;
                    }
#pragma unroll
                for (int i = 0; i < M; ++i)
#pragma unroll
                    for (int j = 0; j < M; ++j) S[i][j] = tmp[i][j];
            }
        }
        // the multipliers at pass precision (as in the scalar path), then y = V x
        C x[M];
#pragma unroll
        for (int j = 0; j < M; ++j) x[j] = h[j * g.item];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            C acc{(R)0, (R)0};
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const double2 v = cscale_rn(V[i][j], p.scale);
                acc = cadd(acc, cmul(C{(R)v.x, (R)v.y}, x[j]));
            }
            h[i * g.item] = acc;
        }
    }
}

// One field (scalar plans on mixed-radix grids): y = V x with the symbol
// factorised along axis 0, as in the column passes of the power-of-two path.
// A thread owns a chunk of kChunk frequencies k_0 of one column (k_1, k_2):
// G[m_0] = sum_{m_1, m_2} w[m_0, m_1, m_2] E_1[m_1 k_1] E_2[m_2 k_2] once in
// FP32 (screen: sum |G| + delta bounds Lambda over the whole column), then
// Lambda(k_0) = sum_{m_0} E_0[m_0 k_0] G[m_0] per element; survivors take the
// FP64 power from the column's FP64 factors (formed once, when needed).
constexpr int kChunk = 64;

template <typename R, int RAD>
__global__ void __launch_bounds__(128)
k_scalar_mult_cols(typename CxOf<R>::T* __restrict__ H, const __grid_constant__ VecGeom g,
                   const __grid_constant__ SymbolParams p) {
    using C = typename CxOf<R>::T;
    constexpr int W = 2 * RAD + 1;
    const int l0 = g.ndim == 1 ? 1 : g.len[0];
    const long long ncols = g.ndim == 1 ? g.nh : g.rows / l0 * g.nh;   // (k1, k2) columns
    const int nchunks = (l0 + kChunk - 1) / kChunk;
    const long long total = ncols * nchunks;
    const float delta = g.delta[0];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long col = e % ncols;
        const int chunk = (int)(e / ncols);
        int k1 = 0, k2 = 0;
        long long base;   // element (k0 = 0) of this column
        if (g.ndim == 1) {
            base = col;   // 1-D: the column is one element, k0 = col
        } else if (g.ndim == 2) {
            k1 = (int)col;
            base = col;
        } else {
            k1 = (int)(col / g.nh);
            k2 = (int)(col % g.nh);
            base = (long long)k1 * g.Mp + k2;
        }
        const long long stride = g.ndim == 2 ? g.Mp : (long long)g.len[1] * g.Mp;
        float2 G[W];
        {
            float2 e1[W], e2[W];
#pragma unroll
            for (int m = -RAD; m <= RAD; ++m) {
                e1[m + RAD] = g.ndim >= 2 ? __ldg(p.E32[1] + axis_index(p, 1, m * k1)) : float2{1.f, 0.f};
                e2[m + RAD] = g.ndim >= 3 ? __ldg(p.E32[2] + axis_index(p, 2, m * k2)) : float2{1.f, 0.f};
            }
            const int W1 = g.ndim >= 2 ? W : 1, W2 = g.ndim >= 3 ? W : 1;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                float2 acc{0.f, 0.f};
                for (int j = 0; j < W1; ++j) {
                    float2 inner{0.f, 0.f};
                    for (int q = 0; q < W2; ++q)
                        inner = cadd(inner, cscale(e2[q], (float)__ldg(g.w + (i * W1 + j) * W2 + q)));
                    acc = cadd(acc, cmul(e1[j], inner));
                }
                G[i] = acc;
            }
        }
        const int kb = g.ndim == 1 ? (int)col : chunk * kChunk;
        const int ke = g.ndim == 1 ? (int)col + 1 : min(l0, kb + kChunk);
        if (p.T > 0) {   // whole-column screen
            float b = 0.f;
#pragma unroll
            for (int i = 0; i < W; ++i) b += sqrtf(G[i].x * G[i].x + G[i].y * G[i].y);
            b = (b + delta) * (1.0f + 0x1p-18f);
            if (b < 1.0f && (float)p.T * log2f(b) < -g.cut) {
                for (int k0 = kb; k0 < ke; ++k0)
                    H[g.ndim == 1 ? base : base + (long long)k0 * stride] = C{(R)0, (R)0};
                continue;
            }
        }
        bool have64 = false;
        ColSymbol64<RAD> cs64;
        for (int k0 = kb; k0 < ke; ++k0) {
            C* h = H + (g.ndim == 1 ? base : base + (long long)k0 * stride);
            const int kk0 = g.ndim == 1 ? (int)col : k0;
            if (p.T > 0) {
                float2 l = G[RAD];
#pragma unroll
                for (int m = 1; m <= RAD; ++m) {
                    const float2 em = __ldg(p.E32[0] + axis_index(p, 0, m * kk0));
                    l = cadd(l, cmul(em, G[RAD + m]));
                    l = cadd(l, cmul(cconj(em), G[RAD - m]));
                }
                const float bound = (sqrtf(l.x * l.x + l.y * l.y) + delta) * (1.0f + 0x1p-18f);
                if (bound < 1.0f && (float)p.T * log2f(bound) < -g.cut) {
                    *h = C{(R)0, (R)0};
                    continue;
                }
            }
            if (!have64) {
                col_symbol_init64<RAD>(p, g.w, k1, k2, cs64);
                have64 = true;
            }
            const double2 v = col_power64<RAD>(p, cs64, kk0);
            *h = cmul(*h, C{(R)v.x, (R)v.y});
        }
    }
}

template <typename R, int M>
cudaError_t launch_mult_m(void* H, const VecGeom& g, const SymbolParams& p, cudaStream_t s) {
    const long long total = g.rows * g.nh;
    const int threads = 128;
    long long blocks = (total + threads - 1) / threads;
    if (blocks > 152 * 32) blocks = 152 * 32;
    using C = typename CxOf<R>::T;
    switch (p.r) {
        case 0: k_vector_mult<R, M, 0><<<(int)blocks, threads, 0, s>>>(static_cast<C*>(H), g, p); break;
        case 1: k_vector_mult<R, M, 1><<<(int)blocks, threads, 0, s>>>(static_cast<C*>(H), g, p); break;
        case 2: k_vector_mult<R, M, 2><<<(int)blocks, threads, 0, s>>>(static_cast<C*>(H), g, p); break;
        default: k_vector_mult<R, M, 3><<<(int)blocks, threads, 0, s>>>(static_cast<C*>(H), g, p); break;
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_mult(void* H, const VecGeom& g, const SymbolParams& p, cudaStream_t s) {
    if (g.m == 1) {
        using C = typename CxOf<R>::T;
        const int l0 = g.ndim == 1 ? 1 : g.len[0];
        const long long ncols = g.ndim == 1 ? g.nh : g.rows / l0 * g.nh;
        const long long total = ncols * ((l0 + kChunk - 1) / kChunk);
        long long blocks = (total + 127) / 128;
        if (blocks > 152 * 64) blocks = 152 * 64;
        switch (p.r) {
            case 0: k_scalar_mult_cols<R, 0><<<(int)blocks, 128, 0, s>>>(static_cast<C*>(H), g, p); break;
            case 1: k_scalar_mult_cols<R, 1><<<(int)blocks, 128, 0, s>>>(static_cast<C*>(H), g, p); break;
            case 2: k_scalar_mult_cols<R, 2><<<(int)blocks, 128, 0, s>>>(static_cast<C*>(H), g, p); break;
            default: k_scalar_mult_cols<R, 3><<<(int)blocks, 128, 0, s>>>(static_cast<C*>(H), g, p); break;
        }
        return cudaGetLastError();
    }
    switch (g.m) {
        case 1: return launch_mult_m<R, 1>(H, g, p, s);
        case 2: return launch_mult_m<R, 2>(H, g, p, s);
        case 3: return launch_mult_m<R, 3>(H, g, p, s);
        default: return launch_mult_m<R, 4>(H, g, p, s);
    }
}

// Column geometry of a strided-axis pass over all fields.
ColGeom col_geom(int log2n, long long S, int outer, long long os, int mid, long long ms, int n,
                 int elem) {
    ColGeom g;
    g.log2n = log2n;
    g.S = S;
    g.outer = outer;
    g.os = os;
    g.mid = mid;
    g.ms = ms;
    g.inner_valid = n + 1;
    g.cols_log2 = cols_log2_for(log2n, elem, elem == 8 ? kMaxThreadsF32 : kMaxThreadsF64);
    return g;
}

// One strided-axis pass over every field: the power-of-two kernels, or the
// mixed-radix ones for other lengths.
template <typename R>
cudaError_t cols_pass(stencil_plan_s* p, int axis, const ColGeom& g, int dir, cudaStream_t s) {
    const int64_t l = p->dims[axis];
    if (ilog2_exact(l) >= 0) return launch_cols<R>(p->H, g, dir, p->tw, p->twn_log2, s);
    return launch_mixed_cols<R>(dir, p->H, g, (int)l, p->mtw[axis], s);
}

template <typename R>
cudaError_t rows_pass(stencil_plan_s* p, R* grid, int rows, int dir, cudaStream_t s) {
    const int d = p->ndim;
    const int64_t L = p->dims[d - 1];
    if (ilog2_exact(L) >= 0) {
        const int n_log2 = ilog2_exact(L) - 1;
        if (dir < 0)
            return launch_rows_r2c<R>(grid, p->H, p->Mp, n_log2, rows, p->tw, p->twn_log2, s);
        return launch_rows_c2r<R>(p->H, grid, p->Mp, n_log2, rows, p->tw, p->twn_log2, p->status,
                                  s);
    }
    if (dir < 0)
        return launch_mixed_rows<R>(-1, grid, p->H, p->Mp, (int)(L / 2), rows, p->mtw[d - 1],
                                    p->status, s);
    return launch_mixed_rows<R>(+1, p->H, grid, p->Mp, (int)(L / 2), rows, p->mtw[d - 1],
                                p->status, s);
}

// Each pass bracketed by the plan's profiler (stencil_profile_*).
#define VPASS(kind, call)         \
    do {                          \
        p->prof.begin(kind, s);   \
        err = (call);             \
        p->prof.end(s);           \
    } while (0)

template <typename R>
cudaError_t vector_solve(stencil_plan_s* p, R* grid, int64_t T, cudaStream_t s) {
    const int d = p->ndim, m = p->nfields;
    const int n = (int)(p->dims[d - 1] / 2);
    const long long Mp = p->Mp;
    const int celem = 2 * sizeof(R);
    long long rows_item = 1;
    for (int a = 0; a < d - 1; ++a) rows_item *= p->dims[a];
    const long long item = rows_item * Mp;
    auto log2_or0 = [](int64_t l) { return ilog2_exact(l) >= 0 ? ilog2_exact(l) : 0; };
    cudaError_t err;
    VPASS(PASS_ROWS_R2C, rows_pass<R>(p, grid, (int)(rows_item * m), -1, s));
    if (err != cudaSuccess) return err;
    ColGeom g0, g1;
    if (d == 2) {
        g0 = col_geom(log2_or0(p->dims[0]), Mp, m, item, 1, 0, n, celem);
        VPASS(PASS_COLS_FWD, cols_pass<R>(p, 0, g0, -1, s));
    } else if (d == 3) {
        g1 = col_geom(log2_or0(p->dims[1]), Mp, (int)(p->dims[0] * m), p->dims[1] * Mp, 1, 0, n,
                      celem);
        g0 = col_geom(log2_or0(p->dims[0]), p->dims[1] * Mp, m, item, (int)p->dims[1], Mp, n,
                      celem);
        VPASS(PASS_COLS_FWD, cols_pass<R>(p, 1, g1, -1, s));
        if (err == cudaSuccess) VPASS(PASS_COLS_FWD, cols_pass<R>(p, 0, g0, -1, s));
    }
    if (err != cudaSuccess) return err;
    VecGeom vg;
    std::memset(&vg, 0, sizeof(vg));
    for (int b = 0; b < m * m; ++b) vg.delta[b] = p->vdelta[b];
    vg.ndim = d;
    for (int a = 0; a < d; ++a) vg.len[a] = (int)p->dims[a];
    vg.nh = n + 1;
    vg.Mp = Mp;
    vg.rows = rows_item;
    vg.item = item;
    vg.m = m;
    vg.w = p->wv_dev;
    vg.nw = p->nweights;
    vg.cut = p->precision == STENCIL_FP32 ? 154.0f : 1080.0f;
    const SymbolParams sp = make_symbol_params(p, p->dims, T, p->E64, p->E32, nullptr);
    VPASS(PASS_VTABLE, launch_mult<R>(p->H, vg, sp, s));
    if (err != cudaSuccess) return err;
    if (d == 2) {
        VPASS(PASS_COLS_INV, cols_pass<R>(p, 0, g0, +1, s));
    } else if (d == 3) {
        VPASS(PASS_COLS_INV, cols_pass<R>(p, 0, g0, +1, s));
        if (err == cudaSuccess) VPASS(PASS_COLS_INV, cols_pass<R>(p, 1, g1, +1, s));
    }
    if (err != cudaSuccess) return err;
    VPASS(PASS_ROWS_C2R, rows_pass<R>(p, grid, (int)(rows_item * m), +1, s));
    return err;
}

}  // namespace

cudaError_t vector_run(stencil_plan_s* p, void* grid, int64_t T, cudaStream_t s) {
    return p->precision == STENCIL_FP32 ? vector_solve<float>(p, static_cast<float*>(grid), T, s)
                                        : vector_solve<double>(p, static_cast<double*>(grid), T, s);
}

int vector_max_fields() { return kMaxFields; }

}  // namespace sfft
