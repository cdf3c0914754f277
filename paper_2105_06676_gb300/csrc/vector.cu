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
};

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
        double2 lam[M][M];
        double norm = 0.0;   // ||Lambda||_inf (max row sum of moduli)
#pragma unroll
        for (int i = 0; i < M; ++i) {
            double rs = 0.0;
#pragma unroll
            for (int j = 0; j < M; ++j) {
                lam[i][j] = block_symbol<RAD>(p, g.w + (i * M + j) * g.nw, k0, k1, k2);
                rs += sqrt(lam[i][j].x * lam[i][j].x + lam[i][j].y * lam[i][j].y);
            }
            norm = fmax(norm, rs);
        }
        C* h = H + row * g.Mp + last;
        // every |V_ij| <= ||Lambda||_inf^T / N: below half the smallest
        // subnormal of the pass precision it rounds to 0 (margin 2^-30 for
        // the rounding of the norm)
        if (p.T > 0 && norm * (1.0 + 0x1p-30) < 1.0 &&
            (double)p.T * log2(norm * (1.0 + 0x1p-30)) < -(double)g.cut) {
#pragma unroll
            for (int i = 0; i < M; ++i) h[i * g.item] = C{(R)0, (R)0};
            continue;
        }
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
    cudaError_t err = rows_pass<R>(p, grid, (int)(rows_item * m), -1, s);
    if (err != cudaSuccess) return err;
    ColGeom g0, g1;
    if (d == 2) {
        g0 = col_geom(log2_or0(p->dims[0]), Mp, m, item, 1, 0, n, celem);
        err = cols_pass<R>(p, 0, g0, -1, s);
    } else if (d == 3) {
        g1 = col_geom(log2_or0(p->dims[1]), Mp, (int)(p->dims[0] * m), p->dims[1] * Mp, 1, 0, n,
                      celem);
        g0 = col_geom(log2_or0(p->dims[0]), p->dims[1] * Mp, m, item, (int)p->dims[1], Mp, n,
                      celem);
        err = cols_pass<R>(p, 1, g1, -1, s);
        if (err == cudaSuccess) err = cols_pass<R>(p, 0, g0, -1, s);
    }
    if (err != cudaSuccess) return err;
    VecGeom vg;
    std::memset(&vg, 0, sizeof(vg));
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
    err = launch_mult<R>(p->H, vg, sp, s);
    if (err != cudaSuccess) return err;
    if (d == 2) {
        err = cols_pass<R>(p, 0, g0, +1, s);
    } else if (d == 3) {
        err = cols_pass<R>(p, 0, g0, +1, s);
        if (err == cudaSuccess) err = cols_pass<R>(p, 1, g1, +1, s);
    }
    if (err != cudaSuccess) return err;
    return rows_pass<R>(p, grid, (int)(rows_item * m), +1, s);
}

}  // namespace

cudaError_t vector_run(stencil_plan_s* p, void* grid, int64_t T, cudaStream_t s) {
    return p->precision == STENCIL_FP32 ? vector_solve<float>(p, static_cast<float*>(grid), T, s)
                                        : vector_solve<double>(p, static_cast<double*>(grid), T, s);
}

int vector_max_fields() { return kMaxFields; }

}  // namespace sfft
