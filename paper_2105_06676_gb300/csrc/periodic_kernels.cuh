#pragma once
// StencilFFT-P kernels (paper Sec. 4, Fig. "stencil-fft-algorithm-dD").
// Templates shared by the FP32 and FP64 translation units.
//
// A real grid of shape l_1 x ... x l_d is solved in place by
//   * rows_r2c   : FFT along the contiguous last axis. A real row of L = 2n
//                  values is read as n complex pairs, transformed, and split
//                  into the half spectrum X[0..n] (Hermitian symmetry of a real
//                  input), written to the workspace H (row stride Mp).
//   * cols       : FFT along a strided axis of H (forward or inverse).
//   * cols_fused : forward FFT along axis 0, multiply by V[k] = Lambda[k]^T / N
//                  (Steps 2 and 3: repeated squaring and the pointwise
//                  product), inverse FFT along axis 0, all in shared memory:
//                  one read and one write of H.
//   * rows_c2r   : inverse of rows_r2c (Step 4), writes the real grid.
//   * fused_1d   : for d = 1 the whole solve (R2C, multiply, C2R) in one CTA
//                  per row.
// The spectrum never needs reordering: every pass returns natural order, so
// V is evaluated at the natural frequency of each element.
#include <cuda_runtime.h>

#include <cstdlib>
#include <map>
#include <mutex>
#include <type_traits>

#include "fft_ct.cuh"
#include "fft_reg.cuh"
#include "internal.h"

namespace sfft {

template <typename R> struct MaxT;
template <> struct MaxT<float> { static constexpr int v = kMaxThreadsF32; };
template <> struct MaxT<double> { static constexpr int v = kMaxThreadsF64; };

// Resident CTAs per SM the column kernels are compiled for: FP32 CTAs below
// 1024 threads keep 64 registers per thread so that 2048 / MAXT CTAs fit.
template <typename R, int MAXT>
struct ColMinBlocks {
    static constexpr int v = (sizeof(R) == 4 && MAXT < 1024) ? 1024 / MAXT : 1;
};

// FFT of one sequence: compile-time length when LOG2N > 0, else runtime.
template <int DIR, int LOG2N, typename C>
__device__ __forceinline__ void seq_fft(C* v, const SeqView<C>& sm, int j, int log2n,
                                        const C* __restrict__ tw, int twn_log2) {
    if constexpr (LOG2N > 0) ct_fft<DIR, LOG2N, 0, 5>(v, sm.base, j, tw, twn_log2);
    else reg_fft<DIR>(v, sm, j, log2n, tw, twn_log2);
}
template <int DIR, int LOG2N, int CL, typename C>
__device__ __forceinline__ void col_fft(C* v, const ColView<C>& sm, int j, int log2n,
                                        const C* __restrict__ tw, int twn_log2) {
    if constexpr (LOG2N > 0) ct_fft<DIR, LOG2N, CL, 4 - CL>(v, sm.base + sm.c, j, tw, twn_log2);
    else reg_fft<DIR>(v, sm, j, log2n, tw, twn_log2);
}

__device__ __forceinline__ bool finite2(float2 v) { return isfinite(v.x) && isfinite(v.y); }
__device__ __forceinline__ bool finite2(double2 v) { return isfinite(v.x) && isfinite(v.y); }

// ---------------------------------------------------------------------------
// fused 1-D solve: rows of L = 2n reals, one CTA holds `rpc` rows
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(MaxT<R>::v)
k_fused_1d(R* __restrict__ grid, int n_log2, int nrows, int rpc,
           const typename CxOf<R>::T* __restrict__ tw, int twn_log2,
           const __grid_constant__ SymbolParams p, int* status) {
    using C = typename CxOf<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int n = 1 << n_log2;
    const int ss = seq_stride(n);
    const int row0 = blockIdx.x * rpc;
    const int rows = min(rpc, nrows - row0);
    C* rowp = reinterpret_cast<C*>(grid) + (size_t)row0 * n;  // row c, pair j at rowp[c*n + j]
    for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
        const int c = e >> n_log2, j = e & (n - 1);
        sm[c * ss + spad(j)] = rowp[e];
    }
    __syncthreads();
    fft_smem<-1, kEPT>(sm, n_log2, rows, tw, twn_log2);
    const int half = n / 2 + 1;
    const int sh = twn_log2 - n_log2 - 1;  // W^k = exp(-2 pi i k / 2n) = tw[k << sh]
    for (int e = threadIdx.x; e < rows * half; e += blockDim.x) {
        const int c = e / half, k = e - c * half;
        C* s = sm + c * ss;
        const int ik = spad(k & (n - 1)), ink = spad((n - k) & (n - 1));
        const C zk = s[ik], znk = s[ink];
        const C xe = cscale(cadd(zk, cconj(znk)), (R)0.5);
        const C xo = cscale(cmul_mi(csub(zk, cconj(znk))), (R)0.5);
        const C wk = tw[k << sh];
        const C t = cmul(wk, xo);
        const C Xk = cadd(xe, t);
        const C Xnk = cconj(csub(xe, t));
        int kk = k;
        const C Vk = spectral_multiplier<C>(p, &kk);
        kk = n - k;
        const C Vnk = spectral_multiplier<C>(p, &kk);
        const C Yk = cmul(Vk, Xk), Ynk = cmul(Vnk, Xnk);
        // inverse pre-processing: Z'[q] = (Y[q] + conj Y[n-q]) + i conj(W^q) (Y[q] - conj Y[n-q])
        const C zpk = cadd(cadd(Yk, cconj(Ynk)), cmul_i(cmul(cconj(wk), csub(Yk, cconj(Ynk)))));
        // conj(W^(n-k)) = -W^k
        const C zpnk = csub(cadd(Ynk, cconj(Yk)), cmul_i(cmul(wk, csub(Ynk, cconj(Yk)))));
        s[ik] = zpk;
        if (k != 0 && 2 * k != n) s[ink] = zpnk;
    }
    __syncthreads();
    fft_smem<+1, kEPT>(sm, n_log2, rows, tw, twn_log2);
    bool bad = false;
    for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
        const int c = e >> n_log2, j = e & (n - 1);
        const C v = sm[c * ss + spad(j)];
        bad |= !finite2(v);
        rowp[e] = v;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, 1);
}

// ---------------------------------------------------------------------------
// real rows -> half spectrum rows (n + 1 complex values, row stride Mp)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(MaxT<R>::v)
k_rows_r2c(const R* __restrict__ grid, typename CxOf<R>::T* __restrict__ H, long long Mp,
           int n_log2, int nrows, int rpc, const typename CxOf<R>::T* __restrict__ tw,
           int twn_log2) {
    using C = typename CxOf<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int n = 1 << n_log2;
    const int ss = seq_stride(n);
    const long long row0 = (long long)blockIdx.x * rpc;
    const int rows = (int)min((long long)rpc, nrows - row0);
    const C* rowp = reinterpret_cast<const C*>(grid) + row0 * n;
    for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
        const int c = e >> n_log2, j = e & (n - 1);
        sm[c * ss + spad(j)] = __ldg(rowp + e);
    }
    __syncthreads();
    fft_smem<-1, kEPT>(sm, n_log2, rows, tw, twn_log2);
    const int sh = twn_log2 - n_log2 - 1;
    const int np1 = n + 1;
    for (int e = threadIdx.x; e < rows * np1; e += blockDim.x) {
        const int c = e / np1, k = e - c * np1;
        const C* s = sm + c * ss;
        const C zk = s[spad(k & (n - 1))], znk = s[spad((n - k) & (n - 1))];
        const C xe = cscale(cadd(zk, cconj(znk)), (R)0.5);
        const C xo = cscale(cmul_mi(csub(zk, cconj(znk))), (R)0.5);
        const C wk = tw[k << sh];
        H[(row0 + c) * Mp + k] = cadd(xe, cmul(wk, xo));
    }
}

// ---------------------------------------------------------------------------
// half spectrum rows -> real rows
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(MaxT<R>::v)
k_rows_c2r(const typename CxOf<R>::T* __restrict__ H, R* __restrict__ grid, long long Mp,
           int n_log2, int nrows, int rpc, const typename CxOf<R>::T* __restrict__ tw,
           int twn_log2, int* status) {
    using C = typename CxOf<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int n = 1 << n_log2;
    const int ss = seq_stride(n);
    const long long row0 = (long long)blockIdx.x * rpc;
    const int rows = (int)min((long long)rpc, nrows - row0);
    const int sh = twn_log2 - n_log2 - 1;
    for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
        const int c = e >> n_log2, k = e & (n - 1);
        const C* h = H + (row0 + c) * Mp;
        const C yk = __ldg(h + k), ynk = __ldg(h + (n - k));
        const C wk = tw[k << sh];
        sm[c * ss + spad(k)] =
            cadd(cadd(yk, cconj(ynk)), cmul_i(cmul(cconj(wk), csub(yk, cconj(ynk)))));
    }
    __syncthreads();
    fft_smem<+1, kEPT>(sm, n_log2, rows, tw, twn_log2);
    C* rowp = reinterpret_cast<C*>(grid) + row0 * n;
    bool bad = false;
    for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
        const int c = e >> n_log2, j = e & (n - 1);
        const C v = sm[c * ss + spad(j)];
        bad |= !finite2(v);
        rowp[e] = v;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, 1);
}

// ---------------------------------------------------------------------------
// strided column FFTs (forward or inverse), and the fused
// forward * V * inverse pass along axis 0
// ---------------------------------------------------------------------------
template <typename C>
__device__ __forceinline__ void load_cols(C* sm, const C* __restrict__ base, const ColGeom& g,
                                          int i0) {
    const int n = 1 << g.log2n;
    const int cols = 1 << g.cols_log2;
    const int ss = seq_stride(n);
    for (int e = threadIdx.x; e < cols * n; e += blockDim.x) {
        const int j = e >> g.cols_log2, c = e & (cols - 1);
        C v{0, 0};
        if (i0 + c < g.inner_valid) v = base[(long long)j * g.S + c];
        sm[c * ss + spad(j)] = v;
    }
}

template <typename C>
__device__ __forceinline__ void store_cols(const C* sm, C* __restrict__ base, const ColGeom& g,
                                           int i0) {
    const int n = 1 << g.log2n;
    const int cols = 1 << g.cols_log2;
    const int ss = seq_stride(n);
    for (int e = threadIdx.x; e < cols * n; e += blockDim.x) {
        const int j = e >> g.cols_log2, c = e & (cols - 1);
        if (i0 + c < g.inner_valid) base[(long long)j * g.S + c] = sm[c * ss + spad(j)];
    }
}

template <typename R, int DIR>
__global__ void __launch_bounds__(MaxT<R>::v)
k_cols(typename CxOf<R>::T* __restrict__ H, const __grid_constant__ ColGeom g,
       const typename CxOf<R>::T* __restrict__ tw, int twn_log2) {
    using C = typename CxOf<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int i0 = blockIdx.x << g.cols_log2;
    C* base = H + (long long)blockIdx.z * g.os + (long long)blockIdx.y * g.ms + i0;
    load_cols(sm, base, g, i0);
    __syncthreads();
    const int cols = min(1 << g.cols_log2, g.inner_valid - i0);
    fft_smem<DIR, kEPT>(sm, g.log2n, cols, tw, twn_log2);
    store_cols(sm, base, g, i0);
}

// Fused pass along axis 0 of the half spectrum. Frequencies: k_0 is the FFT
// index; for d = 2 the inner index is k_1; for d = 3 the mid index is k_1 and
// the inner index k_2.
template <typename R>
__global__ void __launch_bounds__(MaxT<R>::v)
k_cols_fused(typename CxOf<R>::T* __restrict__ H, const __grid_constant__ ColGeom g,
             const typename CxOf<R>::T* __restrict__ tw, int twn_log2,
             const __grid_constant__ SymbolSet ps) {
    const SymbolParams& p = ps.p[ps.orient[blockIdx.z]];
    using C = typename CxOf<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int i0 = blockIdx.x << g.cols_log2;
    C* base = H + (long long)blockIdx.z * g.os + (long long)blockIdx.y * g.ms + i0;
    load_cols(sm, base, g, i0);
    __syncthreads();
    const int cols = min(1 << g.cols_log2, g.inner_valid - i0);
    fft_smem<-1, kEPT>(sm, g.log2n, cols, tw, twn_log2);
    const int n = 1 << g.log2n;
    const int ss = seq_stride(n);
    for (int e = threadIdx.x; e < cols * n; e += blockDim.x) {
        const int c = e >> g.log2n, j = e & (n - 1);
        int k[3];
        k[0] = j;
        if (p.ndim == 2) {
            k[1] = i0 + c;
        } else {
            k[1] = blockIdx.y;
            k[2] = i0 + c;
        }
        const C* vt = static_cast<const C*>(ps.vtab_item[blockIdx.z] ? ps.vtab_item[blockIdx.z]
                                                                       : ps.vtab[ps.orient[blockIdx.z]]);
        const C v = vt ? (i0 + c < g.inner_valid
                              ? vt[(long long)blockIdx.y * g.ms + (long long)j * g.S + i0 + c]
                              : C{0, 0})
                       : spectral_multiplier<C>(p, k);
        C* q = sm + c * ss + spad(j);
        *q = cmul(*q, v);
    }
    __syncthreads();
    fft_smem<+1, kEPT>(sm, g.log2n, cols, tw, twn_log2);
    store_cols(sm, base, g, i0);
}

// ---------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_twiddles(typename CxOf<R>::T* tw, int twn_log2) {
    const int n = 1 << twn_log2;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)m / (double)n, &s, &c);   // exp(-2 pi i m / n)
        tw[m] = typename CxOf<R>::T{(R)c, (R)s};
    }
}



// V[k] = Lambda[k]^T / N at pass precision for one box shape, laid out like
// one item's half spectrum: ((k_0 * l_1 + k_1) * Mp + k_last) (d = 3) or
// (k_0 * Mp + k_1) (d = 2).
template <typename R>
__global__ void k_vtable(typename CxOf<R>::T* __restrict__ V, const __grid_constant__ SymbolParams p,
                         int nhalf, long long Mp, long long total) {
    using C = typename CxOf<R>::T;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int k[3] = {0, 0, 0};
        long long rest = e;
        const int last = (int)(rest % nhalf);
        rest /= nhalf;
        if (p.ndim == 1) {
            k[0] = last;
        } else if (p.ndim == 2) {
            k[0] = (int)rest;
            k[1] = last;
        } else {
            k[1] = (int)(rest % p.len[1]);
            k[0] = (int)(rest / p.len[1]);
            k[2] = last;
        }
        V[rest * Mp + last] = spectral_multiplier<C>(p, k);
    }
}

// ---------------------------------------------------------------------------
// register-resident kernels (transform length n >= 16): q = n/16 threads per
// sequence, 16 elements per thread, two shared-memory exchanges per 4096-point
// transform instead of a shared-memory round trip per stage
// ---------------------------------------------------------------------------
template <typename R, int RAD, int MAXT, int LOG2N>
__global__ void __launch_bounds__(MAXT)
k_fused_1d_reg(R* __restrict__ grid, int n_log2, int nrows, int rpc,
               const typename CxOf<R>::T* __restrict__ tw, int twn_log2,
               const __grid_constant__ SymbolParams p, int* status,
               const __grid_constant__ RowTables rt) {
    using C = typename CxOf<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* small = reinterpret_cast<C*>(smraw);
    if constexpr (LOG2N > 0) n_log2 = LOG2N;
    const int n = 1 << n_log2, q = n >> 4;
    const int ss = seq_stride(n);
    const int c = threadIdx.x / q, j = threadIdx.x - c * q;
    const int row = blockIdx.x * rpc + c;
    const bool live = row < nrows;
    const SeqView<C> sm{small + c * ss};
    C* rowp = reinterpret_cast<C*>(grid) + (size_t)(live ? row : 0) * n;
    C v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) v[s] = live ? rowp[j + q * s] : C{0, 0};
    seq_fft<-1, LOG2N>(v, sm, j, n_log2, tw, twn_log2);
    // real-input split: X[k] from Z[k] and Z[n-k]
#pragma unroll
    for (int r = 0; r < 16; ++r) sm[j + q * r] = v[r];
    __syncthreads();
    const int sh = twn_log2 - n_log2 - 1;  // W^k = exp(-2 pi i k / 2n) = tw[k << sh]
    C xn{0, 0};                             // X[n], thread j = 0 only
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int k = j + q * r;
        const C zk = v[r];
        const C znk = sm[(n - k) & (n - 1)];
        const C xe = cscale(cadd(zk, cconj(znk)), (R)0.5);
        const C xo = cscale(cmul_mi(csub(zk, cconj(znk))), (R)0.5);
        const C t = cmul(tw[k << sh], xo);
        v[r] = cadd(xe, t);
        if (k == 0) xn = csub(xe, xo);
    }
    __syncthreads();
    // Y[k] = V[k] X[k]
    const C* vt = row < kMaxItems ? static_cast<const C*>(rt.t[row]) : nullptr;
    if (vt) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = cmul(v[r], __ldg(vt + j + q * r));
        if (j == 0) xn = cmul(xn, __ldg(vt + n));
    } else {
        ColSymbol<RAD> cs;
        int kz[3] = {0, 0, 0};
        col_symbol_init<RAD>(p, kz, cs);
        apply_multiplier<RAD>(v, sm, j, q, p, cs, 0, 0);
        if (j == 0) xn = multiply_single<C>(xn, p, n, 0, 0);
    }
    __syncthreads();
    // inverse split: Z'[k] = (Y[k] + conj Y[n-k]) + i conj(W^k) (Y[k] - conj Y[n-k])
#pragma unroll
    for (int r = 0; r < 16; ++r) sm[j + q * r] = v[r];
    if (j == 0) sm[n] = xn;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int k = j + q * r;
        const C yk = v[r];
        const C ynk = sm[n - k];
        const C wk = tw[k << sh];
        v[r] = cadd(cadd(yk, cconj(ynk)), cmul_i(cmul(cconj(wk), csub(yk, cconj(ynk)))));
    }
    __syncthreads();
    seq_fft<+1, LOG2N>(v, sm, j, n_log2, tw, twn_log2);
    bool bad = false;
    if (live) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            bad |= !finite2(v[r]);
            rowp[j + q * r] = v[r];
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, 1);
}

template <typename R, int MAXT, int LOG2N>
__global__ void __launch_bounds__(MAXT)
k_rows_r2c_reg(const R* __restrict__ grid, typename CxOf<R>::T* __restrict__ H, long long Mp,
               int n_log2, int nrows, int rpc, const typename CxOf<R>::T* __restrict__ tw,
               int twn_log2) {
    using C = typename CxOf<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* small = reinterpret_cast<C*>(smraw);
    if constexpr (LOG2N > 0) n_log2 = LOG2N;
    const int n = 1 << n_log2, q = n >> 4;
    const int ss = seq_stride(n);
    const int c = threadIdx.x / q, j = threadIdx.x - c * q;
    const long long row = (long long)blockIdx.x * rpc + c;
    const bool live = row < nrows;
    const SeqView<C> sm{small + c * ss};
    const C* rowp = reinterpret_cast<const C*>(grid) + (live ? row : 0) * n;
    C v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) v[s] = live ? __ldg(rowp + j + q * s) : C{0, 0};
    seq_fft<-1, LOG2N>(v, sm, j, n_log2, tw, twn_log2);
#pragma unroll
    for (int r = 0; r < 16; ++r) sm[j + q * r] = v[r];
    __syncthreads();
    if (!live) return;
    const int sh = twn_log2 - n_log2 - 1;
    C* h = H + row * Mp;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int k = j + q * r;
        const C zk = v[r], znk = sm[(n - k) & (n - 1)];
        const C xe = cscale(cadd(zk, cconj(znk)), (R)0.5);
        const C xo = cscale(cmul_mi(csub(zk, cconj(znk))), (R)0.5);
        h[k] = cadd(xe, cmul(tw[k << sh], xo));
        if (k == 0) h[n] = csub(xe, xo);   // X[n] = Xe[0] - Xo[0] (both real)
    }
}

template <typename R, int MAXT, int LOG2N>
__global__ void __launch_bounds__(MAXT)
k_rows_c2r_reg(const typename CxOf<R>::T* __restrict__ H, R* __restrict__ grid, long long Mp,
               int n_log2, int nrows, int rpc, const typename CxOf<R>::T* __restrict__ tw,
               int twn_log2, int* status) {
    using C = typename CxOf<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* small = reinterpret_cast<C*>(smraw);
    if constexpr (LOG2N > 0) n_log2 = LOG2N;
    const int n = 1 << n_log2, q = n >> 4;
    const int ss = seq_stride(n);
    const int c = threadIdx.x / q, j = threadIdx.x - c * q;
    const long long row = (long long)blockIdx.x * rpc + c;
    const bool live = row < nrows;
    const SeqView<C> sm{small + c * ss};
    const C* h = H + (live ? row : 0) * Mp;
    const int sh = twn_log2 - n_log2 - 1;
    C v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int k = j + q * s;
        const C yk = live ? __ldg(h + k) : C{0, 0};
        const C ynk = live ? __ldg(h + (n - k)) : C{0, 0};
        const C wk = tw[k << sh];
        v[s] = cadd(cadd(yk, cconj(ynk)), cmul_i(cmul(cconj(wk), csub(yk, cconj(ynk)))));
    }
    seq_fft<+1, LOG2N>(v, sm, j, n_log2, tw, twn_log2);
    bool bad = false;
    if (live) {
        C* rowp = reinterpret_cast<C*>(grid) + row * n;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            bad |= !finite2(v[r]);
            rowp[j + q * r] = v[r];
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, 1);
}

template <typename R, int DIR, int MAXT, int LOG2N, int CL>
__global__ void __launch_bounds__(MAXT, ColMinBlocks<R, MAXT>::v)
k_cols_reg(typename CxOf<R>::T* __restrict__ H, const __grid_constant__ ColGeom g,
           const typename CxOf<R>::T* __restrict__ tw, int twn_log2) {
    using C = typename CxOf<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* small = reinterpret_cast<C*>(smraw);
    const int log2n = LOG2N > 0 ? LOG2N : g.log2n;
    const int cl = LOG2N > 0 ? CL : g.cols_log2;
    const int n = 1 << log2n, q = n >> 4;
    const int cols = 1 << cl;
    const int c = threadIdx.x & (cols - 1), j = threadIdx.x >> cl;
    const int i0 = blockIdx.x << cl;
    const bool live = i0 + c < g.inner_valid;
    const ColView<C> sm{small, c, cl};
    C* base = H + (long long)blockIdx.z * g.os + (long long)blockIdx.y * g.ms + i0 + c;
    C v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) v[s] = live ? base[(long long)(j + q * s) * g.S] : C{0, 0};
    col_fft<DIR, LOG2N, CL>(v, sm, j, log2n, tw, twn_log2);
    if (live) {
#pragma unroll
        for (int r = 0; r < 16; ++r) base[(long long)(j + q * r) * g.S] = v[r];
    }
}

template <typename R, int RAD, int MAXT, int LOG2N, int CL>
__global__ void __launch_bounds__(MAXT, ColMinBlocks<R, MAXT>::v)
k_cols_fused_reg(typename CxOf<R>::T* __restrict__ H, const __grid_constant__ ColGeom g,
                 const typename CxOf<R>::T* __restrict__ tw, int twn_log2,
                 const __grid_constant__ SymbolSet ps) {
    const SymbolParams& p = ps.p[ps.orient[blockIdx.z]];
    using C = typename CxOf<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* small = reinterpret_cast<C*>(smraw);
    const int log2n = LOG2N > 0 ? LOG2N : g.log2n;
    const int cl = LOG2N > 0 ? CL : g.cols_log2;
    const int n = 1 << log2n, q = n >> 4;
    const int cols = 1 << cl;
    const int c = threadIdx.x & (cols - 1), j = threadIdx.x >> cl;
    const int i0 = blockIdx.x << cl;
    const bool live = i0 + c < g.inner_valid;
    const ColView<C> sm{small, c, cl};
    C* base = H + (long long)blockIdx.z * g.os + (long long)blockIdx.y * g.ms + i0 + c;
    C v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) v[s] = live ? base[(long long)(j + q * s) * g.S] : C{0, 0};
    col_fft<-1, LOG2N, CL>(v, sm, j, log2n, tw, twn_log2);
    int k[3];
    if (p.ndim == 2) {
        k[1] = i0 + c;
        k[2] = 0;
    } else {
        k[1] = blockIdx.y;
        k[2] = i0 + c;
    }
    const C* vt = static_cast<const C*>(ps.vtab_item[blockIdx.z] ? ps.vtab_item[blockIdx.z]
                                                                   : ps.vtab[ps.orient[blockIdx.z]]);
    if (vt) {
        // multipliers shared by every solve of this shape and T, built once per run
        const C* vbase = vt + (long long)blockIdx.y * g.ms + i0 + c;
        if (live) {
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = cmul(v[r], __ldg(vbase + (long long)(j + q * r) * g.S));
        }
    } else {
        ColSymbol<RAD> cs;
        col_symbol_init<RAD>(p, k, cs);
        apply_multiplier<RAD>(v, sm, j, q, p, cs, k[1], k[2]);
    }
    __syncthreads();
    col_fft<+1, LOG2N, CL>(v, sm, j, log2n, tw, twn_log2);
    if (live) {
#pragma unroll
        for (int r = 0; r < 16; ++r) base[(long long)(j + q * r) * g.S] = v[r];
    }
}




// ---------------------------------------------------------------------------
// 1-D real axes longer than one CTA holds (n = L/2 complex > 16 x threads):
// the packed sequence z (z[m] = a[2m] + i a[2m+1]) is viewed as an n1 x n2
// matrix, z[m1 n2 + m2]. A forward column FFT (length n1, k_cols_reg) leaves
// column m2's k1-th output at (k1, m2); this kernel multiplies it by
// w_n^{m2 k1}, transforms each row (length n2) and finds Z[k1 + n1 k2] at
// (k1, k2) -- the Multi-FFT's "transposed" order, never stored transposed.
// The real split pairs Z[k] with Z[n - k], which lies in row n1 - k1 (row 0
// and row n1/2 pair with themselves), so each CTA takes two rows of a pair,
// splits, multiplies by V = Lambda^T / N at the natural frequency k, undoes
// the split, runs the inverse row transforms and the conjugate twiddle; the
// inverse column FFT then returns a_T in natural order.
// ---------------------------------------------------------------------------

// Survivors of a 1-D row-pair thread: element r has frequency row + n1 (j + q r).
template <typename C, typename View>
__device__ __noinline__ void multiply_survivors_1d(View sm, int j, int q, unsigned mask,
                                                   const SymbolParams& p, int row, int n1) {
    using R = decltype(C{}.x);
    while (mask) {
        const int r = __ffs(mask) - 1;
        mask &= mask - 1;
        const int k[3] = {row + n1 * (j + q * r), 0, 0};
        const double2 v = cscale_rn(lambda_pow64(p, k), p.scale);
        const C V{(R)v.x, (R)v.y};
        C& e = sm[j + q * r];
        e = cmul(e, V);
    }
}

template <typename R, int RAD>
__global__ void __launch_bounds__(256)
k_fused_1d_pairs(R* __restrict__ grid, int n1_log2, int n2_log2,
                 const typename CxOf<R>::T* __restrict__ tw, int twn_log2,
                 const __grid_constant__ SymbolParams p, int* status) {
    using C = typename CxOf<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* small = reinterpret_cast<C*>(smraw);
    const int n1 = 1 << n1_log2, n2 = 1 << n2_log2;
    const int n_log2 = n1_log2 + n2_log2;
    const long long n = 1ll << n_log2;
    const int q = n2 >> 4;
    const int ss = seq_stride(n2);
    const int h = threadIdx.x / q, j = threadIdx.x - h * q;
    const int P = blockIdx.x;
    const bool selfp = P == 0;                       // rows 0 and n1/2 pair with themselves
    const int row = selfp ? (h ? n1 / 2 : 0) : (h ? n1 - P : P);
    const int prow_half = selfp ? h : 1 - h;         // half holding the partner row
    const SeqView<C> sm{small + h * ss};
    const SeqView<C> pm{small + prow_half * ss};
    C* xslot = small + 2 * ss;                       // Y[n] for the inverse split
    C* rowp = reinterpret_cast<C*>(grid) + (long long)blockIdx.y * n + (long long)row * n2;
    const int shn = twn_log2 - n_log2;               // w_n^x = tw[x << shn]
    const int sh2 = shn - 1;                         // W^k = exp(-2 pi i k / 2n) = tw[k << sh2]
    const int nmask = (int)(n - 1);
    C v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int m2 = j + q * s;
        v[s] = cmul(rowp[m2], twiddle(tw, ((m2 * row) & nmask) << shn, -1));
    }
    reg_fft<-1>(v, sm, j, n2_log2, tw, twn_log2);
#pragma unroll
    for (int r = 0; r < 16; ++r) sm[j + q * r] = v[r];
    __syncthreads();
    // partner of (row, k2): (0, (n2 - k2) mod n2) in row 0, else (n1 - row, n2 - 1 - k2)
    auto partner = [&](int k2) { return row == 0 ? ((n2 - k2) & (n2 - 1)) : (n2 - 1 - k2); };
    C xn{0, 0};
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int k2 = j + q * r;
        const int k = row + n1 * k2;
        const C zk = v[r];
        const C znk = pm[partner(k2)];
        const C xe = cscale(cadd(zk, cconj(znk)), (R)0.5);
        const C xo = cscale(cmul_mi(csub(zk, cconj(znk))), (R)0.5);
        v[r] = cadd(xe, cmul(twiddle(tw, k << sh2, -1), xo));
        if (k == 0) xn = csub(xe, xo);
    }
    __syncthreads();
    // Y[k] = V[k] X[k]
    if (p.T == 0) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = cscale(v[r], (R)p.scale);
    } else {
        ColSymbol<RAD> cs;
        int kz[3] = {0, 0, 0};
        col_symbol_init<RAD>(p, kz, cs);
        unsigned mask = 0;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const float2 l = col_lambda32<RAD>(p, cs, row + n1 * (j + q * r));
            if (l.x * l.x + l.y * l.y < p.tau2) v[r] = C{(R)0, (R)0};
            else mask |= 1u << r;
        }
        if (mask) {
#pragma unroll
            for (int r = 0; r < 16; ++r) sm[j + q * r] = v[r];
            multiply_survivors_1d<C>(sm, j, q, mask, p, row, n1);
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = mask >> r & 1 ? sm[j + q * r] : C{(R)0, (R)0};
        }
    }
    if (row == 0 && j == 0) xn = multiply_single<C>(xn, p, (int)n, 0, 0);
    __syncthreads();
    // inverse split: Z'[k] = (Y[k] + conj Y[n-k]) + i conj(W^k) (Y[k] - conj Y[n-k])
#pragma unroll
    for (int r = 0; r < 16; ++r) sm[j + q * r] = v[r];
    if (row == 0 && j == 0) *xslot = xn;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int k2 = j + q * r;
        const int k = row + n1 * k2;
        const C yk = v[r];
        const C ynk = k == 0 ? *xslot : pm[partner(k2)];
        const C wk = twiddle(tw, k << sh2, -1);
        v[r] = cadd(cadd(yk, cconj(ynk)), cmul_i(cmul(cconj(wk), csub(yk, cconj(ynk)))));
    }
    __syncthreads();
    reg_fft<+1>(v, sm, j, n2_log2, tw, twn_log2);
    bool bad = false;
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int m2 = j + q * s;
        const C x = cmul(v[s], twiddle(tw, ((m2 * row) & nmask) << shn, +1));
        bad |= !finite2(x);
        rowp[m2] = x;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, 1);
}


static int threads_for(long long elems, int max_threads) {
    long long t = (elems + kEPT - 1) / kEPT;
    t = (t + 31) / 32 * 32;
    if (t < 32) t = 32;
    if (t > max_threads) t = max_threads;
    return (int)t;
}

// Raise a kernel's dynamic shared-memory limit once per (kernel, device); later
// launches (including those recorded into a CUDA graph) make no runtime call.
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return smem_optin(reinterpret_cast<const void*>(kernel), bytes);
}

// rows per CTA of the register kernels: up to 256 threads per CTA
static int reg_rows_per_cta(int n_log2) {
    const int q = 1 << (n_log2 - 4);
    int rpc = 1;
    while (rpc * 2 * q <= 256) rpc *= 2;
    return rpc;
}

// Threads per CTA of the FP32 register column kernels (512 or 1024; the
// environment variable STENCILFFT_COL_THREADS overrides the default of 1024,
// which measured fastest: 4 columns of a 4096-point transform per CTA read
// 32-byte row segments, full sectors).
static int col_threads_cap() {
    static int cap = [] {
        const char* e = std::getenv("STENCILFFT_COL_THREADS");
        const int v = e ? std::atoi(e) : 1024;
        return v == 512 ? 512 : 1024;
    }();
    return pass_variant() == 3 ? 512 : cap;
}

// Transform lengths (log2) with compile-time specialised register kernels;
// other lengths run the runtime-length kernels (LOG2N = 0).
constexpr int kCtLo = 8, kCtHi = 13;

// Calls f(std::integral_constant<int, L>) with L = l if LO <= l <= HI, else L = 0.
template <int LO, int HI, typename F>
static cudaError_t with_log2n(int l, F&& f) {
    if constexpr (LO > HI) {
        return f(std::integral_constant<int, 0>{});
    } else {
        if (l == LO) return f(std::integral_constant<int, LO>{});
        return with_log2n<LO + 1, HI>(l, f);
    }
}

template <typename R, int RAD, int MAXT>
static cudaError_t launch_fused_1d_reg_t(R* grid, int n_log2, int nrows, const void* tw,
                                         int twn_log2, const SymbolParams& p, int* status,
                                         const RowTables& rt, cudaStream_t s) {
    using C = typename CxOf<R>::T;
    const int n = 1 << n_log2;
    const int rpc = reg_rows_per_cta(n_log2);
    const size_t smem = (size_t)rpc * seq_stride(n) * sizeof(C);
    const int threads = rpc * (n >> 4);
    cudaError_t err = set_smem(k_fused_1d_reg<R, RAD, MAXT, 0>, smem);
    if (err != cudaSuccess) return err;
    const int blocks = (nrows + rpc - 1) / rpc;
    k_fused_1d_reg<R, RAD, MAXT, 0><<<blocks, threads, smem, s>>>(
        grid, n_log2, nrows, rpc, static_cast<const C*>(tw), twn_log2, p, status, rt);
    return cudaGetLastError();
}

template <typename R, int RAD>
static cudaError_t launch_fused_1d_reg_r(R* grid, int n_log2, int nrows, const void* tw,
                                         int twn_log2, const SymbolParams& p, int* status,
                                         const RowTables& rt, cudaStream_t s) {
    if ((1 << (n_log2 - 4)) <= 256)
        return launch_fused_1d_reg_t<R, RAD, 256>(grid, n_log2, nrows, tw, twn_log2, p, status, rt,
                                                  s);
    return launch_fused_1d_reg_t<R, RAD, MaxT<R>::v>(grid, n_log2, nrows, tw, twn_log2, p, status,
                                                     rt, s);
}

template <typename R, int MAXT>
static cudaError_t launch_rows_r2c_reg(const R* grid, void* H, long long Mp, int n_log2,
                                       int nrows, const void* tw, int twn_log2, cudaStream_t s) {
    using C = typename CxOf<R>::T;
    const int n = 1 << n_log2;
    const int rpc = reg_rows_per_cta(n_log2);
    const size_t smem = (size_t)rpc * seq_stride(n) * sizeof(C);
    const dim3 blocks((nrows + rpc - 1) / rpc), threads(rpc * (n >> 4));
    return with_log2n<kCtLo, kCtHi>(n_log2, [&](auto tag) {
        constexpr int L = decltype(tag)::value;
        cudaError_t err = set_smem(k_rows_r2c_reg<R, MAXT, L>, smem);
        if (err != cudaSuccess) return err;
        k_rows_r2c_reg<R, MAXT, L><<<blocks, threads, smem, s>>>(
            grid, static_cast<C*>(H), Mp, n_log2, nrows, rpc, static_cast<const C*>(tw), twn_log2);
        return cudaGetLastError();
    });
}

template <typename R, int MAXT>
static cudaError_t launch_rows_c2r_reg(const void* H, R* grid, long long Mp, int n_log2,
                                       int nrows, const void* tw, int twn_log2, int* status,
                                       cudaStream_t s) {
    using C = typename CxOf<R>::T;
    const int n = 1 << n_log2;
    const int rpc = reg_rows_per_cta(n_log2);
    const size_t smem = (size_t)rpc * seq_stride(n) * sizeof(C);
    const dim3 blocks((nrows + rpc - 1) / rpc), threads(rpc * (n >> 4));
    return with_log2n<kCtLo, kCtHi>(n_log2, [&](auto tag) {
        constexpr int L = decltype(tag)::value;
        cudaError_t err = set_smem(k_rows_c2r_reg<R, MAXT, L>, smem);
        if (err != cudaSuccess) return err;
        k_rows_c2r_reg<R, MAXT, L><<<blocks, threads, smem, s>>>(
            static_cast<const C*>(H), grid, Mp, n_log2, nrows, rpc, static_cast<const C*>(tw),
            twn_log2, status);
        return cudaGetLastError();
    });
}

// column count (log2) of the register column kernels for MAXT threads per CTA
static int reg_cols_log2(int log2n, int elem_bytes, int maxt) {
    return ct_cols_log2(log2n, elem_bytes, maxt, kSmemBudget);
}

// The default thread cap of the column kernels for real type R.
template <typename R>
static int col_maxt() {
    return sizeof(R) == 8 ? 512 : col_threads_cap();
}

template <typename R, int DIR, int MAXT>
static cudaError_t launch_cols_reg(void* H, ColGeom g, const void* tw, int twn_log2,
                                   cudaStream_t s) {
    using C = typename CxOf<R>::T;
    const int n = 1 << g.log2n;
    g.cols_log2 = reg_cols_log2(g.log2n, sizeof(C), MAXT);
    const int cols = 1 << g.cols_log2;
    const size_t smem = (size_t)colview_elems(n, cols) * sizeof(C);
    const dim3 grid((g.inner_valid + cols - 1) / cols, g.mid, g.outer);
    const int threads = cols * (n >> 4);
    // compile-time lengths only at the default thread cap
    constexpr bool ct = MAXT == (sizeof(R) == 8 ? 512 : 1024);
    return with_log2n<kCtLo, ct ? kCtHi : 0>(g.log2n, [&](auto tag) {
        constexpr int L = decltype(tag)::value;
        constexpr int CL = L > 0 ? ct_cols_log2(L, sizeof(C), MAXT, kSmemBudget) : 0;
        cudaError_t err = set_smem(k_cols_reg<R, DIR, MAXT, L, CL>, smem);
        if (err != cudaSuccess) return err;
        k_cols_reg<R, DIR, MAXT, L, CL><<<grid, threads, smem, s>>>(
            static_cast<C*>(H), g, static_cast<const C*>(tw), twn_log2);
        return cudaGetLastError();
    });
}

template <typename R, int RAD, int MAXT, int L>
static cudaError_t launch_cols_fused_reg_t(void* H, ColGeom g, const void* tw, int twn_log2,
                                           const SymbolSet& p, cudaStream_t s) {
    using C = typename CxOf<R>::T;
    const int n = 1 << g.log2n;
    g.cols_log2 = reg_cols_log2(g.log2n, sizeof(C), MAXT);
    constexpr int CL = L > 0 ? ct_cols_log2(L, sizeof(C), MAXT, kSmemBudget) : 0;
    const int cols = 1 << g.cols_log2;
    const size_t smem = (size_t)colview_elems(n, cols) * sizeof(C);
    cudaError_t err = set_smem(k_cols_fused_reg<R, RAD, MAXT, L, CL>, smem);
    if (err != cudaSuccess) return err;
    dim3 grid((g.inner_valid + cols - 1) / cols, g.mid, g.outer);
    k_cols_fused_reg<R, RAD, MAXT, L, CL><<<grid, cols * (n >> 4), smem, s>>>(
        static_cast<C*>(H), g, static_cast<const C*>(tw), twn_log2, p);
    return cudaGetLastError();
}

// Stencil radii 1 and 2 at the default thread cap get compile-time lengths.
template <typename R, int RAD, int MAXT>
static cudaError_t launch_cols_fused_reg_m(void* H, const ColGeom& g, const void* tw,
                                           int twn_log2, const SymbolSet& p, cudaStream_t s) {
    constexpr bool ct = (RAD == 1 || RAD == 2) && MAXT == (sizeof(R) == 8 ? 512 : 1024);
    if constexpr (ct) {
        return with_log2n<kCtLo, kCtHi>(g.log2n, [&](auto tag) {
            return launch_cols_fused_reg_t<R, RAD, MAXT, decltype(tag)::value>(H, g, tw, twn_log2,
                                                                                p, s);
        });
    } else {
        return launch_cols_fused_reg_t<R, RAD, MAXT, 0>(H, g, tw, twn_log2, p, s);
    }
}

template <typename R, int RAD>
static cudaError_t launch_cols_fused_reg_r(void* H, const ColGeom& g, const void* tw,
                                           int twn_log2, const SymbolSet& p, cudaStream_t s) {
    if (col_maxt<R>() == 512) return launch_cols_fused_reg_m<R, RAD, 512>(H, g, tw, twn_log2, p, s);
    return launch_cols_fused_reg_m<R, RAD, 1024>(H, g, tw, twn_log2, p, s);
}

template <typename R>
cudaError_t launch_fused_1d(R* grid, int n_log2, int nrows, const void* tw, int twn_log2,
                            const SymbolParams& p, int* status, cudaStream_t s,
                            const RowTables* rtab) {
    using C = typename CxOf<R>::T;
    const int n = 1 << n_log2;
    RowTables rt;
    for (int i = 0; i < kMaxItems; ++i) rt.t[i] = rtab ? rtab->t[i] : nullptr;
    if (n_log2 >= 4 && (n >> 4) <= MaxT<R>::v) {
        switch (p.r) {
            case 0: return launch_fused_1d_reg_r<R, 0>(grid, n_log2, nrows, tw, twn_log2, p, status, rt, s);
            case 1: return launch_fused_1d_reg_r<R, 1>(grid, n_log2, nrows, tw, twn_log2, p, status, rt, s);
            case 2: return launch_fused_1d_reg_r<R, 2>(grid, n_log2, nrows, tw, twn_log2, p, status, rt, s);
            default: return launch_fused_1d_reg_r<R, 3>(grid, n_log2, nrows, tw, twn_log2, p, status, rt, s);
        }
    }
    if (rtab) return cudaErrorInvalidValue;   // tables need the register kernels (n >= 16)
    const int rpc = rows_per_cta_for(n_log2, sizeof(C), MaxT<R>::v);
    const size_t smem = (size_t)rpc * seq_stride(n) * sizeof(C);
    const int threads = threads_for((long long)rpc * n, MaxT<R>::v);
    cudaError_t err = set_smem(k_fused_1d<R>, smem);
    if (err != cudaSuccess) return err;
    const int blocks = (nrows + rpc - 1) / rpc;
    k_fused_1d<R><<<blocks, threads, smem, s>>>(grid, n_log2, nrows, rpc,
                                                 static_cast<const C*>(tw), twn_log2, p, status);
    return cudaGetLastError();
}

// Large 1-D axes: forward column FFT, fused row pairs, inverse column FFT
// (all in place on the grid viewed as n1 x n2 complex, `items` grids stacked).
template <typename R>
cudaError_t launch_fused_1d_pairs(R* grid, int n1_log2, int n2_log2, int items, const void* tw,
                                  int twn_log2, const SymbolParams& p, int* status,
                                  cudaStream_t s) {
    using C = typename CxOf<R>::T;
    const int n2 = 1 << n2_log2;
    if (n1_log2 < 4 || n2_log2 < 4 || n2 / 8 > 256) return cudaErrorInvalidValue;
    ColGeom g;
    g.log2n = n1_log2;
    g.S = n2;
    g.outer = items;
    g.os = (long long)n2 << n1_log2;
    g.mid = 1;
    g.ms = 0;
    g.inner_valid = n2;
    g.cols_log2 = 0;
    cudaError_t err = launch_cols<R>(grid, g, -1, tw, twn_log2, s);
    if (err != cudaSuccess) return err;
    const size_t smem = (size_t)(2 * seq_stride(n2) + 1) * sizeof(C);
    const dim3 blocks(1u << (n1_log2 - 1), items);
    const int threads = n2 / 8;
    switch (p.r) {
#define SFFT_PAIRS(RAD)                                                                            \
    case RAD:                                                                                      \
        err = set_smem(k_fused_1d_pairs<R, RAD>, smem);                                           \
        if (err != cudaSuccess) return err;                                                        \
        k_fused_1d_pairs<R, RAD><<<blocks, threads, smem, s>>>(grid, n1_log2, n2_log2,             \
                                                                static_cast<const C*>(tw),        \
                                                                twn_log2, p, status);              \
        break;
        SFFT_PAIRS(0)
        SFFT_PAIRS(1)
        SFFT_PAIRS(2)
        default:
        SFFT_PAIRS(3)
#undef SFFT_PAIRS
    }
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    return launch_cols<R>(grid, g, +1, tw, twn_log2, s);
}

template <typename R>
cudaError_t launch_rows_r2c(const R* grid, void* H, long long Mp, int n_log2, int nrows,
                            const void* tw, int twn_log2, cudaStream_t s) {
    using C = typename CxOf<R>::T;
    const int n = 1 << n_log2;
    if (n_log2 >= 4 && (n >> 4) <= MaxT<R>::v) {
        if ((n >> 4) <= 256)
            return launch_rows_r2c_reg<R, 256>(grid, H, Mp, n_log2, nrows, tw, twn_log2, s);
        return launch_rows_r2c_reg<R, MaxT<R>::v>(grid, H, Mp, n_log2, nrows, tw, twn_log2, s);
    }
    const int rpc = rows_per_cta_for(n_log2, sizeof(C), MaxT<R>::v);
    const size_t smem = (size_t)rpc * seq_stride(n) * sizeof(C);
    const int threads = threads_for((long long)rpc * n, MaxT<R>::v);
    cudaError_t err = set_smem(k_rows_r2c<R>, smem);
    if (err != cudaSuccess) return err;
    const int blocks = (nrows + rpc - 1) / rpc;
    k_rows_r2c<R><<<blocks, threads, smem, s>>>(grid, static_cast<C*>(H), Mp, n_log2, nrows, rpc,
                                                 static_cast<const C*>(tw), twn_log2);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_rows_c2r(const void* H, R* grid, long long Mp, int n_log2, int nrows,
                            const void* tw, int twn_log2, int* status, cudaStream_t s) {
    using C = typename CxOf<R>::T;
    const int n = 1 << n_log2;
    if (n_log2 >= 4 && (n >> 4) <= MaxT<R>::v) {
        if ((n >> 4) <= 256)
            return launch_rows_c2r_reg<R, 256>(H, grid, Mp, n_log2, nrows, tw, twn_log2, status, s);
        return launch_rows_c2r_reg<R, MaxT<R>::v>(H, grid, Mp, n_log2, nrows, tw, twn_log2, status,
                                                  s);
    }
    const int rpc = rows_per_cta_for(n_log2, sizeof(C), MaxT<R>::v);
    const size_t smem = (size_t)rpc * seq_stride(n) * sizeof(C);
    const int threads = threads_for((long long)rpc * n, MaxT<R>::v);
    cudaError_t err = set_smem(k_rows_c2r<R>, smem);
    if (err != cudaSuccess) return err;
    const int blocks = (nrows + rpc - 1) / rpc;
    k_rows_c2r<R><<<blocks, threads, smem, s>>>(static_cast<const C*>(H), grid, Mp, n_log2, nrows,
                                                 rpc, static_cast<const C*>(tw), twn_log2, status);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_cols(void* H, const ColGeom& g, int dir, const void* tw, int twn_log2,
                        cudaStream_t s) {
    using C = typename CxOf<R>::T;
    const int n = 1 << g.log2n;
    const int cols = 1 << g.cols_log2;
    if (g.log2n >= 4 && (n >> 4) <= MaxT<R>::v) {
        const bool small = sizeof(R) == 8 || col_threads_cap() == 512;
        if (dir < 0)
            return small ? launch_cols_reg<R, -1, 512>(H, g, tw, twn_log2, s)
                         : launch_cols_reg<R, -1, 1024>(H, g, tw, twn_log2, s);
        return small ? launch_cols_reg<R, +1, 512>(H, g, tw, twn_log2, s)
                     : launch_cols_reg<R, +1, 1024>(H, g, tw, twn_log2, s);
    }
    const size_t smem = (size_t)cols * seq_stride(n) * sizeof(C);
    const int threads = threads_for((long long)cols * n, MaxT<R>::v);
    dim3 grid((g.inner_valid + cols - 1) / cols, g.mid, g.outer);
    cudaError_t err;
    if (dir < 0) {
        err = set_smem(k_cols<R, -1>, smem);
        if (err != cudaSuccess) return err;
        k_cols<R, -1><<<grid, threads, smem, s>>>(static_cast<C*>(H), g, static_cast<const C*>(tw),
                                                   twn_log2);
    } else {
        err = set_smem(k_cols<R, +1>, smem);
        if (err != cudaSuccess) return err;
        k_cols<R, +1><<<grid, threads, smem, s>>>(static_cast<C*>(H), g, static_cast<const C*>(tw),
                                                   twn_log2);
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_cols_fused(void* H, const ColGeom& g, const void* tw, int twn_log2,
                              const SymbolSet& p, cudaStream_t s) {
    using C = typename CxOf<R>::T;
    const int n = 1 << g.log2n;
    const int cols = 1 << g.cols_log2;
    if (g.log2n >= 4 && (n >> 4) <= MaxT<R>::v) {
        switch (p.p[0].r) {
            case 0: return launch_cols_fused_reg_r<R, 0>(H, g, tw, twn_log2, p, s);
            case 1: return launch_cols_fused_reg_r<R, 1>(H, g, tw, twn_log2, p, s);
            case 2: return launch_cols_fused_reg_r<R, 2>(H, g, tw, twn_log2, p, s);
            default: return launch_cols_fused_reg_r<R, 3>(H, g, tw, twn_log2, p, s);
        }
    }
    const size_t smem = (size_t)cols * seq_stride(n) * sizeof(C);
    const int threads = threads_for((long long)cols * n, MaxT<R>::v);
    cudaError_t err = set_smem(k_cols_fused<R>, smem);
    if (err != cudaSuccess) return err;
    dim3 grid((g.inner_valid + cols - 1) / cols, g.mid, g.outer);
    k_cols_fused<R><<<grid, threads, smem, s>>>(static_cast<C*>(H), g, static_cast<const C*>(tw),
                                                 twn_log2, p);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_vtable(void* V, const SymbolParams& p, long long Mp, cudaStream_t s) {
    const int nhalf = p.len[p.ndim - 1] / 2 + 1;
    long long total = nhalf;
    for (int a = 0; a < p.ndim - 1; ++a) total *= p.len[a];
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_vtable<R><<<(int)blocks, 256, 0, s>>>(static_cast<typename CxOf<R>::T*>(V), p, nhalf, Mp,
                                            total);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_twiddles(void* tw, int twn_log2, cudaStream_t s) {
    const int n = 1 << twn_log2;
    const int threads = 256;
    const int blocks = (n + threads - 1) / threads;
    k_twiddles<R><<<blocks, threads, 0, s>>>(static_cast<typename CxOf<R>::T*>(tw), twn_log2);
    return cudaGetLastError();
}






// Explicit instantiations, in three groups so that each precision compiles as
// three translation units in parallel.
#define SFFT_INSTANTIATE_ROWS(R)                                                                   \
    template cudaError_t launch_rows_r2c<R>(const R*, void*, long long, int, int, const void*,     \
                                            int, cudaStream_t);                                    \
    template cudaError_t launch_rows_c2r<R>(const void*, R*, long long, int, int, const void*,     \
                                            int, int*, cudaStream_t);                              \
    template cudaError_t launch_twiddles<R>(void*, int, cudaStream_t);                            \
    template cudaError_t launch_vtable<R>(void*, const SymbolParams&, long long, cudaStream_t);

#define SFFT_INSTANTIATE_COLS(R)                                                                   \
    template cudaError_t launch_cols<R>(void*, const ColGeom&, int, const void*, int,              \
                                        cudaStream_t);

#define SFFT_INSTANTIATE_FUSED(R)                                                                  \
    extern template cudaError_t launch_cols<R>(void*, const ColGeom&, int, const void*, int,       \
                                               cudaStream_t);                                      \
    template cudaError_t launch_fused_1d<R>(R*, int, int, const void*, int, const SymbolParams&,   \
                                            int*, cudaStream_t, const RowTables*);                 \
    template cudaError_t launch_cols_fused<R>(void*, const ColGeom&, const void*, int,             \
                                              const SymbolSet&, cudaStream_t);                  \
    template cudaError_t launch_fused_1d_pairs<R>(R*, int, int, int, const void*, int,             \
                                                  const SymbolParams&, int*, cudaStream_t);

}  // namespace sfft
