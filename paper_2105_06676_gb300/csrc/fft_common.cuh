// Device building blocks of the FFT stencil solver: complex arithmetic, radix
// 2..16 DFTs in registers, and radix-16 Stockham stages over shared memory.
//
// The FFT convention is the paper's (Sec. 4, "Reformulating the Final Data"):
// forward F[i,j] = w^(-ij), inverse w^(+ij), w = exp(2 pi i / n), no scaling in
// either direction; the solver folds the inverse's 1/N into the spectral
// multiplier.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sfft {

template <typename R> struct CxOf;
template <> struct CxOf<float> { using T = float2; };
template <> struct CxOf<double> { using T = double2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { return C{a.x * s, a.y * s}; }
// a * (+i)
template <typename C> __device__ __forceinline__ C cmul_i(C a) { return C{-a.y, a.x}; }
// a * (-i)
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { return C{a.y, -a.x}; }

// cos(2 pi q / 16) for integer q: exact mathematical constants.
__host__ __device__ constexpr double cos16(int q) {
    constexpr double c1 = 0.92387953251128675613;  // cos(pi/8)
    constexpr double c2 = 0.70710678118654752440;  // cos(pi/4)
    constexpr double c3 = 0.38268343236508977173;  // cos(3pi/8)
    q = ((q % 16) + 16) % 16;
    return q == 0 ? 1.0 : q == 1 ? c1 : q == 2 ? c2 : q == 3 ? c3 : q == 4 ? 0.0
         : q == 5 ? -c3 : q == 6 ? -c2 : q == 7 ? -c1 : q == 8 ? -1.0
         : q == 9 ? -c1 : q == 10 ? -c2 : q == 11 ? -c3 : q == 12 ? 0.0
         : q == 13 ? c3 : q == 14 ? c2 : c1;
}
__host__ __device__ constexpr double sin16(int q) { return cos16(q - 4); }

// a * exp(DIR * 2 pi i q / 16); DIR = -1 forward, +1 inverse. q is a
// compile-time constant after unrolling, so the special cases fold away.
template <int DIR, typename C>
__device__ __forceinline__ C rot16(C a, int q) {
    using R = decltype(a.x);
    q &= 15;
    if (q == 0) return a;
    if (q == 8) return C{-a.x, -a.y};
    if (q == 4) return DIR < 0 ? cmul_mi(a) : cmul_i(a);
    if (q == 12) return DIR < 0 ? cmul_i(a) : cmul_mi(a);
    const R c = (R)cos16(q);
    const R s = (R)(DIR * sin16(q));
    return C{a.x * c - a.y * s, a.x * s + a.y * c};
}

// In-register DFT of size R (power of two, <= 16), natural order in and out:
// v[k] <- sum_j v[j] exp(DIR 2 pi i jk / R). Radix-2 decimation in time.
template <int R, int DIR, typename C>
__device__ __forceinline__ void dft_reg(C* v) {
    if constexpr (R == 1) {
        return;
    } else if constexpr (R == 2) {
        const C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else {
        C e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        dft_reg<R / 2, DIR>(e);
        dft_reg<R / 2, DIR>(o);
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            const C t = rot16<DIR>(o[k], k * (16 / R));
            v[k] = cadd(e[k], t);
            v[k + R / 2] = csub(e[k], t);
        }
    }
}

// Shared-memory element index with one pad slot every 32 elements, which
// spreads the stride-R stores of the early Stockham stages over the banks.
__device__ __forceinline__ int spad(int p) { return p + (p >> 5); }
// Distance between consecutive sequences in shared memory (odd, so that
// element p of neighbouring sequences lands on different banks).
__host__ __device__ __forceinline__ int seq_stride(int n) { return n + (n >> 5) + 1; }

// Twiddle table: tw[m] = exp(-2 pi i m / TWN), m in [0, TWN), computed with
// FP64 sincospi and stored at pass precision. TWN is the largest transform
// length the plan needs (a power of two).
template <typename C>
__device__ __forceinline__ C twiddle(const C* __restrict__ tw, int m, int dir) {
    C w = __ldg(tw + m);
    if (dir > 0) w.y = -w.y;
    return w;
}

// One radix-R Stockham stage (decimation in time, autosort) over `cols`
// sequences of length n held in shared memory. Ns is the length of the
// sub-transforms already combined (1, R0, R0*16, ...). The R inputs of
// butterfly j sit at j + r*n/R, the outputs go to (j/Ns)*Ns*R + j%Ns + r*Ns,
// and input r is first turned by exp(DIR 2 pi i (j%Ns) r / (Ns R)).
// Every thread loads all of its butterflies into registers before the barrier
// and stores them after it, so the stage runs in place in one buffer.
template <int R, int DIR, int EPT, typename C>
__device__ __forceinline__ void stockham_stage(C* sm, int n, int Ns, int cols, int sstride,
                                               const C* __restrict__ tw, int twn_log2,
                                               int log2n) {
    constexpr int BPT = EPT / R;
    const int nb_log2 = log2n - (R == 16 ? 4 : R == 8 ? 3 : R == 4 ? 2 : 1);
    const int nb = 1 << nb_log2;
    const int total = cols * nb;
    // twiddle step in table units: TWN / (Ns * R)
    const int ns_log2 = __ffs(Ns) - 1;
    const int step_log2 = twn_log2 - ns_log2 - (R == 16 ? 4 : R == 8 ? 3 : R == 4 ? 2 : 1);
    C v[EPT];
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int g = threadIdx.x + b * blockDim.x;
        if (g < total) {
            const int c = g >> nb_log2;
            const int j = g & (nb - 1);
            const int k = j & (Ns - 1);
            const C* src = sm + c * sstride;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                C x = src[spad(j + r * nb)];
                if (r > 0 && Ns > 1) {
                    const C w = twiddle(tw, (k * r) << step_log2, DIR);
                    x = cmul(x, w);
                }
                v[b * R + r] = x;
            }
            dft_reg<R, DIR>(v + b * R);
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int g = threadIdx.x + b * blockDim.x;
        if (g < total) {
            const int c = g >> nb_log2;
            const int j = g & (nb - 1);
            const int k = j & (Ns - 1);
            const int d0 = ((j - k) * R) + k;
            C* dst = sm + c * sstride;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[spad(d0 + r * Ns)] = v[b * R + r];
        }
    }
    __syncthreads();
}

// Full in-place FFT of `cols` sequences of length n = 2^log2n (n >= 2) in
// shared memory; natural order in and out. One radix-2/4/8 stage first when
// log2n is not a multiple of 4, then radix-16 stages. EPT >= 16 elements per
// thread and cols * n <= EPT * blockDim.x. Ends with a barrier.
template <int DIR, int EPT, typename C>
__device__ __forceinline__ void fft_smem(C* sm, int log2n, int cols, const C* __restrict__ tw,
                                         int twn_log2) {
    const int n = 1 << log2n;
    const int ss = seq_stride(n);
    int Ns = 1;
    const int rem = log2n & 3;
    if (rem == 1) {
        stockham_stage<2, DIR, EPT>(sm, n, Ns, cols, ss, tw, twn_log2, log2n);
        Ns = 2;
    } else if (rem == 2) {
        stockham_stage<4, DIR, EPT>(sm, n, Ns, cols, ss, tw, twn_log2, log2n);
        Ns = 4;
    } else if (rem == 3) {
        stockham_stage<8, DIR, EPT>(sm, n, Ns, cols, ss, tw, twn_log2, log2n);
        Ns = 8;
    }
    for (; Ns < n; Ns <<= 4) stockham_stage<16, DIR, EPT>(sm, n, Ns, cols, ss, tw, twn_log2, log2n);
}

}  // namespace sfft
