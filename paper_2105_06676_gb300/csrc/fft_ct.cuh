// Register-resident FFT with the transform length as a compile-time constant
// (same algorithm as fft_reg.cuh: radix-R0 first stage, radix-16 Stockham
// stages, 16 elements per thread, natural order in and out; paper Sec. 4's
// Multi-FFT building block).
//
// Shared memory is addressed through a padded layout addr(p) = p * 2^SL +
// (p >> S) + c: SL = 0, S = 5 for a sequence stored alone, SL = CL, S = 4 - CL
// for column c of 2^CL interleaved sequences. For every exchange of the
// transform the element index splits as p = A(j) + B with B a compile-time
// constant and addr(A + B) = addr(A) + addr(B) exactly (checked for every
// length, layout and stage), so each access is a per-thread base plus an
// immediate offset.
#pragma once

#include "fft_common.cuh"
#include "fft_reg.cuh"

namespace sfft {

template <int SL, int S>
struct PadLayout {
    static __host__ __device__ constexpr int off(int p) { return (p << SL) + (p >> S); }
};

// Exchange through shared memory: thread j writes v[r] at element wbase + wstep(r)
// and reads back elements j + q s into v[s].
template <int SL, int S, int LOG2N, typename C>
__device__ __forceinline__ void ct_read(C* v, const C* sm, int j) {
    using L = PadLayout<SL, S>;
    constexpr int q = (1 << LOG2N) >> 4;
    const C* rd = sm + L::off(j);
#pragma unroll
    for (int s = 0; s < 16; ++s) v[s] = rd[L::off(q * s)];
}

// Radix-16 stages from sub-transform length 2^NSL up to n.
template <int DIR, int LOG2N, int NSL, int SL, int S, typename C>
__device__ __forceinline__ void ct_stages(C* v, C* sm, int j, const C* __restrict__ tw,
                                          int twn_log2) {
    if constexpr (NSL < LOG2N) {
        using L = PadLayout<SL, S>;
        constexpr int Ns = 1 << NSL;
        const int k = j & (Ns - 1);
        // twiddle by w_{16 Ns}^{k s}, then the radix-16 butterfly
        reg_twiddle<DIR>(v, k, twn_log2 - NSL - 4, tw);
        dft_reg<16, DIR>(v);
        if constexpr (NSL + 4 < LOG2N) {
            // output r of butterfly j goes to (j - k) 16 + k + Ns r
            C* w = sm + L::off((j - k) * 16 + k);
#pragma unroll
            for (int r = 0; r < 16; ++r) w[L::off(Ns * r)] = v[r];
            __syncthreads();
            ct_read<SL, S, LOG2N>(v, sm, j);
            __syncthreads();
            ct_stages<DIR, LOG2N, NSL + 4, SL, S>(v, sm, j, tw, twn_log2);
        }
    }
}

template <int DIR, int LOG2N, int SL, int S, typename C>
__device__ __forceinline__ void ct_fft(C* v, C* sm, int j, const C* __restrict__ tw, int twn_log2) {
    using L = PadLayout<SL, S>;
    constexpr int n = 1 << LOG2N;
    constexpr int q = n >> 4;
    constexpr int r0log = (LOG2N & 3) ? (LOG2N & 3) : 4;
    constexpr int R0 = 1 << r0log;
    constexpr int G = 16 / R0;
    reg_first_stage<R0, DIR>(v);
    if constexpr (R0 < n) {
        // output r of first-stage butterfly j + q t goes to (j + q t) R0 + r
        C* w = sm + L::off(j * R0);
#pragma unroll
        for (int t = 0; t < G; ++t)
#pragma unroll
            for (int r = 0; r < R0; ++r) w[L::off(q * t * R0 + r)] = v[t * R0 + r];
        __syncthreads();
        ct_read<SL, S, LOG2N>(v, sm, j);
        __syncthreads();
        ct_stages<DIR, LOG2N, r0log, SL, S>(v, sm, j, tw, twn_log2);
    }
}

// Interleaved-column layout constants for 2^CL columns: SL = CL, S = 4 - CL.
template <int CL>
struct ColLayout {
    static constexpr int SL = CL;
    static constexpr int S = 4 - CL;
};

// Columns per CTA (log2) of the compile-time column kernels: as many as fit
// MAXT threads and the shared-memory budget, at most 16.
__host__ __device__ constexpr int ct_cols_log2(int log2n, int elem_bytes, int maxt, int budget) {
    int cl = 0;
    while (cl < 4 && ((2 << cl) * (1 << (log2n - 4))) <= maxt &&
           (long long)((1 << log2n) * (2 << cl) + (((1 << log2n) * (2 << cl)) >> 4) + 1) * elem_bytes <=
               budget)
        ++cl;
    return cl;
}

}  // namespace sfft
