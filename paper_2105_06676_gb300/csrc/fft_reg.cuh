// Register-resident FFT of length n = 2^log2n >= 16 (paper Sec. 4's Multi-FFT
// building block; convention F[i,j] = w^(-ij), inverse w^(+ij), unscaled).
//
// Each sequence is handled by q = n/16 threads; thread j holds 16 elements.
// On entry v[s] = x[j + q s] (s = 0..15), the layout a coalesced global load of
// a contiguous row produces. The transform is a Stockham decimation in time
// with a radix-R0 first stage (R0 = 2^(log2n mod 4), or 16) and radix-16
// stages after it; between stages the data moves through the sequence's
// shared-memory buffer (one write, one read). On exit v[r] = X[j + q r]: natural
// frequency order with the same stride, so the last forward stage and the first
// inverse stage of a forward-multiply-inverse pass meet in registers.
//
// Twiddles: the FP64-built table tw[m] = exp(-2 pi i m / 2^twn_log2). FP32
// passes load w^k, w^(4k), w^(8k), w^(12k) and form the other powers by at most
// three complex products; FP64 passes load every power (FP64 arithmetic is the
// scarce resource there).
#pragma once

#include "fft_common.cuh"

namespace sfft {

// Shared-memory views of one sequence.
//   SeqView : a sequence stored alone, element p at p + p/32.
//   ColView : sequence c of `cols` column-interleaved sequences, element p at
//             f + f/16 with f = p*cols + c. Lanes that differ in c then hit
//             neighbouring banks, so the column kernels (lanes ordered column
//             first, for coalesced global access) exchange without conflicts.
template <typename C>
struct SeqView {
    C* base;
    __device__ __forceinline__ C& operator[](int p) const { return base[p + (p >> 5)]; }
};
template <typename C>
struct ColView {
    C* base;
    int c, cl;
    __device__ __forceinline__ C& operator[](int p) const {
        const int f = (p << cl) + c;
        return base[f + (f >> 4)];
    }
};
// Elements of shared memory needed by `cols` interleaved sequences of length n.
__host__ __device__ __forceinline__ int colview_elems(int n, int cols) {
    return n * cols + (n * cols >> 4) + 1;
}

// v[t*R0 + r] <- output r of the radix-R0 butterfly over v[t + (16/R0) r].
template <int R0, int DIR, typename C>
__device__ __forceinline__ void reg_first_stage(C* v) {
    constexpr int G = 16 / R0;
    C out[16];
#pragma unroll
    for (int t = 0; t < G; ++t) {
        C sub[R0];
#pragma unroll
        for (int r = 0; r < R0; ++r) sub[r] = v[t + G * r];
        dft_reg<R0, DIR>(sub);
#pragma unroll
        for (int r = 0; r < R0; ++r) out[t * R0 + r] = sub[r];
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = out[i];
}

// v[s] *= w^(k s) for s = 1..15, w = exp(DIR 2 pi i / L), L = 2^twn_log2 >> sh.
template <int DIR, typename C>
__device__ __forceinline__ void reg_twiddle(C* v, int k, int sh, const C* __restrict__ tw) {
    if (k == 0) return;
    if constexpr (sizeof(C) == 8) {
        // FP32: two table loads (w^k, w^4k), the rest by products (<= 3
        // roundings deep); the loads of w^8k and w^12k would touch a sector per
        // lane for the strided k of the last stages
        const C w1 = twiddle(tw, k << sh, DIR);
        const C w4 = twiddle(tw, (4 * k) << sh, DIR);
        const C w8 = cmul(w4, w4);
        const C w12 = cmul(w8, w4);
        const C w2 = cmul(w1, w1);
        const C w3 = cmul(w2, w1);
        const C base[4] = {C{1, 0}, w4, w8, w12};
#pragma unroll
        for (int s = 1; s < 16; ++s) {
            const int hi = s >> 2, lo = s & 3;
            C w;
            if (lo == 0) w = base[hi];
            else if (hi == 0) w = lo == 1 ? w1 : lo == 2 ? w2 : w3;
            else w = cmul(base[hi], lo == 1 ? w1 : lo == 2 ? w2 : w3);
            v[s] = cmul(v[s], w);
        }
    } else {
#pragma unroll
        for (int s = 1; s < 16; ++s) v[s] = cmul(v[s], twiddle(tw, (k * s) << sh, DIR));
    }
}

// Forward (DIR = -1) or inverse (+1) FFT of one sequence held as described
// above. sm is this sequence's shared-memory view; every
// thread of the CTA must call this together (it contains barriers); j is the
// thread's index within its sequence (0 <= j < n/16).
template <int DIR, typename C, typename View>
__device__ __forceinline__ void reg_fft(C* v, const View& sm, int j, int log2n,
                                        const C* __restrict__ tw, int twn_log2) {
    const int n = 1 << log2n;
    const int q = n >> 4;
    const int r0log = (log2n & 3) ? (log2n & 3) : 4;
    const int R0 = 1 << r0log;
    switch (r0log) {
        case 1: reg_first_stage<2, DIR>(v); break;
        case 2: reg_first_stage<4, DIR>(v); break;
        case 3: reg_first_stage<8, DIR>(v); break;
        default: reg_first_stage<16, DIR>(v); break;
    }
    int Ns = R0;
    int prev_first = 1;
    while (Ns < n) {
        // write the previous stage's outputs to their Stockham positions
        if (prev_first) {
            const int G = 16 >> r0log;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int t = i >> r0log;        // i = t*R0 + r
                const int r = i & (R0 - 1);
                if (t < G) sm[(j + q * t) * R0 + r] = v[i];
            }
        } else {
            const int pN = Ns >> 4;
            const int k = j & (pN - 1);
            const int d0 = (j - k) * 16 + k;
#pragma unroll
            for (int r = 0; r < 16; ++r) sm[d0 + pN * r] = v[r];
        }
        prev_first = 0;
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 16; ++s) v[s] = sm[j + q * s];
        __syncthreads();
        // twiddle by w_{16 Ns}^{k s}, then the radix-16 butterfly
        const int k = j & (Ns - 1);
        const int ns_log2 = __ffs(Ns) - 1;
        reg_twiddle<DIR>(v, k, twn_log2 - ns_log2 - 4, tw);
        dft_reg<16, DIR>(v);
        Ns <<= 4;
    }
}

}  // namespace sfft
