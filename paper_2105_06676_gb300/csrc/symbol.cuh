// Spectral multiplier of StencilFFT-P: V[k] = Lambda[k]^T / N, evaluated on the
// GPU per spectral element (paper Sec. 4, Steps 1 (i) and 2; Fig.
// "stencil-fft-algorithm-dD").
//
// Lambda[k] = (F s)[k] with s the first column of S (appendix "Proof of
// Eigenvalue-FFT Relation"); with s[(-m) mod l] = w[m] and the unnormalised
// forward DFT this is
//     Lambda[k] = sum_m w[m] exp(+2 pi i sum_a m_a k_a / l_a),
// evaluated separably from per-axis FP64 tables E_a[q] = exp(2 pi i q / l_a)
// (built with FP64 sincospi). Lambda^T is taken by repeated squaring over the
// bits of T in FP64 (Sec. 4, "Step 2"), then scaled by 1/N (the inverse DFT's
// normalisation, Sec. 4) and rounded once to the pass precision.
//
// Underflow shortcut: a FP32 evaluation of Lambda plus a rigorous bound delta on
// its error gives an upper bound B >= |Lambda|. When T log2 B is below the
// cut, |Lambda^T / N| is below half the smallest subnormal of the output
// precision, so the FP64 result would round to exactly 0; the element is set to
// 0 without the FP64 work. This changes no output bit.
#pragma once

#include "fft_common.cuh"

namespace sfft {

constexpr int kMaxRadius = 3;
constexpr int kMaxWeights = (2 * kMaxRadius + 1) * (2 * kMaxRadius + 1) * (2 * kMaxRadius + 1);

struct SymbolParams {
    int ndim;
    int r;
    long long T;
    double scale;          // 1 / N
    int real_symbol;       // weights symmetric under m -> -m: Lambda is real
    int use_cut;
    float delta;           // bound on |Lambda - Lambda_fp32|
    float cut;             // skip when T log2(|Lambda_fp32| + delta) < -cut
    int len[3];            // axis lengths l_a of the solved box (full length of the halved last axis)
    int tshift[3];         // tables hold exp(2 pi i q / (l_a << tshift)): index scale of this box
    int tmask[3];          // l_a - 1
    const double2* E64[3];
    const float2* E32[3];
    double w[kMaxWeights];
    float w32[kMaxWeights];
};

// sum_m w[m] prod_a E_a[(m_a k_a) mod l_a], separably; k[a] in [0, l_a).
// RAD is the stencil radius as a compile-time constant so the phase factors
// stay in registers.
template <int RAD, typename R, typename C>
__device__ __forceinline__ C lambda_eval_r(const SymbolParams& p, const C* const* E, const R* w,
                                           const int* k) {
    constexpr int W = 2 * RAD + 1;
    C e0[W], e1[W], e2[W];
#pragma unroll
    for (int m = -RAD; m <= RAD; ++m) e0[m + RAD] = __ldg(E[0] + (((m * k[0]) & p.tmask[0]) << p.tshift[0]));
    if (p.ndim == 1) {
        C acc{0, 0};
#pragma unroll
        for (int i = 0; i < W; ++i) acc = cadd(acc, cscale(e0[i], w[i]));
        return acc;
    }
#pragma unroll
    for (int m = -RAD; m <= RAD; ++m) e1[m + RAD] = __ldg(E[1] + (((m * k[1]) & p.tmask[1]) << p.tshift[1]));
    if (p.ndim == 2) {
        C acc{0, 0};
#pragma unroll
        for (int i = 0; i < W; ++i) {
            C inner{0, 0};
#pragma unroll
            for (int j = 0; j < W; ++j) inner = cadd(inner, cscale(e1[j], w[i * W + j]));
            acc = cadd(acc, cmul(e0[i], inner));
        }
        return acc;
    }
#pragma unroll
    for (int m = -RAD; m <= RAD; ++m) e2[m + RAD] = __ldg(E[2] + (((m * k[2]) & p.tmask[2]) << p.tshift[2]));
    C acc{0, 0};
#pragma unroll
    for (int i = 0; i < W; ++i) {
        C mid{0, 0};
#pragma unroll
        for (int j = 0; j < W; ++j) {
            C inner{0, 0};
#pragma unroll
            for (int q = 0; q < W; ++q) inner = cadd(inner, cscale(e2[q], w[(i * W + j) * W + q]));
            mid = cadd(mid, cmul(e1[j], inner));
        }
        acc = cadd(acc, cmul(e0[i], mid));
    }
    return acc;
}

template <typename R, typename C>
__device__ __forceinline__ C lambda_eval(const SymbolParams& p, const C* const* E, const R* w,
                                         const int* k) {
    switch (p.r) {
        case 0: return lambda_eval_r<0, R, C>(p, E, w, k);
        case 1: return lambda_eval_r<1, R, C>(p, E, w, k);
        case 2: return lambda_eval_r<2, R, C>(p, E, w, k);
        default: return lambda_eval_r<3, R, C>(p, E, w, k);
    }
}

// z^T by repeated squaring over the bits of T (T >= 0).
__device__ __forceinline__ double2 cpow_sq(double2 z, long long T) {
    double2 v{1.0, 0.0};
    double2 s = z;
    while (T > 0) {
        if (T & 1) v = cmul(v, s);
        T >>= 1;
        if (T > 0) s = cmul(s, s);
    }
    return v;
}
__device__ __forceinline__ double rpow_sq(double x, long long T) {
    double v = 1.0, s = x;
    while (T > 0) {
        if (T & 1) v *= s;
        T >>= 1;
        if (T > 0) s *= s;
    }
    return v;
}

// Lambda[k]^T in FP64 (no scale, no shortcut).
static __device__ __noinline__ double2 lambda_pow64(const SymbolParams& p, const int* k) {
    const double2 lam = lambda_eval<double, double2>(p, p.E64, p.w, k);
    if (p.real_symbol) return double2{rpow_sq(lam.x, p.T), 0.0};
    return cpow_sq(lam, p.T);
}

// V[k] = Lambda[k]^T / N rounded to the pass precision (with the exact
// underflow shortcut).
template <typename C>
__device__ __forceinline__ C spectral_multiplier(const SymbolParams& p, const int* k) {
    using R = decltype(C{}.x);
    if (p.T == 0) return C{(R)p.scale, (R)0};
    if (p.use_cut) {
        const float2 l32 = lambda_eval<float, float2>(p, p.E32, p.w32, k);
        const float bound = hypotf(l32.x, l32.y) + p.delta;
        if (bound < 1.0f) {
            const float lg = (float)p.T * log2f(bound);
            if (lg < -p.cut) return C{(R)0, (R)0};
        }
    }
    const double2 v = lambda_pow64(p, k);
    return C{(R)(v.x * p.scale), (R)(v.y * p.scale)};
}

}  // namespace sfft
