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
    float tau2;            // same test as |Lambda_fp32|^2 < tau2, tau = 2^(-cut/T) - delta
                           // (with a relative margin for the rounding of the square);
                           // negative when no element can be skipped
    int len[3];            // axis lengths l_a of the solved box (full length of the halved last axis)
    int tshift[3];         // tables hold exp(2 pi i q / (l_a << tshift)): index scale of this box
    int tmask[3];          // l_a - 1, or -1 for a length that is not a power of two (modulo)
    const double2* E64[3];
    const float2* E32[3];
    double w[kMaxWeights];
    float w32[kMaxWeights];
    // implicit stencils Q a_{t+1} = S a_t (w holds S): Q's weights in device
    // memory (null for explicit stencils) and the magnitude at or below which
    // Lambda_Q counts as zero
    const double* wq;
    double qzero;
};

// Table index of exp(2 pi i (m k mod l_a) / l_a) along axis a.
__device__ __forceinline__ int axis_index(const SymbolParams& p, int a, int mk) {
    if (p.tmask[a] >= 0) return (mk & p.tmask[a]) << p.tshift[a];
    const int v = mk % p.len[a];
    return v < 0 ? v + p.len[a] : v;
}

// Symbol parameters for a batch of boxes solved by one launch: up to
// kMaxOrient orientations (box axes mapped to grid axes by a permutation) and
// the orientation of each batch item.
constexpr int kMaxOrient = 3;
constexpr int kMaxItems = 8;
struct SymbolSet {
    SymbolParams p[kMaxOrient];
    int orient[kMaxItems];
    // optional precomputed multipliers V = Lambda^T / N per orientation, laid
    // out like one item's half spectrum (null: evaluate on the fly)
    const void* vtab[kMaxOrient];
    // optional per-item tables (each item its own weights and T); override vtab
    const void* vtab_item[kMaxItems];
    // set when vtab[0] is a blocked-layout table (FP32 2-D, one item): one flag
    // per column block, 0 when every multiplier of the block is zero
    const int* vflags;
};

// Per-row multiplier tables of a batched 1-D solve (row r uses t[r] when set).
struct RowTables {
    const void* t[kMaxItems];
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
    for (int m = -RAD; m <= RAD; ++m) e0[m + RAD] = __ldg(E[0] + axis_index(p, 0, m * k[0]));
    if (p.ndim == 1) {
        C acc{0, 0};
#pragma unroll
        for (int i = 0; i < W; ++i) acc = cadd(acc, cscale(e0[i], w[i]));
        return acc;
    }
#pragma unroll
    for (int m = -RAD; m <= RAD; ++m) e1[m + RAD] = __ldg(E[1] + axis_index(p, 1, m * k[1]));
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
    for (int m = -RAD; m <= RAD; ++m) e2[m + RAD] = __ldg(E[2] + axis_index(p, 2, m * k[2]));
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

// FP64 complex arithmetic with every rounding spelled out (no contraction left
// to the compiler), so that every kernel that evaluates a multiplier -- inside a
// pass or into a table -- produces the same bits.
__device__ __forceinline__ double2 cmul_rn(double2 a, double2 b) {
    return double2{__fma_rn(a.x, b.x, -__dmul_rn(a.y, b.y)), __fma_rn(a.x, b.y, __dmul_rn(a.y, b.x))};
}
__device__ __forceinline__ double2 cadd_rn(double2 a, double2 b) {
    return double2{__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)};
}
__device__ __forceinline__ double2 cscale_rn(double2 a, double s) {
    return double2{__dmul_rn(a.x, s), __dmul_rn(a.y, s)};
}

// z^T by repeated squaring over the bits of T (T >= 0).
__device__ __forceinline__ double2 cpow_sq(double2 z, long long T) {
    double2 v{1.0, 0.0};
    double2 s = z;
    while (T > 0) {
        if (T & 1) v = cmul_rn(v, s);
        T >>= 1;
        if (T > 0) s = cmul_rn(s, s);
    }
    return v;
}
__device__ __forceinline__ double rpow_sq(double x, long long T) {
    double v = 1.0, s = x;
    while (T > 0) {
        if (T & 1) v = __dmul_rn(v, s);
        T >>= 1;
        if (T > 0) s = __dmul_rn(s, s);
    }
    return v;
}

// FP64 factorisation of Lambda along axis 0 for fixed k_1, k_2:
// G64[m_0] = sum_{m_1..} w[m_0, m_1, ..] prod_{a >= 1} E64_a[m_a k_a], so that
// Lambda(k) = sum_{m_0} E64_0[m_0 k_0] G64[m_0]. A column pass forms it once
// per thread and reuses it for every element of the column it evaluates.
template <int RAD>
struct ColSymbol64 {
    double2 g[2 * RAD + 1];
};

template <int RAD>
__device__ __forceinline__ void col_symbol_init64(const SymbolParams& p, const double* w, int k1,
                                                  int k2, ColSymbol64<RAD>& cs) {
    constexpr int W = 2 * RAD + 1;
    if (p.ndim == 1) {
#pragma unroll
        for (int i = 0; i < W; ++i) cs.g[i] = double2{w[i], 0.0};
        return;
    }
    double2 e1[W];
#pragma unroll
    for (int m = -RAD; m <= RAD; ++m)
        e1[m + RAD] = __ldg(p.E64[1] + axis_index(p, 1, m * k1));
    if (p.ndim == 2) {
#pragma unroll
        for (int i = 0; i < W; ++i) {
            double2 inner{0.0, 0.0};
#pragma unroll
            for (int jj = 0; jj < W; ++jj) inner = cadd_rn(inner, cscale_rn(e1[jj], w[i * W + jj]));
            cs.g[i] = inner;
        }
        return;
    }
    double2 e2[W];
#pragma unroll
    for (int m = -RAD; m <= RAD; ++m)
        e2[m + RAD] = __ldg(p.E64[2] + axis_index(p, 2, m * k2));
#pragma unroll
    for (int i = 0; i < W; ++i) {
        double2 mid{0.0, 0.0};
#pragma unroll
        for (int jj = 0; jj < W; ++jj) {
            double2 inner{0.0, 0.0};
#pragma unroll
            for (int qq = 0; qq < W; ++qq)
                inner = cadd_rn(inner, cscale_rn(e2[qq], w[(i * W + jj) * W + qq]));
            mid = cadd_rn(mid, cmul_rn(e1[jj], inner));
        }
        cs.g[i] = mid;
    }
}

// Lambda at k_0 for the column of cs, in FP64.
template <int RAD>
__device__ __forceinline__ double2 col_lambda64(const SymbolParams& p, const ColSymbol64<RAD>& cs,
                                                int k0) {
    double2 lam{0.0, 0.0};
#pragma unroll
    for (int i = 0; i < 2 * RAD + 1; ++i) {
        const int m = i - RAD;
        const double2 e = __ldg(p.E64[0] + axis_index(p, 0, m * k0));
        lam = cadd_rn(lam, cmul_rn(e, cs.g[i]));
    }
    return lam;
}

// Lambda^T (real when the weights are symmetric: only the real part is kept).
__device__ __forceinline__ double2 symbol_pow64(const SymbolParams& p, double2 lam) {
    if (p.real_symbol) return double2{rpow_sq(lam.x, p.T), 0.0};
    return cpow_sq(lam, p.T);
}

// Lambda_R = Lambda_Q^+ Lambda_S of an implicit stencil at one frequency
// (appendix "Supporting Implicit Stencils": the pseudoinverse is 1 / Lambda_Q
// where Lambda_Q is not zero, 0 where it is).
__device__ __forceinline__ double2 implicit_ratio(const SymbolParams& p, double2 ls, double2 lq) {
    const double q2 = __fma_rn(lq.x, lq.x, __dmul_rn(lq.y, lq.y));
    if (q2 <= __dmul_rn(p.qzero, p.qzero)) return double2{0.0, 0.0};
    if (p.real_symbol) return double2{__ddiv_rn(ls.x, lq.x), 0.0};
    // ls conj(lq) / |lq|^2
    const double2 num = cmul_rn(ls, double2{lq.x, -lq.y});
    return double2{__ddiv_rn(num.x, q2), __ddiv_rn(num.y, q2)};
}

// V[k] = Lambda[k]^T / N in FP64 for the column of cs at k_0 (explicit stencils).
template <int RAD>
__device__ __forceinline__ double2 col_power64(const SymbolParams& p, const ColSymbol64<RAD>& cs,
                                               int k0) {
    return cscale_rn(symbol_pow64(p, col_lambda64<RAD>(p, cs, k0)), p.scale);
}

template <int RAD>
__device__ __forceinline__ double2 lambda_pow64_r(const SymbolParams& p, const int* k) {
    ColSymbol64<RAD> cs;
    col_symbol_init64<RAD>(p, p.w, k[1], k[2], cs);
    double2 lam = col_lambda64<RAD>(p, cs, k[0]);
    if (p.wq) {
        ColSymbol64<RAD> cq;
        col_symbol_init64<RAD>(p, p.wq, k[1], k[2], cq);
        lam = implicit_ratio(p, lam, col_lambda64<RAD>(p, cq, k[0]));
    }
    return symbol_pow64(p, lam);
}

// Lambda[k]^T in FP64 (no scale, no shortcut); Lambda_R^T for implicit stencils.
static __device__ __noinline__ double2 lambda_pow64(const SymbolParams& p, const int* k) {
    switch (p.r) {
        case 0: return lambda_pow64_r<0>(p, k);
        case 1: return lambda_pow64_r<1>(p, k);
        case 2: return lambda_pow64_r<2>(p, k);
        default: return lambda_pow64_r<3>(p, k);
    }
}

// V[k] = Lambda[k]^T / N rounded to the pass precision (with the exact
// underflow shortcut).
template <typename C>
__device__ __forceinline__ C spectral_multiplier(const SymbolParams& p, const int* k) {
    using R = decltype(C{}.x);
    if (p.T == 0) return C{(R)p.scale, (R)0};
    if (p.use_cut && !p.wq) {
        const float2 l32 = lambda_eval<float, float2>(p, p.E32, p.w32, k);
        const float bound = hypotf(l32.x, l32.y) + p.delta;
        if (bound < 1.0f) {
            const float lg = (float)p.T * log2f(bound);
            if (lg < -p.cut) return C{(R)0, (R)0};
        }
    }
    const double2 v = cscale_rn(lambda_pow64(p, k), p.scale);
    return C{(R)v.x, (R)v.y};
}

// Per-column part of Lambda for a pass along axis 0: with k_0 the transform
// index and k_1.. fixed for the column,
//   Lambda(k) = sum_{m_0} E_0[m_0 k_0] G[m_0],
//   G[m_0]    = sum_{m_1..} w[m_0, m_1, ..] prod_{a >= 1} E_a[m_a k_a]      (FP32).
template <int RAD>
struct ColSymbol {
    float2 g[2 * RAD + 1];
};

template <int RAD>
__device__ __forceinline__ void col_symbol_init(const SymbolParams& p, const int* k,
                                                ColSymbol<RAD>& cs) {
    constexpr int W = 2 * RAD + 1;
    if (p.ndim == 1) {
#pragma unroll
        for (int i = 0; i < W; ++i) cs.g[i] = float2{p.w32[i], 0.f};
        return;
    }
    float2 e1[W], e2[W];
#pragma unroll
    for (int m = -RAD; m <= RAD; ++m)
        e1[m + RAD] = __ldg(p.E32[1] + (((m * k[1]) & p.tmask[1]) << p.tshift[1]));
    if (p.ndim == 2) {
#pragma unroll
        for (int i = 0; i < W; ++i) {
            float2 acc{0.f, 0.f};
#pragma unroll
            for (int jj = 0; jj < W; ++jj) acc = cadd(acc, cscale(e1[jj], p.w32[i * W + jj]));
            cs.g[i] = acc;
        }
        return;
    }
#pragma unroll
    for (int m = -RAD; m <= RAD; ++m)
        e2[m + RAD] = __ldg(p.E32[2] + (((m * k[2]) & p.tmask[2]) << p.tshift[2]));
#pragma unroll
    for (int i = 0; i < W; ++i) {
        float2 acc{0.f, 0.f};
#pragma unroll
        for (int jj = 0; jj < W; ++jj) {
            float2 inner{0.f, 0.f};
#pragma unroll
            for (int qq = 0; qq < W; ++qq)
                inner = cadd(inner, cscale(e2[qq], p.w32[(i * W + jj) * W + qq]));
            acc = cadd(acc, cmul(e1[jj], inner));
        }
        cs.g[i] = acc;
    }
}

// FP32 value of Lambda at k_0 for the column described by cs; E[-q] is
// conj(E[q]) and E[0] = 1, so RAD table loads suffice.
template <int RAD>
__device__ __forceinline__ float2 col_lambda32(const SymbolParams& p, const ColSymbol<RAD>& cs,
                                               int k0) {
    float2 l = cs.g[RAD];
#pragma unroll
    for (int m = 1; m <= RAD; ++m) {
        const float2 e = __ldg(p.E32[0] + (((m * k0) & p.tmask[0]) << p.tshift[0]));
        l = cadd(l, cmul(e, cs.g[RAD + m]));
        l = cadd(l, cmul(cconj(e), cs.g[RAD - m]));
    }
    return l;
}

// Multiply the survivors (bits of mask) of a thread's 16 elements, parked in
// shared memory at sm[j + q r], by V = Lambda^T / N in FP64. Kept out of line
// so the caller's registers are not held across it; the column's FP64 factors
// are formed once here and serve every survivor.
template <int RAD, typename C, typename View>
__device__ __noinline__ void multiply_survivors(View sm, int j, int q, unsigned mask,
                                                const SymbolParams& p, int k1, int k2) {
    using R = decltype(C{}.x);
    ColSymbol64<RAD> cs;
    col_symbol_init64<RAD>(p, p.w, k1, k2, cs);
    while (mask) {
        const int r = __ffs(mask) - 1;
        mask &= mask - 1;
        const double2 v = col_power64<RAD>(p, cs, j + q * r);
        const C V{(R)v.x, (R)v.y};
        C& e = sm[j + q * r];
        e = cmul(e, V);
    }
}

// x * V[k] for a single frequency k (out of line; used for the one Nyquist
// element of a real axis).
template <typename C>
__device__ __noinline__ C multiply_single(C x, const SymbolParams& p, int k0, int k1, int k2) {
    const int k[3] = {k0, k1, k2};
    return cmul(x, spectral_multiplier<C>(p, k));
}

// True when every element of the column described by cs is below the cut:
// |Lambda(k_0)| <= sum_m |G[m]| for every k_0 (|E| = 1), so when that sum
// (raised by 2^-18 for the rounding of the sum and of any per-element
// evaluation) passes the per-element test, every element does.
template <int RAD>
__device__ __forceinline__ bool col_below_cut(const SymbolParams& p, const ColSymbol<RAD>& cs) {
    if (!(p.tau2 > 0.f)) return false;
    float b = 0.f;
#pragma unroll
    for (int i = 0; i < 2 * RAD + 1; ++i) b += sqrtf(cs.g[i].x * cs.g[i].x + cs.g[i].y * cs.g[i].y);
    b *= 1.0f + 0x1p-18f;
    return b * b < p.tau2;
}

// v[r] <- V[k] v[r] for the thread's elements k_0 = j + q r of one column whose
// other frequencies are (k1, k2) and whose FP32 factorisation is cs. Elements
// whose FP32 bound shows |V| below half the smallest subnormal become 0; the
// rest get the FP64 multiplier. sm (this sequence's shared buffer) is used as
// scratch at the thread's own positions; the caller must place a barrier
// between this and the next use of sm by other threads.
//
// When the column is a full transform (16 q = l_0), E_0[m (j + q r)] =
// E_0[m j] exp(2 pi i m r / 16): one table load per m and thread, the rest
// exact-constant rotations (their rounding is far inside the bound delta).
template <int RAD, typename C, typename View>
__device__ __forceinline__ void apply_multiplier(C* v, const View& sm, int j, int q,
                                                 const SymbolParams& p, const ColSymbol<RAD>& cs,
                                                 int k1, int k2) {
    using R = decltype(C{}.x);
    if (p.T == 0) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = cscale(v[r], (R)p.scale);
        return;
    }
    if (col_below_cut<RAD>(p, cs)) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = C{(R)0, (R)0};
        return;
    }
    unsigned mask = 0;
    if (RAD > 0 && q * 16 == p.len[0]) {
        float2 e[RAD > 0 ? RAD : 1];
#pragma unroll
        for (int m = 1; m <= RAD; ++m)
            e[m - 1] = __ldg(p.E32[0] + (((m * j) & p.tmask[0]) << p.tshift[0]));
        if (p.real_symbol) {
            // Lambda real: G[-m] = conj(G[m]), Lambda = G[0] + 2 sum_m Re(E_m G[m])
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                float l = cs.g[RAD].x;
#pragma unroll
                for (int m = 1; m <= RAD; ++m) {
                    const float2 em = rot16<+1>(e[m - 1], m * r);
                    l += 2.f * (em.x * cs.g[RAD + m].x - em.y * cs.g[RAD + m].y);
                }
                if (l * l < p.tau2) v[r] = C{(R)0, (R)0};
                else mask |= 1u << r;
            }
        } else {
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                float2 l = cs.g[RAD];
#pragma unroll
                for (int m = 1; m <= RAD; ++m) {
                    const float2 em = rot16<+1>(e[m - 1], m * r);
                    l = cadd(l, cmul(em, cs.g[RAD + m]));
                    l = cadd(l, cmul(cconj(em), cs.g[RAD - m]));
                }
                if (l.x * l.x + l.y * l.y < p.tau2) v[r] = C{(R)0, (R)0};
                else mask |= 1u << r;
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const float2 l = col_lambda32<RAD>(p, cs, j + q * r);
            if (l.x * l.x + l.y * l.y < p.tau2) v[r] = C{(R)0, (R)0};
            else mask |= 1u << r;
        }
    }
    if (mask) {
#pragma unroll
        for (int r = 0; r < 16; ++r) sm[j + q * r] = v[r];
        multiply_survivors<RAD, C, View>(sm, j, q, mask, p, k1, k2);
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = mask >> r & 1 ? sm[j + q * r] : C{(R)0, (R)0};
    }
}

}  // namespace sfft
