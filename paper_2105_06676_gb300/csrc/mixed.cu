// Mixed-radix Multi-FFT passes for axis lengths whose prime factors are 2, 3,
// 5 and 7 (the paper's experiments use 1.6e6, 8000^2 and 800^3 cells, Sec. 6
// and Tab. "experimental-results"). Same convention as the power-of-two
// passes (paper Sec. 4: forward w^(-ij), inverse w^(+ij), unscaled).
//
// A pass holds whole sequences in shared memory and runs Stockham stages of
// radix 8, 4, 2, 5, 3 or 7 in place: every thread loads its butterflies of a
// stage into registers, the CTA synchronises, and the results go back to
// their autosorted positions (output index (j / Ns) Ns R + j mod Ns + r Ns for
// butterfly j over inputs j + r n/R, inputs turned by exp(DIR 2 pi i (j mod Ns)
// r / (Ns R)) first). Twiddles come from a per-length table
// exp(-2 pi i m / len) built with FP64 sincospi and stored at pass precision.
//
// Passes: real rows -> half spectra (R2C: the packed n = L/2 complex
// transform and the real-input split), strided C2C columns, and the inverse
// C2R. The multiply by Lambda^T / N runs between them (vector.cu).
#include <cuda_runtime.h>

#include <cstring>

#include "internal.h"

namespace sfft {

namespace {

constexpr int kMaxStages = 24;
constexpr int kMixEPT = 16;   // elements per thread a CTA is sized for

struct RadixPlan {
    int nst;
    int radix[kMaxStages];
};

// cos / sin(2 pi q / R) for R = 3, 5, 7, q = 0..R-1 (exact constants,
// rounded); chained conditionals so that constant arguments fold away.
__host__ __device__ constexpr double cos_r(int R, int q) {
    return q == 0 ? 1.0
         : R == 3 ? -0.5
         : R == 5 ? (q == 1 || q == 4 ? 0.3090169943749474241023 : -0.8090169943749474241023)
         : (q == 1 || q == 6 ? 0.6234898018587335305250
            : q == 2 || q == 5 ? -0.2225209339563144042889 : -0.9009688679024191262361);
}
__host__ __device__ constexpr double sin_r(int R, int q) {
    return q == 0 ? 0.0
         : R == 3 ? (q == 1 ? 0.8660254037844386467637 : -0.8660254037844386467637)
         : R == 5 ? (q == 1 ? 0.9510565162951535721164 : q == 2 ? 0.5877852522924731291687
                     : q == 3 ? -0.5877852522924731291687 : -0.9510565162951535721164)
         : (q == 1 ? 0.7818314824680298087084 : q == 2 ? 0.9749279121818236070181
            : q == 3 ? 0.4338837391175581204758 : q == 4 ? -0.4338837391175581204758
            : q == 5 ? -0.9749279121818236070181 : -0.7818314824680298087084);
}

// In-register DFT of odd prime size R (3, 5, 7) by its definition:
// out[k] = sum_j v[j] exp(DIR 2 pi i j k / R).
template <int R, int DIR, typename C>
__device__ __forceinline__ void dft_odd(C* v) {
    using Re = decltype(C{}.x);
    C out[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        C acc = v[0];
#pragma unroll
        for (int j = 1; j < R; ++j) {
            const int q = (j * k) % R;
            const Re c = (Re)cos_r(R, q), s = (Re)(DIR * sin_r(R, q));
            acc.x += v[j].x * c - v[j].y * s;
            acc.y += v[j].x * s + v[j].y * c;
        }
        out[k] = acc;
    }
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = out[k];
}

template <int R, int DIR, typename C>
__device__ __forceinline__ void dft_any(C* v) {
    if constexpr (R == 3 || R == 5 || R == 7) dft_odd<R, DIR>(v);
    else dft_reg<R, DIR>(v);
}

// x / d and x mod d for 0 <= x < 2^24 through a float reciprocal (rcp = 1/d
// rounded): the quotient is off by at most one and corrected exactly.
__device__ __forceinline__ void divmod_small(int x, int d, float rcp, int& q, int& r) {
    q = __float2int_rz((float)x * rcp);
    r = x - q * d;
    if (r < 0) { --q; r += d; }
    else if (r >= d) { ++q; r -= d; }
}

// One in-place Stockham stage of radix R over nseq sequences of length n held
// at sm + s * ss. tw: table of exp(-2 pi i m / (n * twmul)) (read at m *
// twmul). A butterfly j (k = j mod Ns) loads w = exp(-2 pi i k / (Ns R)) once
// and forms w^r by products (r <= 7: a few roundings). Contains a CTA barrier.
template <int R, int DIR, typename C>
__device__ __forceinline__ void mixed_stage(C* sm, int n, int nseq, int ss, int Ns,
                                            const C* __restrict__ tw, int twmul) {
    constexpr int MAXB = (kMixEPT + R - 1) / R + 1;   // butterflies per thread
    const int nb = n / R;
    const int total = nseq * nb;
    const int span = n / (Ns * R);   // w^k = exp(-2 pi i k span / n)
    const float rnb = 1.0f / (float)nb, rns = 1.0f / (float)Ns;
    C v[MAXB * R];
    int pos[MAXB];
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        const int g = threadIdx.x + b * blockDim.x;
        pos[b] = -1;
        if (g < total) {
            int s, j, jq, k;
            if (nseq == 1) {
                s = 0;
                j = g;
            } else {
                divmod_small(g, nb, rnb, s, j);
            }
            divmod_small(j, Ns, rns, jq, k);
            pos[b] = s * ss + jq * Ns * R + k;   // first output position
            const C* src = sm + s * ss;
            C w1 = tw[k * span * twmul];
            if (DIR > 0) w1.y = -w1.y;
            C wr = w1;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                C x = src[j + r * nb];
                if (r > 0 && k > 0) {
                    x = cmul(x, wr);
                    if (r + 1 < R) wr = cmul(wr, w1);
                }
                v[b * R + r] = x;
            }
            dft_any<R, DIR>(v + b * R);
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        if (pos[b] >= 0) {
            C* dst = sm + pos[b];
#pragma unroll
            for (int r = 0; r < R; ++r) dst[r * Ns] = v[b * R + r];
        }
    }
    __syncthreads();
}

// Full transform of nseq sequences of length n in shared memory (natural order
// in and out). Ends with a barrier.
template <int DIR, typename C>
__device__ void mixed_fft(C* sm, int n, int nseq, int ss, const RadixPlan& rp,
                          const C* __restrict__ tw, int twmul) {
    int Ns = 1;
    for (int i = 0; i < rp.nst; ++i) {
        switch (rp.radix[i]) {
            case 8: mixed_stage<8, DIR>(sm, n, nseq, ss, Ns, tw, twmul); break;
            case 4: mixed_stage<4, DIR>(sm, n, nseq, ss, Ns, tw, twmul); break;
            case 2: mixed_stage<2, DIR>(sm, n, nseq, ss, Ns, tw, twmul); break;
            case 5: mixed_stage<5, DIR>(sm, n, nseq, ss, Ns, tw, twmul); break;
            case 3: mixed_stage<3, DIR>(sm, n, nseq, ss, Ns, tw, twmul); break;
            default: mixed_stage<7, DIR>(sm, n, nseq, ss, Ns, tw, twmul); break;
        }
        Ns *= rp.radix[i];
    }
}

// R2C / C2R rows: one CTA per row of L = 2n reals; twL = table of length L.
template <typename R>
__global__ void __launch_bounds__(512)
k_mixed_rows_r2c(const R* __restrict__ grid, typename CxOf<R>::T* __restrict__ H, long long Mp,
                 int n, int nrows, const typename CxOf<R>::T* __restrict__ twL,
                 const __grid_constant__ RadixPlan rp) {
    using C = typename CxOf<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const long long row = blockIdx.x;
    const C* src = reinterpret_cast<const C*>(grid) + row * n;   // z[m] = a[2m] + i a[2m+1]
    for (int e = threadIdx.x; e < n; e += blockDim.x) sm[e] = src[e];
    __syncthreads();
    mixed_fft<-1>(sm, n, 1, n, rp, twL, 2);
    C* h = H + row * Mp;
    for (int k = threadIdx.x; k <= n; k += blockDim.x) {
        const C zk = sm[k % n], znk = sm[(n - k) % n];
        const C xe = cscale(cadd(zk, cconj(znk)), (R)0.5);
        const C xo = cscale(cmul_mi(csub(zk, cconj(znk))), (R)0.5);
        // X[k] = Xe[k] + W^k Xo[k], W = exp(-2 pi i / L); X[n] = Xe[0] - Xo[0]
        h[k] = k == n ? csub(xe, xo) : cadd(xe, cmul(twL[k], xo));
    }
}

template <typename R>
__global__ void __launch_bounds__(512)
k_mixed_rows_c2r(const typename CxOf<R>::T* __restrict__ H, R* __restrict__ grid, long long Mp,
                 int n, int nrows, const typename CxOf<R>::T* __restrict__ twL,
                 const __grid_constant__ RadixPlan rp, int* status) {
    using C = typename CxOf<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const long long row = blockIdx.x;
    const C* h = H + row * Mp;
    // Z'[k] = (Y[k] + conj Y[n-k]) + i conj(W^k) (Y[k] - conj Y[n-k])
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const C yk = h[k], ynk = h[n - k];
        const C wk = twL[k];
        sm[k] = cadd(cadd(yk, cconj(ynk)), cmul_i(cmul(cconj(wk), csub(yk, cconj(ynk)))));
    }
    __syncthreads();
    mixed_fft<+1>(sm, n, 1, n, rp, twL, 2);
    C* out = reinterpret_cast<C*>(grid) + row * n;
    bool bad = false;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const C v = sm[e];
        bad |= !(isfinite(v.x) && isfinite(v.y));
        out[e] = v;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, 1);
}

// Strided C2C transforms of length n (ColGeom): cols adjacent sequences per
// CTA, held sequence-major in shared memory (stride n + 1).
template <typename R, int DIR>
__global__ void __launch_bounds__(512)
k_mixed_cols(typename CxOf<R>::T* __restrict__ H, const __grid_constant__ ColGeom g, int n,
             int cols, const typename CxOf<R>::T* __restrict__ tw,
             const __grid_constant__ RadixPlan rp) {
    using C = typename CxOf<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int ss = n + 1;
    const int i0 = blockIdx.x * cols;
    C* base = H + (long long)blockIdx.z * g.os + (long long)blockIdx.y * g.ms + i0;
    for (int e = threadIdx.x; e < cols * n; e += blockDim.x) {
        const int j = e / cols, c = e - j * cols;
        sm[c * ss + j] = i0 + c < g.inner_valid ? base[(long long)j * g.S + c] : C{0, 0};
    }
    __syncthreads();
    mixed_fft<DIR>(sm, n, cols, ss, rp, tw, 1);
    for (int e = threadIdx.x; e < cols * n; e += blockDim.x) {
        const int j = e / cols, c = e - j * cols;
        if (i0 + c < g.inner_valid) base[(long long)j * g.S + c] = sm[c * ss + j];
    }
}

template <typename R>
__global__ void k_mixed_table(typename CxOf<R>::T* tw, int len) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < len; m += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)m / (double)len, &s, &c);   // exp(-2 pi i m / len)
        tw[m] = typename CxOf<R>::T{(R)c, (R)s};
    }
}

bool factor(int n, RadixPlan& rp) {
    rp.nst = 0;
    while (n % 8 == 0 && rp.nst < kMaxStages) { rp.radix[rp.nst++] = 8; n /= 8; }
    while (n % 4 == 0 && rp.nst < kMaxStages) { rp.radix[rp.nst++] = 4; n /= 4; }
    while (n % 2 == 0 && rp.nst < kMaxStages) { rp.radix[rp.nst++] = 2; n /= 2; }
    while (n % 5 == 0 && rp.nst < kMaxStages) { rp.radix[rp.nst++] = 5; n /= 5; }
    while (n % 3 == 0 && rp.nst < kMaxStages) { rp.radix[rp.nst++] = 3; n /= 3; }
    while (n % 7 == 0 && rp.nst < kMaxStages) { rp.radix[rp.nst++] = 7; n /= 7; }
    return n == 1;
}

int threads_for_mixed(long long elems, int maxt) {
    long long t = (elems + kMixEPT - 1) / kMixEPT;
    t = (t + 31) / 32 * 32;
    if (t < 64) t = 64;
    if (t > maxt) t = maxt;
    return (int)t;
}

template <typename R>
int max_threads_mixed() { return 512; }

}  // namespace

bool mixed_length_ok(int64_t len, int precision) {
    if (len < 2) return false;
    RadixPlan rp;
    if (!factor((int)len, rp) || len > (1 << 24)) return false;
    // one sequence per CTA in shared memory, kMixEPT elements per thread
    (void)precision;
    return len <= (int64_t)kMixEPT * 512;
}

template <typename R>
cudaError_t launch_mixed_table(void* tw, int len, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (len + threads - 1) / threads;
    k_mixed_table<R><<<blocks, threads, 0, s>>>(static_cast<typename CxOf<R>::T*>(tw), len);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_mixed_rows(int dir, const void* src, void* dst, long long Mp, int n, int nrows,
                              const void* twL, int* status, cudaStream_t s) {
    using C = typename CxOf<R>::T;
    RadixPlan rp;
    if (!factor(n, rp)) return cudaErrorInvalidValue;
    const size_t smem = (size_t)n * sizeof(C);
    const int threads = threads_for_mixed(n, max_threads_mixed<R>());
    if ((long long)threads * kMixEPT < n) return cudaErrorInvalidValue;
    cudaError_t err;
    if (dir < 0) {
        err = smem_optin(reinterpret_cast<const void*>(k_mixed_rows_r2c<R>), smem);
        if (err != cudaSuccess) return err;
        k_mixed_rows_r2c<R><<<nrows, threads, smem, s>>>(static_cast<const R*>(src),
                                                         static_cast<C*>(dst), Mp, n, nrows,
                                                         static_cast<const C*>(twL), rp);
    } else {
        err = smem_optin(reinterpret_cast<const void*>(k_mixed_rows_c2r<R>), smem);
        if (err != cudaSuccess) return err;
        k_mixed_rows_c2r<R><<<nrows, threads, smem, s>>>(static_cast<const C*>(src),
                                                         static_cast<R*>(dst), Mp, n, nrows,
                                                         static_cast<const C*>(twL), rp, status);
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_mixed_cols(int dir, void* H, const ColGeom& g, int n, const void* tw,
                              cudaStream_t s) {
    using C = typename CxOf<R>::T;
    RadixPlan rp;
    if (!factor(n, rp)) return cudaErrorInvalidValue;
    const int maxt = max_threads_mixed<R>();
    // columns per CTA: up to 8 (64-byte row segments for FP32) within the
    // thread and shared-memory budgets
    int cols = 8;
    while (cols > 1 && ((long long)cols * n > (long long)kMixEPT * maxt ||
                        (size_t)cols * (n + 1) * sizeof(C) > (size_t)kSmemBudget))
        cols /= 2;
    if ((long long)cols * n > (long long)kMixEPT * maxt) return cudaErrorInvalidValue;
    const size_t smem = (size_t)cols * (n + 1) * sizeof(C);
    const int threads = threads_for_mixed((long long)cols * n, maxt);
    dim3 grid((g.inner_valid + cols - 1) / cols, g.mid, g.outer);
    cudaError_t err;
    if (dir < 0) {
        err = smem_optin(reinterpret_cast<const void*>(k_mixed_cols<R, -1>), smem);
        if (err != cudaSuccess) return err;
        k_mixed_cols<R, -1><<<grid, threads, smem, s>>>(static_cast<C*>(H), g, n, cols,
                                                        static_cast<const C*>(tw), rp);
    } else {
        err = smem_optin(reinterpret_cast<const void*>(k_mixed_cols<R, +1>), smem);
        if (err != cudaSuccess) return err;
        k_mixed_cols<R, +1><<<grid, threads, smem, s>>>(static_cast<C*>(H), g, n, cols,
                                                        static_cast<const C*>(tw), rp);
    }
    return cudaGetLastError();
}

#define SFFT_MIXED_INST(R)                                                                       \
    template cudaError_t launch_mixed_table<R>(void*, int, cudaStream_t);                        \
    template cudaError_t launch_mixed_rows<R>(int, const void*, void*, long long, int, int,       \
                                              const void*, int*, cudaStream_t);                  \
    template cudaError_t launch_mixed_cols<R>(int, void*, const ColGeom&, int, const void*,      \
                                              cudaStream_t);
SFFT_MIXED_INST(float)
SFFT_MIXED_INST(double)

}  // namespace sfft
