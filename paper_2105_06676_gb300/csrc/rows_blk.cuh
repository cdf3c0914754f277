#pragma once
// Contiguous-axis passes of StencilFFT-P for FP32 2-D grids that keep the half
// spectrum in column blocks (paper Sec. 4, Fig. "stencil-fft-algorithm-dD":
// the forward Multi-FFT along the stored-contiguous axis with the real-input
// split, Step 1; its inverse, Step 4). The strided-axis pass between them
// (cols_tma.cuh, BLK = 1) then reads and writes one contiguous 64 KB block per
// tile.
//
// Layout: an item of l0 rows has its half spectrum X[i][k] (k = 0..n, n = l1/2)
// at  (k >> CL) * l0 * CPT + i * CPT + (k & (CPT - 1)),  CPT = 2^CL columns per
// block, NX = ceil((n + 1) / CPT) blocks; items follow each other every
// NX * l0 * CPT elements. Columns n+1 .. NX*CPT-1 hold zeros.
//
// A CTA transforms RPT consecutive rows of one item (q = n/16 threads per row,
// 16 elements per thread, the register FFT of fft_ct.cuh), so for every block x
// its rows form one contiguous run of RPT * CPT values (RPT >= 2, CPT >= 2:
// at least 32 bytes, whole sectors). The runs pass through a shared staging
// area so that global memory sees 16-byte accesses with lane pairs covering
// whole 32-byte sectors.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_ct.cuh"
#include "internal.h"

namespace sfft {

constexpr int kBlkLog2Lo = 8, kBlkLog2Hi = 12;

// Threads and rows per CTA of the blocked row passes: at least two rows, at
// least 256 threads. (Four rows per CTA -- 64-byte runs, 512 threads for
// 2048-point rows -- measured slower on GB300: 4096^2 R2C 53.5 -> 55.7 us, C2R
// 49.0 -> 53.8 us.)
__host__ __device__ constexpr int blk_threads(int log2n) {
    return ((1 << log2n) >> 4) * 2 > 256 ? ((1 << log2n) >> 4) * 2 : 256;
}
__host__ __device__ constexpr int blk_rows(int log2n) {
    return blk_threads(log2n) / ((1 << log2n) >> 4);
}
// Sequence stride of the exchange buffer: the FFT's exchanges use one pad
// slot per 16 elements (PadLayout<0, 4>), which keeps every exchange of every
// stage free of bank conflicts for 8-byte elements, half a warp per wavefront
// (one pad per 32 left the stride-R0 stores of the first exchange and the
// Ns = 8 stores of a 2048-point transform two-way conflicted).
__host__ __device__ constexpr int blk_seq_stride(int log2n) {
    return (1 << log2n) + ((1 << log2n) >> 4) + 1;
}
__host__ __device__ constexpr int blk_nx(int log2n, int cl) {
    return ((1 << log2n) + 1 + (1 << cl) - 1) >> cl;
}
__host__ __device__ constexpr size_t blk_smem(int log2n, int cl) {
    const size_t ex = (size_t)blk_rows(log2n) * blk_seq_stride(log2n);
    // staging, rounded up to whole 128-byte rows (the swizzle permutes within them)
    const size_t st = ((size_t)blk_nx(log2n, cl) * blk_rows(log2n) * (1 << cl) + 15) / 16 * 16;
    return (ex > st ? ex : st) * 8;
}

// The staging area holds 16-byte pieces (two complex values) in the order of
// the global runs; piece p lives at slot p ^ (3 (p / 8) mod 8), a permutation
// within each 128-byte row. A warp's element accesses (one row of the CTA,
// 32 consecutive columns: every RPT-th run of CPT values) then spread over all
// banks instead of hitting the same RPT-th of them, while a warp's 16-byte
// piece accesses (32 consecutive pieces, four whole rows) stay conflict-free.
__device__ __forceinline__ int blk_piece(int p) { return p ^ ((3 * (p >> 3)) & 7); }

// Staging position (in complex values) of X[c][k], row c of the CTA: block-major,
// rows within a block, columns within a row, pieces swizzled as above.
template <int CL, int RPT>
__device__ __forceinline__ int blk_stage(int c, int k) {
    const int s = ((k >> CL) * RPT + c) * (1 << CL) + (k & ((1 << CL) - 1));
    return (blk_piece(s >> 1) << 1) | (s & 1);
}

// R2C: rows of the real grid (viewed as n complex pairs) -> blocked half spectra.
template <int LOG2N, int CL>
__global__ void __launch_bounds__(blk_threads(LOG2N), 1024 / blk_threads(LOG2N))
k_rows_r2c_blk(const float2* __restrict__ grid, float2* __restrict__ H, int l0_log2, long long os,
               int nrows, const float2* __restrict__ tw, int twn_log2) {
    constexpr int n = 1 << LOG2N, q = n >> 4;
    constexpr int RPT = blk_rows(LOG2N), CPT = 1 << CL, NX = blk_nx(LOG2N, CL);
    constexpr int SS = blk_seq_stride(LOG2N);
    extern __shared__ __align__(16) unsigned char smraw[];
    float2* buf = reinterpret_cast<float2*>(smraw);
    const int c = threadIdx.x / q, j = threadIdx.x - c * q;
    const long long row0 = (long long)blockIdx.x * RPT;   // first row of the CTA (all items)
    const long long row = row0 + c;
    const bool live = row < nrows;
    const SeqView<float2> sv{buf + c * SS};
    const float2* rowp = grid + (live ? row : 0) * n;
    float2 v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) v[s] = live ? __ldg(rowp + j + q * s) : float2{0.f, 0.f};
    ct_fft<-1, LOG2N, 0, 4>(v, buf + c * SS, j, tw, twn_log2);
#pragma unroll
    for (int r = 0; r < 16; ++r) sv[j + q * r] = v[r];
    __syncthreads();
    // real-input split: X[k] from Z[k] and Z[n-k]. W^k = exp(-2 pi i k / 2n)
    // = tw[k << sh] is taken as W^j W^(q r): one per-thread load and sixteen
    // loads that are the same for the whole warp
    const int sh = twn_log2 - LOG2N - 1;
    const float2 wj = __ldg(tw + (j << sh));
    float2 xn{0.f, 0.f};
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int k = j + q * r;
        const float2 zk = v[r], znk = sv[(n - k) & (n - 1)];
        const float2 xe = cscale(cadd(zk, cconj(znk)), 0.5f);
        const float2 xo = cscale(cmul_mi(csub(zk, cconj(znk))), 0.5f);
        const float2 wk = r == 0 ? wj : cmul(wj, __ldg(tw + ((q * r) << sh)));
        v[r] = cadd(xe, cmul(wk, xo));
        if (k == 0) xn = csub(xe, xo);   // X[n] = Xe[0] - Xo[0]
    }
    __syncthreads();   // every partner read is done: the buffer becomes the staging area
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[blk_stage<CL, RPT>(c, j + q * r)] = v[r];
    if (j == 0) {
        buf[blk_stage<CL, RPT>(c, n)] = xn;
#pragma unroll
        for (int k = n + 1; k < NX * CPT; ++k) buf[blk_stage<CL, RPT>(c, k)] = float2{0.f, 0.f};
    }
    __syncthreads();
    // copy-out: block x's run of RPT * CPT values goes to item z, rows i0..
    const int l0 = 1 << l0_log2;
    const long long z = row0 >> l0_log2;
    const int i0 = (int)(row0 & (l0 - 1));
    const int rows_live = nrows - row0 < RPT ? (int)(nrows - row0) : RPT;
    constexpr int PPR = CPT / 2;              // 16-byte pieces per row of a run
    constexpr int PIECES = NX * RPT * PPR;
    float4* hz = reinterpret_cast<float4*>(H + z * os + (long long)i0 * CPT);
    const float4* st = reinterpret_cast<const float4*>(buf);
    constexpr int PER = (PIECES + blk_threads(LOG2N) - 1) / blk_threads(LOG2N);
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int p = threadIdx.x + u * blk_threads(LOG2N);
        if (p < PIECES) {
            const int x = p / (RPT * PPR);
            const int rem = p - x * (RPT * PPR);
            if (rem / PPR < rows_live) hz[(long long)x * (l0 * PPR) + rem] = st[blk_piece(p)];
        }
    }
}

// C2R: blocked half spectra -> real rows (Z'[k] = (Y[k] + conj Y[n-k]) + i
// conj(W^k) (Y[k] - conj Y[n-k]), inverse FFT). Non-finite output sets bit 0
// of *status.
template <int LOG2N, int CL>
__global__ void __launch_bounds__(blk_threads(LOG2N), 1024 / blk_threads(LOG2N))
k_rows_c2r_blk(const float2* __restrict__ H, float2* __restrict__ grid, int l0_log2, long long os,
               int nrows, const float2* __restrict__ tw, int twn_log2, int* status) {
    constexpr int n = 1 << LOG2N, q = n >> 4;
    constexpr int RPT = blk_rows(LOG2N), CPT = 1 << CL, NX = blk_nx(LOG2N, CL);
    constexpr int SS = blk_seq_stride(LOG2N);
    extern __shared__ __align__(16) unsigned char smraw[];
    float2* buf = reinterpret_cast<float2*>(smraw);
    const int c = threadIdx.x / q, j = threadIdx.x - c * q;
    const long long row0 = (long long)blockIdx.x * RPT;
    const long long row = row0 + c;
    const bool live = row < nrows;
    const int l0 = 1 << l0_log2;
    const long long z = row0 >> l0_log2;
    const int i0 = (int)(row0 & (l0 - 1));
    const int rows_live = nrows - row0 < RPT ? (int)(nrows - row0) : RPT;
    constexpr int PPR = CPT / 2;
    constexpr int PIECES = NX * RPT * PPR;
    {
        // every piece of the CTA in flight at once, then into the staging area
        const float4* hz = reinterpret_cast<const float4*>(H + z * os + (long long)i0 * CPT);
        float4* st = reinterpret_cast<float4*>(buf);
        constexpr int PER = (PIECES + blk_threads(LOG2N) - 1) / blk_threads(LOG2N);
        float4 t[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int p = threadIdx.x + u * blk_threads(LOG2N);
            const int x = p / (RPT * PPR);
            const int rem = p - x * (RPT * PPR);
            t[u] = p < PIECES && rem / PPR < rows_live ? __ldg(hz + (long long)x * (l0 * PPR) + rem)
                                                        : float4{0.f, 0.f, 0.f, 0.f};
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int p = threadIdx.x + u * blk_threads(LOG2N);
            if (p < PIECES) st[blk_piece(p)] = t[u];
        }
    }
    __syncthreads();
    const int sh = twn_log2 - LOG2N - 1;
    const float2 wj = __ldg(tw + (j << sh));   // W^k = W^j W^(q s), as in the R2C split
    float2 v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int k = j + q * s;
        const float2 yk = buf[blk_stage<CL, RPT>(c, k)];
        const float2 ynk = buf[blk_stage<CL, RPT>(c, n - k)];
        const float2 wk = s == 0 ? wj : cmul(wj, __ldg(tw + ((q * s) << sh)));
        v[s] = cadd(cadd(yk, cconj(ynk)), cmul_i(cmul(cconj(wk), csub(yk, cconj(ynk)))));
    }
    __syncthreads();   // staging read: the buffer becomes the exchange buffer
    ct_fft<+1, LOG2N, 0, 4>(v, buf + c * SS, j, tw, twn_log2);
    bool bad = false;
    if (live) {
        float2* out = grid + row * n;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            bad |= !(isfinite(v[r].x) && isfinite(v[r].y));
            out[j + q * r] = v[r];
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, 1);
}

}  // namespace sfft
