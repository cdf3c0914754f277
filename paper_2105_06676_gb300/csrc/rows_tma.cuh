#pragma once
// Contiguous-axis passes of StencilFFT-P for FP32 grids (paper Sec. 4, Fig.
// "stencil-fft-algorithm-dD": the forward Multi-FFT's transform along the
// stored-contiguous axis with the real-input split, and its inverse) as
// persistent kernels fed by bulk copies. The library launches the inverse
// (C2R) form; the forward form measured slower than the register row kernel
// on GB300 and is not launched.
//
// A real row of L = 2n values is read as n complex pairs and transformed by
// the register-resident FFT of fft_ct.cuh (n = 2^LOG2N, 256 <= n <= 4096, q =
// n/16 threads per row, 16 elements per thread). A tile is RPT = 256 / q rows
// (32 KB). Four 256-thread CTAs per SM each walk the tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ...:
//   * one elected thread issues one cp.async.bulk per row of the next tile
//     (row r lands at the start of its padded region in shared memory),
//     completing on the CTA's mbarrier (expect-tx);
//   * every thread waits (bounded) for the tile and reads its elements into
//     registers; the same buffer then serves as the transform's exchange
//     buffer (one padded sequence per row);
//   * once the tile's last shared-memory read is done the elected thread
//     issues the next tile, which lands while this CTA finishes and stores and
//     while the SM's other CTAs compute.
// R2C writes the half spectrum X[0..n] of each row (row stride Mp); C2R reads
// Y[0..n+1] of each row (one padding element beyond Y[n], inside the row
// stride) and writes the real row. A wait that gives up after kWaitLimitNs
// records kGemmTimeout (bit 2 of the status word) and ends the CTA.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cols_tma.cuh"   // mbarrier helpers
#include "fft_ct.cuh"
#include "internal.h"

namespace sfft {

constexpr int kRowThreads = 256;
constexpr int kRowTmaLog2Lo = 8, kRowTmaLog2Hi = 12;

// Padded sequence stride of the row buffers: n + n/32 rounded up to a whole
// 16-byte unit (every row's landing address stays 16-byte aligned).
__host__ __device__ constexpr int row_tma_stride(int log2n) {
    return (((1 << log2n) + ((1 << log2n) >> 5)) + 1) & ~1;
}
__host__ __device__ constexpr int row_tma_rows(int log2n) {
    return kRowThreads / ((1 << log2n) >> 4);
}
__host__ __device__ constexpr size_t row_tma_smem(int log2n) {
    return (size_t)row_tma_rows(log2n) * row_tma_stride(log2n) * 8 + 16;
}


// DIR = -1: rows of the real grid -> half spectra (R2C); +1: half spectra ->
// real rows (C2R). src / dst are the grid (complex view of its rows) or H.
template <int DIR, int LOG2N>
__global__ void __launch_bounds__(kRowThreads, 4)
k_rows_tma(const float2* __restrict__ src, float2* __restrict__ dst, long long Mp, int nrows,
           const float2* __restrict__ tw, int twn_log2, int* status) {
    constexpr int n = 1 << LOG2N;
    constexpr int q = n >> 4;
    constexpr int RPT = row_tma_rows(LOG2N);
    constexpr int SS = row_tma_stride(LOG2N);
    constexpr uint32_t kInBytes = DIR < 0 ? n * 8 : (n + 2) * 8;   // per row
    extern __shared__ __align__(1024) unsigned char smraw[];
    float2* buf = reinterpret_cast<float2*>(smraw);
    const uint32_t bar = smem_u32(smraw + row_tma_smem(LOG2N) - 16);
    const uint32_t bufa = smem_u32(buf);
    const int c = threadIdx.x / q;   // row within the tile
    const int j = threadIdx.x - c * q;
    const bool leader = threadIdx.x == 0;
    const int ntiles = (nrows + RPT - 1) / RPT;

    auto issue = [&](int tile) {
        const int r0 = tile * RPT;
        const int rows = min(RPT, nrows - r0);
        mbar_expect_tx(bar, kInBytes * rows);
        for (int i = 0; i < rows; ++i) {
            const float2* s = DIR < 0 ? src + (long long)(r0 + i) * n : src + (long long)(r0 + i) * Mp;
            bulk_load(bufa + i * SS * 8, s, kInBytes, bar);
        }
    };

    if (leader) {
        mbar_init(bar, 1);
        mbar_fence_init();
        fence_async_shared();
    }
    __syncthreads();
    if (leader && (int)blockIdx.x < ntiles) issue(blockIdx.x);
    const SeqView<float2> sv{buf + c * SS};
    const int sh = twn_log2 - LOG2N - 1;   // W^k = exp(-2 pi i k / 2n) = tw[k << sh]
    bool bad = false;
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const bool ok = mbar_wait(bar, it & 1);
        if (__syncthreads_or(!ok)) {
            if (leader) {
                atomicOr(status, kGemmTimeout);
                mbar_wait(bar, it & 1);
            }
            return;
        }
        const long long row = (long long)tile * RPT + c;
        const bool live = row < nrows;
        const int next = tile + (int)gridDim.x;
        float2 v[16];
        const float2* rowbuf = buf + c * SS;   // the row as it landed (dense)
        if constexpr (DIR < 0) {
#pragma unroll
            for (int s = 0; s < 16; ++s) v[s] = live ? rowbuf[j + q * s] : float2{0.f, 0.f};
            __syncthreads();
            ct_fft<-1, LOG2N, 0, 5>(v, sv.base, j, tw, twn_log2);
            // real-input split: X[k] from Z[k] and Z[n-k]
#pragma unroll
            for (int r = 0; r < 16; ++r) sv[j + q * r] = v[r];
            __syncthreads();
            float2* h = dst + (live ? row : 0) * Mp;
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const int k = j + q * r;
                const float2 zk = v[r], znk = sv[(n - k) & (n - 1)];
                const float2 xe = cscale(cadd(zk, cconj(znk)), 0.5f);
                const float2 xo = cscale(cmul_mi(csub(zk, cconj(znk))), 0.5f);
                if (live) {
                    h[k] = cadd(xe, cmul(__ldg(tw + (k << sh)), xo));
                    if (k == 0) h[n] = csub(xe, xo);   // X[n] = Xe[0] - Xo[0]
                }
            }
            __syncthreads();   // the tile's last shared-memory read
            if (leader && next < ntiles) {
                fence_async_shared();
                issue(next);
            }
        } else {
            // Z'[k] = (Y[k] + conj Y[n-k]) + i conj(W^k) (Y[k] - conj Y[n-k])
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                const int k = j + q * s;
                const float2 yk = live ? rowbuf[k] : float2{0.f, 0.f};
                const float2 ynk = live ? rowbuf[n - k] : float2{0.f, 0.f};
                const float2 wk = __ldg(tw + (k << sh));
                v[s] = cadd(cadd(yk, cconj(ynk)), cmul_i(cmul(cconj(wk), csub(yk, cconj(ynk)))));
            }
            __syncthreads();
            ct_fft<+1, LOG2N, 0, 5>(v, sv.base, j, tw, twn_log2);
            // ct_fft ends after a barrier that follows its last shared-memory read
            if (leader && next < ntiles) {
                fence_async_shared();
                issue(next);
            }
            if (live) {
                float2* out = dst + row * n;
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    bad |= !(isfinite(v[r].x) && isfinite(v[r].y));
                    out[j + q * r] = v[r];
                }
            }
        }
    }
    if (DIR > 0 && __syncthreads_or(bad) && leader) atomicOr(status, 1);
}

}  // namespace sfft
