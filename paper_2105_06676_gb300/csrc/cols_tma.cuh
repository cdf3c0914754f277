#pragma once
// Strided-axis FFT passes of StencilFFT-P (paper Sec. 4, Fig.
// "stencil-fft-algorithm-dD": the Multi-FFT along every axis but the
// contiguous one, and Steps 2-3 fused between the forward and the inverse
// transform along axis 0) as persistent, TMA-fed kernels for FP32 half spectra.
//
// Work unit: a tile of 8192 complex values = CPT = 8192 / n adjacent columns of
// one transform axis of length n = 2^LOG2N (512 <= n <= 4096), 64 KB. Two
// 512-thread CTAs per SM each walk the tiles t = blockIdx.x, blockIdx.x +
// gridDim.x, ...; thread (c, j) = (tid mod CPT, tid / CPT) owns column c and
// the 16 elements j + (n/16) s of the tile.
//
// Pipeline per CTA (shared memory: one padded tile buffer, the stage twiddle
// tables, one mbarrier):
//   * one elected thread issues a single 5-D cp.async.bulk.tensor load per tile
//     into the buffer, completing on the mbarrier (expect-tx);
//   * every thread waits (bounded) for the tile and copies its 16 elements into
//     registers; the buffer then serves as the exchange buffer of the
//     transforms (radix-R0 first stage, two radix-16 stages, two exchanges
//     each; stage twiddles from shared tables filled once per CTA);
//   * after the last exchange of the tile the elected thread issues the next
//     tile's load, which lands while this CTA finishes its last butterflies and
//     stores and while the SM's other CTA computes;
//   * results go straight from registers to global memory.
// A wait that gives up after kWaitLimitNs records kGemmTimeout (bit 2 of
// the status word) and ends the CTA (no load is then in flight).
//
// Blocked half spectra (BLK = 1, 2-D solves): the row passes store the half
// spectrum of an item as column blocks, element (row i, column k) at
// (k / CPT) n CPT + i CPT + k mod CPT, so a tile is one contiguous 64 KB block:
// it arrives by a single cp.async.bulk and leaves by stores that cover whole
// 256-byte runs per warp (the row-major layout moves 16-byte pieces of 4096
// rows both ways).
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dft_gemm.cuh"   // smem_u32, mbar_init, mbar_wait (time-bounded), fence_async_shared
#include "fft_ct.cuh"
#include "internal.h"
#include "symbol.cuh"

namespace sfft {

constexpr int kTileElems = 8192;          // complex values per tile (64 KB FP32)
constexpr int kTileThreads = 512;         // 16 elements per thread
constexpr int kTmaLog2Lo = 9, kTmaLog2Hi = 12;

// Shared memory of the TMA column kernels for a transform of 2^log2n: the
// tile buffer in the padded exchange layout (the tile lands dense in its first
// 64 KB), the two stage twiddle tables, the mbarrier.
__host__ __device__ constexpr int tma_cols_log2(int log2n) { return 13 - log2n; }
constexpr size_t kTmaBufBytes = ((size_t)(kTileElems + (kTileElems >> 4) + 1) * 8 + 127) / 128 * 128;
constexpr size_t kTmaTwABytes = 15 * 16 * 8;
__host__ __device__ constexpr size_t tma_twb_bytes(int log2n) {
    return (size_t)15 * ((1 << log2n) >> 4) * 8;
}
__host__ __device__ constexpr size_t tma_smem_bytes(int log2n) {
    return kTmaBufBytes + kTmaTwABytes + tma_twb_bytes(log2n) + 16;
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
                 : "memory");
}

// One 5-D tiled tensor load into shared memory, completing on mbar.
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, int c4, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
        "r"(mbar)
        : "memory");
}

// One contiguous bulk copy (untiled) into shared memory, completing on mbar;
// both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(mbar)
        : "memory");
}

// Twiddles of the two radix-16 stages after the first stage of an n = 2^LOG2N
// transform, forward direction, exact entries of the FP64-built table
// tw[m] = exp(-2 pi i m / TWN), in shared tables filled once per CTA:
//   stage Ns = R0 = 2^(LOG2N-8): a[(s-1) R0 + k1] = exp(-2 pi i k1 s / (16 R0)),
//     k1 = j mod R0;
//   stage Ns = q = n/16 (where k = j): b[(s-1) q + j] = exp(-2 pi i j s / n);
// s = 1..15. A warp's lanes read distinct consecutive entries (or the same
// entry): no bank conflicts.
template <int LOG2N>
struct StageTwiddles {
    const float2* a;   // a + k1: entry s at a[(s-1) R0]
    const float2* b;   // b + j:  entry s at b[(s-1) q]
};

template <int LOG2N>
__device__ __forceinline__ StageTwiddles<LOG2N> fill_stage_twiddles(float2* ta, float2* tb, int j,
                                                                   const float2* __restrict__ tw,
                                                                   int twn_log2) {
    constexpr int r0log = LOG2N - 8;
    constexpr int R0 = 1 << r0log;
    constexpr int q = (1 << LOG2N) >> 4;
    const int sh1 = twn_log2 - r0log - 4;
    for (int e = threadIdx.x; e < 15 * R0; e += blockDim.x) {
        const int s = e / R0 + 1, k1 = e % R0;
        ta[e] = __ldg(tw + ((k1 * s) << sh1));
    }
    const int sh2 = twn_log2 - LOG2N;
    for (int e = threadIdx.x; e < 15 * q; e += blockDim.x) {
        const int s = e / q + 1, jj = e % q;
        tb[e] = __ldg(tw + ((jj * s) << sh2));
    }
    return StageTwiddles<LOG2N>{ta + (j & (R0 - 1)), tb + j};
}

// v[s] *= w[(s-1) STEP] (forward) or its conjugate (inverse), s = 1..15.
template <int DIR, int STEP>
__device__ __forceinline__ void apply_stage_twiddles(float2* v, const float2* w) {
#pragma unroll
    for (int s = 1; s < 16; ++s) {
        const float2 t = w[(s - 1) * STEP];
        v[s] = DIR < 0 ? cmul(v[s], t) : cmul(v[s], cconj(t));
    }
}

// fft_ct.cuh's ct_fft for 9 <= LOG2N <= 12 (three stages: radix-R0, radix-16
// at Ns = R0, radix-16 at Ns = n/16; natural order in and out, x[j + q s] in
// v[s] on entry, X[j + q r] in v[r] on exit), stage twiddles from the shared
// tables. sm is this column's view of the padded exchange buffer
// (PadLayout<SL, S> from base + c); contains CTA barriers;
// after_last_exchange() runs on every thread once the buffer is no longer read.
template <int DIR, int LOG2N, int SL, int S, typename F>
__device__ __forceinline__ void tw_fft(float2* v, float2* sm, int j, const StageTwiddles<LOG2N>& t,
                                       F&& after_last_exchange) {
    using L = PadLayout<SL, S>;
    constexpr int q = (1 << LOG2N) >> 4;
    constexpr int r0log = LOG2N - 8;
    constexpr int R0 = 1 << r0log;
    constexpr int G = 16 / R0;
    reg_first_stage<R0, DIR>(v);
    {
        // output r of first-stage butterfly j + q t goes to (j + q t) R0 + r
        float2* w = sm + L::off(j * R0);
#pragma unroll
        for (int tt = 0; tt < G; ++tt)
#pragma unroll
            for (int r = 0; r < R0; ++r) w[L::off(q * tt * R0 + r)] = v[tt * R0 + r];
    }
    __syncthreads();
    ct_read<SL, S, LOG2N>(v, sm, j);
    __syncthreads();
    apply_stage_twiddles<DIR, R0>(v, t.a);
    dft_reg<16, DIR>(v);
    {
        // output r of butterfly j goes to (j - k) 16 + k + R0 r, k = j mod R0
        const int k = j & (R0 - 1);
        float2* w = sm + L::off((j - k) * 16 + k);
#pragma unroll
        for (int r = 0; r < 16; ++r) w[L::off(R0 * r)] = v[r];
    }
    __syncthreads();
    ct_read<SL, S, LOG2N>(v, sm, j);
    __syncthreads();
    after_last_exchange();
    apply_stage_twiddles<DIR, q>(v, t.b);
    dft_reg<16, DIR>(v);
}

// MODE: -1 forward FFT, +1 inverse FFT, 0 the fused forward x V x inverse pass
// along axis 0 (V = Lambda^T / N, from a table or evaluated per element).
// Tile t covers column group x = t mod gx (columns x*CPT ..), mid index
// y = (t / gx) mod g.mid and outer index z = t / (gx g.mid), as in ColGeom.
template <int MODE, int RAD, int LOG2N, int BLK>
__global__ void __launch_bounds__(kTileThreads, 2)
k_cols_tma(float2* __restrict__ H, const __grid_constant__ CUtensorMap map,
           const __grid_constant__ ColGeom g, const float2* __restrict__ tw, int twn_log2,
           const __grid_constant__ SymbolSet ps, int* status, int gx, int ntiles) {
    constexpr int n = 1 << LOG2N;
    constexpr int q = n >> 4;
    constexpr int CL = tma_cols_log2(LOG2N);
    constexpr int CPT = 1 << CL;
    constexpr uint32_t kTileBytes = kTileElems * 8;
    extern __shared__ __align__(1024) unsigned char smraw[];
    float2* buf = reinterpret_cast<float2*>(smraw);
    float2* ta = reinterpret_cast<float2*>(smraw + kTmaBufBytes);
    float2* tb = reinterpret_cast<float2*>(smraw + kTmaBufBytes + kTmaTwABytes);
    const uint32_t bar = smem_u32(smraw + tma_smem_bytes(LOG2N) - 16);
    const uint32_t bufa = smem_u32(buf);
    const int c = threadIdx.x & (CPT - 1);
    const int j = threadIdx.x >> CL;
    const bool leader = threadIdx.x == 0;

    auto issue = [&](int tile) {
        const int x = tile % gx;
        const int rest = tile / gx;
        const int y = rest % g.mid;
        const int z = rest / g.mid;
        mbar_expect_tx(bar, kTileBytes);
        if constexpr (BLK)
            bulk_load(bufa, H + (long long)z * g.os + (long long)x * kTileElems, kTileBytes, bar);
        else
            tma_load_5d(bufa, &map, x * 2 * CPT, y, 0, 0, z, bar);
    };

    if (leader) {
        mbar_init(bar, 1);
        mbar_fence_init();
        fence_async_shared();
    }
    __syncthreads();
    if (leader && (int)blockIdx.x < ntiles) issue(blockIdx.x);
    const StageTwiddles<LOG2N> tws = fill_stage_twiddles<LOG2N>(ta, tb, j, tw, twn_log2);
    float2* sm = buf + c;   // this column's view: PadLayout<CL, 4 - CL> from base + c

    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const bool ok = mbar_wait(bar, it & 1);
        if (__syncthreads_or(!ok)) {
            // give up: record it, let the load in flight land (bounded), end the CTA
            if (leader) {
                atomicOr(status, kGemmTimeout);
                mbar_wait(bar, it & 1);
            }
            return;
        }
        float2 v[16];
        {
            const float2* src = buf + j * CPT + c;   // dense [row][CPT] as the tile landed
#pragma unroll
            for (int s = 0; s < 16; ++s) v[s] = src[s * q * CPT];
        }
        __syncthreads();   // every thread has its elements: the buffer is the exchange buffer now
        const int next = tile + (int)gridDim.x;
        auto refill = [&]() {
            if (leader && next < ntiles) {
                fence_async_shared();
                issue(next);
            }
        };
        auto nothing = [] {};
        const int x = tile % gx;
        const int rest = tile / gx;
        const int y = rest % g.mid;
        const int z = rest / g.mid;
        const int i0 = x * CPT;
        const bool live = i0 + c < g.inner_valid;
        if constexpr (MODE == 0) {
            tw_fft<-1, LOG2N, CL, 4 - CL>(v, sm, j, tws, nothing);
            const SymbolParams& p = ps.p[ps.orient[z]];
            const float2* vt = static_cast<const float2*>(ps.vtab_item[z] ? ps.vtab_item[z]
                                                                          : ps.vtab[ps.orient[z]]);
            if (BLK && vt && ps.vflags) {
                // blocked table: this tile's 64 KB block, or nothing at all when
                // every multiplier of the block is zero
                if (__ldg(ps.vflags + x)) {
                    const float2* vb = vt + (long long)x * kTileElems + c;
#pragma unroll
                    for (int r = 0; r < 16; ++r) v[r] = cmul(v[r], __ldg(vb + (j + q * r) * CPT));
                } else {
#pragma unroll
                    for (int r = 0; r < 16; ++r) v[r] = float2{0.f, 0.f};
                }
            } else if (vt) {
                // multipliers shared by every solve of this shape and T
                const float2* vb = vt + (long long)y * g.ms + i0 + c;
                const long long vs = BLK ? g.vS : g.S;   // tables keep the row-major layout
                if (live) {
#pragma unroll
                    for (int r = 0; r < 16; ++r)
                        v[r] = cmul(v[r], __ldg(vb + (long long)(j + q * r) * vs));
                }
            } else {
                int k[3];
                if (p.ndim == 2) {
                    k[1] = i0 + c;
                    k[2] = 0;
                } else {
                    k[1] = y;
                    k[2] = i0 + c;
                }
                ColSymbol<RAD> cs;
                col_symbol_init<RAD>(p, k, cs);
                const ColView<float2> cv{buf, c, CL};
                apply_multiplier<RAD>(v, cv, j, q, p, cs, k[1], k[2]);
            }
            __syncthreads();
            tw_fft<+1, LOG2N, CL, 4 - CL>(v, sm, j, tws, refill);
        } else {
            tw_fft<MODE, LOG2N, CL, 4 - CL>(v, sm, j, tws, refill);
        }
        if constexpr (BLK) {
            // the whole block goes back (a ragged block's extra columns are
            // finite padding that no pass reads as data)
            float2* dst = H + (long long)z * g.os + (long long)x * kTileElems + c;
#pragma unroll
            for (int r = 0; r < 16; ++r) dst[(j + q * r) * CPT] = v[r];
        } else if (live) {
            float2* dst = H + (long long)z * g.os + (long long)y * g.ms + i0 + c;
#pragma unroll
            for (int r = 0; r < 16; ++r) dst[(long long)(j + q * r) * g.S] = v[r];
        }
    }
}

}  // namespace sfft
