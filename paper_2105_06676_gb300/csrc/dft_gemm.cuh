// Radix-16 DFT butterflies as tensor-core GEMMs (tcgen05, sm_103a).
//
// The 16-point DFT of paper Sec. 4's Multi-FFT, y_u = sum_t x_t w^(t u) with
// w = exp(DIR 2 pi i / 16), is a dense contraction. For a CTA whose 256 threads
// each hold one butterfly's 16 complex inputs, the stage is one real GEMM
//   D[256 x 32] = A[256 x 32] . B[32 x 32]^T,
//   A row  = (Re x_0..15, Im x_0..15)            (the thread's inputs),
//   B rows = (Re y_u | Im y_u) as linear forms of that row (cos / sin of the DFT),
// run as two M = 128, N = 32 tiles of tcgen05.mma kind::f16 with K = 2 x 16,
// operands in shared memory (K-major, no swizzle), FP32 accumulators in tensor
// memory, read back one row per thread with tcgen05.ld.
//
// Operand precision (both operands the same type):
//   kGemmBF16   : A, B rounded to bf16, one product;
//   kGemmFP16   : fp16, one product;
//   kGemmBF16x3 : x = hi + lo split in bf16, products hi.hi + lo.hi + hi.lo.
// Each row is scaled by a power of two (exact) so that its largest component
// lies in [0.5, 1) before rounding, which keeps fp16 in range; the outputs are
// scaled back.
//
// Synchronisation per stage: every thread writes its A row, makes it visible
// to the tensor core's async proxy (fence.proxy.async) and meets the others at
// a barrier; thread 0 issues the MMAs and commits them to an mbarrier; all
// threads wait on it, then load their row. Waits are bounded in time
// (kWaitLimitNs of %globaltimer): a CTA whose wait runs out records kGemmTimeout
// in its status word and sets its abandoned flag; from then on it issues no
// MMA and waits on nothing (its remaining butterflies return whatever tensor
// memory holds, and the status word reports the failure), and before releasing
// tensor memory it waits once more (bounded) for the abandoned stage's MMAs.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "fft_common.cuh"

namespace sfft {

constexpr int kGemmBF16 = 0;
constexpr int kGemmFP16 = 1;
constexpr int kGemmBF16x3 = 2;

constexpr int kGemmRows = 256;            // butterflies (threads) per CTA
constexpr int kGemmTmemCols = 64;         // two 128-row tiles x 32 FP32 columns
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s per bounded wait
constexpr int kGemmTimeout = 4;           // status bit for an abandoned wait

// Shared-memory operand layout, K-major without swizzle: 8-row x 16-byte core
// matrices; element (row, k) of a 16-bit operand at
//   (row / 8) * kSbo + (k / 8) * kLbo + (row % 8) * 16 + (k % 8) * 2.
constexpr uint32_t kLbo = 128;            // next core matrix along K
constexpr uint32_t kSbo = 512;            // next 8-row group (K = 32 per row)
constexpr uint32_t kOperandRowBytes = 64;
constexpr uint32_t kABytes = kGemmRows * kOperandRowBytes;   // 16 KB per term
constexpr uint32_t kBBytes = 32 * kOperandRowBytes;          // 2 KB per term

__device__ __forceinline__ uint32_t operand_offset(int row, int k) {
    return (uint32_t)(row >> 3) * kSbo + (uint32_t)(k >> 3) * kLbo + (uint32_t)(row & 7) * 16 +
           (uint32_t)(k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start, leading (K) and stride (M/N)
// byte offsets in 16-byte units, the fixed 0b001 field at bit 46, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(kLbo >> 4) << 16) |
           ((uint64_t)(kSbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator, A and B of type fmt
// (0 = f16, 1 = bf16), both K-major, N = 32, M = 128.
__host__ __device__ constexpr uint32_t gemm_idesc(int fmt) {
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((32u >> 3) << 17) |
           ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     mbar)
                 : "memory");
}

__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait for the mbarrier phase with parity `parity`, bounded in time
// (kWaitLimitNs of the global nanosecond timer); false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    unsigned long long start = 0;
    for (unsigned i = 0;; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if (i == 0) start = global_ns();
        else if ((i & 63) == 0 && global_ns() - start > kWaitLimitNs) return false;
        if (i == 0xFFFFFFFFu) return false;   // backstop should the timer not advance
    }
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* out) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) out[i] = __uint_as_float(r[i]);
}

// 16-bit operand element of type MODE's format.
template <int MODE>
__device__ __forceinline__ uint16_t to_op(float x) {
    if constexpr (MODE == kGemmFP16) return __half_as_ushort(__float2half_rn(x));
    else return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
template <int MODE>
__device__ __forceinline__ float from_op(uint16_t h) {
    if constexpr (MODE == kGemmFP16) return __half2float(__ushort_as_half(h));
    else return __bfloat162float(__ushort_as_bfloat16(h));
}

// Per-CTA state of the GEMM butterflies. Shared memory (carved by the kernel):
// A terms (hi, lo), B terms for the forward and the inverse DFT (hi, lo), one
// mbarrier, the tensor-memory base address.
template <int MODE>
struct DftGemm {
    static constexpr int kTerms = MODE == kGemmBF16x3 ? 2 : 1;
    unsigned char* a;        // kTerms x kABytes
    unsigned char* b;        // 2 directions x kTerms x kBBytes
    uint32_t mbar;           // shared address of the mbarrier
    uint32_t tmem;           // tensor-memory base (lane 0, column 0)
    uint32_t phase;          // parity of the next mbarrier phase
    int* status;
    // shared words: [0] abandoned (a wait ran out), [1] an MMA commit of the
    // abandoned stage was issued, [2] that stage's phase
    uint32_t* flags;
    // test hook: issue no MMA and no commit, so that every wait runs out
    bool skip_commit;

    static constexpr size_t smem_bytes() {
        return (size_t)kTerms * kABytes + 2 * (size_t)kTerms * kBBytes + 32;
    }

    // Builds B (both directions), initialises the mbarrier and allocates
    // tensor memory. Every thread of the CTA calls it; it ends with a barrier.
    __device__ void init(unsigned char* smem, uint32_t* tmem_slot, int* st, bool no_commit) {
        a = smem;
        b = smem + kTerms * kABytes;
        unsigned char* mb = b + 2 * kTerms * kBBytes;
        mbar = smem_u32(mb);
        flags = reinterpret_cast<uint32_t*>(mb + 16);
        status = st;
        phase = 0;
        skip_commit = no_commit;
        if (threadIdx.x < 3) flags[threadIdx.x] = 0;
        // B[n][k] for n < 16: Re y_n from (Re x_k | Im x_k); n >= 16: Im y_(n-16)
        for (int e = threadIdx.x; e < 2 * 32 * 32; e += blockDim.x) {
            const int dir = e >> 10;             // 0: forward (w = e^{-2 pi i/16}), 1: inverse
            const int n = (e >> 5) & 31, k = e & 31;
            const int t = k & 15, u = n & 15;
            const int q = (t * u) & 15;
            const double c = cos16(q);
            const double s = (dir ? 1.0 : -1.0) * sin16(q);
            double v;
            if (n < 16) v = k < 16 ? c : -s;     // Re y_u = sum Re x_t c - Im x_t s
            else v = k < 16 ? s : c;             // Im y_u = sum Re x_t s + Im x_t c
            const float vf = (float)v;
            const uint16_t hi = to_op<MODE>(vf);
            unsigned char* bd = b + (size_t)dir * kTerms * kBBytes;
            *reinterpret_cast<uint16_t*>(bd + operand_offset(n, k)) = hi;
            if constexpr (kTerms == 2) {
                const uint16_t lo = to_op<MODE>(vf - from_op<MODE>(hi));
                *reinterpret_cast<uint16_t*>(bd + kBBytes + operand_offset(n, k)) = lo;
            }
        }
        if (threadIdx.x == 0) mbar_init(mbar, 1);
        if (threadIdx.x < 32) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"((uint32_t)kGemmTmemCols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        fence_async_shared();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        tmem = *tmem_slot;
    }

    // Releases tensor memory. Every thread calls it after its last dft16. After
    // an abandoned wait whose MMAs were issued, first waits once more (bounded)
    // for them.
    __device__ void finish() {
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (flags[0] && flags[1]) mbar_wait(mbar, flags[2]);
        if (threadIdx.x < 32)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                         "r"((uint32_t)kGemmTmemCols)
                         : "memory");
    }

    // v[u] <- sum_t v[t] exp(DIR 2 pi i t u / 16) for this thread's butterfly
    // (row threadIdx.x of the GEMM). Every thread of the CTA calls it together.
    template <int DIR>
    __device__ void dft16(float2* v) {
        const int row = threadIdx.x;
        // power-of-two row scale: largest component into [0.5, 1)
        float m = 0.f;
#pragma unroll
        for (int t = 0; t < 16; ++t) m = fmaxf(m, fmaxf(fabsf(v[t].x), fabsf(v[t].y)));
        int e = 0;
        if (m > 0.f) frexpf(m, &e);
        uint32_t hi_re[8], hi_im[8], lo_re[8], lo_im[8];
#pragma unroll
        for (int t = 0; t < 16; t += 2) {
            float xr0 = ldexpf(v[t].x, -e), xr1 = ldexpf(v[t + 1].x, -e);
            float xi0 = ldexpf(v[t].y, -e), xi1 = ldexpf(v[t + 1].y, -e);
            const uint16_t hr0 = to_op<MODE>(xr0), hr1 = to_op<MODE>(xr1);
            const uint16_t hi0 = to_op<MODE>(xi0), hi1 = to_op<MODE>(xi1);
            hi_re[t / 2] = (uint32_t)hr0 | ((uint32_t)hr1 << 16);
            hi_im[t / 2] = (uint32_t)hi0 | ((uint32_t)hi1 << 16);
            if constexpr (kTerms == 2) {
                const uint16_t lr0 = to_op<MODE>(xr0 - from_op<MODE>(hr0));
                const uint16_t lr1 = to_op<MODE>(xr1 - from_op<MODE>(hr1));
                const uint16_t li0 = to_op<MODE>(xi0 - from_op<MODE>(hi0));
                const uint16_t li1 = to_op<MODE>(xi1 - from_op<MODE>(hi1));
                lo_re[t / 2] = (uint32_t)lr0 | ((uint32_t)lr1 << 16);
                lo_im[t / 2] = (uint32_t)li0 | ((uint32_t)li1 << 16);
            }
        }
        // row = (Re x_0..15 | Im x_0..15): four 16-byte chunks along K
#pragma unroll
        for (int term = 0; term < kTerms; ++term) {
            const uint32_t* re = term ? lo_re : hi_re;
            const uint32_t* im = term ? lo_im : hi_im;
            unsigned char* ad = a + (size_t)term * kABytes;
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                const uint32_t* src = ch < 2 ? re + 4 * ch : im + 4 * (ch - 2);
                *reinterpret_cast<uint4*>(ad + operand_offset(row, 8 * ch)) =
                    make_uint4(src[0], src[1], src[2], src[3]);
            }
        }
        fence_async_shared();
        tc_fence_before();
        __syncthreads();
        const bool abandoned = flags[0] != 0;   // set before the barrier above
        if (threadIdx.x == 0 && !abandoned && !skip_commit) {
            tc_fence_after();
            constexpr uint32_t idesc = gemm_idesc(MODE == kGemmFP16 ? 0 : 1);
            const unsigned char* bd = b + (size_t)(DIR < 0 ? 0 : 1) * kTerms * kBBytes;
#pragma unroll
            for (int tile = 0; tile < 2; ++tile) {
                const uint32_t d = tmem + 32u * tile;
                uint32_t acc = 0;
                // products: A_hi B_hi (+ A_lo B_hi + A_hi B_lo)
#pragma unroll
                for (int prod = 0; prod < (kTerms == 2 ? 3 : 1); ++prod) {
                    const int ta = prod == 1 ? 1 : 0, tb = prod == 2 ? 1 : 0;
                    const uint32_t a0 = smem_u32(a + (size_t)ta * kABytes + (size_t)tile * 16 * kSbo);
                    const uint32_t b0 = smem_u32(bd + (size_t)tb * kBBytes);
#pragma unroll
                    for (int kh = 0; kh < 2; ++kh) {
                        mma_f16(d, smem_desc(a0 + kh * 2 * kLbo), smem_desc(b0 + kh * 2 * kLbo),
                                idesc, acc);
                        acc = 1;
                    }
                }
            }
            mma_commit(mbar);
        }
        const bool ok = abandoned || mbar_wait(mbar, phase);
        if (__syncthreads_or(!ok) && !abandoned) {
            // the first abandoned wait of this CTA: record it; later stages issue
            // nothing and wait on nothing (flags are read after the next barrier)
            if (threadIdx.x == 0) {
                atomicOr(status, kGemmTimeout);
                flags[0] = 1;
                flags[1] = skip_commit ? 0u : 1u;
                flags[2] = phase;
            }
        }
        phase ^= 1;
        tc_fence_after();
        // warp w reads lanes 32 (w % 4) .. of tile w / 4
        const uint32_t warp = threadIdx.x >> 5;
        const uint32_t taddr = tmem + ((32u * (warp & 3)) << 16) + 32u * (warp >> 2);
        float out[32];
        tmem_ld32(taddr, out);
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = float2{ldexpf(out[u], e), ldexpf(out[16 + u], e)};
        // the next stage's MMAs overwrite these accumulators
        tc_fence_before();
    }
};

}  // namespace sfft
