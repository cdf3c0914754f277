// Launchers of the persistent TMA-fed column passes (cols_tma.cuh) for FP32
// half spectra: tensor-map encoding, eligibility and the kernel dispatch.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "cols_tma.cuh"
#include "rows_tma.cuh"
#include "rows_blk.cuh"
#include "internal.h"

namespace sfft {

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (the library
// links only the CUDA runtime); null when the driver does not provide it.
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

int sm_count() {
    static std::mutex mu;
    static int count[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lock(mu);
    if (!count[dev]) cudaDeviceGetAttribute(&count[dev], cudaDevAttrMultiProcessorCount, dev);
    return count[dev];
}

// STENCILFFT_COLS=reg selects the register column kernels instead (A/B timing).
bool tma_enabled() {
    static bool on = [] {
        const char* e = std::getenv("STENCILFFT_COLS");
        return !(e && std::strcmp(e, "reg") == 0);
    }();
    return on && pass_variant() < 2;
}

// 5-D view of the passes' geometry: (floats of a row of columns, mid, 256 rows,
// n/256 row blocks, outer); box = one tile.
cudaError_t make_map(CUtensorMap* map, void* H, const ColGeom& g) {
    const int n = 1 << g.log2n;
    const int cpt = 1 << tma_cols_log2(g.log2n);
    const long long srow = g.S * 8;                       // bytes between rows of the axis
    const long long smid = g.mid > 1 ? g.ms * 8 : srow;   // unused extent-1 axis: any valid stride
    cuuint64_t dim[5] = {(cuuint64_t)(2 * g.inner_valid), (cuuint64_t)g.mid, 256,
                         (cuuint64_t)(n / 256), (cuuint64_t)g.outer};
    cuuint64_t stride[4] = {(cuuint64_t)smid, (cuuint64_t)srow, (cuuint64_t)(256 * srow),
                            (cuuint64_t)(g.outer > 1 ? g.os * 8 : (long long)n * srow)};
    cuuint32_t box[5] = {(cuuint32_t)(2 * cpt), 1, 256, (cuuint32_t)(n / 256), 1};
    cuuint32_t estride[5] = {1, 1, 1, 1, 1};
    const CUresult r = encode_tiled()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, H, dim, stride, box,
                                      estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int L, typename F>
cudaError_t with_len(int l, F&& f) {
    if constexpr (L > kTmaLog2Hi) {
        return cudaErrorNotSupported;
    } else {
        if (l == L) return f(std::integral_constant<int, L>{});
        return with_len<L + 1>(l, f);
    }
}

template <int MODE, int RAD, int LOG2N, int BLK = 0>
cudaError_t launch_t(void* H, const ColGeom& g, const CUtensorMap& map, const void* tw,
                     int twn_log2, const SymbolSet& ps, int* status, cudaStream_t s) {
    const size_t smem = tma_smem_bytes(LOG2N);
    auto kern = k_cols_tma<MODE, RAD, LOG2N, BLK>;
    cudaError_t err = smem_optin(reinterpret_cast<const void*>(kern), smem);
    if (err != cudaSuccess) return err;
    const int cpt = 1 << tma_cols_log2(LOG2N);
    const int gx = (g.inner_valid + cpt - 1) / cpt;
    const long long ntiles = (long long)gx * g.mid * g.outer;
    const int nsm = sm_count();
    const long long slots = 2ll * nsm;   // two CTAs per SM
    const int grid = (int)(ntiles < slots ? ntiles : slots);
    kern<<<grid, kTileThreads, smem, s>>>(static_cast<float2*>(H), map, g,
                                          static_cast<const float2*>(tw), twn_log2, ps, status, gx,
                                          (int)ntiles);
    return cudaGetLastError();
}

template <int DIR, int LOG2N>
cudaError_t launch_rows_t(const void* src, void* dst, long long Mp, int nrows, const void* tw,
                          int twn_log2, int* status, cudaStream_t s) {
    const size_t smem = row_tma_smem(LOG2N);
    auto kern = k_rows_tma<DIR, LOG2N>;
    cudaError_t err = smem_optin(reinterpret_cast<const void*>(kern), smem);
    if (err != cudaSuccess) return err;
    const int rpt = row_tma_rows(LOG2N);
    const long long ntiles = (nrows + rpt - 1) / rpt;
    const long long slots = 4ll * sm_count();   // four CTAs per SM
    const int grid = (int)(ntiles < slots ? ntiles : slots);
    kern<<<grid, kRowThreads, smem, s>>>(static_cast<const float2*>(src), static_cast<float2*>(dst),
                                         Mp, nrows, static_cast<const float2*>(tw), twn_log2,
                                         status);
    return cudaGetLastError();
}

template <int L, typename F>
cudaError_t with_row_len(int l, F&& f) {
    if constexpr (L > kRowTmaLog2Hi) {
        return cudaErrorNotSupported;
    } else {
        if (l == L) return f(std::integral_constant<int, L>{});
        return with_row_len<L + 1>(l, f);
    }
}

}  // namespace

bool rows_tma_ok(const void* grid, const void* H, long long Mp, int n_log2, int nrows) {
    if (!tma_enabled() || sm_count() <= 0) return false;
    if (n_log2 < kRowTmaLog2Lo || n_log2 > kRowTmaLog2Hi || nrows < 1) return false;
    const long long n = 1ll << n_log2;
    return reinterpret_cast<uintptr_t>(grid) % 16 == 0 && reinterpret_cast<uintptr_t>(H) % 16 == 0 &&
           Mp % 2 == 0 && Mp >= n + 2;
}

cudaError_t launch_rows_tma(int dir, const void* src, void* dst, long long Mp, int n_log2,
                            int nrows, const void* tw, int twn_log2, int* status, cudaStream_t s) {
    const void* grid = dir < 0 ? src : dst;
    const void* H = dir < 0 ? dst : src;
    if (!rows_tma_ok(grid, H, Mp, n_log2, nrows)) return cudaErrorNotSupported;
    return with_row_len<kRowTmaLog2Lo>(n_log2, [&](auto tag) -> cudaError_t {
        constexpr int L = decltype(tag)::value;
        if (dir < 0) return cudaErrorNotSupported;   // R2C: the register row kernel
        return launch_rows_t<+1, L>(src, dst, Mp, nrows, tw, twn_log2, status, s);
    });
}

// Blocked-layout row passes (rows_blk.cuh) for packed row length 2^n_log2 and
// 2^cl columns per block.
template <int L, int CL, bool R2C>
cudaError_t launch_blk_t(const void* src, void* dst, int l0_log2, long long os, int nrows,
                         const void* tw, int twn_log2, int* status, cudaStream_t s) {
    const size_t smem = blk_smem(L, CL);
    const int rpt = blk_rows(L);
    const int grid = (nrows + rpt - 1) / rpt;
    if (R2C) {
        auto kern = k_rows_r2c_blk<L, CL>;
        cudaError_t err = smem_optin(reinterpret_cast<const void*>(kern), smem);
        if (err != cudaSuccess) return err;
        kern<<<grid, blk_threads(L), smem, s>>>(static_cast<const float2*>(src),
                                                static_cast<float2*>(dst), l0_log2, os, nrows,
                                                static_cast<const float2*>(tw), twn_log2);
    } else {
        auto kern = k_rows_c2r_blk<L, CL>;
        cudaError_t err = smem_optin(reinterpret_cast<const void*>(kern), smem);
        if (err != cudaSuccess) return err;
        kern<<<grid, blk_threads(L), smem, s>>>(static_cast<const float2*>(src),
                                                static_cast<float2*>(dst), l0_log2, os, nrows,
                                                static_cast<const float2*>(tw), twn_log2, status);
    }
    return cudaGetLastError();
}

template <int L, typename F>
cudaError_t with_blk_len(int l, F&& f) {
    if constexpr (L > kBlkLog2Hi) {
        return cudaErrorNotSupported;
    } else {
        if (l == L) return f(std::integral_constant<int, L>{});
        return with_blk_len<L + 1>(l, f);
    }
}

template <int CL, typename F>
cudaError_t with_cl(int cl, F&& f) {
    if constexpr (CL > 4) {
        return cudaErrorNotSupported;
    } else {
        if (cl == CL) return f(std::integral_constant<int, CL>{});
        return with_cl<CL + 1>(cl, f);
    }
}

bool cols_tma_ok(const void* H, const ColGeom& g) {
    if (!tma_enabled() || !encode_tiled() || sm_count() <= 0) return false;
    if (g.log2n < kTmaLog2Lo || g.log2n > kTmaLog2Hi) return false;
    if (reinterpret_cast<uintptr_t>(H) % 16) return false;
    // strides are whole 16-byte units (two FP32 complex values)
    if ((g.S & 1) || (g.mid > 1 && (g.ms & 1)) || (g.outer > 1 && (g.os & 1))) return false;
    const long long tiles = (long long)((g.inner_valid + (1 << tma_cols_log2(g.log2n)) - 1) >>
                                        tma_cols_log2(g.log2n)) *
                            g.mid * g.outer;
    return g.inner_valid > 0 && tiles < (1ll << 31);
}

cudaError_t launch_cols_tma(void* H, const ColGeom& g, int mode, const void* tw, int twn_log2,
                            const SymbolSet* ps, int* status, cudaStream_t s) {
    if (!cols_tma_ok(H, g) || (mode == 0 && !ps)) return cudaErrorNotSupported;
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    cudaError_t err = make_map(&map, H, g);
    if (err != cudaSuccess) return cudaErrorNotSupported;
    static const SymbolSet kNone = [] {
        SymbolSet z;
        std::memset(&z, 0, sizeof(z));
        return z;
    }();
    const SymbolSet& set = ps ? *ps : kNone;
    return with_len<kTmaLog2Lo>(g.log2n, [&](auto tag) -> cudaError_t {
        constexpr int L = decltype(tag)::value;
        if (mode < 0) return launch_t<-1, 0, L>(H, g, map, tw, twn_log2, set, status, s);
        if (mode > 0) return launch_t<+1, 0, L>(H, g, map, tw, twn_log2, set, status, s);
        switch (set.p[0].r) {
            case 0: return launch_t<0, 0, L>(H, g, map, tw, twn_log2, set, status, s);
            case 1: return launch_t<0, 1, L>(H, g, map, tw, twn_log2, set, status, s);
            case 2: return launch_t<0, 2, L>(H, g, map, tw, twn_log2, set, status, s);
            default: return launch_t<0, 3, L>(H, g, map, tw, twn_log2, set, status, s);
        }
    });
}

// STENCILFFT_BLOCKED=0 keeps row-major half spectra for 2-D solves (A/B timing).
static bool blocked_enabled() {
    static bool on = [] {
        const char* e = std::getenv("STENCILFFT_BLOCKED");
        return !(e && std::strcmp(e, "0") == 0);
    }();
    return on && pass_variant() < 1;
}

// V = Lambda^T / N in the blocked layout of the half spectrum (one 2-D item)
// and one flag per column block: set when a multiplier of the block is not 0.
__global__ void k_vtable_blk(float2* __restrict__ V, int* __restrict__ flags,
                             const __grid_constant__ SymbolParams p, int l0_log2, int cl, int n,
                             long long total) {
    const int l0 = 1 << l0_log2, cpt = 1 << cl;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(e >> 13);              // 8192 values per block
        const int rem = (int)(e & 8191);
        const int i = rem >> cl, c = rem & (cpt - 1);
        const int k1 = x * cpt + c;
        float2 v{0.f, 0.f};
        if (k1 <= n) {
            const int k[3] = {i, k1, 0};
            v = spectral_multiplier<float2>(p, k);
        }
        V[e] = v;
        if (v.x != 0.f || v.y != 0.f) flags[x] = 1;
    }
    (void)l0;
}

static int log2_or_neg(int64_t v) {
    if (v <= 0 || (v & (v - 1))) return -1;
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return l;
}

bool blocked_shape(int ndim, const int64_t* dims) {
    if (ndim != 2) return false;
    const int l0 = log2_or_neg(dims[0]), l1 = log2_or_neg(dims[1]);
    if (l0 < 0 || l1 < 0) return false;
    return l0 >= kTmaLog2Lo && l0 <= kTmaLog2Hi && l1 - 1 >= kBlkLog2Lo && l1 - 1 <= kBlkLog2Hi;
}

cudaError_t launch_vtable_blk(void* V, int* flags, const SymbolParams& p, int l0_log2, int n_log2,
                              cudaStream_t s) {
    const long long total = blocked_item_elems(l0_log2, n_log2);
    const int nx = (int)(total >> 13);
    cudaError_t err = cudaMemsetAsync(flags, 0, nx * sizeof(int), s);
    if (err != cudaSuccess) return err;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_vtable_blk<<<(int)blocks, 256, 0, s>>>(static_cast<float2*>(V), flags, p, l0_log2,
                                             tma_cols_log2(l0_log2), 1 << n_log2, total);
    return cudaGetLastError();
}

bool blocked_ok(const void* grid, const void* H, int l0_log2, int n_log2) {
    if (!tma_enabled() || !blocked_enabled() || sm_count() <= 0) return false;
    if (l0_log2 < kTmaLog2Lo || l0_log2 > kTmaLog2Hi) return false;
    if (n_log2 < kBlkLog2Lo || n_log2 > kBlkLog2Hi) return false;
    return reinterpret_cast<uintptr_t>(grid) % 16 == 0 && reinterpret_cast<uintptr_t>(H) % 16 == 0;
}

long long blocked_item_elems(int l0_log2, int n_log2) {
    const int cl = tma_cols_log2(l0_log2);
    const long long nx = (((long long)1 << n_log2) + 1 + (1 << cl) - 1) >> cl;
    return nx << 13;   // nx blocks of 8192 values
}

cudaError_t launch_rows_blk(int dir, const void* src, void* dst, int l0_log2, int n_log2,
                            int nrows, const void* tw, int twn_log2, int* status, cudaStream_t s) {
    const void* grid = dir < 0 ? src : dst;
    const void* H = dir < 0 ? dst : src;
    if (!blocked_ok(grid, H, l0_log2, n_log2) || nrows % (1 << l0_log2)) return cudaErrorNotSupported;
    const long long os = blocked_item_elems(l0_log2, n_log2);
    return with_blk_len<kBlkLog2Lo>(n_log2, [&](auto tl) -> cudaError_t {
        constexpr int L = decltype(tl)::value;
        return with_cl<1>(tma_cols_log2(l0_log2), [&](auto tc) -> cudaError_t {
            constexpr int CL = decltype(tc)::value;
            if (dir < 0)
                return launch_blk_t<L, CL, true>(src, dst, l0_log2, os, nrows, tw, twn_log2,
                                                  status, s);
            return launch_blk_t<L, CL, false>(src, dst, l0_log2, os, nrows, tw, twn_log2, status,
                                              s);
        });
    });
}

cudaError_t launch_cols_tma_blk(void* H, const ColGeom& g, const void* tw, int twn_log2,
                                const SymbolSet& ps, int* status, cudaStream_t s) {
    if (!tma_enabled() || sm_count() <= 0 || g.log2n < kTmaLog2Lo || g.log2n > kTmaLog2Hi ||
        g.mid != 1 || reinterpret_cast<uintptr_t>(H) % 16)
        return cudaErrorNotSupported;
    CUtensorMap map;   // unused by the blocked kernels
    std::memset(&map, 0, sizeof(map));
    return with_len<kTmaLog2Lo>(g.log2n, [&](auto tag) -> cudaError_t {
        constexpr int L = decltype(tag)::value;
        switch (ps.p[0].r) {
            case 0: return launch_t<0, 0, L, 1>(H, g, map, tw, twn_log2, ps, status, s);
            case 1: return launch_t<0, 1, L, 1>(H, g, map, tw, twn_log2, ps, status, s);
            case 2: return launch_t<0, 2, L, 1>(H, g, map, tw, twn_log2, ps, status, s);
            default: return launch_t<0, 3, L, 1>(H, g, map, tw, twn_log2, ps, status, s);
        }
    });
}

}  // namespace sfft
