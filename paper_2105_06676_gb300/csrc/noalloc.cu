// stencil_periodic_run_noalloc: the periodic solve without any device
// allocation (declared in include/stencilfft.h).
//
// Some callers cannot allocate device memory at the point where they solve:
// a latency-critical loop cannot afford cudaMalloc's implicit device
// synchronisation and unbounded cost, and a host program whose allocator has
// reserved the device memory up front (a framework's caching pool) would see a
// raw cudaMalloc fail or fragment that pool. For them this entry point takes
// all of its scratch -- twiddle and symbol tables, the half-spectrum workspace
// and the status word -- from one file-scope device array of fixed size,
// g_noalloc_scratch, which every GPU that loads this library holds until the
// process exits. The caller still passes the grid.
//
// Host code may not use g_noalloc_scratch's name as a device address: on the
// host it is only a stand-in. Every call looks the array's address up with
// cudaGetSymbolAddress on the current device (so a device reset, after which
// the module and the array are loaded again, never leaves a stale address).
// The first call on a device loads the module there and should therefore come
// before any stream capture on that device.
// Every call shares the one array and leaves its contents behind: calls whose
// work overlaps on the GPU (on different streams, or from different host
// threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "../../include/stencilfft.h"
#include "internal.h"
#include "plan_impl.h"

using namespace sfft;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the current device.
cudaError_t scratch_address(void** out) {
    void* p = nullptr;
    const cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess) return err;
    *out = p;
    return cudaSuccess;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

bool weights_symmetric(const double* w, int ndim, int r) {
    const int W = 2 * r + 1;
    int count = 1;
    for (int a = 0; a < ndim; ++a) count *= W;
    for (int i = 0; i < count; ++i) {
        int rest = i, mirror = 0, mul = 1;
        for (int a = 0; a < ndim; ++a) {
            mirror += (W - 1 - rest % W) * mul;
            rest /= W;
            mul *= W;
        }
        if (w[i] != w[mirror]) return false;
    }
    return true;
}

}  // namespace

extern "C" size_t stencil_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

extern "C" int stencil_periodic_run_noalloc(int ndim, const int64_t* dims, int radius,
                                            const double* weights, int precision, void* grid,
                                            int64_t T, void* stream) {
    if (ndim < 1 || ndim > 3 || !dims || !weights || !grid || radius < 0 || radius > kMaxRadius ||
        T < 0 || (precision != STENCIL_FP32 && precision != STENCIL_FP64))
        return STENCIL_EINVAL;
    if (reinterpret_cast<uintptr_t>(grid) % 16) return STENCIL_EINVAL;
    for (int a = 0; a < ndim; ++a) {
        if (dims[a] < 2 * radius + 1 || dims[a] < 4) return STENCIL_EINVAL;
        if (ilog2_exact(dims[a]) < 0 || dims[a] > max_axis(ndim, precision, a))
            return STENCIL_EUNSUPPORTED;
    }
    int nweights = 1;
    for (int a = 0; a < ndim; ++a) nweights *= 2 * radius + 1;
    for (int i = 0; i < nweights; ++i)
        if (!std::isfinite(weights[i])) return STENCIL_EINVAL;

    // carve the scratch array: status | twiddles | E64 | E32 | half spectrum
    const size_t celem = precision == STENCIL_FP32 ? sizeof(float2) : sizeof(double2);
    int64_t tmax = 4;
    for (int a = 0; a < ndim; ++a) tmax = dims[a] > tmax ? dims[a] : tmax;
    const int twn_log2 = ilog2_exact(tmax);
    size_t off_tw = 256;
    size_t off = align256(off_tw + (celem << twn_log2));
    size_t off_e64[3] = {0, 0, 0}, off_e32[3] = {0, 0, 0};
    for (int a = 0; a < ndim; ++a) {
        off_e64[a] = off;
        off = align256(off + sizeof(double2) * dims[a]);
        off_e32[a] = off;
        off = align256(off + sizeof(float2) * dims[a]);
    }
    const size_t off_H = off;
    const size_t H_bytes = periodic_workspace_bytes(ndim, dims, precision);
    if (off_H + H_bytes > kNoAllocScratchBytes) return STENCIL_EUNSUPPORTED;
    if (T == 0) return STENCIL_OK;

    void* base = nullptr;
    cudaError_t err = scratch_address(&base);
    if (err != cudaSuccess) return STENCIL_ECUDA;
    unsigned char* sb = static_cast<unsigned char*>(base);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    stencil_plan_s p;   // host-side description only; owns no device memory
    p.ndim = ndim;
    p.radius = radius;
    p.boundary = STENCIL_PERIODIC;
    p.precision = precision;
    p.nweights = nweights;
    p.n_cells = 1;
    for (int a = 0; a < ndim; ++a) {
        p.dims[a] = dims[a];
        p.n_cells *= dims[a];
    }
    for (int i = 0; i < nweights; ++i) p.weights[i] = weights[i];
    p.real_symbol = weights_symmetric(p.weights, ndim, radius);
    p.elem = precision == STENCIL_FP32 ? sizeof(float) : sizeof(double);
    p.status = reinterpret_cast<int*>(sb);
    p.twn_log2 = twn_log2;
    p.tw = sb + off_tw;
    for (int a = 0; a < ndim; ++a) {
        p.E64[a] = reinterpret_cast<double2*>(sb + off_e64[a]);
        p.E32[a] = reinterpret_cast<float2*>(sb + off_e32[a]);
    }
    p.H = H_bytes ? sb + off_H : nullptr;
    p.H_bytes = H_bytes;
    const int64_t n = dims[ndim - 1] / 2;
    const int64_t align = precision == STENCIL_FP32 ? 16 : 8;
    p.Mp = (n + 1 + align - 1) / align * align;

    // the array keeps the previous call's contents: reset the status word and
    // rebuild the tables for this call's sizes
    err = cudaMemsetAsync(p.status, 0, sizeof(int), s);
    if (err == cudaSuccess)
        err = precision == STENCIL_FP32 ? launch_twiddles<float>(p.tw, twn_log2, s)
                                        : launch_twiddles<double>(p.tw, twn_log2, s);
    for (int a = 0; a < ndim && err == cudaSuccess; ++a)
        err = launch_axis_table(p.E64[a], p.E32[a], (int)dims[a], s);
    if (err == cudaSuccess)
        err = precision == STENCIL_FP32
                  ? periodic_solve<float>(&p, static_cast<float*>(grid), p.dims, T, p.H, p.Mp,
                                          p.tw, p.twn_log2, p.E64, p.E32, p.status, s)
                  : periodic_solve<double>(&p, static_cast<double*>(grid), p.dims, T, p.H, p.Mp,
                                           p.tw, p.twn_log2, p.E64, p.E32, p.status, s);
    return err == cudaSuccess ? STENCIL_OK : STENCIL_ECUDA;
}
