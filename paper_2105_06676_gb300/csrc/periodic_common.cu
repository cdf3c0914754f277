// Non-template kernels and helpers of the periodic path: per-axis symbol
// tables, the FP64 Lambda^T table, launch-shape helpers.
#include <cuda_runtime.h>

#include <cstdlib>
#include <map>
#include <mutex>

#include "fft_reg.cuh"
#include "internal.h"

namespace sfft {

__global__ void k_axis_table(double2* E64, float2* E32, int len) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < len; q += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)q / (double)len, &s, &c);  // exp(+2 pi i q / len)
        E64[q] = double2{c, s};
        E32[q] = float2{(float)c, (float)s};
    }
}

// V[k] = Lambda[k]^T (FP64, natural order of the half spectrum).
__global__ void k_symbol_table(double2* out, const __grid_constant__ SymbolParams p,
                               int nlast_half, long long total) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int k[3];
        long long rest = e;
        k[p.ndim - 1] = (int)(rest % nlast_half);
        rest /= nlast_half;
        for (int a = p.ndim - 2; a >= 0; --a) {
            k[a] = (int)(rest % p.len[a]);
            rest /= p.len[a];
        }
        out[e] = lambda_pow64(p, k);
    }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
static thread_local int t_pass_variant = -1;
int pass_variant() { return t_pass_variant; }
PassVariantScope::PassVariantScope(int v) : saved(t_pass_variant) { t_pass_variant = v; }
PassVariantScope::~PassVariantScope() { t_pass_variant = saved; }

cudaError_t smem_optin(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    size_t& have = done[{kernel, dev}];
    if (bytes <= have) return cudaSuccess;
    cudaError_t err =
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (err == cudaSuccess) have = bytes;
    return err;
}

int cols_log2_for(int log2n, int elem_bytes, int max_threads) {
    const int n = 1 << log2n;
    int cl = 0;
    while (cl < 4) {
        const int next = 1 << (cl + 1);
        const long long smem = (long long)next * seq_stride(n) * elem_bytes;
        if (smem > kSmemBudget || (long long)next * n > (long long)kEPT * max_threads) break;
        ++cl;
    }
    return cl;
}

int rows_per_cta_for(int n_log2, int elem_bytes, int max_threads) {
    const int n = 1 << n_log2;
    int rpc = 1;
    while (rpc * 2 * n <= 4096 && (long long)rpc * 2 * seq_stride(n) * elem_bytes <= kSmemBudget &&
           rpc * 2 * n <= kEPT * max_threads)
        rpc *= 2;
    return rpc;
}

cudaError_t launch_axis_table(double2* E64, float2* E32, int len, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (len + threads - 1) / threads;
    k_axis_table<<<blocks, threads, 0, s>>>(E64, E32, len);
    return cudaGetLastError();
}

cudaError_t launch_symbol_table(double2* out, const SymbolParams& p, int nlast_half,
                                long long total, cudaStream_t s) {
    const int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    if (blocks > 65535) blocks = 65535;
    if (blocks < 1) blocks = 1;
    k_symbol_table<<<(int)blocks, threads, 0, s>>>(out, p, nlast_half, total);
    return cudaGetLastError();
}

}  // namespace sfft
