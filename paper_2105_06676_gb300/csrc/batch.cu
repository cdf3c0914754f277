// Batched small periodic solves of mixed shapes in one persistent launch
// (declared in include/stencilfft.h as stencil_batch_*).
//
// The paper solves the strips of a node "in parallel" and the Multi-FFT runs
// one transform per axis with every other index in parallel (Sec. 4, Fig.
// "stencil-fft-algorithm-dD"; Sec. 5.2). For many small requests -- each too
// small to fill the GPU, each of its own shape, stencil and T -- the executor
// keeps a device work list of request descriptors and launches ONE persistent
// kernel: every CTA takes the next request from a device counter and runs its
// whole StencilFFT-P in shared memory: R2C rows (packed complex FFT and the
// real-input split), the strided FFTs along every other axis, the multiply by
// Lambda^T / N (FP64 power with the exact underflow shortcut, per element),
// the inverse transforms, and the C2R rows, in place on the request's grid.
//
// Transforms are radix-16 Stockham stages over shared memory (one radix-2/4/8
// stage first when log2 n is not a multiple of 4), on sequences with any
// element and sequence strides, so the column passes need no transposes.
// Twiddles and per-axis symbol tables are built once per executor for the
// longest supported axis (2^13) and indexed with a shift for shorter axes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/stencilfft.h"
#include "internal.h"
#include "plan_impl.h"

using namespace sfft;

namespace {

constexpr int kBatchLog2Max = 13;            // longest axis 8192
constexpr int kBatchThreads = 512;
constexpr int kBatchEPT = 16;                 // elements per thread of a stage
constexpr size_t kBatchSmem = 200 * 1024;     // shared memory of one request

struct BatchItem {
    void* grid;          // device grid of the request (in place)
    int ndim;
    int dims[3];
    int log2[3];
    int param;           // index of the request's SymbolParams
};

// One radix-R Stockham stage over nseq sequences of length n in shared memory;
// element j of sequence s at sm[base(s) + j * es], base(s) = (s / inner) *
// outer_stride + (s % inner) * inner_stride. In place (all loads, barrier, all
// stores); ends with a barrier.
template <int R, int DIR, typename C>
__device__ __forceinline__ void bstage(C* sm, int log2n, int nseq, int es, int inner, int istr,
                                       int ostr, int Ns, const C* __restrict__ tw, int twn_log2) {
    constexpr int RL = R == 16 ? 4 : R == 8 ? 3 : R == 4 ? 2 : 1;
    constexpr int BPT = kBatchEPT / R;
    const int nb_log2 = log2n - RL;
    const int nb = 1 << nb_log2;
    const int total = nseq * nb;
    const int ns_log2 = __ffs(Ns) - 1;
    const int step_log2 = twn_log2 - ns_log2 - RL;
    C v[kBatchEPT];
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int g = threadIdx.x + b * blockDim.x;
        if (g < total) {
            const int s = g >> nb_log2, j = g & (nb - 1);
            const int k = j & (Ns - 1);
            const C* src = sm + (s / inner) * ostr + (s % inner) * istr;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                C x = src[(j + r * nb) * es];
                if (r > 0 && Ns > 1) x = cmul(x, twiddle(tw, (k * r) << step_log2, DIR));
                v[b * R + r] = x;
            }
            dft_reg<R, DIR>(v + b * R);
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int g = threadIdx.x + b * blockDim.x;
        if (g < total) {
            const int s = g >> nb_log2, j = g & (nb - 1);
            const int k = j & (Ns - 1);
            C* dst = sm + (s / inner) * ostr + (s % inner) * istr;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[((j - k) * R + k + r * Ns) * es] = v[b * R + r];
        }
    }
    __syncthreads();
}

template <int DIR, typename C>
__device__ void bfft(C* sm, int log2n, int nseq, int es, int inner, int istr, int ostr,
                     const C* __restrict__ tw, int twn_log2) {
    int Ns = 1;
    const int rem = log2n & 3;
    if (rem == 1) bstage<2, DIR>(sm, log2n, nseq, es, inner, istr, ostr, Ns, tw, twn_log2), Ns = 2;
    else if (rem == 2) bstage<4, DIR>(sm, log2n, nseq, es, inner, istr, ostr, Ns, tw, twn_log2), Ns = 4;
    else if (rem == 3) bstage<8, DIR>(sm, log2n, nseq, es, inner, istr, ostr, Ns, tw, twn_log2), Ns = 8;
    for (; Ns < (1 << log2n); Ns <<= 4)
        bstage<16, DIR>(sm, log2n, nseq, es, inner, istr, ostr, Ns, tw, twn_log2);
}

// Half-spectrum row stride in shared memory for rows of n + 1 values.
__host__ __device__ inline int brow_stride(int n) { return n + 1 + ((n + 1) & 1 ? 0 : 1); }

template <typename R>
__global__ void __launch_bounds__(kBatchThreads)
k_batch_solve(const BatchItem* __restrict__ items, const SymbolParams* __restrict__ params,
              int count, int* counter, const typename CxOf<R>::T* __restrict__ tw, int twn_log2,
              int* status) {
    using C = typename CxOf<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    __shared__ int next;
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);
        __syncthreads();
        const int q = next;
        __syncthreads();
        if (q >= count) return;
        const BatchItem it = items[q];
        const SymbolParams& p = params[it.param];
        const int d = it.ndim;
        const int L = it.dims[d - 1];
        const int n = L >> 1, nl = it.log2[d - 1] - 1;
        int rows = 1;
        for (int a = 0; a < d - 1; ++a) rows *= it.dims[a];
        const int SS = brow_stride(n);
        C* g = static_cast<C*>(it.grid);   // z[m] = a[2m] + i a[2m+1]
        // rows: packed complex FFT of n values, then the real-input split
        for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
            const int r = e >> nl, m = e & (n - 1);
            sm[r * SS + m] = g[e];
        }
        __syncthreads();
        if (n > 1) bfft<-1>(sm, nl, rows, 1, 1, 0, SS, tw, twn_log2);
        const int sh = twn_log2 - nl - 1;   // W^k = exp(-2 pi i k / 2n) = tw[k << sh]
        for (int e = threadIdx.x; e < rows * (n / 2 + 1); e += blockDim.x) {
            const int r = e / (n / 2 + 1), k = e - r * (n / 2 + 1);
            C* row = sm + r * SS;
            const int nk = (n - k) & (n - 1);
            const C zk = row[k], znk = row[nk];
            const C xe = cscale(cadd(zk, cconj(znk)), (R)0.5);
            const C xo = cscale(cmul_mi(csub(zk, cconj(znk))), (R)0.5);
            const C xk = cadd(xe, cmul(twiddle(tw, k << sh, -1), xo));
            if (k == 0) {
                row[0] = xk;
                row[n] = csub(xe, xo);
            } else {
                // X[n-k] from the same pair: Z[n-k] and Z[k] swap roles
                const C xe2 = cscale(cadd(znk, cconj(zk)), (R)0.5);
                const C xo2 = cscale(cmul_mi(csub(znk, cconj(zk))), (R)0.5);
                const C xnk = cadd(xe2, cmul(twiddle(tw, nk << sh, -1), xo2));
                row[k] = xk;
                row[nk] = xnk;
            }
        }
        __syncthreads();
        // strided axes: along axis d-2 (and axis 0 for d = 3), every column k
        if (d == 2) {
            bfft<-1>(sm, it.log2[0], n + 1, SS, n + 1, 1, 0, tw, twn_log2);
        } else if (d == 3) {
            const int l1 = it.dims[1];
            bfft<-1>(sm, it.log2[1], it.dims[0] * (n + 1), SS, n + 1, 1, l1 * SS, tw, twn_log2);
            bfft<-1>(sm, it.log2[0], l1 * (n + 1), l1 * SS, n + 1, 1, SS, tw, twn_log2);
        }
        // y = V x, V = Lambda^T / N (FP64 power; exact zero below the cut)
        for (int e = threadIdx.x; e < rows * (n + 1); e += blockDim.x) {
            const int r = e / (n + 1), kl = e - r * (n + 1);
            int k[3] = {0, 0, 0};
            if (d == 1) {
                k[0] = kl;
            } else if (d == 2) {
                k[0] = r;
                k[1] = kl;
            } else {
                k[0] = r / it.dims[1];
                k[1] = r % it.dims[1];
                k[2] = kl;
            }
            C* x = sm + r * SS + kl;
            *x = cmul(*x, spectral_multiplier<C>(p, k));
        }
        __syncthreads();
        if (d == 2) {
            bfft<+1>(sm, it.log2[0], n + 1, SS, n + 1, 1, 0, tw, twn_log2);
        } else if (d == 3) {
            const int l1 = it.dims[1];
            bfft<+1>(sm, it.log2[0], l1 * (n + 1), l1 * SS, n + 1, 1, SS, tw, twn_log2);
            bfft<+1>(sm, it.log2[1], it.dims[0] * (n + 1), SS, n + 1, 1, l1 * SS, tw, twn_log2);
        }
        // inverse split, Z'[k] = (Y[k] + conj Y[n-k]) + i conj(W^k) (Y[k] - conj Y[n-k]),
        // in place by pairs (k, n-k)
        for (int e = threadIdx.x; e < rows * (n / 2 + 1); e += blockDim.x) {
            const int r = e / (n / 2 + 1), k = e - r * (n / 2 + 1);
            C* row = sm + r * SS;
            const int nk = n - k;   // Y[n] is stored at row[n]
            const C yk = row[k], ynk = row[nk];
            const C wk = twiddle(tw, k << sh, -1);
            const C zk = cadd(cadd(yk, cconj(ynk)), cmul_i(cmul(cconj(wk), csub(yk, cconj(ynk)))));
            if (k == 0) {
                row[0] = zk;
            } else if (nk != k) {
                const C wnk = twiddle(tw, nk << sh, -1);
                const C znk =
                    cadd(cadd(ynk, cconj(yk)), cmul_i(cmul(cconj(wnk), csub(ynk, cconj(yk)))));
                row[k] = zk;
                row[nk] = znk;
            } else {
                row[k] = zk;
            }
        }
        __syncthreads();
        if (n > 1) bfft<+1>(sm, nl, rows, 1, 1, 0, SS, tw, twn_log2);
        bool bad = false;
        for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
            const int r = e >> nl, m = e & (n - 1);
            const C v = sm[r * SS + m];
            bad |= !(isfinite(v.x) && isfinite(v.y));
            g[e] = v;
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, 1);
    }
}

}  // namespace

struct stencil_batch_s {
    int precision = STENCIL_FP32;
    int capacity = 0;
    int device = 0;
    void* tw = nullptr;                  // exp(-2 pi i m / 2^13) at pass precision
    double2* E64 = nullptr;              // exp(+2 pi i q / 2^13)
    float2* E32 = nullptr;
    BatchItem* d_items = nullptr;
    SymbolParams* d_params = nullptr;
    int* d_counter = nullptr;
    int* d_status = nullptr;
    BatchItem* h_items = nullptr;        // pinned staging
    SymbolParams* h_params = nullptr;
    cudaEvent_t staged = nullptr;        // the last upload has read the staging
    cudaEvent_t done = nullptr;          // the last run's kernel has finished
    bool pending = false;
};

namespace {

// Bytes of shared memory a request needs (0: not batchable).
size_t request_smem(int ndim, const int64_t* dims, int precision) {
    if (ndim < 1 || ndim > 3) return 0;
    int64_t rows = 1;
    for (int a = 0; a < ndim; ++a) {
        if (ilog2_exact(dims[a]) < 0 || dims[a] > (1 << kBatchLog2Max) || dims[a] < 4) return 0;
        if (a < ndim - 1) rows *= dims[a];
    }
    const int64_t n = dims[ndim - 1] / 2;
    // every stage's butterflies must fit kBatchEPT elements per thread
    if (rows * (n + 1) > (int64_t)kBatchEPT * kBatchThreads / 2 * 2) return 0;
    const size_t elem = precision == STENCIL_FP32 ? 8 : 16;
    const size_t bytes = (size_t)rows * brow_stride((int)n) * elem;
    return bytes <= kBatchSmem ? bytes : 0;
}

}  // namespace

extern "C" {

size_t stencil_batch_smem_bytes(int ndim, const int64_t* dims, int precision) {
    if (!dims || (precision != STENCIL_FP32 && precision != STENCIL_FP64)) return 0;
    return request_smem(ndim, dims, precision);
}

int stencil_batch_create(stencil_batch_t* out, int capacity, int precision) {
    if (!out || capacity < 1 || capacity > (1 << 20)) return STENCIL_EINVAL;
    if (precision != STENCIL_FP32 && precision != STENCIL_FP64) return STENCIL_EINVAL;
    *out = nullptr;
    stencil_batch_s* b = new (std::nothrow) stencil_batch_s();
    if (!b) return STENCIL_ENOMEM;
    b->precision = precision;
    b->capacity = capacity;
    cudaGetDevice(&b->device);
    const int L = 1 << kBatchLog2Max;
    const size_t celem = precision == STENCIL_FP32 ? sizeof(float2) : sizeof(double2);
    const cudaStream_t ts = cudaStreamPerThread;
    cudaError_t err = cudaMalloc(&b->tw, celem * L);
    if (err == cudaSuccess)
        err = precision == STENCIL_FP32 ? launch_twiddles<float>(b->tw, kBatchLog2Max, ts)
                                        : launch_twiddles<double>(b->tw, kBatchLog2Max, ts);
    if (err == cudaSuccess) err = cudaMalloc(&b->E64, sizeof(double2) * L);
    if (err == cudaSuccess) err = cudaMalloc(&b->E32, sizeof(float2) * L);
    if (err == cudaSuccess) err = launch_axis_table(b->E64, b->E32, L, ts);
    if (err == cudaSuccess) err = cudaMalloc(&b->d_items, sizeof(BatchItem) * capacity);
    if (err == cudaSuccess) err = cudaMalloc(&b->d_params, sizeof(SymbolParams) * capacity);
    if (err == cudaSuccess) err = cudaMalloc(&b->d_counter, sizeof(int));
    if (err == cudaSuccess) err = cudaMalloc(&b->d_status, sizeof(int));
    if (err == cudaSuccess) err = cudaMemsetAsync(b->d_status, 0, sizeof(int), ts);
    if (err == cudaSuccess) err = cudaMallocHost(&b->h_items, sizeof(BatchItem) * capacity);
    if (err == cudaSuccess) err = cudaMallocHost(&b->h_params, sizeof(SymbolParams) * capacity);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaStreamSynchronize(ts);
    if (err != cudaSuccess) {
        stencil_batch_destroy(b);
        note_cuda_error(err);
        return err == cudaErrorMemoryAllocation ? STENCIL_ENOMEM : STENCIL_ECUDA;
    }
    *out = b;
    return STENCIL_OK;
}

int stencil_batch_run(stencil_batch_t b, int count, const stencil_request* reqs, void* stream) {
    if (!b || count < 0 || (count > 0 && !reqs)) return STENCIL_EINVAL;
    if (count > b->capacity) return STENCIL_EINVAL;
    if (count == 0) return STENCIL_OK;
    // validate everything before touching the staging buffers
    for (int i = 0; i < count; ++i) {
        const stencil_request& r = reqs[i];
        if (!r.grid || !r.weights || r.T < 0 || r.radius < 0 || r.radius > kMaxRadius ||
            r.boundary != STENCIL_PERIODIC || r.precision != b->precision ||
            reinterpret_cast<uintptr_t>(r.grid) % 16)
            return STENCIL_EINVAL;
        for (int a = 0; a < r.ndim; ++a)
            if (r.dims[a] < 2 * r.radius + 1) return STENCIL_EINVAL;
        if (!request_smem(r.ndim, r.dims, r.precision)) return STENCIL_EUNSUPPORTED;
        int nw = 1;
        for (int a = 0; a < r.ndim; ++a) nw *= 2 * r.radius + 1;
        for (int k = 0; k < nw; ++k)
            if (!std::isfinite(r.weights[k])) return STENCIL_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the previous upload must have read the staging buffers
    if (b->pending && cudaEventSynchronize(b->staged) != cudaSuccess) return STENCIL_ECUDA;
    size_t smem = 0;
    for (int i = 0; i < count; ++i) {
        const stencil_request& r = reqs[i];
        BatchItem& it = b->h_items[i];
        std::memset(&it, 0, sizeof(it));
        it.grid = r.grid;
        it.ndim = r.ndim;
        for (int a = 0; a < r.ndim; ++a) {
            it.dims[a] = (int)r.dims[a];
            it.log2[a] = ilog2_exact(r.dims[a]);
        }
        it.param = i;
        smem = std::max(smem, request_smem(r.ndim, r.dims, r.precision));
        // the request's symbol over the executor's 2^13-point axis tables
        stencil_plan_s tmp;
        tmp.ndim = r.ndim;
        tmp.precision = r.precision;
        for (int a = 0; a < r.ndim; ++a) tmp.dims[a] = (int64_t)1 << kBatchLog2Max;
        plan_set_weights(&tmp, r.radius, r.weights);
        const double2* E64[3] = {b->E64, b->E64, b->E64};
        const float2* E32[3] = {b->E32, b->E32, b->E32};
        b->h_params[i] = make_symbol_params(&tmp, r.dims, r.T, E64, E32, nullptr);
    }
    cudaError_t err = cudaMemcpyAsync(b->d_items, b->h_items, sizeof(BatchItem) * count,
                                      cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(b->d_params, b->h_params, sizeof(SymbolParams) * count,
                              cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) err = cudaEventRecord(b->staged, s);
    if (err == cudaSuccess) b->pending = true;
    if (err == cudaSuccess) err = cudaMemsetAsync(b->d_counter, 0, sizeof(int), s);
    if (err == cudaSuccess) {
        int nsm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
        const int per_sm = std::max<int>(1, (int)(228 * 1024 / (smem + 1024)));
        const int grid = std::min<int>(count, std::max(1, nsm) * std::min(per_sm, 2));
        if (b->precision == STENCIL_FP32) {
            err = smem_optin(reinterpret_cast<const void*>(k_batch_solve<float>), smem);
            if (err == cudaSuccess)
                k_batch_solve<float><<<grid, kBatchThreads, smem, s>>>(
                    b->d_items, b->d_params, count, b->d_counter, static_cast<const float2*>(b->tw),
                    kBatchLog2Max, b->d_status);
        } else {
            err = smem_optin(reinterpret_cast<const void*>(k_batch_solve<double>), smem);
            if (err == cudaSuccess)
                k_batch_solve<double><<<grid, kBatchThreads, smem, s>>>(
                    b->d_items, b->d_params, count, b->d_counter, static_cast<const double2*>(b->tw),
                    kBatchLog2Max, b->d_status);
        }
        if (err == cudaSuccess) err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaEventRecord(b->done, s);
    }
    if (err != cudaSuccess) {
        note_cuda_error(err);
        return STENCIL_ECUDA;
    }
    return STENCIL_OK;
}

int stencil_batch_status(stencil_batch_t b, void* stream) {
    if (!b) return STENCIL_EINVAL;
    cudaError_t err = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (err != cudaSuccess) {
        note_cuda_error(err);
        return STENCIL_ECUDA;
    }
    int st = 0;
    if (cudaMemcpy(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return STENCIL_ECUDA;
    if (st) {
        cudaMemset(b->d_status, 0, sizeof(int));
        return STENCIL_ENONFINITE;
    }
    return STENCIL_OK;
}

int stencil_batch_destroy(stencil_batch_t b) {
    if (!b) return STENCIL_EINVAL;
    // the last run's kernel (and with it every upload) has finished: no
    // device-wide synchronisation
    if (b->done) {
        if (b->pending) cudaEventSynchronize(b->done);
        cudaEventDestroy(b->done);
    }
    if (b->staged) cudaEventDestroy(b->staged);
    cudaFree(b->tw);
    cudaFree(b->E64);
    cudaFree(b->E32);
    cudaFree(b->d_items);
    cudaFree(b->d_params);
    cudaFree(b->d_counter);
    cudaFree(b->d_status);
    cudaFreeHost(b->h_items);
    cudaFreeHost(b->h_params);
    delete b;
    return STENCIL_OK;
}

}  // extern "C"
