// Internal interfaces between the host plan code and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "symbol.cuh"

namespace sfft {

// Elements per thread held in registers by the shared-memory FFT.
constexpr int kEPT = 16;
// Threads per CTA upper bounds (launch bounds of the FFT kernels).
constexpr int kMaxThreadsF32 = 1024;
constexpr int kMaxThreadsF64 = 512;
// Largest per-CTA dynamic shared memory the FFT kernels request.
constexpr int kSmemBudget = 200 * 1024;

// A batch of strided columns: the FFT runs along an axis of length n = 2^log2n
// with element stride S; the batch is (outer, mid, inner) with
// address = base + o*os + m*ms + j*S + i for i < inner_valid, and `cols`
// consecutive inner indices per CTA.
struct ColGeom {
    int log2n;
    long long S;
    int outer;
    long long os;
    int mid;
    long long ms;
    int inner_valid;
    int cols_log2;
    long long vS = 0;   // row stride of multiplier tables where it differs from S (blocked H)
};

// Launchers (templated on the real type; instantiated for float and double).
template <typename R>
cudaError_t launch_fused_1d(R* grid, int n_log2, int nrows, const void* tw, int twn_log2,
                            const SymbolParams& p, int* status, cudaStream_t s,
                            const RowTables* rtab = nullptr);
// 1-D axes whose packed length n = 2^(n1_log2 + n2_log2) exceeds one CTA:
// column FFT, fused row pairs (split, multiplier, inverse split), inverse
// column FFT, in place on `items` stacked grids.
template <typename R>
cudaError_t launch_fused_1d_pairs(R* grid, int n1_log2, int n2_log2, int items, const void* tw,
                                  int twn_log2, const SymbolParams& p, int* status,
                                  cudaStream_t s);
template <typename R>
cudaError_t launch_rows_r2c(const R* grid, void* H, long long Mp, int n_log2, int nrows,
                            const void* tw, int twn_log2, cudaStream_t s);
template <typename R>
cudaError_t launch_rows_c2r(const void* H, R* grid, long long Mp, int n_log2, int nrows,
                            const void* tw, int twn_log2, int* status, cudaStream_t s);
template <typename R>
cudaError_t launch_cols(void* H, const ColGeom& g, int dir, const void* tw, int twn_log2,
                        cudaStream_t s);
template <typename R>
cudaError_t launch_cols_fused(void* H, const ColGeom& g, const void* tw, int twn_log2,
                              const SymbolSet& p, cudaStream_t s);
template <typename R>
cudaError_t launch_twiddles(void* tw, int twn_log2, cudaStream_t s);
template <typename R>
cudaError_t launch_vtable(void* V, const SymbolParams& p, long long Mp, cudaStream_t s);
cudaError_t launch_axis_table(double2* E64, float2* E32, int len, cudaStream_t s);
cudaError_t launch_symbol_table(double2* out, const SymbolParams& p, int nlast_half,
                                long long total, cudaStream_t s);

// Strided-axis transforms with the radix-16 DFTs on the tensor cores (FP32
// data; mode kGemmBF16 / kGemmFP16 / kGemmBF16x3; 2^8 <= n <= 2^12). Device
// waits that give up set bit 4 of *status.
bool gemm_axis_ok(int log2n);
cudaError_t launch_cols_gemm(void* H, const ColGeom& g, int dir, const void* tw, int twn_log2,
                             int mode, int* status, cudaStream_t s);
cudaError_t launch_cols_fused_gemm(void* H, const ColGeom& g, const void* tw, int twn_log2,
                                   const SymbolSet& p, int mode, int* status, cudaStream_t s);

// Persistent TMA-fed strided-axis passes for FP32 half spectra (cols_tma.cuh),
// transform lengths 2^9..2^12: mode -1 forward, +1 inverse, 0 the fused
// forward x V x inverse pass along axis 0 (ps required). Returns
// cudaErrorNotSupported when the geometry or the driver does not allow it (the
// caller then uses the register column kernels). Abandoned waits set bit 2 of
// *status.
bool cols_tma_ok(const void* H, const ColGeom& g);
cudaError_t launch_cols_tma(void* H, const ColGeom& g, int mode, const void* tw, int twn_log2,
                            const SymbolSet* ps, int* status, cudaStream_t s);

// Persistent bulk-copy-fed passes along the contiguous axis for FP32 grids
// (rows_tma.cuh), packed row lengths n = 2^8..2^12: dir +1 half spectra ->
// real rows (src H, dst grid; non-finite output sets bit 0 of *status); dir -1
// (real rows -> half spectra) is not dispatched. Returns cudaErrorNotSupported when
// not applicable (the caller then uses the register row kernels).
bool rows_tma_ok(const void* grid, const void* H, long long Mp, int n_log2, int nrows);
cudaError_t launch_rows_tma(int dir, const void* src, void* dst, long long Mp, int n_log2,
                            int nrows, const void* tw, int twn_log2, int* status, cudaStream_t s);

// Blocked half spectra of FP32 2-D solves (rows_blk.cuh, cols_tma.cuh with
// BLK = 1): an item of 2^l0_log2 rows stores its half spectrum as column blocks
// of 8192 values (2^(13 - l0_log2) columns x all rows). blocked_ok: the three
// passes apply (2^9 <= l0 <= 2^12, packed row length 2^8..2^12, aligned);
// blocked_item_elems: complex values per item (at most l0 * Mp for Mp >= n + 16).
// launch_rows_blk: dir -1 grid rows -> blocked H, +1 blocked H -> grid rows
// (non-finite output sets bit 0 of *status); launch_cols_tma_blk: the fused
// forward x V x inverse pass over the blocks (g.os = item stride, g.vS = row
// stride of multiplier tables). All return cudaErrorNotSupported when not
// applicable.
bool blocked_ok(const void* grid, const void* H, int l0_log2, int n_log2);
// The blocked path applies to a 2-D shape (dims only; pointers aside), and its
// repeated-T multiplier table: V = Lambda^T / N laid out like the blocked half
// spectrum of one item plus one flag per column block (0: all zero).
bool blocked_shape(int ndim, const int64_t* dims);
cudaError_t launch_vtable_blk(void* V, int* flags, const SymbolParams& p, int l0_log2, int n_log2,
                              cudaStream_t s);
long long blocked_item_elems(int l0_log2, int n_log2);
cudaError_t launch_rows_blk(int dir, const void* src, void* dst, int l0_log2, int n_log2,
                            int nrows, const void* tw, int twn_log2, int* status, cudaStream_t s);
cudaError_t launch_cols_tma_blk(void* H, const ColGeom& g, const void* tw, int twn_log2,
                                const SymbolSet& ps, int* status, cudaStream_t s);

// Mixed-radix passes (mixed.cu) for transform lengths with prime factors 2, 3,
// 5, 7 up to 8192: mixed_length_ok says whether a length is covered;
// launch_mixed_table builds exp(-2 pi i m / len) at pass precision;
// launch_mixed_rows: dir -1 real rows of 2n values -> half spectra (row
// stride Mp), +1 back (non-finite output sets bit 0 of *status), twL the table
// of length 2n; launch_mixed_cols: C2C along a strided axis of length n (tw of
// length n).
bool mixed_length_ok(int64_t len, int precision);
template <typename R>
cudaError_t launch_mixed_table(void* tw, int len, cudaStream_t s);
template <typename R>
cudaError_t launch_mixed_rows(int dir, const void* src, void* dst, long long Mp, int n, int nrows,
                              const void* twL, int* status, cudaStream_t s);
template <typename R>
cudaError_t launch_mixed_cols(int dir, void* H, const ColGeom& g, int n, const void* tw,
                              cudaStream_t s);

// Pass variant of the periodic solve running on this host thread (set by
// batched_solve from the plan, chosen by stencil_plan_autotune): 0 the default
// (FP32 2-D: blocked half spectrum; TMA-fed column and C2R passes), 1 the
// row-major half spectrum with the TMA-fed passes, 2 the register kernels
// only (1024-thread FP32 column CTAs), 3 the register kernels with 512-thread
// column CTAs. -1 leaves the selection to the defaults.
int pass_variant();
struct PassVariantScope {
    int saved;
    explicit PassVariantScope(int v);
    ~PassVariantScope();
};
constexpr int kPassVariants = 4;

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per kernel and device.
cudaError_t smem_optin(const void* kernel, size_t bytes);

// Number of columns per CTA the column kernels use for a transform of 2^log2n.
int cols_log2_for(int log2n, int elem_bytes, int max_threads);
// Rows per CTA of the row kernels.
int rows_per_cta_for(int n_log2, int elem_bytes, int max_threads);

}  // namespace sfft
