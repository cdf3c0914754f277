// Instantiation of the periodic-path kernels and launchers for double.
#include "periodic_kernels.cuh"

namespace sfft {

#define SFFT_INSTANTIATE(R)                                                                        \
    template cudaError_t launch_fused_1d<R>(R*, int, int, const void*, int, const SymbolParams&,   \
                                            int*, cudaStream_t, const RowTables*);                 \
    template cudaError_t launch_rows_r2c<R>(const R*, void*, long long, int, int, const void*,     \
                                            int, cudaStream_t);                                    \
    template cudaError_t launch_rows_c2r<R>(const void*, R*, long long, int, int, const void*,     \
                                            int, int*, cudaStream_t);                              \
    template cudaError_t launch_cols<R>(void*, const ColGeom&, int, const void*, int,              \
                                        cudaStream_t);                                             \
    template cudaError_t launch_cols_fused<R>(void*, const ColGeom&, const void*, int,             \
                                              const SymbolSet&, cudaStream_t);                  \
    template cudaError_t launch_twiddles<R>(void*, int, cudaStream_t);                            \
    template cudaError_t launch_vtable<R>(void*, const SymbolParams&, long long, cudaStream_t);


SFFT_INSTANTIATE(double)

}  // namespace sfft
