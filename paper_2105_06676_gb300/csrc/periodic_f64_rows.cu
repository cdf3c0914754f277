// Instantiation of the periodic-path rows launchers for double.
#include "periodic_kernels.cuh"

namespace sfft {

SFFT_INSTANTIATE_ROWS(double)

}  // namespace sfft
