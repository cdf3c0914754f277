// Instantiation of the periodic-path rows launchers for float.
#include "periodic_kernels.cuh"

namespace sfft {

SFFT_INSTANTIATE_ROWS(float)

}  // namespace sfft
