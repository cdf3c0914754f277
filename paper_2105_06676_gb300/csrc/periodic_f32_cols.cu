// Instantiation of the periodic-path cols launchers for float.
#include "periodic_kernels.cuh"

namespace sfft {

SFFT_INSTANTIATE_COLS(float)

}  // namespace sfft
