// Instantiation of the periodic-path cols launchers for double.
#include "periodic_kernels.cuh"

namespace sfft {

SFFT_INSTANTIATE_COLS(double)

}  // namespace sfft
