// Instantiation of the periodic-path fused launchers for double.
#include "periodic_kernels.cuh"

namespace sfft {

SFFT_INSTANTIATE_FUSED(double)

}  // namespace sfft
