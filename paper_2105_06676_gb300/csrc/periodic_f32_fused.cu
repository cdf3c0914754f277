// Instantiation of the periodic-path fused launchers for float.
#include "periodic_kernels.cuh"

namespace sfft {

SFFT_INSTANTIATE_FUSED(float)

}  // namespace sfft
