// StencilFFT-A (paper Sec. 5): placeholder until the RecursiveBoundary schedule lands.
#include "../../include/stencilfft.h"
#include "plan_impl.h"

int aperiodic_run(stencil_plan_s* p, void* grid, int64_t T, cudaStream_t s) {
    (void)p; (void)grid; (void)T; (void)s;
    return STENCIL_EUNSUPPORTED;
}

void aperiodic_release(stencil_plan_s* p) { (void)p; }
