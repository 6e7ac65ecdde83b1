// Fused persistent step kernel (all SSP-RK(3,3) stages of many steps in one
// launch, teuk_stage_kernels.cuh) on r* grids, in a translation unit of its
// own so that it compiles in parallel with the stage kernels.
#include "teuk_stage_kernels.cuh"

namespace teuk {

cudaError_t launch_fused_rstar(const FusedArgs& F, int wprec, int theta, int seg, int cap,
                               cudaStream_t st) {
    return launch_fused_h<false>(F, wprec, theta, seg, cap, st);
}

cudaError_t fused_occupancy_rstar(int wprec, int theta, int* per_sm) {
    return fused_occupancy_h<false>(wprec, theta, per_sm);
}

}  // namespace teuk
