// Fused persistent step kernel on the hyperboloidal slices (the pi rows' own
// speed, quartic ghosts), in a translation unit of its own.
#include "teuk_stage_kernels.cuh"

namespace teuk {

cudaError_t launch_fused_hyp(const FusedArgs& F, int wprec, int theta, int seg, int cap,
                             cudaStream_t st) {
    return launch_fused_h<true>(F, wprec, theta, seg, cap, st);
}

cudaError_t fused_occupancy_hyp(int wprec, int theta, int* per_sm) {
    return fused_occupancy_h<true>(wprec, theta, per_sm);
}

}  // namespace teuk
