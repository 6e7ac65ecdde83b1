// Hyperboloidal-slice instantiations of the fused stage kernel, single
// evolution and batches (the pi rows' own speed, quartic ghosts;
// teuk_stage_kernels.cuh), in a translation unit of their own so that they
// compile in parallel with the r* kernels.
#include "teuk_stage_kernels.cuh"

namespace teuk {

template <int W>
static cudaError_t launch_hyp_w(const StageArgs& A, int theta, int stage, cudaStream_t st) {
    return theta == TEUK_THETA_WENO5 ? launch_stage_wt<W, TEUK_THETA_WENO5, true>(A, stage, st)
                                     : launch_stage_wt<W, TEUK_THETA_CENTERED4, true>(A, stage, st);
}

cudaError_t launch_stage_hyp(const StageArgs& A, int wprec, int theta, int stage,
                             cudaStream_t st) {
    switch (wprec) {
    case TEUK_W_FP64: return launch_hyp_w<TEUK_W_FP64>(A, theta, stage, st);
    case TEUK_W_FP32: return launch_hyp_w<TEUK_W_FP32>(A, theta, stage, st);
    case TEUK_W_FP16: return launch_hyp_w<TEUK_W_FP16>(A, theta, stage, st);
    default: return launch_hyp_w<TEUK_W_BF16>(A, theta, stage, st);
    }
}

cudaError_t launch_batch_stage_hyp(int wprec, int theta, int stage, int segv,
                                   const BatchDesc* d, int n, long long items, int grid,
                                   cudaStream_t st) {
    switch (wprec) {
    case TEUK_W_FP64:
        return launch_batch_w<TEUK_W_FP64, true>(stage, segv, theta, d, n, items, grid, st);
    case TEUK_W_FP32:
        return launch_batch_w<TEUK_W_FP32, true>(stage, segv, theta, d, n, items, grid, st);
    case TEUK_W_FP16:
        return launch_batch_w<TEUK_W_FP16, true>(stage, segv, theta, d, n, items, grid, st);
    default:
        return launch_batch_w<TEUK_W_BF16, true>(stage, segv, theta, d, n, items, grid, st);
    }
}

}  // namespace teuk
