// Step-kernel instances for FP16 population storage.
#include "lbm_launch.h"

namespace lbm {

cudaError_t launch_step_fp16(const StepArgs& a, int mode, bool walls, bool langmuir, dim3 grid, int pipe,
                           cudaStream_t s) {
    return launch_step_impl<kFP16>(a, mode, walls, langmuir, grid, pipe, s);
}

cudaError_t prepare_step_fp16(int* blocks_per_sm, int* pipe_blocks_per_sm) {
    return prepare_step_impl<kFP16>(blocks_per_sm, pipe_blocks_per_sm);
}

cudaError_t launch_batch_fp16(const BatchArgs& b, bool walls, bool langmuir, unsigned ntiles, cudaStream_t s) {
    return launch_batch_impl<kFP16>(b, walls, langmuir, ntiles, s);
}

cudaError_t prepare_batch_fp16() { return prepare_batch_impl<kFP16>(); }

}  // namespace lbm
