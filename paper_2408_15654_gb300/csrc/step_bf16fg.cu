// Step-kernel instances for BF16 storage of the (f, g) pairs, FP32 storage of h.
#include "lbm_launch.h"

namespace lbm {

cudaError_t launch_step_bf16fg(const StepArgs& a, int mode, bool walls, bool langmuir, dim3 grid, int pipe,
                           cudaStream_t s) {
    return launch_step_impl<kBF16FG>(a, mode, walls, langmuir, grid, pipe, s);
}

cudaError_t prepare_step_bf16fg(int* blocks_per_sm, int* pipe_blocks_per_sm) {
    return prepare_step_impl<kBF16FG>(blocks_per_sm, pipe_blocks_per_sm);
}

cudaError_t launch_batch_bf16fg(const BatchArgs& b, bool walls, bool langmuir, unsigned ntiles, cudaStream_t s) {
    return launch_batch_impl<kBF16FG>(b, walls, langmuir, ntiles, s);
}

cudaError_t prepare_batch_bf16fg() { return prepare_batch_impl<kBF16FG>(); }

}  // namespace lbm
