// Step-kernel instances for BF16 population storage.
#include "lbm_launch.h"

namespace lbm {

cudaError_t launch_step_bf16(const StepArgs& a, int mode, bool walls, bool langmuir, dim3 grid, cudaStream_t s) {
    return launch_step_impl<kBF16>(a, mode, walls, langmuir, grid, s);
}

cudaError_t prepare_step_bf16(int* blocks_per_sm) { return prepare_step_impl<kBF16>(blocks_per_sm); }

}  // namespace lbm
