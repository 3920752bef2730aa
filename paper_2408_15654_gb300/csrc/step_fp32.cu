// Step-kernel instances for FP32 population storage.
#include "lbm_launch.h"

namespace lbm {

cudaError_t launch_step_fp32(const StepArgs& a, int mode, bool walls, bool langmuir, dim3 grid, cudaStream_t s) {
    return launch_step_impl<kFP32>(a, mode, walls, langmuir, grid, s);
}

cudaError_t prepare_step_fp32(int* blocks_per_sm) { return prepare_step_impl<kFP32>(blocks_per_sm); }

}  // namespace lbm
