// Step-kernel instances for FP32 population storage.
#include "lbm_launch.h"

namespace lbm {

cudaError_t launch_step_fp32(const StepArgs& a, int mode, bool walls, bool langmuir, dim3 grid, int pipe,
                           cudaStream_t s) {
    return launch_step_impl<kFP32>(a, mode, walls, langmuir, grid, pipe, s);
}

cudaError_t prepare_step_fp32(int* blocks_per_sm, int* pipe_blocks_per_sm) {
    return prepare_step_impl<kFP32>(blocks_per_sm, pipe_blocks_per_sm);
}

cudaError_t launch_batch_fp32(const BatchArgs& b, bool walls, bool langmuir, unsigned ntiles, cudaStream_t s) {
    return launch_batch_impl<kFP32>(b, walls, langmuir, ntiles, s);
}

cudaError_t prepare_batch_fp32() { return prepare_batch_impl<kFP32>(); }

// Dispatch of the many-lattice kernel by storage mode.
cudaError_t launch_batch(int st, const BatchArgs& b, bool walls, bool langmuir, unsigned ntiles, cudaStream_t s) {
    switch (st) {
        case kFP16: return launch_batch_fp16(b, walls, langmuir, ntiles, s);
        case kBF16: return launch_batch_bf16(b, walls, langmuir, ntiles, s);
        case kFP16FG: return launch_batch_fp16fg(b, walls, langmuir, ntiles, s);
        case kBF16FG: return launch_batch_bf16fg(b, walls, langmuir, ntiles, s);
        default: return launch_batch_fp32(b, walls, langmuir, ntiles, s);
    }
}

cudaError_t prepare_batch(int st) {
    switch (st) {
        case kFP16: return prepare_batch_fp16();
        case kBF16: return prepare_batch_bf16();
        case kFP16FG: return prepare_batch_fp16fg();
        case kBF16FG: return prepare_batch_bf16fg();
        default: return prepare_batch_fp32();
    }
}

}  // namespace lbm
