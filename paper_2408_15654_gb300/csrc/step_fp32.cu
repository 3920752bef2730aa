// Step-kernel instances for FP32 population storage.
#include "lbm_launch.h"

namespace lbm {

LBM_DEFINE_STORAGE(fp32, kFP32)

// Dispatch by storage mode.
cudaError_t launch_step(int st, const StepArgs& a, int mode, const Variant& v, dim3 grid, int pipe, cudaStream_t s) {
    switch (st) {
        case kFP16: return launch_step_fp16(a, mode, v, grid, pipe, s);
        case kBF16: return launch_step_bf16(a, mode, v, grid, pipe, s);
        case kFP16FG: return launch_step_fp16fg(a, mode, v, grid, pipe, s);
        case kBF16FG: return launch_step_bf16fg(a, mode, v, grid, pipe, s);
        default: return launch_step_fp32(a, mode, v, grid, pipe, s);
    }
}

cudaError_t prepare_step(int st, const Variant& v, int* blocks_per_sm, int* pipe_blocks_per_sm) {
    switch (st) {
        case kFP16: return prepare_step_fp16(v, blocks_per_sm, pipe_blocks_per_sm);
        case kBF16: return prepare_step_bf16(v, blocks_per_sm, pipe_blocks_per_sm);
        case kFP16FG: return prepare_step_fp16fg(v, blocks_per_sm, pipe_blocks_per_sm);
        case kBF16FG: return prepare_step_bf16fg(v, blocks_per_sm, pipe_blocks_per_sm);
        default: return prepare_step_fp32(v, blocks_per_sm, pipe_blocks_per_sm);
    }
}

cudaError_t launch_batch(int st, const BatchArgs& b, const Variant& v, unsigned ntiles, cudaStream_t s) {
    switch (st) {
        case kFP16: return launch_batch_fp16(b, v, ntiles, s);
        case kBF16: return launch_batch_bf16(b, v, ntiles, s);
        case kFP16FG: return launch_batch_fp16fg(b, v, ntiles, s);
        case kBF16FG: return launch_batch_bf16fg(b, v, ntiles, s);
        default: return launch_batch_fp32(b, v, ntiles, s);
    }
}

cudaError_t prepare_batch(int st, int* ws_blocks_per_sm) {
    switch (st) {
        case kFP16: return prepare_batch_fp16(ws_blocks_per_sm);
        case kBF16: return prepare_batch_bf16(ws_blocks_per_sm);
        case kFP16FG: return prepare_batch_fp16fg(ws_blocks_per_sm);
        case kBF16FG: return prepare_batch_bf16fg(ws_blocks_per_sm);
        default: return prepare_batch_fp32(ws_blocks_per_sm);
    }
}

}  // namespace lbm
