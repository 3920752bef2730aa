// Launch helpers of the step kernel, one translation unit per storage mode
// (step_fp32.cu, step_fp16.cu, step_bf16.cu, step_fp16fg.cu, step_bf16fg.cu) so that the
// instances compile in parallel.
#pragma once
#include <cstring>

#include "lbm_kernels.cuh"

namespace lbm {

// Every step launch uses programmatic dependent launch: the kernel waits (griddepcontrol.wait)
// for the previous grid before touching memory, so the next launch may be scheduled during the
// tail of this one.
// grid = (tiles along x, tiles along y).  A step (mode kStep) with pipe_ctas > 0 runs the
// persistent pipelined kernel on pipe_ctas CTAs instead of one CTA per tile.
template <int ST>
cudaError_t launch_step_impl(const StepArgs& a, int mode, bool walls, bool langmuir, dim3 grid, int pipe_ctas,
                             cudaStream_t stream) {
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = grid;
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = Smem<ST>::BYTES;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (mode == kStep && pipe_ctas > 0) {
        const int ntx = (int)grid.x, nty = (int)grid.y;
        cfg.gridDim = dim3((unsigned)pipe_ctas);
        cfg.dynamicSmemBytes = Smem<ST>::BYTES_PIPE;
        if (walls && langmuir) return cudaLaunchKernelEx(&cfg, step_kernel_pipe<ST, true, true>, a, ntx, nty);
        if (walls) return cudaLaunchKernelEx(&cfg, step_kernel_pipe<ST, true, false>, a, ntx, nty);
        if (langmuir) return cudaLaunchKernelEx(&cfg, step_kernel_pipe<ST, false, true>, a, ntx, nty);
        return cudaLaunchKernelEx(&cfg, step_kernel_pipe<ST, false, false>, a, ntx, nty);
    }
#define LBM_LAUNCH_CASE(W_, L_)                                                              \
    do {                                                                                     \
        if (mode == kStep) return cudaLaunchKernelEx(&cfg, step_kernel<ST, W_, L_, kStep>, a);      \
        return cudaLaunchKernelEx(&cfg, step_kernel<ST, W_, L_, kMoments>, a);               \
    } while (0)
    if (walls && langmuir) LBM_LAUNCH_CASE(true, true);
    if (walls) LBM_LAUNCH_CASE(true, false);
    if (langmuir) LBM_LAUNCH_CASE(false, true);
    LBM_LAUNCH_CASE(false, false);
#undef LBM_LAUNCH_CASE
}

template <int ST, bool W_, bool L_, int M_>
cudaError_t prepare_one(int* bps) {
    auto k = step_kernel<ST, W_, L_, M_>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<ST>::BYTES);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, NT, Smem<ST>::BYTES);
}

template <int ST, bool W_, bool L_>
cudaError_t prepare_pipe_one(int* bps) {
    auto k = step_kernel_pipe<ST, W_, L_>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<ST>::BYTES_PIPE);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, NT, Smem<ST>::BYTES_PIPE);
}

// Opt the instances of storage mode ST into their dynamic shared memory; resident CTAs per SM of
// the one-tile kernels and of the pipelined kernels (the minimum over the instances).
template <int ST>
cudaError_t prepare_step_impl(int* blocks_per_sm, int* pipe_blocks_per_sm) {
    int b[8] = {0};
    cudaError_t e = prepare_one<ST, false, false, kStep>(&b[0]);
    if (e == cudaSuccess) e = prepare_one<ST, false, true, kStep>(&b[1]);
    if (e == cudaSuccess) e = prepare_one<ST, true, false, kStep>(&b[2]);
    if (e == cudaSuccess) e = prepare_one<ST, true, true, kStep>(&b[3]);
    if (e == cudaSuccess) e = prepare_one<ST, false, false, kMoments>(&b[4]);
    if (e == cudaSuccess) e = prepare_one<ST, false, true, kMoments>(&b[5]);
    if (e == cudaSuccess) e = prepare_one<ST, true, false, kMoments>(&b[6]);
    if (e == cudaSuccess) e = prepare_one<ST, true, true, kMoments>(&b[7]);
    int m = b[0];
    for (int k = 1; k < 8; ++k) m = b[k] < m ? b[k] : m;
    *blocks_per_sm = m;
    int q[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = prepare_pipe_one<ST, false, false>(&q[0]);
    if (e == cudaSuccess) e = prepare_pipe_one<ST, false, true>(&q[1]);
    if (e == cudaSuccess) e = prepare_pipe_one<ST, true, false>(&q[2]);
    if (e == cudaSuccess) e = prepare_pipe_one<ST, true, true>(&q[3]);
    m = q[0];
    for (int k = 1; k < 4; ++k) m = q[k] < m ? q[k] : m;
    *pipe_blocks_per_sm = m;
    return e;
}

// One launch of the many-lattice kernel over `ntiles` tiles (all lattices of one storage mode,
// boundary kind and EOS).
template <int ST>
cudaError_t launch_batch_impl(const BatchArgs& b, bool walls, bool langmuir, unsigned ntiles, cudaStream_t stream) {
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(ntiles);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = Smem<ST>::BYTES_BATCH;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (walls && langmuir) return cudaLaunchKernelEx(&cfg, batch_step_kernel<ST, true, true>, b);
    if (walls) return cudaLaunchKernelEx(&cfg, batch_step_kernel<ST, true, false>, b);
    if (langmuir) return cudaLaunchKernelEx(&cfg, batch_step_kernel<ST, false, true>, b);
    return cudaLaunchKernelEx(&cfg, batch_step_kernel<ST, false, false>, b);
}

template <int ST, bool W_, bool L_>
cudaError_t prepare_batch_one() {
    return cudaFuncSetAttribute(batch_step_kernel<ST, W_, L_>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Smem<ST>::BYTES_BATCH);
}

template <int ST>
cudaError_t prepare_batch_impl() {
    cudaError_t e = prepare_batch_one<ST, false, false>();
    if (e == cudaSuccess) e = prepare_batch_one<ST, false, true>();
    if (e == cudaSuccess) e = prepare_batch_one<ST, true, false>();
    if (e == cudaSuccess) e = prepare_batch_one<ST, true, true>();
    return e;
}

// Entry points of the per-storage translation units; st is the storage mode.
cudaError_t launch_batch(int st, const BatchArgs& b, bool walls, bool langmuir, unsigned ntiles, cudaStream_t s);
cudaError_t prepare_batch(int st);

cudaError_t launch_step_fp32(const StepArgs& a, int mode, bool walls, bool langmuir, dim3 grid, int pipe, cudaStream_t s);
cudaError_t launch_step_fp16(const StepArgs& a, int mode, bool walls, bool langmuir, dim3 grid, int pipe, cudaStream_t s);
cudaError_t launch_step_bf16(const StepArgs& a, int mode, bool walls, bool langmuir, dim3 grid, int pipe, cudaStream_t s);
cudaError_t launch_step_fp16fg(const StepArgs& a, int mode, bool walls, bool langmuir, dim3 grid, int pipe, cudaStream_t s);
cudaError_t launch_step_bf16fg(const StepArgs& a, int mode, bool walls, bool langmuir, dim3 grid, int pipe, cudaStream_t s);
cudaError_t prepare_step_fp32(int* blocks_per_sm, int* pipe_blocks_per_sm);
cudaError_t prepare_step_fp16(int* blocks_per_sm, int* pipe_blocks_per_sm);
cudaError_t prepare_step_bf16(int* blocks_per_sm, int* pipe_blocks_per_sm);
cudaError_t prepare_step_fp16fg(int* blocks_per_sm, int* pipe_blocks_per_sm);
cudaError_t prepare_step_bf16fg(int* blocks_per_sm, int* pipe_blocks_per_sm);
cudaError_t launch_batch_fp32(const BatchArgs& b, bool walls, bool langmuir, unsigned ntiles, cudaStream_t s);
cudaError_t launch_batch_fp16(const BatchArgs& b, bool walls, bool langmuir, unsigned ntiles, cudaStream_t s);
cudaError_t launch_batch_bf16(const BatchArgs& b, bool walls, bool langmuir, unsigned ntiles, cudaStream_t s);
cudaError_t launch_batch_fp16fg(const BatchArgs& b, bool walls, bool langmuir, unsigned ntiles, cudaStream_t s);
cudaError_t launch_batch_bf16fg(const BatchArgs& b, bool walls, bool langmuir, unsigned ntiles, cudaStream_t s);
cudaError_t prepare_batch_fp32();
cudaError_t prepare_batch_fp16();
cudaError_t prepare_batch_bf16();
cudaError_t prepare_batch_fp16fg();
cudaError_t prepare_batch_bf16fg();

}  // namespace lbm
