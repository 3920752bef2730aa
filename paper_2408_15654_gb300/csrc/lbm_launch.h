// Launch helpers of the step kernels, one translation unit per storage mode
// (step_fp32.cu, step_fp16.cu, step_bf16.cu, step_fp16fg.cu, step_bf16fg.cu) so that the
// instances compile in parallel.  Each storage mode has ten kernel variants: walls or periodic y
// and Langmuir or linear EOS with the flow solved at uniform density or with a density ratio, and
// walls or periodic y with the velocity prescribed (no flow populations; the EOS is unused).
#pragma once
#include <cstring>

#include "lbm_kernels.cuh"

namespace lbm {

// Tile geometry of storage mode st, for the host: tile width and height in cells, the pair box
// (BW x BH) that TMA stages per plane, and the width of the h boxes in (h_i, h_i+1) pairs.
struct TileDims {
    int tx, ty, bw, bh, hbw;
};
inline TileDims tile_dims(int st) {
    const int hx0 = h_is_16bit(st) ? Traits<kFP16>::H_X0 : Traits<kFP32>::H_X0;
    if (cpt_of(st) == 1) return TileDims{Geo<1>::TX, Geo<1>::TY, Geo<1>::BW, Geo<1>::BH, Geo<1>::TX + 2 * hx0};
    return TileDims{Geo<2>::TX, Geo<2>::TY, Geo<2>::BW, Geo<2>::BH, Geo<2>::TX + 2 * hx0};
}

// Runtime flags of a launch, mapped to the kernel variant.
struct Variant {
    bool walls, langmuir, flow, var_rho;
};

// Calls f.template operator()<WALLS, LANGMUIR, FLOW>() for the variant's template arguments (the
// EOS is unused with a prescribed velocity).
template <typename F>
cudaError_t dispatch_variant(const Variant& v, F&& f) {
    if (v.flow && v.var_rho) {
        if (v.walls && v.langmuir) return f.template operator()<true, true, kFlowVarRho>();
        if (v.walls) return f.template operator()<true, false, kFlowVarRho>();
        if (v.langmuir) return f.template operator()<false, true, kFlowVarRho>();
        return f.template operator()<false, false, kFlowVarRho>();
    }
    if (v.flow) {
        if (v.walls && v.langmuir) return f.template operator()<true, true, kFlowUniform>();
        if (v.walls) return f.template operator()<true, false, kFlowUniform>();
        if (v.langmuir) return f.template operator()<false, true, kFlowUniform>();
        return f.template operator()<false, false, kFlowUniform>();
    }
    if (v.walls) return f.template operator()<true, false, kFlowPrescribed>();
    return f.template operator()<false, false, kFlowPrescribed>();
}

// The ten variants, for set-up loops.
inline Variant variant_of(int k) {
    if (k < 8) return Variant{(k & 1) != 0, (k & 2) != 0, true, k >= 4};
    return Variant{k == 8, false, false, false};
}
constexpr int kVariants = 10;

inline cudaLaunchConfig_t pdl_config(dim3 grid, size_t smem, cudaStream_t stream, cudaLaunchAttribute* attr,
                                     unsigned threads) {
    // Every launch uses programmatic dependent launch: the kernel waits (griddepcontrol.wait) for
    // the previous grid before touching memory, so the next launch may be scheduled during the
    // tail of this one.
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// grid = (tiles along x, tiles along y).  A step (mode kStep) with pipe_ctas > 0 runs the
// persistent warp-specialised kernel on pipe_ctas CTAs of nt_pipe<ST>() threads instead of one CTA per tile.
template <int ST>
cudaError_t launch_step_impl(const StepArgs& a, int mode, const Variant& v, dim3 grid, int pipe_ctas,
                             cudaStream_t stream) {
    cudaLaunchAttribute attr[1];
    if (mode == kStep && pipe_ctas > 0) {
        const int ntx = (int)grid.x, nty = (int)grid.y;
        cudaLaunchConfig_t cfg = pdl_config(dim3((unsigned)pipe_ctas), Smem<ST>::BYTES_PIPE, stream, attr, nt_pipe<ST>());
        return dispatch_variant(v, [&]<bool W, bool L, int F>() {
            return cudaLaunchKernelEx(&cfg, pipe_kernel<ST, W, L, F>(), a, ntx, nty);
        });
    }
    cudaLaunchConfig_t cfg = pdl_config(grid, Smem<ST>::BYTES, stream, attr, GeoOf<ST>::NT);
    return dispatch_variant(v, [&]<bool W, bool L, int F>() {
        if (mode == kStep) return cudaLaunchKernelEx(&cfg, step_kernel<ST, W, L, kStep, F>, a);
        return cudaLaunchKernelEx(&cfg, step_kernel<ST, W, L, kMoments, F>, a);
    });
}

// Opt every variant of storage mode ST into its dynamic shared memory; resident CTAs per SM of the
// one-tile kernels (the minimum over the variants) and of the pipelined kernel of variant `use`
// (its register use differs between the variants: a minimum would hold every variant to the
// density-ratio update's 128 registers).
template <int ST>
cudaError_t prepare_step_impl(const Variant& use, int* blocks_per_sm, int* pipe_blocks_per_sm) {
    int tile = 1 << 30, pipe = 0;
    auto one = [&]<bool W, bool L, int F>() -> cudaError_t {
        int b = 0;
        auto k0 = step_kernel<ST, W, L, kStep, F>;
        auto k1 = step_kernel<ST, W, L, kMoments, F>;
        auto kp = pipe_kernel<ST, W, L, F>();
        cudaError_t e = cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<ST>::BYTES);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<ST>::BYTES);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<ST>::BYTES_PIPE);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k0, GeoOf<ST>::NT, Smem<ST>::BYTES);
        tile = b < tile ? b : tile;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k1, GeoOf<ST>::NT, Smem<ST>::BYTES);
        tile = b < tile ? b : tile;
        return e;
    };
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kVariants && e == cudaSuccess; ++k) e = dispatch_variant(variant_of(k), one);
    if (e == cudaSuccess)
        e = dispatch_variant(use, [&]<bool W, bool L, int F>() {
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pipe, pipe_kernel<ST, W, L, F>(), nt_pipe<ST>(),
                                                                 Smem<ST>::BYTES_PIPE);
        });
    *blocks_per_sm = tile;
    *pipe_blocks_per_sm = pipe;
    return e;
}

// One launch of the many-lattice kernel over `ntiles` tiles (all lattices of one variant): one CTA
// per tile, or (b.ws_ctas > 0) the persistent warp-specialised kernel on b.ws_ctas CTAs.
template <int ST>
cudaError_t launch_batch_impl(const BatchArgs& b, const Variant& v, unsigned ntiles, cudaStream_t stream) {
    cudaLaunchAttribute attr[1];
    if (b.ws_ctas > 0) {
        cudaLaunchConfig_t cfg = pdl_config(dim3((unsigned)b.ws_ctas), Smem<ST>::BYTES_BWS, stream, attr, nt_pipe<ST>());
        return dispatch_variant(v, [&]<bool W, bool L, int F>() {
            return cudaLaunchKernelEx(&cfg, batch_ws_kernel<ST, W, L, F>(), b);
        });
    }
    cudaLaunchConfig_t cfg = pdl_config(dim3(ntiles), Smem<ST>::BYTES_BATCH, stream, attr, GeoOf<ST>::NT);
    return dispatch_variant(v, [&]<bool W, bool L, int F>() {
        return cudaLaunchKernelEx(&cfg, batch_step_kernel<ST, W, L, F>, b);
    });
}

// Opt both batch kernels of storage mode ST into their shared memory; resident CTAs per SM of the
// warp-specialised one (the minimum over the variants).
template <int ST>
cudaError_t prepare_batch_impl(int* ws_blocks_per_sm) {
    cudaError_t e = cudaSuccess;
    int ws = 1 << 30;
    for (int k = 0; k < kVariants && e == cudaSuccess; ++k) {
        e = dispatch_variant(variant_of(k), [&]<bool W, bool L, int F>() {
            cudaError_t r = cudaFuncSetAttribute(batch_step_kernel<ST, W, L, F>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<ST>::BYTES_BATCH);
            auto kw = batch_ws_kernel<ST, W, L, F>();
            if (r == cudaSuccess)
                r = cudaFuncSetAttribute(kw, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<ST>::BYTES_BWS);
            int bl = 0;
            if (r == cudaSuccess) r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, kw, nt_pipe<ST>(), Smem<ST>::BYTES_BWS);
            ws = bl < ws ? bl : ws;
            return r;
        });
    }
    *ws_blocks_per_sm = ws;
    return e;
}

// Entry points of the per-storage translation units; st is the storage mode.
cudaError_t launch_step(int st, const StepArgs& a, int mode, const Variant& v, dim3 grid, int pipe, cudaStream_t s);
cudaError_t prepare_step(int st, const Variant& v, int* blocks_per_sm, int* pipe_blocks_per_sm);
cudaError_t launch_batch(int st, const BatchArgs& b, const Variant& v, unsigned ntiles, cudaStream_t s);
cudaError_t prepare_batch(int st, int* ws_blocks_per_sm);

#define LBM_DECLARE_STORAGE(name)                                                                                  \
    cudaError_t launch_step_##name(const StepArgs& a, int mode, const Variant& v, dim3 grid, int pipe,              \
                                   cudaStream_t s);                                                                \
    cudaError_t prepare_step_##name(const Variant& v, int* blocks_per_sm, int* pipe_blocks_per_sm);                 \
    cudaError_t launch_batch_##name(const BatchArgs& b, const Variant& v, unsigned ntiles, cudaStream_t s);         \
    cudaError_t prepare_batch_##name(int* ws_blocks_per_sm);
LBM_DECLARE_STORAGE(fp32)
LBM_DECLARE_STORAGE(fp16)
LBM_DECLARE_STORAGE(bf16)
LBM_DECLARE_STORAGE(fp16fg)
LBM_DECLARE_STORAGE(bf16fg)
#undef LBM_DECLARE_STORAGE

// Body of a per-storage translation unit.
#define LBM_DEFINE_STORAGE(name, ST)                                                                               \
    cudaError_t launch_step_##name(const StepArgs& a, int mode, const Variant& v, dim3 grid, int pipe,              \
                                   cudaStream_t s) {                                                               \
        return launch_step_impl<ST>(a, mode, v, grid, pipe, s);                                                   \
    }                                                                                                              \
    cudaError_t prepare_step_##name(const Variant& v, int* blocks_per_sm, int* pipe_blocks_per_sm) {                \
        return prepare_step_impl<ST>(v, blocks_per_sm, pipe_blocks_per_sm);                                       \
    }                                                                                                              \
    cudaError_t launch_batch_##name(const BatchArgs& b, const Variant& v, unsigned ntiles, cudaStream_t s) {        \
        return launch_batch_impl<ST>(b, v, ntiles, s);                                                            \
    }                                                                                                              \
    cudaError_t prepare_batch_##name(int* ws_blocks_per_sm) { return prepare_batch_impl<ST>(ws_blocks_per_sm); }

}  // namespace lbm
