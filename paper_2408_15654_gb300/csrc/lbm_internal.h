// Host-side definitions shared by the single-lattice API (lbm_api.cu) and the many-lattice
// runtime (lbm_batch.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>

#include "lbm.h"
#include "lbm_launch.h"

namespace lbm_host {

extern thread_local std::string g_err;  // message of the last failing call of this thread
int fail(int code, const char* fmt, ...);

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    int pitch;
    size_t plane;       // cells per plane
    size_t pops_bytes;  // one population buffer
    size_t off_pops[2], off_hist[2], off_shist[2], shist_bytes, off_status, off_partials, total;
};

}  // namespace lbm_host

#define LBM_CUDA(call)                                                                                   \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return lbm_host::fail(LBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

struct lbm_handle {
    lbm_params prm;
    lbm_host::Layout L;
    lbm::Phys phys;
    cudaStream_t stream;
    char* ws;
    void* pops[2];
    float2* hist[2];         // u history, alternating with the population buffers
    float2* shist[2];        // mass-flux history (density ratio != 1), else null
    unsigned* status;
    unsigned* tile_ctr;      // two tile counters of the pipelined kernel (status region + 8 bytes)
    int64_t last_pipe_step;  // step index of the last pipelined launch (-2: none since a reset)
    double* partials;
    CUtensorMap tm_fg[2];    // TMA descriptors of the (f, g) pair planes of each buffer
    CUtensorMap tm_h[2];     // TMA descriptors of the h planes of each buffer
    CUtensorMap tm_hist[2];  // TMA descriptors of the u history buffers
    int tiles_x, tiles_y;    // step-kernel grid: one tile per CTA (lbm::tile_dims of the storage mode)
    int kernel;              // LBM_KERNEL_TILE or LBM_KERNEL_PIPELINED
    int pipe_ctas;           // CTAs of the pipelined kernel (0: it does not fit)
    int cur;          // buffer holding the current state
    int initialized;
    int first;        // 1 until the first step after lbm_init_fields
    int64_t steps;
};
