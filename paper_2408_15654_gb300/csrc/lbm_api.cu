// Host implementation of the C ABI declared in include/lbm.h.
//
// The library owns no device memory: the caller passes one workspace, carved here into
//   [pops A | pops B | u history A | u history B | (S history A | S history B) | status word | reduction partials]
// every part 256-byte aligned.  Between steps the population buffer that is not current is dead
// (the next step overwrites all of it), so host transfers stage through it.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "lbm_internal.h"

static_assert(LBM_STORE_FP32 == lbm::kFP32 && LBM_STORE_FP16 == lbm::kFP16 && LBM_STORE_BF16 == lbm::kBF16 &&
                  LBM_STORE_FP16_FG == lbm::kFP16FG && LBM_STORE_BF16_FG == lbm::kBF16FG,
              "storage codes of the ABI and the kernels agree");

namespace lbm_host {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

}  // namespace lbm_host

using namespace lbm_host;

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (no -lcuda).
int get_encoder(EncodeTiledFn* fn) {
    static EncodeTiledFn cached = nullptr;
    if (!cached) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !ptr)
            return fail(LBM_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
        cached = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    *fn = cached;
    return LBM_OK;
}

// 3-D tensor map {nx, ny, planes} of elements of es bytes (8: float pairs, 4: floats or
// 16-bit pairs, 2: 16-bit values); pitch and plane stride counted in elements.  The step's load
// maps cover whole planes including the ghost frame (nx = pitch, ny = rows of a plane); its store
// maps end at the grid's last column and row.
int encode_map(CUtensorMap* tm, void* base, int es, int nx, int ny, int planes, int pitch, size_t plane,
               unsigned bw, unsigned bh, unsigned bp) {
    EncodeTiledFn enc;
    int rc = get_encoder(&enc);
    if (rc) return rc;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * es, (cuuint64_t)plane * es};
    const cuuint32_t box[3] = {bw, bh, bp};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = es == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64
                                   : (es == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16);
    CUresult r = enc(tm, dt, 3, base, dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(LBM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return LBM_OK;
}

// Opt the step-kernel instances of storage mode st into their shared memory; CTAs per SM of the
// one-tile and of the pipelined kernels.
// The kernel variant of a lattice's parameters (the EOS is unused with a prescribed velocity).
lbm::Variant variant_of(const lbm_params& p, bool var_rho) {
    const bool flow = p.velocity == LBM_VELOCITY_SOLVED;
    return lbm::Variant{p.bc_y == LBM_BC_WALLS, flow && p.eos == LBM_EOS_LANGMUIR, flow, var_rho};
}

int prepare_kernels(int st, const lbm::Variant& v, int* blocks_per_sm, int* pipe_blocks_per_sm) {
    cudaError_t e = lbm::prepare_step(st, v, blocks_per_sm, pipe_blocks_per_sm);
    if (e != cudaSuccess) return fail(LBM_ECUDA, "kernel setup: %s", cudaGetErrorString(e));
    if (*blocks_per_sm < 1) return fail(LBM_ECUDA, "the step kernel does not fit on an SM");
    return LBM_OK;
}

bool rate_ok(double s) { return s > 0.0 && s < 2.0; }

int validate(const lbm_params* p) {
    if (!p) return fail(LBM_EINVAL, "params is NULL");
    if (p->nx < 2 || p->ny < 2) return fail(LBM_EINVAL, "nx and ny must be >= 2 (got %d x %d)", p->nx, p->ny);
    if ((long long)p->nx * p->ny > (1LL << 30)) return fail(LBM_EINVAL, "grid too large");
    // the one-tile, moments and initialisation kernels run one CTA row per 8 cell rows, and a
    // launch has at most 65535 rows of CTAs
    if (p->ny > 65535 * 8) return fail(LBM_EINVAL, "ny = %d exceeds 524280 rows", p->ny);
    if (p->bc_y != LBM_BC_PERIODIC && p->bc_y != LBM_BC_WALLS) return fail(LBM_EINVAL, "bad bc_y");
    if (p->eos != LBM_EOS_LINEAR && p->eos != LBM_EOS_LANGMUIR) return fail(LBM_EINVAL, "bad eos");
    if (p->storage < LBM_STORE_FP32 || p->storage > LBM_STORE_BF16_FG)
        return fail(LBM_EINVAL, "storage mode %d not supported", p->storage);
    if (p->velocity != LBM_VELOCITY_SOLVED && p->velocity != LBM_VELOCITY_PRESCRIBED)
        return fail(LBM_EINVAL, "bad velocity mode %d", p->velocity);
    if (!(p->phiA != p->phiB) || !(p->W > 0) || !(p->M_phi > 0) || !(p->D > 0))
        return fail(LBM_EINVAL, "need phiA != phiB, W > 0, M_phi > 0, D > 0");
    if (!(p->rhoA > 0) || !(p->rhoB > 0)) return fail(LBM_EINVAL, "densities must be > 0");
    if (!(p->muA > 0) || !(p->muB > 0)) return fail(LBM_EINVAL, "viscosities must be > 0");
    const double* rs[3] = {p->s_f, p->s_g, p->s_h};
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 5; ++j) {
            if ((k == 0 || k == 1) && j == 1) continue;  // transport rates of f, g: recomputed
            if (k == 2 && j == 2) continue;              // viscous rate of h: recomputed
            if (k == 2 && (j == 0)) continue;            // s0^h acts only on the dead h_0
            if (k == 2 && j == 4 && p->s_h[4] <= 0.0) continue;  // tied to s2^h
            if ((k == 0 || k == 1) && j == 0) continue;  // conserved zeroth moment
            if (!rate_ok(rs[k][j])) return fail(LBM_EINVAL, "relaxation rate %d of population %d outside (0, 2)", j, k);
        }
    const double s1f = 1.0 / (3.0 * p->M_phi + 0.5), s1g = 1.0 / (3.0 * p->D + 0.5);
    if (!rate_ok(s1f) || !rate_ok(s1g)) return fail(LBM_EINVAL, "M_phi or D gives a rate outside (0, 2)");
    if (!std::isfinite(p->sigma0) || !std::isfinite(p->E0) || !std::isfinite(p->gx) || !std::isfinite(p->gy) ||
        !std::isfinite(p->u_top) || !std::isfinite(p->u_bot) || !(p->n_eps >= 0))
        return fail(LBM_EINVAL, "non-finite physical parameter");
    return LBM_OK;
}

// Plane geometry: the grid inside its ghost frame (lbm::kGX columns left, at least 2 right,
// lbm::kGY rows above and below), pitch a multiple of 32 cells.
void frame_of(int nx, int ny, int* pitch, size_t* plane, long long* org) {
    *pitch = (nx + lbm::kGX + 2 + 31) / 32 * 32;
    *plane = (size_t)(ny + 2 * lbm::kGY) * (size_t)*pitch;
    *org = (long long)lbm::kGY * *pitch + lbm::kGX;
}

Layout layout_of(const lbm_params* p) {
    Layout L;
    long long org = 0;
    frame_of(p->nx, p->ny, &L.pitch, &L.plane, &org);
    // a population buffer also stages, while it is not the current one, the five FP64 fields that
    // lbm_init_fields and lbm_get_moments move through host memory: 40 bytes per cell, more than
    // the 36 of 16-bit storage with a prescribed velocity
    const size_t pops = L.plane * (size_t)lbm::pop_bytes_per_cell(p->storage, p->velocity == LBM_VELOCITY_SOLVED);
    const size_t stage = (size_t)p->nx * (size_t)p->ny * 5 * sizeof(double);
    L.pops_bytes = align_up(pops > stage ? pops : stage);
    size_t off = 0;
    L.off_pops[0] = off; off += L.pops_bytes;
    L.off_pops[1] = off; off += L.pops_bytes;
    L.off_hist[0] = off; off += align_up(L.plane * sizeof(float2));
    L.off_hist[1] = off; off += align_up(L.plane * sizeof(float2));
    // mass-flux history, only with a density ratio (and a solved flow)
    L.shist_bytes = (p->rhoA != p->rhoB && p->velocity == LBM_VELOCITY_SOLVED) ? align_up(L.plane * sizeof(float2)) : 0;
    L.off_shist[0] = off; off += L.shist_bytes;
    L.off_shist[1] = off; off += L.shist_bytes;
    L.off_status = off; off += kAlign;
    L.off_partials = off; off += align_up(lbm::kMaxPartials * sizeof(double) + sizeof(double));
    L.total = off;
    return L;
}

// Step kernel of a new handle: the warp-specialised persistent kernel where it is faster (16-bit
// storage, and any storage with a density ratio != 1), else the one-tile kernel.
int default_kernel(int storage, const lbm::Variant& v, int pipe_blocks_per_sm) {
    // Measured on GB300 (us per step, one-tile / warp-specialised), sheared drop 2048 x 1024: FP32
    // 72.8 / 73.7 (HBM-bound either way); two cells per thread in 32 x 8 tiles: FP16 51.5 / 50.6,
    // BF16 52.0 / 50.7, FP16_FG 55.8 / 54.9, BF16_FG 55.9 / 54.9 (one-tile kernel: five CTAs per
    // SM; warp-specialised: four CTAs of four compute warps and a copy warp, which stages one tile
    // ahead); prescribed velocity, the same grid: FP32 52.5 / 55.1, FP16 40.1 / 37.5; rising bubble
    // 1024 x 2048 (density ratio 10): FP32 81.0 / 80.1, FP16 62.6 / 57.9.
    if (pipe_blocks_per_sm < 1) return LBM_KERNEL_TILE;
    if (v.var_rho || storage != LBM_STORE_FP32) return LBM_KERNEL_PIPELINED;
    return LBM_KERNEL_TILE;
}

lbm::Phys make_phys(const lbm_params* p, const Layout& L) {
    lbm::Phys f;
    std::memset(&f, 0, sizeof(f));
    const double dphi = p->phiA - p->phiB;
    f.nx = p->nx;
    f.ny = p->ny;
    f.pitch = L.pitch;
    f.plane = (long long)L.plane;
    f.org = (long long)lbm::kGY * L.pitch + lbm::kGX;
    f.phiA = (float)p->phiA;
    f.phiB = (float)p->phiB;
    f.inv_dphi = (float)(1.0 / dphi);
    f.cA = (float)(4.0 / (p->W * dphi));
    f.cap_k = (float)(3.0 / (2.0 * dphi * dphi));
    f.c16W = (float)(16.0 / p->W);
    f.W = (float)p->W;
    f.mar_k = (float)(3.0 * p->W / (2.0 * dphi * dphi));
    f.sigma0 = (float)p->sigma0;
    f.E0 = (float)p->E0;
    f.rho = (float)p->rhoA;
    f.inv_rho = (float)(1.0 / p->rhoA);
    f.var_rho = p->rhoA != p->rhoB ? 1 : 0;
    f.rhoB = (float)p->rhoB;
    f.drho = (float)((p->rhoA - p->rhoB) / dphi);
    f.sfac = (float)(p->M_phi * (p->rhoA - p->rhoB) / dphi);
    f.muB = (float)p->muB;
    f.dmu = (float)(p->muA - p->muB);
    f.s2h = (float)(1.0 / (3.0 * p->muB / p->rhoA + 0.5));
    f.gx = (float)p->gx;
    f.gy = (float)p->gy;
    const double s1f = 1.0 / (3.0 * p->M_phi + 0.5), s1g = 1.0 / (3.0 * p->D + 0.5);
    const double sf[4] = {s1f, p->s_f[2], p->s_f[3], p->s_f[4]}, sg[4] = {s1g, p->s_g[2], p->s_g[3], p->s_g[4]};
    float* nS[4] = {f.nS1, f.nS2, f.nS3, f.nS4};
    for (int k = 0; k < 4; ++k) {
        nS[k][0] = (float)(-sf[k]);
        nS[k][1] = (float)(-sg[k]);
    }
    f.K1[0] = (float)(1.0 - 0.5 * sf[0]);
    f.K1[1] = (float)(1.0 - 0.5 * sg[0]);
    f.K3[0] = (float)(1.0 - 0.5 * sf[2]);
    f.K3[1] = (float)(1.0 - 0.5 * sg[2]);
    const double s2h = 1.0 / (3.0 * p->muB / p->rhoA + 0.5);
    const double s4h = p->s_h[4] <= 0.0 ? s2h : p->s_h[4];
    f.s1h = (float)p->s_h[1];
    f.s3h = (float)p->s_h[3];
    f.s4h = (float)p->s_h[4];
    f.k1h = (float)(1.0 - 0.5 * p->s_h[1]);
    f.k3h = (float)(1.0 - 0.5 * p->s_h[3]);
    f.k2h = (float)(1.0 - 0.5 * s2h);
    f.s4h_eff = (float)s4h;
    f.k4h = (float)(1.0 - 0.5 * s4h);
    f.tie_s4h = p->s_h[4] <= 0.0 ? 1 : 0;
    // 16-bit storage: references of the stored deviations (the scales are compile-time
    // constants of each mode)
    f.phi_ref = (float)(0.5 * (p->phiA + p->phiB));
    // 16-bit h: the velocity part removed before storage uses one reference density, so that the
    // decoder reproduces it exactly (with a density ratio it only approximates the local
    // 3 w_i rho c_i.u, which costs accuracy, not correctness)
    const double rho_ref = 0.5 * (p->rhoA + p->rhoB);
    f.kh_axis = (float)(3.0 / 9.0 * rho_ref);
    f.kh_diag = (float)(3.0 / 36.0 * rho_ref);
    f.kh3 = (float)(3.0 * rho_ref);
    f.u_top = (float)p->u_top;
    f.u_bot = (float)p->u_bot;
    f.n_eps2 = (float)(p->n_eps * p->n_eps);
    return f;
}

}  // namespace


namespace {

int launch_step(lbm_handle* h, int mode, double* const out[5]) {
    lbm::StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.tm_fg = h->tm_fg[h->cur];
    a.tm_h = h->tm_h[h->cur];
    a.tm_hist = h->tm_hist[h->cur];
    a.p = h->phys;
    a.io.first = h->first;
    a.io.src = h->pops[h->cur];
    a.io.dst = h->pops[h->cur ^ 1];
    a.io.hist_src = h->hist[h->cur];
    a.io.hist_dst = h->hist[h->cur ^ 1];
    a.io.shist_src = h->shist[h->cur];
    a.io.shist_dst = h->shist[h->cur ^ 1];
    a.io.status = h->status;
    // salt of the stochastic rounding: a function of the step count, so a restored checkpoint
    // continues bit for bit
    a.io.seed = lbm::step_seed(h->steps);
    if (out)
        for (int k = 0; k < 5; ++k) a.io.out[k] = out[k];
    const dim3 grid(h->tiles_x, h->tiles_y);
    const int pipe = (mode == lbm::kStep && h->kernel == LBM_KERNEL_PIPELINED) ? h->pipe_ctas : 0;
    if (pipe) {
        // tile counters: launch s counts on counter s mod 2 and zeroes the other for launch s + 1;
        // after any other launch both start from zero
        if (h->last_pipe_step != h->steps - 1)
            LBM_CUDA(cudaMemsetAsync(h->tile_ctr, 0, 2 * sizeof(unsigned), h->stream));
        a.tile_ctr = h->tile_ctr + (h->steps & 1);
        a.tile_ctr_next = h->tile_ctr + ((h->steps + 1) & 1);
        h->last_pipe_step = h->steps;
    }
    cudaError_t e = lbm::launch_step(h->prm.storage, a, mode, variant_of(h->prm, h->phys.var_rho != 0), grid, pipe,
                                     h->stream);
    if (e != cudaSuccess) return fail(LBM_ECUDA, "step launch: %s", cudaGetErrorString(e));
    return LBM_OK;
}

// FP64 sum of phi (lane 0) or psi (lane 1) of a population buffer into partials[0..blocks),
// then partials[blocks] ... written to *dres.
int launch_reduce(int st, const void* pops, int lane, bool pulled, int nx, int ny, int pitch, size_t plane, long long org,
                  const lbm::Phys& ph,
                  int blocks, double* partials, double* dres, cudaStream_t stream) {
    // the pair planes of the FG modes are stored like those of the all-16-bit modes
    const long long pl = (long long)plane;
    if (st == LBM_STORE_FP16 || st == LBM_STORE_FP16_FG)
        lbm::reduce_partial_kernel<lbm::kFP16><<<blocks, lbm::kReduceThreads, 0, stream>>>(pops, lane, pulled, nx, ny,
                                                                                           pitch, pl, org, ph, partials);
    else if (st == LBM_STORE_BF16 || st == LBM_STORE_BF16_FG)
        lbm::reduce_partial_kernel<lbm::kBF16><<<blocks, lbm::kReduceThreads, 0, stream>>>(pops, lane, pulled, nx, ny,
                                                                                           pitch, pl, org, ph, partials);
    else
        lbm::reduce_partial_kernel<lbm::kFP32><<<blocks, lbm::kReduceThreads, 0, stream>>>(pops, lane, pulled, nx, ny,
                                                                                           pitch, pl, org, ph, partials);
    LBM_CUDA(cudaGetLastError());
    lbm::reduce_final_kernel<<<1, lbm::kReduceThreads, 0, stream>>>(partials, blocks, dres);
    LBM_CUDA(cudaGetLastError());
    return LBM_OK;
}

// The address by which a kernel reaches host memory p, or nullptr: page-locked host memory
// (cudaHostAlloc, cudaHostRegister) is mapped into the device's address space, so the
// initialisation and moments kernels read and write it directly over the CPU-GPU link instead of
// through a staging copy.  Pageable memory returns nullptr and is staged.
const void* mapped_host(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear the error of an unknown pointer
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int read_status(lbm_handle* h, unsigned* st) {
    LBM_CUDA(cudaMemcpyAsync(st, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

// LBM_OK, LBM_ETIMEOUT (a staging copy did not arrive within its bounded wait) or LBM_EUNSTABLE.
int status_code(unsigned st) {
    if (st & lbm::kStatusTimeout) return fail(LBM_ETIMEOUT, "a bounded wait for a tile copy gave up");
    if (st & lbm::kStatusUnstable) return fail(LBM_EUNSTABLE, "the device flagged an unstable state");
    return LBM_OK;
}

}  // namespace

// Fixed scratch of lbm_reduce_noalloc: one FP64 partial per row plus the result.
static __device__ __align__(256) double g_noalloc_partials[LBM_NOALLOC_MAX_ROWS + 1];

namespace {

// The scratch's device address differs per CUDA context (the library's module is loaded into each
// context that uses it), so the cache is keyed by the context current at the call: the primary
// context of each device, or any context the caller has made current.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
std::mutex g_noalloc_mu;
std::vector<std::pair<CUcontext, double*>> g_noalloc_ptr;

int current_context(CUcontext* ctx) {
    static CtxGetCurrentFn fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &ptr, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !ptr)
            return fail(LBM_ECUDA, "cuCtxGetCurrent is not available from the driver");
        fn = reinterpret_cast<CtxGetCurrentFn>(ptr);
    }
    *ctx = nullptr;
    if (fn(ctx) != CUDA_SUCCESS) return fail(LBM_ECUDA, "cuCtxGetCurrent failed");
    return LBM_OK;
}

// Device address of the fixed scratch in the current context, looked up once per context (the
// lookup makes the device's primary context current if no context is).
int noalloc_scratch(double** out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    CUcontext ctx = nullptr;
    int rc = current_context(&ctx);
    if (rc) return rc;
    if (ctx)
        for (const auto& e : g_noalloc_ptr)
            if (e.first == ctx) {
                *out = e.second;
                return LBM_OK;
            }
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
    if (e != cudaSuccess) return fail(LBM_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    rc = current_context(&ctx);
    if (rc) return rc;
    g_noalloc_ptr.emplace_back(ctx, static_cast<double*>(ptr));
    *out = static_cast<double*>(ptr);
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_selftest_wait(unsigned* d_word, void* cuda_stream) {
    g_err.clear();
    if (!d_word) return fail(LBM_EINVAL, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    LBM_CUDA(cudaMemsetAsync(d_word, 0xFF, sizeof(unsigned), st));
    lbm::selftest_wait_kernel<<<1, 32, 0, st>>>(d_word);
    LBM_CUDA(cudaGetLastError());
    unsigned w = 0;
    LBM_CUDA(cudaMemcpyAsync(&w, d_word, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    LBM_CUDA(cudaStreamSynchronize(st));
    if (w == lbm::kStatusTimeout) return fail(LBM_ETIMEOUT, "the bounded wait gave up, as it should");
    return fail(LBM_ECUDA, "the self-test wait did not report a timeout (word %u)", w);
}

int lbm_reduce_noalloc(const void* d_pops, int nx, int ny, int what, void* cuda_stream, double* out) {
    g_err.clear();
    if (!d_pops || !out) return fail(LBM_EINVAL, "d_pops and out are required");
    if (nx < 2 || ny < 2 || (long long)nx * ny > (1LL << 30))
        return fail(LBM_EINVAL, "grid %d x %d outside 2 <= nx, ny and nx * ny <= 2^30", nx, ny);
    if (ny > LBM_NOALLOC_MAX_ROWS)
        return fail(LBM_EINVAL, "ny = %d exceeds the %d rows that the fixed scratch of lbm_reduce_noalloc holds", ny,
                    LBM_NOALLOC_MAX_ROWS);
    if (what != LBM_SUM_PHI && what != LBM_SUM_PSI) return fail(LBM_EINVAL, "bad reduction selector");
    double* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    int pitch = 0;
    size_t plane = 0;
    long long org = 0;
    frame_of(nx, ny, &pitch, &plane, &org);
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    lbm::Phys ph;
    std::memset(&ph, 0, sizeof(ph));
    rc = launch_reduce(LBM_STORE_FP32, d_pops, what == LBM_SUM_PSI ? 1 : 0, false, nx, ny, pitch, plane, org, ph, ny,
                       scratch, scratch + LBM_NOALLOC_MAX_ROWS, stream);
    if (rc) return rc;
    LBM_CUDA(cudaMemcpyAsync(out, scratch + LBM_NOALLOC_MAX_ROWS, sizeof(double), cudaMemcpyDeviceToHost, stream));
    LBM_CUDA(cudaStreamSynchronize(stream));
    return LBM_OK;
}

int lbm_workspace_bytes(const lbm_params* p, size_t* bytes) {
    g_err.clear();
    int rc = validate(p);
    if (rc) return rc;
    if (!bytes) return fail(LBM_EINVAL, "bytes is NULL");
    *bytes = layout_of(p).total;
    return LBM_OK;
}

int lbm_create(const lbm_params* p, void* d_workspace, size_t bytes, void* cuda_stream, lbm_handle** out) {
    g_err.clear();
    int rc = validate(p);
    if (rc) return rc;
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!d_workspace) return fail(LBM_EINVAL, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(d_workspace) % kAlign) return fail(LBM_EINVAL, "workspace not 256-byte aligned");
    const Layout L = layout_of(p);
    if (bytes < L.total) return fail(LBM_ENOMEM, "workspace of %zu bytes < %zu needed", bytes, L.total);
    cudaPointerAttributes attr;
    LBM_CUDA(cudaPointerGetAttributes(&attr, d_workspace));
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return fail(LBM_EINVAL, "workspace is not device memory");
    lbm_handle* h = new (std::nothrow) lbm_handle;
    if (!h) return fail(LBM_ENOMEM, "host allocation failed");
    std::memset(h, 0, sizeof(*h));
    h->prm = *p;
    h->L = L;
    h->phys = make_phys(p, L);
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->ws = static_cast<char*>(d_workspace);
    h->pops[0] = h->ws + L.off_pops[0];
    h->pops[1] = h->ws + L.off_pops[1];
    h->hist[0] = reinterpret_cast<float2*>(h->ws + L.off_hist[0]);
    h->hist[1] = reinterpret_cast<float2*>(h->ws + L.off_hist[1]);
    h->shist[0] = L.shist_bytes ? reinterpret_cast<float2*>(h->ws + L.off_shist[0]) : nullptr;
    h->shist[1] = L.shist_bytes ? reinterpret_cast<float2*>(h->ws + L.off_shist[1]) : nullptr;
    h->status = reinterpret_cast<unsigned*>(h->ws + L.off_status);
    h->tile_ctr = h->status + 2;
    h->last_pipe_step = -2;
    h->partials = reinterpret_cast<double*>(h->ws + L.off_partials);
    int bps = 0, bps_pipe = 0, sms = 0;
    rc = prepare_kernels(p->storage, variant_of(*p, h->phys.var_rho != 0), &bps, &bps_pipe);
    if (!rc && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, attr.device) != cudaSuccess)
        rc = fail(LBM_ECUDA, "cudaDeviceGetAttribute failed");
    const bool pair16 = lbm::pair_is_16bit(p->storage), h16 = lbm::h_is_16bit(p->storage);
    const lbm::TileDims td = lbm::tile_dims(p->storage);
    const int es_pair = pair16 ? 4 : 8;
    // h boxes: one plane per pair of links (elements of two values: 4 bytes for 16-bit h, 8 for
    // FP32 h), TY + 1 rows to cover both links' source rows
    const unsigned hbw = (unsigned)td.hbw;
    const unsigned hbh = (unsigned)td.ty + 1;
    const int h_planes = lbm::kHPlanes / 2, es_hbox = h16 ? 4 : 8;
    for (int b = 0; b < 2 && !rc; ++b) {
        rc = encode_map(&h->tm_fg[b], h->pops[b], es_pair, L.pitch, p->ny + 2 * lbm::kGY, lbm::kPairs, L.pitch, L.plane,
                        (unsigned)td.bw, (unsigned)td.bh, 1);
        char* hbase = static_cast<char*>(h->pops[b]) + (size_t)lbm::kPairs * L.plane * es_pair;
        if (!rc && p->velocity == LBM_VELOCITY_SOLVED)  // no h planes with a prescribed velocity
            rc = encode_map(&h->tm_h[b], hbase, es_hbox, L.pitch, p->ny + 2 * lbm::kGY, h_planes, L.pitch, L.plane, hbw, hbh, 1);
    }
    for (int b = 0; b < 2 && !rc; ++b)
        rc = h16 ? encode_map(&h->tm_hist[b], h->hist[b], 8, L.pitch, p->ny + 2 * lbm::kGY, 1, L.pitch, L.plane,
                              (unsigned)td.bw, (unsigned)td.bh, 1)
                 : encode_map(&h->tm_hist[b], h->hist[b], 8, L.pitch, p->ny + 2 * lbm::kGY, 1, L.pitch, L.plane,
                              (unsigned)td.tx, (unsigned)td.ty, 1);
    if (rc) {
        delete h;
        return rc;
    }
    h->tiles_x = (p->nx + td.tx - 1) / td.tx;
    h->tiles_y = (p->ny + td.ty - 1) / td.ty;
    {
        const long long ntiles = (long long)h->tiles_x * h->tiles_y, slots = (long long)bps_pipe * sms;
        h->pipe_ctas = (int)(ntiles < slots ? ntiles : slots);
        h->kernel = default_kernel(p->storage, variant_of(*p, h->phys.var_rho != 0), bps_pipe);
    }
    cudaError_t e = cudaMemsetAsync(h->ws, 0, L.total, h->stream);
    if (e != cudaSuccess) {
        delete h;
        return fail(LBM_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
    *out = h;
    return LBM_OK;
}

int lbm_init_fields(lbm_handle* h, const double* phi, const double* psi, const double* ux, const double* uy,
                    const double* P, int mem) {
    g_err.clear();
    if (!h) return fail(LBM_EINVAL, "handle is NULL");
    if (!phi || !psi || !ux || !uy || !P) return fail(LBM_EINVAL, "all five fields are required");
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) return fail(LBM_EINVAL, "bad mem kind");
    const size_t n = (size_t)h->prm.nx * h->prm.ny;
    const double* d[5] = {phi, psi, ux, uy, P};
    const int tgt = 0;
    if (mem == LBM_MEM_HOST) {
        const void* m[5];
        bool mapped = true;
        for (int k = 0; k < 5; ++k) mapped = mapped && (m[k] = mapped_host(d[k])) != nullptr;
        if (mapped) {
            // page-locked: the initialisation kernel reads the fields where they are
            for (int k = 0; k < 5; ++k) d[k] = static_cast<const double*>(m[k]);
        } else {
            // stage through the buffer that becomes dead (sized for 5 doubles per cell, see layout_of)
            double* stage = reinterpret_cast<double*>(h->pops[tgt ^ 1]);
            for (int k = 0; k < 5; ++k) {
                LBM_CUDA(cudaMemcpyAsync(stage + k * n, d[k], n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
                d[k] = stage + k * n;
            }
        }
    }
    LBM_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    LBM_CUDA(cudaMemsetAsync(h->pops[tgt], 0, h->L.pops_bytes, h->stream));
    lbm::InitArgs a;
    std::memset(&a, 0, sizeof(a));
    a.p = h->phys;
    a.phi = d[0]; a.psi = d[1]; a.ux = d[2]; a.uy = d[3]; a.P = d[4];
    a.dst = h->pops[tgt];
    a.hist = h->hist[tgt];
    a.status = h->status;
    a.langmuir = h->prm.eos == LBM_EOS_LANGMUIR;
    a.walls = h->prm.bc_y == LBM_BC_WALLS;
    a.flow = h->prm.velocity == LBM_VELOCITY_SOLVED;
    const dim3 block(32, 8), grid((h->prm.nx + 31) / 32, (h->prm.ny + 7) / 8);
    switch (h->prm.storage) {
        case LBM_STORE_FP16: lbm::init_kernel<lbm::kFP16><<<grid, block, 0, h->stream>>>(a); break;
        case LBM_STORE_BF16: lbm::init_kernel<lbm::kBF16><<<grid, block, 0, h->stream>>>(a); break;
        case LBM_STORE_FP16_FG: lbm::init_kernel<lbm::kFP16FG><<<grid, block, 0, h->stream>>>(a); break;
        case LBM_STORE_BF16_FG: lbm::init_kernel<lbm::kBF16FG><<<grid, block, 0, h->stream>>>(a); break;
        default: lbm::init_kernel<lbm::kFP32><<<grid, block, 0, h->stream>>>(a); break;
    }
    LBM_CUDA(cudaGetLastError());
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    h->cur = tgt;
    h->first = 1;
    h->steps = 0;
    h->last_pipe_step = -2;
    h->initialized = 0;
    unsigned st = 0;
    int rc = read_status(h, &st);
    if (rc) return rc;
    if (st) return fail(LBM_EINVAL, "initial fields contain non-finite values (or psi >= 1 with the Langmuir EOS)");
    h->initialized = 1;
    return LBM_OK;
}

int lbm_step(lbm_handle* h, int64_t n) {
    g_err.clear();
    if (!h) return fail(LBM_EINVAL, "handle is NULL");
    if (!h->initialized) return fail(LBM_ESTATE, "lbm_step before lbm_init_fields");
    if (n < 0) return fail(LBM_EINVAL, "negative step count");
    for (int64_t k = 0; k < n; ++k) {
        int rc = launch_step(h, lbm::kStep, nullptr);
        if (rc) return rc;
        h->cur ^= 1;
        h->first = 0;
        h->steps++;
    }
    return LBM_OK;
}

int lbm_get_moments(lbm_handle* h, unsigned mask, double* const out[5], int mem) {
    g_err.clear();
    if (!h) return fail(LBM_EINVAL, "handle is NULL");
    if (!h->initialized) return fail(LBM_ESTATE, "lbm_get_moments before lbm_init_fields");
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) return fail(LBM_EINVAL, "bad mem kind");
    if (mask & ~31u) return fail(LBM_EINVAL, "bad mask");
    if (!out && mask) return fail(LBM_EINVAL, "out is NULL");
    const size_t n = (size_t)h->prm.nx * h->prm.ny;
    double* dev_out[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    double* stage = reinterpret_cast<double*>(h->pops[h->cur ^ 1]);
    bool mapped = mem == LBM_MEM_HOST;  // every requested output page-locked: written where it is
    for (int k = 0; k < 5; ++k) {
        if (!(mask & (1u << k))) continue;
        if (!out[k]) return fail(LBM_EINVAL, "out[%d] is NULL but requested by mask", k);
        if (mem == LBM_MEM_HOST) {
            void* m = const_cast<void*>(mapped_host(out[k]));
            mapped = mapped && m != nullptr;
            dev_out[k] = m ? static_cast<double*>(m) : stage + k * n;
        } else {
            dev_out[k] = out[k];
        }
    }
    if (mem == LBM_MEM_HOST && !mapped)
        for (int k = 0; k < 5; ++k)
            if (mask & (1u << k)) dev_out[k] = stage + k * n;
    int rc = launch_step(h, lbm::kMoments, dev_out);
    if (rc) return rc;
    if (mem == LBM_MEM_HOST && !mapped)
        for (int k = 0; k < 5; ++k)
            if (mask & (1u << k))
                LBM_CUDA(cudaMemcpyAsync(out[k], dev_out[k], n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    unsigned st = 0;
    rc = read_status(h, &st);
    if (rc) return rc;
    return status_code(st);
}

int lbm_reduce(lbm_handle* h, int what, double* out) {
    g_err.clear();
    if (!h) return fail(LBM_EINVAL, "handle is NULL");
    if (!h->initialized) return fail(LBM_ESTATE, "lbm_reduce before lbm_init_fields");
    if (what != LBM_SUM_PHI && what != LBM_SUM_PSI) return fail(LBM_EINVAL, "bad reduction selector");
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    const int blocks = h->prm.ny < lbm::kMaxPartials ? h->prm.ny : lbm::kMaxPartials;
    double* dres = h->partials + lbm::kMaxPartials;
    // before the first step the buffer is staged for the first pull (see reduce_partial_kernel)
    int rc = launch_reduce(h->prm.storage, h->pops[h->cur], what == LBM_SUM_PSI ? 1 : 0, h->first != 0, h->prm.nx,
                           h->prm.ny, h->L.pitch, h->L.plane, h->phys.org, h->phys, blocks, h->partials, dres, h->stream);
    if (rc) return rc;
    LBM_CUDA(cudaMemcpyAsync(out, dres, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    unsigned st = 0;
    rc = read_status(h, &st);
    if (rc) return rc;
    return status_code(st);
}

int lbm_status(lbm_handle* h) {
    g_err.clear();
    if (!h) return fail(LBM_EINVAL, "handle is NULL");
    unsigned st = 0;
    int rc = read_status(h, &st);
    if (rc) return rc;
    return status_code(st);
}

// State blob: header, then the current population buffer, then the u history (and, with a
// density ratio, the mass-flux history).
struct StateHeader {
    uint64_t magic;
    int32_t nx, ny, pitch, first;
    int64_t steps;
    int32_t storage, velocity, var_rho, pad;  // what the population buffer's bytes mean
};
// Names the population layout of the blob ("LBM4STAT": h stored in link pairs, the storage and
// flow modes in the header); blobs written with another layout are refused by lbm_set_state.
static const uint64_t kStateMagic = 0x4c424d3453544154ull;  // "LBM4STAT"

int lbm_state_bytes(const lbm_handle* h, size_t* bytes) {
    g_err.clear();
    if (!h || !bytes) return fail(LBM_EINVAL, "NULL argument");
    *bytes = sizeof(StateHeader) +
             h->L.plane * (size_t)lbm::pop_bytes_per_cell(h->prm.storage, h->prm.velocity == LBM_VELOCITY_SOLVED) +
             h->L.plane * sizeof(float2) * (h->shist[0] ? 2 : 1);
    return LBM_OK;
}

int lbm_get_state(lbm_handle* h, void* host_blob, size_t bytes) {
    g_err.clear();
    if (!h || !host_blob) return fail(LBM_EINVAL, "NULL argument");
    if (!h->initialized) return fail(LBM_ESTATE, "no state before lbm_init_fields");
    size_t need = 0;
    lbm_state_bytes(h, &need);
    if (bytes < need) return fail(LBM_EINVAL, "blob of %zu bytes < %zu needed", bytes, need);
    StateHeader hd{kStateMagic, h->prm.nx, h->prm.ny, h->L.pitch, h->first, h->steps,
                   h->prm.storage, h->prm.velocity, h->phys.var_rho, 0};
    char* b = static_cast<char*>(host_blob);
    std::memcpy(b, &hd, sizeof(hd));
    const size_t pb = h->L.plane * (size_t)lbm::pop_bytes_per_cell(h->prm.storage, h->prm.velocity == LBM_VELOCITY_SOLVED);
    LBM_CUDA(cudaMemcpyAsync(b + sizeof(hd), h->pops[h->cur], pb, cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(cudaMemcpyAsync(b + sizeof(hd) + pb, h->hist[h->cur], h->L.plane * sizeof(float2), cudaMemcpyDeviceToHost,
                             h->stream));
    if (h->shist[0])
        LBM_CUDA(cudaMemcpyAsync(b + sizeof(hd) + pb + h->L.plane * sizeof(float2), h->shist[h->cur],
                                 h->L.plane * sizeof(float2), cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_set_state(lbm_handle* h, const void* host_blob, size_t bytes) {
    g_err.clear();
    if (!h || !host_blob) return fail(LBM_EINVAL, "NULL argument");
    size_t need = 0;
    lbm_state_bytes(h, &need);
    if (bytes < need) return fail(LBM_EINVAL, "blob of %zu bytes < %zu needed", bytes, need);
    StateHeader hd;
    const char* b = static_cast<const char*>(host_blob);
    std::memcpy(&hd, b, sizeof(hd));
    if (hd.magic != kStateMagic || hd.nx != h->prm.nx || hd.ny != h->prm.ny || hd.pitch != h->L.pitch)
        return fail(LBM_EINVAL, "state blob does not match this handle");
    if (hd.storage != h->prm.storage || hd.velocity != h->prm.velocity || hd.var_rho != h->phys.var_rho)
        return fail(LBM_EINVAL, "state blob has another storage, velocity or density mode than this handle");
    const size_t pb = h->L.plane * (size_t)lbm::pop_bytes_per_cell(h->prm.storage, h->prm.velocity == LBM_VELOCITY_SOLVED);
    const int cur = (int)(hd.steps & 1);  // the current state after k steps is buffer k mod 2
    LBM_CUDA(cudaMemcpyAsync(h->pops[cur], b + sizeof(hd), pb, cudaMemcpyHostToDevice, h->stream));
    LBM_CUDA(cudaMemcpyAsync(h->hist[cur], b + sizeof(hd) + pb, h->L.plane * sizeof(float2), cudaMemcpyHostToDevice,
                             h->stream));
    if (h->shist[0])
        LBM_CUDA(cudaMemcpyAsync(h->shist[cur], b + sizeof(hd) + pb + h->L.plane * sizeof(float2),
                                 h->L.plane * sizeof(float2), cudaMemcpyHostToDevice, h->stream));
    LBM_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    h->cur = cur;
    h->first = hd.first;
    h->steps = hd.steps;
    h->last_pipe_step = -2;
    h->initialized = 1;
    return LBM_OK;
}

int lbm_set_kernel(lbm_handle* h, int variant) {
    g_err.clear();
    if (!h) return fail(LBM_EINVAL, "handle is NULL");
    if (variant == LBM_KERNEL_AUTO) {
        int bps = 0, bps_pipe = 0;
        int rc = prepare_kernels(h->prm.storage, variant_of(h->prm, h->phys.var_rho != 0), &bps, &bps_pipe);
        if (rc) return rc;
        h->kernel = default_kernel(h->prm.storage, variant_of(h->prm, h->phys.var_rho != 0), bps_pipe);
        return LBM_OK;
    }
    if (variant != LBM_KERNEL_TILE && variant != LBM_KERNEL_PIPELINED) return fail(LBM_EINVAL, "bad kernel variant");
    if (variant == LBM_KERNEL_PIPELINED && h->pipe_ctas < 1)
        return fail(LBM_EINVAL, "the pipelined kernel does not fit on an SM for this storage mode");
    h->kernel = variant;
    return LBM_OK;
}

int lbm_get_kernel(const lbm_handle* h, int* variant) {
    g_err.clear();
    if (!h || !variant) return fail(LBM_EINVAL, "NULL argument");
    *variant = h->kernel;
    return LBM_OK;
}

int lbm_steps_taken(const lbm_handle* h, int64_t* steps) {
    g_err.clear();
    if (!h || !steps) return fail(LBM_EINVAL, "NULL argument");
    *steps = h->steps;
    return LBM_OK;
}

int lbm_destroy(lbm_handle* h) {
    g_err.clear();
    if (!h) return LBM_OK;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    delete h;
    if (e != cudaSuccess) return fail(LBM_ECUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e));
    return LBM_OK;
}

const char* lbm_last_error(void) { return g_err.c_str(); }

}  // extern "C"
