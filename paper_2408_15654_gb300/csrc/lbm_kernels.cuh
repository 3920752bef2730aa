// Device code of the fused three-population lattice-Boltzmann step (arXiv 2408.15654).
//
// Data layout in HBM (one population buffer; each plane ny + 4 rows x `pitch` cells, the grid
// inside a ghost frame, see kGX / kGY):
//   9 pair planes  (f_i, g_i), i = 0..8      phase field (Sec. 3.1) and surfactant (Sec. 3.2)
//   4 pair planes  (h_1, h_2) .. (h_7, h_8)   flow (Sec. 3.3; absent with a prescribed velocity)
// f_i and g_i stream along the same link, so they travel and collide together: one access per
// pair, and Blackwell's packed FP32x2 arithmetic runs both collisions at once.  h_0 is never
// stored: column 0 of M^-1 is e_0 and rows 1..8 of M do not see h_0, so h_0 feeds only itself
// (Sec. 3.3, Sec. 4).  The u history is one float2 plane (u_x, u_y) per buffer.
// A buffer holds the post-collision populations of the previous step at the cell that produced
// them; a step pulls q_i(x) = q*_i(x - c_i) ("pull" streaming), so it writes only its own cell
// (and the ghost-frame copies of it) and two buffers alternate.  Across a wall the missing link
// is the puller's own opposite slot, with the moving-wall term folded in (half-way bounce-back,
// Sec. 4), which the previous step also wrote into the wall's ghost row.
//
// Storage modes: FP32; FP16 or BF16 for all 26 populations; FP16 or BF16 for the 18 of f and g
// with h kept in FP32.  16-bit values are stored divided by their lattice weight, as scaled
// deviations from a reference:
//   (f_i, g_i):  ((f_i / w_i - phi_ref) S_f, (g_i / w_i) S_g)   phi_ref = (phiA + phiB)/2
//   h_i:         (h_i / w_i - 3 rho c_i.u(x_s)) S_h                x_s = the cell that stored the slot,
// where u(x_s) is the velocity that cell wrote to the u history in the same step.  Dividing by
// w_i makes the bulk equilibria (phi = phiA or phiB, psi = 0, u = 0) exactly representable, so
// the bulk does not drift by repeated rounding; taking away the first-order velocity part keeps
// the pressure (1e-5 against a velocity part of 1e-3) above the 16-bit rounding.  The step
// stores with stochastic rounding (Blackwell's cvt.rs, random bits from a hash of cell and step):
// in a steady flow a cell rounds nearly the same values every step, and round-to-nearest would
// then add the same error every step.  All arithmetic stays in FP32; f and g are collided as the
// deviations f_i - w_i phi_ref that the storage holds (the reference enters only the even
// moments, through phi - phi_ref), and the stored pair values are updated in place by the
// scaled increment of the collision rather than decoded and re-encoded (see kdec / kenc).
//
// Velocity order (the columns of the printed moment matrix M, Sec. 4):
//   0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1)
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbm {

__host__ __device__ constexpr int cx(int i) { return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0); }
__host__ __device__ constexpr int cy(int i) { return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0); }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5); }
__host__ __device__ constexpr float wgt(int i) { return i == 0 ? 4.f / 9.f : (i <= 4 ? 1.f / 9.f : 1.f / 36.f); }

static_assert(opp(1) == 3 && opp(3) == 1 && opp(2) == 4 && opp(4) == 2, "axis opposites");
static_assert(opp(5) == 7 && opp(7) == 5 && opp(6) == 8 && opp(8) == 6, "diagonal opposites");

constexpr int kPairs = 9;       // (f_i, g_i) planes
constexpr int kHPlanes = 8;     // h_1..h_8 planes

enum Storage { kFP32 = 0, kFP16 = 1, kBF16 = 2, kFP16FG = 3, kBF16FG = 4 };

// Storage traits: element types, compile-time scales, and the x origin / width of the h boxes in
// (h_i, h_i+1) pairs (TMA x coordinates must be multiples of 16 bytes: 2 pairs of 8 bytes, 4 of
// 4 bytes; box columns x0 - H_X0 + kGX onwards).
template <int ST> struct Traits;
template <> struct Traits<kFP32> {
    using P = float2;
    using H = float;
    static constexpr bool kPair16 = false, kH16 = false;
    static constexpr int H_X0 = 2, H_BW = 36;  // in (h_i, h_i+1) pairs
    static constexpr float SF = 1.f, SG = 1.f, SH = 1.f;
};
template <> struct Traits<kFP16> {
    using P = __half2;
    using H = __half;
    static constexpr bool kPair16 = true, kH16 = true;
    static constexpr int H_X0 = 4, H_BW = 40;  // in (h_i, h_i+1) pairs
    static constexpr float SF = 1.f, SG = 256.f, SH = 4096.f;  // keep the deviations normal in FP16
};
template <> struct Traits<kBF16> {
    using P = __nv_bfloat162;
    using H = __nv_bfloat16;
    static constexpr bool kPair16 = true, kH16 = true;
    static constexpr int H_X0 = 4, H_BW = 40;  // in (h_i, h_i+1) pairs
    static constexpr float SF = 1.f, SG = 1.f, SH = 1.f;        // BF16 has the FP32 exponent range
};
template <> struct Traits<kFP16FG> {
    using P = __half2;
    using H = float;
    static constexpr bool kPair16 = true, kH16 = false;
    static constexpr int H_X0 = 2, H_BW = 36;  // in (h_i, h_i+1) pairs
    static constexpr float SF = 1.f, SG = 256.f, SH = 1.f;
};
template <> struct Traits<kBF16FG> {
    using P = __nv_bfloat162;
    using H = float;
    static constexpr bool kPair16 = true, kH16 = false;
    static constexpr int H_X0 = 2, H_BW = 36;  // in (h_i, h_i+1) pairs
    static constexpr float SF = 1.f, SG = 1.f, SH = 1.f;
};

// Bytes of one population buffer per cell: 9 (f, g) pairs + 8 h values (no h when the velocity
// is prescribed).
__host__ __device__ constexpr int pop_bytes_per_cell(int st, bool flow = true) {
    return !flow ? (st == kFP32 ? 9 * 8 : 9 * 4)
                 : (st == kFP32 ? 9 * 8 + 8 * 4 : (st == kFP16 || st == kBF16 ? 9 * 4 + 8 * 2 : 9 * 4 + 8 * 4));
}
__host__ __device__ constexpr bool pair_is_16bit(int st) { return st != kFP32; }
__host__ __device__ constexpr bool h_is_16bit(int st) { return st == kFP16 || st == kBF16; }

// Ghost frame of every plane: cell (x, y) sits at row y + kGY, column x + kGX of a plane of
// (ny + 2 kGY) rows x pitch columns.  Columns -2, -1, nx, nx + 1 and, for periodic y, rows -2,
// -1, ny, ny + 1 hold the periodic images of the cells they stand for; with walls, rows -1 and
// ny hold, in the planes of the links that cross the wall, the bounce-back value for the pull
// (the puller's own post-collision opposite slot).  Every value a pull or the one-cell ring of a
// tile reads is then at its plain position, and the TMA boxes need no patching.  kGX = 8 keeps
// the x coordinate of every box a multiple of 16 bytes (boxes start 4 or 8 cells left of a tile).
constexpr int kGX = 8, kGY = 2;

// Index, in h values, of link i's slot at cell k of a buffer's h planes (plane stride `plane`
// cells).  h is stored as pairs (h_2j+1, h_2j+2) in plane j, link 2j+1 first, so that a cell's
// eight values leave in four stores (32-bit for 16-bit h, 64-bit for FP32 h) and the flow
// collision's FP32x2 pairs go out as they are.
__host__ __device__ __forceinline__ long long h_index(int i, long long k, long long plane) {
    return (((long long)((i - 1) >> 1) * plane + k) << 1) + ((i - 1) & 1);
}
// First row of h box j relative to the tile's first row: the lower source row of its links.
__host__ __device__ constexpr int h_row0(int j) {
    return -(cy(2 * j + 1) > cy(2 * j + 2) ? cy(2 * j + 1) : cy(2 * j + 2));
}

// Physical constants in FP32, precomputed on the host from lbm_params.  16-byte aligned and sized
// so that the batched kernel can stage a lattice's copy with one bulk copy.
struct alignas(16) Phys {
    int nx, ny, pitch, pad0;
    long long plane;          // cells per plane ((ny + 2 kGY) * pitch)
    long long org;            // index of cell (0, 0): kGY * pitch + kGX
    float phiA, phiB, inv_dphi;
    float cA;                 // 4 / (W dphi):  A = cA (phiA - phi)(phi - phiB), B = cA psi (phiA + phiB - 2 phi)
    float cap_k, c16W, W;     // capillary: cap_k sigma [c16W (phiA-phi)(phi-phiB)(phiA+phiB-2phi) - W lap phi]
    float mar_k;              // Marangoni: mar_k [|grad phi|^2 grad sigma - (grad sigma . grad phi) grad phi]
    float sigma0, E0;
    float rho, inv_rho;
    float muB, dmu;           // mu(phi) = muB + (phi - phiB)/dphi * dmu
    float s2h;                // 1/s2^h when the viscosity is uniform (dmu == 0)
    float gx, gy;
    float nS1[2], nS2[2], nS3[2], nS4[2];  // -s_k of (f, g) for k = 1..4
    float K1[2], K3[2];                    // 1 - s_k/2 of (f, g) for k = 1, 3
    float s1h, s3h, s4h, k1h, k3h;         // flow rates and 1 - s/2
    float k2h, s4h_eff, k4h;               // with uniform viscosity: 1 - s2/2, s4, 1 - s4/2
    int tie_s4h;              // 1: s4^h = s2^h
    float u_top, u_bot;
    float n_eps2;             // n_eps^2
    // 16-bit storage (unused for FP32)
    float phi_ref;            // (phiA + phiB) / 2
    float kh_axis, kh_diag;   // 3 w_i rho for axis and diagonal links (h decode)
    float kh3;                // 3 rho (h encode, before the scale)
    // density ratio != 1 (Sec. 2.3): rho = rhoB + (phi - phiB) drho, S = sfac [grad phi - A n]
    int var_rho;              // 1: rhoA != rhoB (rho, inv_rho above unused by its kernels)
    float rhoB, drho, sfac;   // drho = (rhoA - rhoB) / dphi; sfac = M_phi drho
};

enum Mode { kStep = 0, kMoments = 1 };

// Flow variant of a kernel (template argument FLOW): the velocity prescribed (no h), solved by h
// with a uniform density, or solved with a density ratio (mass flux S and the grad rho terms).
enum Flow { kFlowPrescribed = 0, kFlowUniform = 1, kFlowVarRho = 2 };

// Tile geometry.  A CTA of NT threads owns a TX x TY tile, one cell per thread.  TMA stages:
//   pair plane i: box of BW x BH pairs,    row r, col c <-> (x0 - 4 + c, y0 - 1 - cy(i) + r)
//   h plane i:    box of H_BW x TY values, row r, col c <-> (x0 - H_X0 + c, y0 - cy(i) + r)
//   u history:    box of TX x TY, or BW x BH (one-cell ring) when h is 16-bit, float2
// so extended-tile cell (ex, ey) (global (x0 - 1 + ex, y0 - 1 + ey)) pulls pair i from
// [ey][ex + 3 - cx(i)], the own cell (tx, ty) pulls h_i from [ty][tx + H_X0 - cx(i)], and the
// own cell's unshifted post-collision pair i sits at [ty + 1 + cy(i)][tx + 4].
constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int BW = TX + 8, BH = TY + 2;
constexpr int FG_BOX = BW * BH;            // pairs per pair-plane box
constexpr int EX = TX + 2, EY = TY + 2, NE = EX * EY;
constexpr int NRING = 2 * EX + 2 * TY;
constexpr unsigned kSuspendNs = 200000;    // sleep hint of one wait attempt
constexpr unsigned kWaitLimit = 5000;      // attempts: the wait ends within ~1 s
constexpr unsigned kStatusUnstable = 1u, kStatusTimeout = 2u;
static_assert(NRING <= NT, "one thread per ring cell");

__host__ __device__ constexpr int round128(int b) { return (b + 127) / 128 * 128; }

// Buffers of one step of one lattice.
struct TileIO {
    const void* __restrict__ src;
    void* __restrict__ dst;
    const float2* __restrict__ hist_src;  // (u_x, u_y) of the previous step
    float2* __restrict__ hist_dst;        // (u_x, u_y) of this step (the other history buffer)
    const float2* __restrict__ shist_src; // mass flux (S_x, S_y) of the previous step (density ratio != 1)
    float2* __restrict__ shist_dst;       // (S_x, S_y) of this step
    unsigned* __restrict__ status;
    double* __restrict__ out[5];  // kMoments: phi, psi, ux, uy, P (dense ny x nx), may be null
    unsigned seed;                // per-step salt of the stochastic rounding
    int first;                    // 1 on the first step after initialisation (zero d/dt terms)
};

// Shared-memory layout (bytes) of one tile for storage mode ST.
template <int ST> struct Smem {
    using T = Traits<ST>;
    static constexpr bool kHalo = T::kH16;  // the 16-bit h decode needs the source cell's u
    static constexpr int FG_SLOT = round128(FG_BOX * (int)sizeof(typename T::P));
    // h boxes: one per plane of pairs (h_2j+1, h_2j+2), spanning the rows of both links (TY + 1)
    static constexpr int H_SLOTS = kHPlanes / 2;
    static constexpr int H_ES = 2 * (int)sizeof(typename T::H);
    static constexpr int H_BH = TY + 1;
    static constexpr int H_BOX = T::H_BW * H_BH;
    static constexpr int H_SLOT = round128(H_BOX * H_ES);
    static constexpr int HIST_W = kHalo ? BW : TX, HIST_H = kHalo ? BH : TY;
    static constexpr int HIST_BYTES = HIST_W * HIST_H * 8;
    static constexpr int FG = 0;
    static constexpr int H = FG + kPairs * FG_SLOT;
    static constexpr int HIST = H + H_SLOTS * H_SLOT;
    static constexpr int PP = HIST + round128(HIST_BYTES);
    static constexpr int BAR = PP + NE * 8;
    static constexpr int BYTES = BAR + 16;
    // batched kernel: the lattice's constants
    static constexpr int PHYS = BYTES;
    static constexpr int BYTES_BATCH = PHYS + (int)((sizeof(Phys) + 15) / 16 * 16);
    // warp-specialised persistent kernel: two stages of the TMA boxes ([0, PP) each), two
    // (phi, psi) tiles (alternating with the tile count), a full and an empty mbarrier per stage,
    // the tile origin (x0, y0) of each stage
    static constexpr int STAGE = PP;
    static constexpr int PIPE_PP = 2 * STAGE;
    static constexpr int PIPE_BAR = PIPE_PP + 2 * NE * 8;
    static constexpr int PIPE_SLOT = PIPE_BAR + 32;
    // 16-bit pairs with FP32 h (FP16_FG, BF16_FG): per compute warp a staging row of its cells'
    // post-collision pairs, [plane][TX] as the bulk tensor store reads it; h goes out with plain
    // stores (staging it too would cost the third CTA per SM).  The all-16-bit modes keep plain
    // stores: with the pairs and h staged their step issued more instructions, not fewer.
    static constexpr bool kTS = T::kPair16 && !T::kH16;
    static constexpr int STG_W = kPairs * TX * (int)sizeof(typename T::P);
    static constexpr int PIPE_STG = round128(PIPE_SLOT + 16);
    static constexpr int BYTES_PIPE = kTS ? PIPE_STG + TY * STG_W : PIPE_SLOT + 16;
    static_assert(STG_W % 128 == 0, "staging rows keep 128-byte alignment");
    // warp-specialised batch kernel: the same buffers and barriers, a 4-word slot per buffer
    // (x0, y0, lattice, current population buffer) and per buffer the lattice's constants
    static constexpr int PHYS_BYTES = (int)sizeof(Phys);
    static constexpr int BWS_SLOT = PIPE_BAR + 32;
    static constexpr int BWS_PHYS = BWS_SLOT + 32;
    static constexpr int BYTES_BWS = BWS_PHYS + 2 * PHYS_BYTES;
    static constexpr unsigned TX_BYTES =
        (unsigned)(kPairs * FG_BOX * sizeof(typename T::P) + H_SLOTS * H_BOX * H_ES + HIST_BYTES);
    static constexpr unsigned TX_BYTES_NOH = (unsigned)(kPairs * FG_BOX * sizeof(typename T::P) + HIST_BYTES);
};


struct StepArgs {
    CUtensorMap tm_fg;            // {nx, ny, 9} pairs, box {BW, BH, 1}
    CUtensorMap tm_h;             // {nx, ny, 4} h pairs, box {H_BW, TY + 1, 1}
    CUtensorMap tm_hist;          // {nx, ny, 1} float2, box {TX, TY, 1} or {BW, BH, 1}
    CUtensorMap tm_st_fg;         // destination pairs {kGX + nx, kGY + ny, 9}, box {TX, 1, 9} (16-bit pairs, FP32 h)
    Phys p;
    TileIO io;
    unsigned* tile_ctr;           // pipelined kernel: tile counter of this launch (zero at start)
    unsigned* tile_ctr_next;      // and of the next launch, zeroed by this one
};

// Salt of the stochastic rounding of step number `steps` (steps taken since initialisation), a
// splitmix64 finaliser: the same on host and device, so any launch path gives the same bits.
__host__ __device__ inline unsigned step_seed(long long steps) {
    unsigned long long z = (unsigned long long)steps * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;
    return (unsigned)(z ^ (z >> 29));
}

__device__ __forceinline__ int wrapg(int a, int n) {
    const int r = a % n;
    return r < 0 ? r + n : r;
}

// packed FP32x2 arithmetic (one instruction for both lanes)
__device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// explicitly rounded scalar arithmetic (never contracted): the density-ratio terms are written
// with these, so that every kernel instantiating them rounds in the one order written here
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// ---- storage conversions ----
__device__ __forceinline__ float2 raw2(float2 v) { return v; }
__device__ __forceinline__ float2 raw2(__half2 v) { return __half22float2(v); }
__device__ __forceinline__ float2 raw2(__nv_bfloat162 v) { return __bfloat1622float2(v); }
__device__ __forceinline__ float raw1(float v) { return v; }
__device__ __forceinline__ float raw1(__half v) { return __half2float(v); }
__device__ __forceinline__ float raw1(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ T pack2(float2 v);
template <> __device__ __forceinline__ float2 pack2<float2>(float2 v) { return v; }
template <> __device__ __forceinline__ __half2 pack2<__half2>(float2 v) { return __float22half2_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat162 pack2<__nv_bfloat162>(float2 v) { return __float22bfloat162_rn(v); }
template <typename T> __device__ __forceinline__ T pack1(float v);
template <> __device__ __forceinline__ float pack1<float>(float v) { return v; }
template <> __device__ __forceinline__ __half pack1<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 pack1<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
// a 16-bit pattern as a storage value
template <typename T> __device__ __forceinline__ T bits_to(uint32_t b);
template <> __device__ __forceinline__ __half bits_to<__half>(uint32_t b) { return __ushort_as_half((unsigned short)b); }
template <> __device__ __forceinline__ __nv_bfloat16 bits_to<__nv_bfloat16>(uint32_t b) {
    return __ushort_as_bfloat16((unsigned short)b);
}
template <> __device__ __forceinline__ float bits_to<float>(uint32_t b) { return __uint_as_float(b); }

// 16-bit storage holds r_i = (f_i / w_i - phi_ref) S_f and g_i / w_i S_g.  The decode constant
// w_i / S is not a binary fraction (w_i = 4/9, 1/9, 1/36), so the stored state is never decoded
// and re-encoded: the step computes its moments from r (each weight class summed raw and scaled
// once; the constant's ~1e-8 relative error then only touches the physics) and writes
// r* = r + (S / w_i) dq_i, the increment of the collision scaled by the exact constant S / w_i.
// A resting bulk, whose increments are below half an FP32 ulp of r, keeps its stored values
// exactly, and the totals of phi and psi carry no coherent decode error.
__host__ __device__ constexpr double wgt_d(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }
// decode constant w_i / S of link i as one (f, g) pair
template <int ST, int I> __device__ __forceinline__ float2 kdec() {
    using T = Traits<ST>;
    return make_float2((float)(wgt_d(I) / T::SF), (float)(wgt_d(I) / T::SG));
}
// c S / w_i of link i (exact in FP32: 1 / w_i is 9/4, 9 or 36 and S a power of two)
template <int ST, int I> __device__ __forceinline__ float2 kenc(double c) {
    using T = Traits<ST>;
    return make_float2((float)(c * T::SF / wgt_d(I)), (float)(c * T::SG / wgt_d(I)));
}
// (phi, psi) of a cell from its nine stored pairs, converted to FP32 (r): FP32 storage sums the
// values; 16-bit storage sums the raw values of each weight class and scales each class sum once
template <int ST> __device__ __forceinline__ float2 pair_sum(const float2 (&r)[9], float2 ref) {
    if constexpr (!Traits<ST>::kPair16) {
        float2 s = ref;
#pragma unroll
        for (int i = 0; i < 9; ++i) s = add2(s, r[i]);
        return s;
    } else {
        const float2 ax = add2(add2(r[1], r[3]), add2(r[2], r[4]));
        const float2 dg = add2(add2(r[5], r[7]), add2(r[6], r[8]));
        return fma2(dg, kdec<ST, 5>(), fma2(ax, kdec<ST, 1>(), fma2(r[0], kdec<ST, 0>(), ref)));
    }
}
// 3 w_i rho c_i.u: the first-order velocity part of h_eq removed before 16-bit storage
template <int I> __device__ __forceinline__ float h_vel(float2 u, const Phys& p) {
    const float k = I <= 4 ? p.kh_axis : p.kh_diag;
    return k * ((float)cx(I) * u.x + (float)cy(I) * u.y);
}

// Two FP32 values to a 16-bit pair with stochastic rounding (lo in the low half).
template <typename T> __device__ __forceinline__ uint32_t cvt_rs2(float lo, float hi, uint32_t rbits) {
    uint32_t out;
    if constexpr (__is_same(T, __half2))
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(out) : "f"(hi), "f"(lo), "r"(rbits));
    else
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(out) : "f"(hi), "f"(lo), "r"(rbits));
    return out;
}
// Per-cell random word for the stochastic rounding of one step (multiply-xorshift hash).
__device__ __forceinline__ uint32_t cell_key(uint32_t cell, uint32_t seed) {
    uint32_t h = cell * 0x9E3779B1u ^ seed;
    h ^= h >> 16;
    h *= 0x7FEB352Du;
    h ^= h >> 15;
    h *= 0x846CA68Bu;
    h ^= h >> 16;
    return h;
}
// Random bits of conversion k of a cell: a rotation of the cell's word.  Every rounding stays
// unbiased; conversions of one cell share bits, which correlates their errors but adds no bias.
__device__ __forceinline__ uint32_t rbits_of(uint32_t key, int k) { return __funnelshift_l(key, key, 5 * k + 1); }
// a scaled (f_i, g_i) pair r* to stochastically rounded 16-bit storage
template <int ST, int I> __device__ __forceinline__ typename Traits<ST>::P enc_pair_rs(float2 v, uint32_t key) {
    using T = Traits<ST>;
    const uint32_t bits = cvt_rs2<typename T::P>(v.x, v.y, rbits_of(key, I));
    return *reinterpret_cast<const typename T::P*>(&bits);
}

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}
__device__ __forceinline__ void mbar_init(unsigned long long* m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
// One bounded wait attempt: the thread may sleep until the phase completes or kSuspendNs pass.
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2, %3;\n selp.u32 %0, 1, 0, P1;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity), "n"(kSuspendNs)
        : "memory");
    return ok != 0;
}
// Wait for a phase of the mbarrier with an iteration limit; false if the limit was reached.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* m, uint32_t parity) {
    for (unsigned it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(m, parity)) return true;
    return false;
}
// Raise the transaction count of the current phase without arriving (for a copy issued before the
// arrival that completes the phase's expectations).
__device__ __forceinline__ void mbar_expect_tx_only(unsigned long long* m, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
// Untiled bulk copy global -> shared on an mbarrier (both addresses 16-byte aligned, size a
// multiple of 16 bytes).
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(m))
        : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* m) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(m)) : "memory");
}
// Named barrier 1 of the NT compute threads of a warp-specialised CTA (its copy warp never takes
// part); the OR form also tells every thread whether any of them passed true.
__device__ __forceinline__ void compute_sync() { asm volatile("bar.sync 1, %0;\n" ::"n"(NT) : "memory"); }
__device__ __forceinline__ bool compute_sync_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 1, %2, q;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(NT)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            unsigned long long* m) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(m))
        : "memory");
}
// Bulk tensor store shared -> global of one box (source 128-byte aligned); the writes that fall
// outside the tensor map's extents are dropped.  The issuing thread tracks it in its bulk group.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* tm, const void* src, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];\n" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// The issuing thread's bulk stores have read their shared-memory source (it may be rewritten).
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
// The issuing thread's bulk stores are complete.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// Generic-proxy writes to shared memory made visible to a later bulk copy (async proxy).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Moment-space MRT collision of the (f, g) pair, applied as an increment so that FP32 rounding
// stays at the scale of the departure from equilibrium (in a uniform bulk nothing changes):
//   m = M q;  dm_k = -s_k (m_k - m_eq_k) + (1 - s_k/2) m_src_k;  q* = q + M^-1 dm.
// For a scalar s (phi or psi) the equilibrium w_i s (1 + c_i.u/cs2) has moments
// (s, s ux, s uy, s/3, s/3, 0, s ux/3, s uy/3, s/9); the source w_i c_i.V has moments
// (0, cs2 Vx, cs2 Vy, 0, 0, 0, Vx/9, Vy/9, 0) with cs2 V = (vx, vy).  dm_0 = 0.
// q may hold deviations q_i - w_i r (r per lane): the odd moments are unchanged, the even ones
// drop r times (1, 1/3, 1/3, 1/9), so they are compared with sr = s - r.
// nS_k = -s_k and K_k = 1 - s_k/2 per lane (f, g).
// FP32 storage: q holds the values and becomes q*.  16-bit storage: q holds the raw stored values r
// and becomes r* = r + (S / w_i) (M^-1 dm)_i (the moments come from r, each weight class scaled by
// its decode constant once).
template <int ST>
__device__ __forceinline__ void collide_pair(float2 q[9], float2 s, float2 sr, float ux, float uy, float2 vx,
                                             float2 vy, float2 nS1, float2 nS2, float2 nS3, float2 nS4, float2 K1,
                                             float2 K3) {
    constexpr bool raw = Traits<ST>::kPair16;
    const float2 third = bc(1.f / 3.f);
    const float2 a = add2(q[5], q[7]), b = add2(q[6], q[8]), c = sub2(q[5], q[7]), d = sub2(q[6], q[8]);
    float2 m1, m2, m3, m4, m5, m6, m7, m8;
    if constexpr (!raw) {
        m5 = sub2(a, b), m8 = add2(a, b), m6 = sub2(c, d), m7 = add2(c, d);
        m1 = add2(sub2(q[1], q[3]), m6), m2 = add2(sub2(q[2], q[4]), m7);
        m3 = add2(add2(q[1], q[3]), m8), m4 = add2(add2(q[2], q[4]), m8);
    } else {
        const float2 kax = kdec<ST, 1>(), kdg = kdec<ST, 5>();
        m5 = mul2(kdg, sub2(a, b)), m8 = mul2(kdg, add2(a, b)), m6 = mul2(kdg, sub2(c, d)), m7 = mul2(kdg, add2(c, d));
        m1 = fma2(kax, sub2(q[1], q[3]), m6), m2 = fma2(kax, sub2(q[2], q[4]), m7);
        m3 = fma2(kax, add2(q[1], q[3]), m8), m4 = fma2(kax, add2(q[2], q[4]), m8);
    }
    const float2 su = mul2(s, bc(ux)), sv = mul2(s, bc(uy)), s3 = mul2(sr, third);
    const float2 d1 = fma2(nS1, sub2(m1, su), mul2(K1, vx));
    const float2 d2 = fma2(nS1, sub2(m2, sv), mul2(K1, vy));
    const float2 d3 = mul2(nS2, sub2(m3, s3));
    const float2 d4 = mul2(nS2, sub2(m4, s3));
    const float2 d5 = mul2(nS2, m5);
    const float2 d6 = fma2(nS3, fma2(su, bc(-1.f / 3.f), m6), mul2(K3, mul2(vx, third)));
    const float2 d7 = fma2(nS3, fma2(sv, bc(-1.f / 3.f), m7), mul2(K3, mul2(vy, third)));
    const float2 d8 = mul2(nS4, fma2(sr, bc(-1.f / 9.f), m8));
    const float2 A = sub2(d1, d6), B = sub2(d3, d8), C = sub2(d2, d7), D = sub2(d4, d8);
    const float2 E = add2(d8, d5), F = sub2(d8, d5), G = add2(d6, d7), H = sub2(d7, d6);
    if constexpr (!raw) {
        const float2 half = bc(0.5f), quarter = bc(0.25f);
        q[0] = add2(q[0], sub2(sub2(d8, d3), d4));
        q[1] = fma2(half, add2(A, B), q[1]);
        q[3] = fma2(half, sub2(B, A), q[3]);
        q[2] = fma2(half, add2(C, D), q[2]);
        q[4] = fma2(half, sub2(D, C), q[4]);
        q[5] = fma2(quarter, add2(E, G), q[5]);
        q[7] = fma2(quarter, sub2(E, G), q[7]);
        q[6] = fma2(quarter, add2(F, H), q[6]);
        q[8] = fma2(quarter, sub2(F, H), q[8]);
    } else {
        q[0] = fma2(kenc<ST, 0>(1.0), sub2(sub2(d8, d3), d4), q[0]);
        q[1] = fma2(kenc<ST, 1>(0.5), add2(A, B), q[1]);
        q[3] = fma2(kenc<ST, 3>(0.5), sub2(B, A), q[3]);
        q[2] = fma2(kenc<ST, 2>(0.5), add2(C, D), q[2]);
        q[4] = fma2(kenc<ST, 4>(0.5), sub2(D, C), q[4]);
        q[5] = fma2(kenc<ST, 5>(0.25), add2(E, G), q[5]);
        q[7] = fma2(kenc<ST, 7>(0.25), sub2(E, G), q[7]);
        q[6] = fma2(kenc<ST, 6>(0.25), add2(F, H), q[6]);
        q[8] = fma2(kenc<ST, 8>(0.25), sub2(F, H), q[8]);
    }
}

template <int ST, int I>
__device__ __forceinline__ float load_h(const unsigned char* sm, const float2* Hist, const Phys& p, int tx, int ty,
                                        bool bb, float2 uown) {
    using T = Traits<ST>;
    using S = Smem<ST>;
    constexpr int j = (I - 1) / 2;                  // the box (pair plane) holding link I
    constexpr int dr = -cy(I) - h_row0(j);          // the source row's offset inside it
    const int e = (ty + dr) * T::H_BW + tx + T::H_X0 - cx(I);
    const typename T::H* box = reinterpret_cast<const typename T::H*>(sm + S::H + j * S::H_SLOT);
    const typename T::H v = box[2 * e + ((I - 1) & 1)];
    if constexpr (!T::kH16) {
        return v;
    } else {
        // the slot was stored with the first-order velocity part of the cell that stored it:
        // the source cell x - c_i, or across a wall the own cell (whose opposite slot it is)
        const float2 us = bb ? make_float2(-uown.x, -uown.y) : Hist[(ty + 1 - cy(I)) * BW + tx + 4 - cx(I)];
        // one FP32 decode constant: h has no conserved zeroth moment, and the collision relaxes the
        // constant's ~1e-8 relative error away every step
        constexpr float dh = (float)(wgt_d(I) / T::SH);
        return fmaf(raw1(v), dh, h_vel<I>(us, p));
    }
}

// Stage the boxes of tile (x0, y0) with TMA on one mbarrier (called by one thread).
template <int ST, int FLOW>
__device__ __forceinline__ void issue_tile_loads(unsigned char* sm, const CUtensorMap* tm_fg, const CUtensorMap* tm_h,
                                                 const CUtensorMap* tm_hist, int x0, int y0, unsigned long long* mbar) {
    using T = Traits<ST>;
    using S = Smem<ST>;
    mbar_expect_tx(mbar, FLOW ? S::TX_BYTES : S::TX_BYTES_NOH);
#pragma unroll
    for (int i = 0; i < kPairs; ++i)
        tma_load_3d(sm + S::FG + i * S::FG_SLOT, tm_fg, x0 - 4 + kGX, y0 - 1 - cy(i) + kGY, i, mbar);
    if constexpr (FLOW) {
#pragma unroll
        for (int j = 0; j < S::H_SLOTS; ++j)
            tma_load_3d(sm + S::H + j * S::H_SLOT, tm_h, x0 - T::H_X0 + kGX, y0 + h_row0(j) + kGY, j, mbar);
    }
    if constexpr (S::kHalo) tma_load_3d(sm + S::HIST, tm_hist, x0 - 4 + kGX, y0 - 1 + kGY, 0, mbar);
    else tma_load_3d(sm + S::HIST, tm_hist, x0 + kGX, y0 + kGY, 0, mbar);
}

// One fused step (kStep) or the macroscopic fields of the current level (kMoments) for one tile,
// after one thread has issued the tile's TMA loads into `stage` on `mbar`, whose phase of this
// tile has parity `parity`; PP holds the tile's (phi, psi).  Returns true (uniformly) if a copy
// did not arrive within its bounded wait (nothing stored).  The pulled (f, g) of the tile and of a one-cell ring give (phi, psi) for the
// 9-point stencils; the same boxes hold the own cell's unshifted post-collision values, whose sums
// are phi and psi of the previous level (m*_0 = phi exactly, Sec. 3.1), so only u of the
// previous level is stored.
// WS: called by the compute warps of a warp-specialised CTA, which synchronise among themselves
// with named barrier 1 only (the copy warp has staged the tile and waits on its own barriers).
template <int ST, bool WALLS, bool LANGMUIR, int MODE, int FLOW, bool WS = false, bool TS = false>
__device__ __forceinline__ bool step_tile(const Phys& p, const TileIO& io, unsigned char* sm, float2* PP,
                                          unsigned long long* mbar, uint32_t parity, int x0, int y0,
                                          unsigned char* stg = nullptr) {
    using T = Traits<ST>;
    using S = Smem<ST>;
    using P = typename T::P;
    const P* FG = reinterpret_cast<const P*>(sm + S::FG);
    const float2* Hist = reinterpret_cast<const float2*>(sm + S::HIST);
    const int t = threadIdx.x;
    if constexpr (!WS) __syncthreads();
    bool abort = !mbar_wait_bounded(mbar, parity);

    const int tx = t % TX, ty = t / TX;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = (x < p.nx) && (y < p.ny);
    // mass flux of the previous step (density ratio != 1 only; the own cell's, read early so that
    // its latency overlaps the stencil work)
    float2 Sp = make_float2(0.f, 0.f);
    if (FLOW == kFlowVarRho && !io.first && active) Sp = io.shist_src[p.org + (long long)y * p.pitch + x];
    // (phi, psi) references of the stored deviations (zero for FP32 storage)
    const float2 ref = T::kPair16 ? make_float2(p.phi_ref, 0.f) : make_float2(0.f, 0.f);

    // ---- (phi, psi) of the extended tile: the own cell (pulled pairs kept for the collision)
    //      and the ring; cells beyond a wall take the value of the adjacent fluid row ----
    const int eo = (ty + 1) * EX + (tx + 1);
    constexpr int SLOT = S::FG_SLOT / (int)sizeof(P);
    float2 q[9];
    {
        int row = ty + 1;
        if (WALLS && y >= p.ny) row = p.ny - y0;
        const P* base = FG + row * BW + tx + 4;
#pragma unroll
        for (int i = 0; i < 9; ++i) q[i] = raw2(base[i * SLOT - cx(i)]);  // the values, or the raw 16-bit deviations
        PP[eo] = pair_sum<ST>(q, ref);
    }
    if (t < NRING) {
        int ex, ey;
        if (t < EX) { ex = t; ey = 0; }
        else if (t < 2 * EX) { ex = t - EX; ey = EY - 1; }
        else if (t < 2 * EX + TY) { ex = 0; ey = 1 + t - 2 * EX; }
        else { ex = EX - 1; ey = 1 + t - 2 * EX - TY; }
        int row = ey;
        if (WALLS) {
            const int gy = y0 - 1 + ey;
            if (gy < 0) row = 1 - y0;
            else if (gy >= p.ny) row = p.ny - y0;
        }
        const P* base = FG + row * BW + ex + 3;
        float2 r[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) r[i] = raw2(base[i * SLOT - cx(i)]);
        PP[ey * EX + ex] = pair_sum<ST>(r, ref);
    }
    if (WS ? compute_sync_or(abort) : __syncthreads_or(abort)) {
        // a staging copy did not arrive in time: report it, wait (bounded) for it, store nothing
        if (t == 0) {
            atomicOr(io.status, kStatusTimeout);
            mbar_wait_bounded(mbar, parity);
        }
        if constexpr (WS) compute_sync();
        else __syncthreads();
        return true;
    }
    if (!active) return false;

    const float2 pp = PP[eo];          // (phi, psi)
    const float phi = pp.x, psi = pp.y;

    // isotropic stencils of (phi, psi) at once:
    //   d_a = (1/cs2) sum w_i c_ia q(x+c_i);  lap = (2/cs2) sum_{i>0} w_i (q_i - q)
    float2 gX, gY, lap2;
    {
        const float2 E = PP[eo + 1], Wn = PP[eo - 1], N = PP[eo + EX], S_ = PP[eo - EX];
        const float2 NE_ = PP[eo + EX + 1], NW = PP[eo + EX - 1], SE = PP[eo - EX + 1], SW = PP[eo - EX - 1];
        const float2 third = bc(1.f / 3.f), twelfth = bc(1.f / 12.f);
        gX = fma2(sub2(add2(NE_, SE), add2(NW, SW)), twelfth, mul2(sub2(E, Wn), third));
        gY = fma2(sub2(add2(NE_, NW), add2(SE, SW)), twelfth, mul2(sub2(N, S_), third));
        const float2 axis = add2(add2(E, Wn), add2(N, S_)), diag = add2(add2(NE_, NW), add2(SE, SW));
        lap2 = mul2(fma2(bc(4.f), axis, fma2(bc(-20.f), pp, diag)), bc(1.f / 6.f));
    }
    const float gpx = gX.x, gpy = gY.x, gsx = gX.y, gsy = gY.y, lap = lap2.x;

    // interface normal and the delta-function terms (Sec. 2.2, Secs. 3.1-3.2)
    const float g2 = gpx * gpx + gpy * gpy;
    float nx_ = 0.f, ny_ = 0.f;
    if (g2 > p.n_eps2) {
        const float r = rsqrtf(g2);
        nx_ = gpx * r;
        ny_ = gpy * r;
    }
    const float dA = p.phiA - phi, dB = phi - p.phiB, sym = p.phiA + p.phiB - 2.f * phi;
    const float Aterm = p.cA * dA * dB;
    const float Bterm = p.cA * psi * sym;

    // EOS and surface-tension force: capillary + Marangoni, expanded form (Sec. 2.3); F_b = rho g
    float sigma, dsig;
    if (LANGMUIR) {
        const float om = 1.f - psi;
        sigma = p.sigma0 * (1.f + p.E0 * __logf(om));
        dsig = __fdividef(-p.sigma0 * p.E0, om);
    } else {
        sigma = p.sigma0 * (1.f - p.E0 * psi);
        dsig = -p.sigma0 * p.E0;
    }
    // density (Sec. 2.3): rho(phi), its gradient by the chain rule, and the mass flux S
    constexpr bool var = FLOW == kFlowVarRho;
    const float rho_v = var ? rfma(rsub(phi, p.phiB), p.drho, p.rhoB) : 0.f;  // local density (ratio != 1)
    float grx = 0.f, gry = 0.f, Sx = 0.f, Sy = 0.f;
    if (var) {
        grx = rmul(p.drho, gpx);
        gry = rmul(p.drho, gpy);
        Sx = rmul(p.sfac, rfma(-Aterm, nx_, gpx));
        Sy = rmul(p.sfac, rfma(-Aterm, ny_, gpy));
    }
    const float gsgx = dsig * gsx, gsgy = dsig * gsy;
    const float cap = p.cap_k * sigma * (p.c16W * dA * dB * sym - p.W * lap);
    const float sdg = gsgx * gpx + gsgy * gpy;
    float Fx, Fy;
    if constexpr (!var) {
        Fx = cap * gpx + p.mar_k * (g2 * gsgx - sdg * gpx) + p.rho * p.gx;
        Fy = cap * gpy + p.mar_k * (g2 * gsgy - sdg * gpy) + p.rho * p.gy;
    } else {
        Fx = rfma(rho_v, p.gx, rfma(cap, gpx, rmul(p.mar_k, rfma(g2, gsgx, -rmul(sdg, gpx)))));
        Fy = rfma(rho_v, p.gy, rfma(cap, gpy, rmul(p.mar_k, rfma(g2, gsgy, -rmul(sdg, gpy)))));
    }

    // own u of the previous level (also the encoding velocity of the own slots across a wall)
    const float2 uown = S::kHalo ? Hist[(ty + 1) * BW + tx + 4] : Hist[ty * TX + tx];

    // flow populations pulled from the staged boxes (16-bit: plus the source cell's 3 w rho c.u)
    float h[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if constexpr (FLOW) {
        const bool bb_up = WALLS && y == 0;           // links 2, 5, 6 come from below the bottom wall
        const bool bb_dn = WALLS && y == p.ny - 1;    // links 4, 7, 8 come from above the top wall
        h[1] = load_h<ST, 1>(sm, Hist, p, tx, ty, false, uown);
        h[2] = load_h<ST, 2>(sm, Hist, p, tx, ty, bb_up, uown);
        h[3] = load_h<ST, 3>(sm, Hist, p, tx, ty, false, uown);
        h[4] = load_h<ST, 4>(sm, Hist, p, tx, ty, bb_dn, uown);
        h[5] = load_h<ST, 5>(sm, Hist, p, tx, ty, bb_up, uown);
        h[6] = load_h<ST, 6>(sm, Hist, p, tx, ty, bb_up, uown);
        h[7] = load_h<ST, 7>(sm, Hist, p, tx, ty, bb_dn, uown);
        h[8] = load_h<ST, 8>(sm, Hist, p, tx, ty, bb_dn, uown);
    }

    // velocity: rho u = sum c_i h_i + F/2 (Sec. 3.3), or the imposed velocity (kept in the history)
    // the links paired as (1, 2), (3, 4), (5, 6), (7, 8) for packed FP32x2 arithmetic
    float2 X = make_float2(h[1], h[2]), Y = make_float2(h[3], h[4]), U = make_float2(h[5], h[6]),
           V = make_float2(h[7], h[8]);
    const float2 dXY = sub2(X, Y), dUV = sub2(U, V);  // (h1 - h3, h2 - h4), (h5 - h7, h6 - h8)
    const float h57 = dUV.x, h68 = dUV.y;
    const float jx = dXY.x + (h57 - h68);
    const float jy = dXY.y + (h57 + h68);
    const float inv_rho = var ? __frcp_rn(rho_v) : p.inv_rho;
    const float ux = FLOW ? (jx + 0.5f * Fx) * inv_rho : uown.x;
    const float uy = FLOW ? (jy + 0.5f * Fy) * inv_rho : uown.y;

    // previous level: (phi, psi) from the own cell's post-collision pairs, u from history
    float2 pprev = pp;
    float uxp = ux, uyp = uy;
    if (!io.first) {
        const P* base = FG + (ty + 1) * BW + tx + 4;
        float2 r[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) r[i] = raw2(base[i * SLOT + cy(i) * BW]);
        pprev = pair_sum<ST>(r, ref);
        uxp = uown.x;
        uyp = uown.y;
    }

    // time derivatives, backward difference over one step: d_t(phi u), d_t(psi u) as pairs, and
    // d_t(rho u u - (S u + u S)/2) (Sec. 3.3)
    const float rho = var ? rho_v : p.rho;
    const float2 dtX = fma2(pp, bc(ux), mul2(pprev, bc(-uxp)));
    const float2 dtY = fma2(pp, bc(uy), mul2(pprev, bc(-uyp)));
    float dt_xx, dt_yy, dt_xy, ugr = 0.f;
    // Q = (rho u - S) u of this level (density ratio only): diagonal and symmetrised off-diagonal
    float Jx = 0.f, Jy = 0.f, qxx = 0.f, qyy = 0.f, qxy = 0.f;
    if (!var) {
        dt_xx = rho * (ux * ux - uxp * uxp);
        dt_yy = rho * (uy * uy - uyp * uyp);
        dt_xy = rho * (ux * uy - uxp * uyp);
    } else {
        Jx = rmul(rho, ux);
        Jy = rmul(rho, uy);
        qxx = rmul(rsub(Jx, Sx), ux);
        qyy = rmul(rsub(Jy, Sy), uy);
        qxy = rfma(Jx, uy, -rmul(0.5f, rfma(Sx, uy, rmul(Sy, ux))));
        const float rp = rfma(rsub(pprev.x, p.phiB), p.drho, p.rhoB);  // rho of the previous level
        const float Sxp = io.first ? Sx : Sp.x, Syp = io.first ? Sy : Sp.y;
        const float Jxp = rmul(rp, uxp), Jyp = rmul(rp, uyp);
        dt_xx = rsub(qxx, rmul(rsub(Jxp, Sxp), uxp));
        dt_yy = rsub(qyy, rmul(rsub(Jyp, Syp), uyp));
        dt_xy = rsub(qxy, rfma(Jxp, uyp, -rmul(0.5f, rfma(Sxp, uyp, rmul(Syp, uxp)))));
        ugr = rfma(ux, grx, rmul(uy, gry));
    }

    // pressure (Eq. for P, Sec. 3.3) with K = w0/(c^2 - cs2) = 2/3:
    //   P = 3/5 [sum_{i>0} h_i + u.grad rho / 2 - (2/3) (rho u - S).u + (1/3) d_t(rho u.u - S.u)]
    const float2 sXY = add2(X, Y), sUV = add2(U, V);  // (h1 + h3, h2 + h4), (h5 + h7, h6 + h8)
    const float hsum = (sXY.x + sXY.y) + (sUV.x + sUV.y);
    float P_ = 0.f;
    if (FLOW) {
        if (!var)
            P_ = 0.6f * (hsum - (2.f / 3.f) * rho * (ux * ux + uy * uy) + (1.f / 3.f) * (dt_xx + dt_yy));
        else
            P_ = rmul(0.6f, rfma(1.f / 3.f, radd(dt_xx, dt_yy),
                                 rfma(-2.f / 3.f, radd(qxx, qyy), rfma(0.5f, ugr, hsum))));
    }

    {
        // |u| >= 0.3, or a non-finite value (NaN fails every comparison; a NaN anywhere in the
        // cell reaches u, phi or psi within a step), or psi >= 1 under the Langmuir EOS
        bool bad = !(fabsf(ux) < 0.3f) | !(fabsf(uy) < 0.3f) | !(fabsf(phi) < 1e30f) | !(fabsf(psi) < 1e30f);
        if (LANGMUIR) bad |= !(psi < 1.f);
        if (bad) atomicOr(io.status, kStatusUnstable);
    }

    const size_t cell = (size_t)(p.org + (long long)y * p.pitch + x);
    if constexpr (MODE == kMoments) {
        const size_t o = (size_t)y * p.nx + x;
        if (io.out[0]) io.out[0][o] = phi;
        if (io.out[1]) io.out[1][o] = psi;
        if (io.out[2]) io.out[2][o] = ux;
        if (io.out[3]) io.out[3][o] = uy;
        if (io.out[4]) io.out[4][o] = P_;
    } else {
        using Hv = typename T::H;
        uint32_t key = 0;
        if constexpr (T::kPair16) key = cell_key((uint32_t)cell, io.seed);
        P outp[9];  // the stored (f_i, g_i)
        float2 outhp[4];   // FP32 h: the stored pairs (h_1, h_2), (h_3, h_4), (h_5, h_6), (h_7, h_8)
        uint32_t outw[4];  // 16-bit h: the stored pairs (h_1, h_2), (h_3, h_4), (h_5, h_6), (h_7, h_8)
        // ---- f (Sec. 3.1) and g (Sec. 3.2) together; sources cs2 V = d_t(s u) + cs2 (A or B) n ----
        {
            const float2 vx = fma2(make_float2(Aterm, Bterm), bc(nx_ * (1.f / 3.f)), dtX);
            const float2 vy = fma2(make_float2(Aterm, Bterm), bc(ny_ * (1.f / 3.f)), dtY);
            collide_pair<ST>(q, pp, sub2(pp, ref), ux, uy, vx, vy, make_float2(p.nS1[0], p.nS1[1]),
                         make_float2(p.nS2[0], p.nS2[1]), make_float2(p.nS3[0], p.nS3[1]),
                         make_float2(p.nS4[0], p.nS4[1]), make_float2(p.K1[0], p.K1[1]), make_float2(p.K3[0], p.K3[1]));
            if constexpr (!T::kPair16) {
#pragma unroll
                for (int i = 0; i < 9; ++i) outp[i] = q[i];
            } else {
                outp[0] = enc_pair_rs<ST, 0>(q[0], key);
                outp[1] = enc_pair_rs<ST, 1>(q[1], key);
                outp[2] = enc_pair_rs<ST, 2>(q[2], key);
                outp[3] = enc_pair_rs<ST, 3>(q[3], key);
                outp[4] = enc_pair_rs<ST, 4>(q[4], key);
                outp[5] = enc_pair_rs<ST, 5>(q[5], key);
                outp[6] = enc_pair_rs<ST, 6>(q[6], key);
                outp[7] = enc_pair_rs<ST, 7>(q[7], key);
                outp[8] = enc_pair_rs<ST, 8>(q[8], key);
            }
        }
        // ---- flow h (Sec. 3.3); none when the velocity is prescribed ----
        if constexpr (FLOW) {
            float s2, k2, s4, k4;
            if (p.dmu == 0.f && !var) {
                s2 = p.s2h;
                k2 = p.k2h;
                s4 = p.s4h_eff;
                k4 = p.k4h;
            } else {
                if constexpr (!var)
                    s2 = __frcp_rn(3.f * (p.muB + (phi - p.phiB) * p.inv_dphi * p.dmu) * p.inv_rho + 0.5f);
                else  // nu = mu(phi) / rho(phi)
                    s2 = __frcp_rn(rfma(rmul(3.f, rfma(rmul(rsub(phi, p.phiB), p.inv_dphi), p.dmu, p.muB)), inv_rho, 0.5f));
                k2 = 1.f - 0.5f * s2;
                s4 = p.tie_s4h ? s2 : p.s4h;
                k4 = 1.f - 0.5f * s4;
            }
            const float s1 = p.s1h, s3 = p.s3h, k1 = p.k1h, k3 = p.k3h;
            if constexpr (!var) {
                Jx = rho * ux;
                Jy = rho * uy;
            }
            // equilibrium moments, Q = (rho u - S) u:
            //   (., Jx, Jy, P + Q_xx, P + Q_yy, (Q_xy + Q_yx)/2, Jx/3, Jy/3, P/3 + (Q_xx + Q_yy)/3)
            // source moments of H, m2H = d_t(rho u u - (S u + u S)/2) + cs2 (u grad rho + grad rho u):
            //   (., Fx, Fy, m2H_xx + u.grad rho/3, m2H_yy + u.grad rho/3, m2H_xy, Fx/3, Fy/3,
            //    (m2H_xx + m2H_yy)/3 + u.grad rho/9)
            const float m5 = sUV.x - sUV.y, m8 = sUV.x + sUV.y;
            const float2 m67 = make_float2(h57 - h68, h57 + h68);  // (m6, m7)
            const float2 m34 = add2(sXY, bc(m8));                   // (m3, m4)
            const float2 Fv = make_float2(Fx, Fy), Jv = make_float2(Jx, Jy), uv = make_float2(ux, uy);
            // increments dm_k = -s_k (m_k - m_eq_k) + (1 - s_k/2) m_src_k, then h* = h + M^-1 dm; the
            // x and y moments of each order as one pair
            float2 d12, d34, d67;
            float d5, d8;
            if constexpr (!var) {
                d12 = fma2(bc(k1), Fv, mul2(bc(-s1), sub2(make_float2(jx, jy), Jv)));
                d34 = fma2(bc(k2), make_float2(dt_xx, dt_yy), mul2(bc(-s2), sub2(m34, fma2(Jv, uv, bc(P_)))));
                d5 = k2 * dt_xy - s2 * (m5 - Jx * uy);
                d67 = mul2(bc(1.f / 3.f), fma2(bc(k3), Fv, mul2(bc(-s3), fma2(bc(3.f), m67, make_float2(-Jx, -Jy)))));
                d8 = (1.f / 3.f) * (k4 * (dt_xx + dt_yy) - s4 * (3.f * m8 - (P_ + Jx * ux + Jy * uy)));
            } else {
                d12 = make_float2(rfma(k1, Fx, -rmul(s1, rsub(jx, Jx))), rfma(k1, Fy, -rmul(s1, rsub(jy, Jy))));
                const float mxx = rfma(2.f / 3.f, rmul(ux, grx), dt_xx);
                const float myy = rfma(2.f / 3.f, rmul(uy, gry), dt_yy);
                const float mxy = rfma(1.f / 3.f, rfma(ux, gry, rmul(uy, grx)), dt_xy);
                d34 = make_float2(rfma(k2, rfma(1.f / 3.f, ugr, mxx), -rmul(s2, rsub(m34.x, radd(P_, qxx)))),
                                  rfma(k2, rfma(1.f / 3.f, ugr, myy), -rmul(s2, rsub(m34.y, radd(P_, qyy)))));
                d5 = rfma(k2, mxy, -rmul(s2, rsub(m5, qxy)));
                d67 = make_float2(rmul(1.f / 3.f, rfma(k3, Fx, -rmul(s3, rfma(3.f, m67.x, -Jx)))),
                                  rmul(1.f / 3.f, rfma(k3, Fy, -rmul(s3, rfma(3.f, m67.y, -Jy)))));
                // 3 x the eighth source moment (mxx + myy)/3 + u.grad rho/9
                d8 = rmul(1.f / 3.f, rfma(k4, rfma(1.f / 3.f, ugr, radd(mxx, myy)),
                                          -rmul(s4, rfma(3.f, m8, -radd(P_, radd(qxx, qyy))))));
            }
            // (A, C) = (d1 - d6, d2 - d7), (B, D) = (d3 - d8, d4 - d8), (E, F) = (d8 + d5, d8 - d5),
            // (G, H) = (d6 + d7, d7 - d6)
            const float2 AC = sub2(d12, d67), BD = sub2(d34, bc(d8));
            const float2 EF = make_float2(d8 + d5, d8 - d5), GH = make_float2(d67.x + d67.y, d67.y - d67.x);
            X = fma2(bc(0.5f), add2(AC, BD), X);     // h1 += (A + B)/2, h2 += (C + D)/2
            Y = fma2(bc(0.5f), sub2(BD, AC), Y);     // h3 += (B - A)/2, h4 += (D - C)/2
            U = fma2(bc(0.25f), add2(EF, GH), U);    // h5 += (E + G)/4, h6 += (F + H)/4
            V = fma2(bc(0.25f), sub2(EF, GH), V);    // h7 += (E - G)/4, h8 += (F - H)/4
            if (WALLS) {
                // moving-wall term for the links that leave through a wall, folded in before storing:
                // h_ibar(x_b, t+1) = h*_i(x_b, t) - 2 w_i rho c_i.u_w / cs2
                if (y == 0) {
                    V.x -= 6.f * wgt(7) * rho * (-1.f) * p.u_bot;
                    V.y -= 6.f * wgt(8) * rho * (1.f) * p.u_bot;
                }
                if (y == p.ny - 1) {
                    U.x -= 6.f * wgt(5) * rho * (1.f) * p.u_top;
                    U.y -= 6.f * wgt(6) * rho * (-1.f) * p.u_top;
                }
            }
            if constexpr (!T::kH16) {
                outhp[0] = X, outhp[1] = Y, outhp[2] = U, outhp[3] = V;
            } else {
                // every slot is stored relative to this cell's new u (what the next step reads back):
                // raw = (h_i / w_i - 3 rho c_i.u) S_h, two links per stochastic conversion
                const float vx = p.kh3 * T::SH * ux, vy = p.kh3 * T::SH * uy;
                constexpr float e1 = (float)(T::SH / wgt_d(1)), e5 = (float)(T::SH / wgt_d(5));  // exact
                const float2 r12 = fma2(X, bc(e1), make_float2(-vx, -vy));
                const float2 r34 = fma2(Y, bc(e1), make_float2(vx, vy));
                const float2 r56 = fma2(U, bc(e5), make_float2(-(vx + vy), vx - vy));
                const float2 r78 = fma2(V, bc(e5), make_float2(vx + vy, vy - vx));
                outw[0] = cvt_rs2<typename T::P>(r12.x, r12.y, rbits_of(key, 9));
                outw[1] = cvt_rs2<typename T::P>(r34.x, r34.y, rbits_of(key, 10));
                outw[2] = cvt_rs2<typename T::P>(r56.x, r56.y, rbits_of(key, 11));
                outw[3] = cvt_rs2<typename T::P>(r78.x, r78.y, rbits_of(key, 12));
            }
        }
        // ---- stores: the own cell, its periodic images in the ghost frame, and at a wall the
        //      bounce-back ghosts of the links that cross it ----
        P* __restrict__ dfg = static_cast<P*>(io.dst);
        Hv* __restrict__ dh = reinterpret_cast<Hv*>(dfg + (size_t)kPairs * p.plane);
        const long long pl = p.plane;
        auto put = [&](long long c) {
#pragma unroll
            for (int i = 0; i < 9; ++i) dfg[i * pl + c] = outp[i];
            if constexpr (FLOW && T::kH16) {
                uint32_t* dw = reinterpret_cast<uint32_t*>(dh);
#pragma unroll
                for (int j = 0; j < 4; ++j) dw[j * pl + c] = outw[j];
            } else if constexpr (FLOW) {
                float2* dp = reinterpret_cast<float2*>(dh);
#pragma unroll
                for (int j = 0; j < 4; ++j) dp[j * pl + c] = outhp[j];
            }
        };
        const bool xl = x <= 1, xr = x >= p.nx - 2;
        const bool yl = !WALLS && y <= 1, yr = !WALLS && y >= p.ny - 2;
        const long long DX = p.nx, DY = (long long)p.ny * p.pitch;
        if constexpr (TS) {
            // the own cell into the warp's staging row (the warp is the tile row, tx the lane); the
            // caller writes the row out (store_staged_row)
            P* sp = reinterpret_cast<P*>(stg) + tx;
#pragma unroll
            for (int i = 0; i < 9; ++i) sp[i * TX] = outp[i];
            if constexpr (FLOW && T::kH16) {
                uint32_t* dw = reinterpret_cast<uint32_t*>(dh);
#pragma unroll
                for (int j = 0; j < 4; ++j) dw[j * pl + cell] = outw[j];
            } else if constexpr (FLOW) {
                float2* dp = reinterpret_cast<float2*>(dh);
#pragma unroll
                for (int j = 0; j < 4; ++j) dp[j * pl + cell] = outhp[j];
            }
        } else {
            put((long long)cell);
        }
        if (xl | xr | yl | yr) {
            if (xl) put(cell + DX);
            if (xr) put(cell - DX);
            if (yl) {
                put(cell + DY);
                if (xl) put(cell + DY + DX);
                if (xr) put(cell + DY - DX);
            }
            if (yr) {
                put(cell - DY);
                if (xl) put(cell - DY + DX);
                if (xr) put(cell - DY - DX);
            }
        }
        if (WALLS && (y == 0 || y == p.ny - 1)) {
            // the pull of link i across the wall, at (x - c_ix, -1) or (x - c_ix, ny) in plane i,
            // reads this cell's post-collision opposite slot (half-way bounce-back, Sec. 4)
            auto bb = [&](int i, int io_, int col, long long c) {
                const int nx = p.nx;
                auto one = [&](long long d) {
                    dfg[i * pl + d] = outp[io_];
                    if constexpr (FLOW && T::kH16) {
                        const uint32_t w = outw[(io_ - 1) >> 1];
                        dh[h_index(i, d, pl)] = bits_to<Hv>(((io_ - 1) & 1) ? (w >> 16) : (w & 0xFFFFu));
                    } else if constexpr (FLOW) {
                        const float2 w = outhp[(io_ - 1) >> 1];
                        dh[h_index(i, d, pl)] = ((io_ - 1) & 1) ? w.y : w.x;
                    }
                };
                one(c);
                if (col <= 1) one(c + nx);
                if (col >= nx - 2) one(c - nx);
            };
            const long long pt = p.pitch;
            if (y == 0) {
                bb(2, 4, x, cell - pt);
                bb(5, 7, x - 1, cell - pt - 1);
                bb(6, 8, x + 1, cell - pt + 1);
            } else {
                bb(4, 2, x, cell + pt);
                bb(7, 5, x + 1, cell + pt + 1);
                bb(8, 6, x - 1, cell + pt - 1);
            }
        }
        const float2 un = make_float2(ux, uy);
        io.hist_dst[cell] = un;
        if (var) io.shist_dst[cell] = make_float2(Sx, Sy);
        if constexpr (S::kHalo) {
            // the 16-bit h decode reads the neighbours' u, across periodic edges too
            if (xl) io.hist_dst[cell + DX] = un;
            if (xr) io.hist_dst[cell - DX] = un;
            if (yl) {
                io.hist_dst[cell + DY] = un;
                if (xl) io.hist_dst[cell + DY + DX] = un;
                if (xr) io.hist_dst[cell + DY - DX] = un;
            }
            if (yr) {
                io.hist_dst[cell - DY] = un;
                if (xl) io.hist_dst[cell - DY + DX] = un;
                if (xr) io.hist_dst[cell - DY - DX] = un;
            }
        }
    }
    return false;
}

// One step (or the moments) of one lattice: one TX x TY tile per CTA.  Four CTAs per SM; with FP32
// storage and a prescribed velocity (no h) the cell update fits 48 registers without spills and
// the boxes 33 KB, so five (convection test 2048 x 1024: 54.3 -> 52.5 us per step).
template <int ST, bool WALLS, bool LANGMUIR, int MODE, int FLOW>
__global__ void __launch_bounds__(NT, FLOW == kFlowPrescribed && ST == kFP32 ? 5 : 4) step_kernel(const __grid_constant__ StepArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(sm + Smem<ST>::BAR);
    // The first and the last tile row (whose cells also write the ghost frame, and so run longest)
    // are launched first, so that the last wave holds interior tiles only.
    const int ntr = gridDim.y;
    const int tr = blockIdx.y == 0 ? 0 : (blockIdx.y == 1 ? ntr - 1 : (int)blockIdx.y - 1);
    const int x0 = blockIdx.x * TX, y0 = tr * TY;
    if (threadIdx.x == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
    }
    // Programmatic dependent launch: let the next step's CTAs be scheduled into the slots this
    // grid frees, and wait here until the previous step's writes are complete and visible.
    cudaTriggerProgrammaticLaunchCompletion();
    cudaGridDependencySynchronize();
    if (threadIdx.x == 0) issue_tile_loads<ST, FLOW>(sm, &a.tm_fg, &a.tm_h, &a.tm_hist, x0, y0, mbar);
    step_tile<ST, WALLS, LANGMUIR, MODE, FLOW>(a.p, a.io, sm, reinterpret_cast<float2*>(sm + Smem<ST>::PP), mbar, 0, x0,
                                               y0);
}

// Tile k of a grid of ntx x nty tiles: rows in the order first, last, then the interior (the two
// edge rows, whose cells also write the ghost frame, run first).
__device__ __forceinline__ void tile_origin(int k, int ntx, int nty, int& x0, int& y0) {
    const int r = k / ntx, c = k - r * ntx;
    const int tr = r == 0 ? 0 : (r == 1 ? nty - 1 : r - 1);
    x0 = c * TX;
    y0 = tr * TY;
}

// One step of one lattice by a persistent, warp-specialised grid.  Each CTA has NT compute threads
// (eight warps, one cell each, as in step_kernel) and one copy warp.  One lane of the copy warp
// claims tiles from an atomic counter (one at a time, which balances the longer edge tiles across
// the CTAs; each claim one iteration ahead, so its latency overlaps the wait for a buffer) and
// stages each into one of two buffers with TMA, on that buffer's "full" mbarrier;
// the compute warps release a buffer on its "empty" mbarrier (one arrival per warp) once the tile
// is done, so the copy of the next tile overlaps the arithmetic of the current one and the copy
// warp never joins a block-wide barrier.  After the last tile the copy lane arrives on a full
// barrier without a copy; the compute warps read the stop mark (x0 = -1) and stop.  Every
// wait is bounded: a copy lane that gives up waits (bounded) for the copies it has in flight.
// Three CTAs per SM with 16-bit storage; two with FP32, whose two stages fill the shared memory of
// two, so its bound lets the compiler use up to 112 registers (rising bubble, FP32: 81.6 -> 80.6 us).
constexpr int NT_PIPE = NT + 32;

// Writes the staged own pairs of tile row y0 + warp (see Smem::kTS).  A tile that lies wholly
// inside the grid in x goes out as one bulk tensor store, issued by lane 0 and tracked in its bulk
// group.  The ragged last tile column ends next
// to the ghost columns that hold the periodic images of x = 0, 1, which plain stores write in the
// same step; its lanes copy their own cells with plain stores, so no bulk store depends on
// clipping at the map's extent.
template <int ST>
__device__ __forceinline__ void store_staged_row(const StepArgs& a, const unsigned char* stg, int x0, int y0,
                                                 int warp, int lane) {
    using P = typename Traits<ST>::P;
    const int y = y0 + warp;
    if (x0 + TX <= a.p.nx) {
        fence_proxy_async();
        __syncwarp();
        if (lane == 0 && y < a.p.ny) {
            tma_store_3d(&a.tm_st_fg, stg, kGX + x0, kGY + y, 0);
            bulk_commit();
        }
    } else if (x0 + lane < a.p.nx && y < a.p.ny) {
        const long long pl = a.p.plane, cell = a.p.org + (long long)y * a.p.pitch + x0 + lane;
        P* dfg = static_cast<P*>(a.io.dst);
        const P* sp = reinterpret_cast<const P*>(stg) + lane;
#pragma unroll
        for (int i = 0; i < 9; ++i) dfg[i * pl + cell] = sp[i * TX];
    }
}

template <int ST, bool WALLS, bool LANGMUIR, int FLOW>
__global__ void __launch_bounds__(NT_PIPE, ST == kFP32 ? 2 : 3) step_kernel_pipe(const __grid_constant__ StepArgs a, int ntx, int nty) {
    using S = Smem<ST>;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned long long* full = reinterpret_cast<unsigned long long*>(sm + S::PIPE_BAR);
    unsigned long long* empty = full + 2;
    volatile int* slot = reinterpret_cast<volatile int*>(sm + S::PIPE_SLOT);  // (x0, y0) per buffer
    const unsigned ntiles = (unsigned)(ntx * nty);
    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&empty[0], NT / 32);
        mbar_init(&empty[1], NT / 32);
        fence_mbar_init();
    }
    __syncthreads();
    cudaTriggerProgrammaticLaunchCompletion();
    cudaGridDependencySynchronize();  // also: the previous launch no longer uses its counter

    if (threadIdx.x >= NT) {
        // ---- copy warp ----
        if (threadIdx.x != NT) return;
        if (blockIdx.x == 0) *a.tile_ctr_next = 0u;
        bool pending[2] = {false, false};   // a copy into the buffer that no release has confirmed
        uint32_t issued[2] = {0u, 0u};      // parity of the full barrier's phase of that copy
        unsigned k = atomicAdd(a.tile_ctr, 1u);  // claimed one iteration ahead of its use
        for (int it = 0;; ++it) {
            const int b = it & 1;
            const unsigned kn = k < ntiles ? atomicAdd(a.tile_ctr, 1u) : ntiles;  // the next claim, early
            if (it >= 2) {
                if (!mbar_wait_bounded(&empty[b], (uint32_t)((it >> 1) - 1) & 1u)) {
                    atomicOr(a.io.status, kStatusTimeout);
                    for (int q = 0; q < 2; ++q)
                        if (pending[q]) mbar_wait_bounded(&full[q], issued[q]);
                    return;
                }
                pending[b] = false;
            }
            if (k >= ntiles) {
                slot[2 * b] = -1;
                mbar_arrive(&full[b]);  // no copy: the compute warps read x0 = -1 and stop
                return;
            }
            int x0, y0;
            tile_origin((int)k, ntx, nty, x0, y0);
            slot[2 * b] = x0;
            slot[2 * b + 1] = y0;
            issue_tile_loads<ST, FLOW>(sm + b * S::STAGE, &a.tm_fg, &a.tm_h, &a.tm_hist, x0, y0, &full[b]);
            pending[b] = true;
            issued[b] = (uint32_t)(it >> 1) & 1u;
            k = kn;
        }
    }

    // ---- compute warps ----
    const int warp = (int)threadIdx.x / 32, lane = (int)threadIdx.x % 32;
    unsigned char* stg = sm + S::PIPE_STG + warp * S::STG_W;  // this warp's staging row (see Smem::kTS)
    for (int it = 0;; ++it) {
        const int b = it & 1;
        const uint32_t parity = (uint32_t)(it >> 1) & 1u;
        // the previous tile's bulk stores have read the staging row before the barrier below, so
        // the warp may rewrite it after the barrier
        if (S::kTS && lane == 0) bulk_wait_read();
        const bool late = !mbar_wait_bounded(&full[b], parity);
        if (compute_sync_or(late)) {  // uniform: a copy (or the stop mark) did not come in time
            if (threadIdx.x == 0) {
                atomicOr(a.io.status, kStatusTimeout);
                // wait (bounded) for the copies that may still be in flight into either buffer
                mbar_wait_bounded(&full[b], parity);
                mbar_wait_bounded(&full[b ^ 1], (uint32_t)((it + 1) >> 1) & 1u);
            }
            break;
        }
        const int x0 = slot[2 * b], y0 = slot[2 * b + 1];
        if (x0 < 0) break;  // uniform: every compute thread reads the same slot
        float2* PP = reinterpret_cast<float2*>(sm + S::PIPE_PP) + b * NE;
        if (step_tile<ST, WALLS, LANGMUIR, kStep, FLOW, true, S::kTS>(a.p, a.io, sm + b * S::STAGE, PP, &full[b],
                                                                      parity, x0, y0, stg))
            break;  // uniform (decided by the OR barrier inside)
        if constexpr (S::kTS) store_staged_row<ST>(a, stg, x0, y0, warp, lane);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);  // this warp is done with buffer b
    }
    // the bulk stores are complete before the CTA's shared memory goes away
    if (S::kTS && lane == 0) bulk_wait_all();
}

// ---- many lattices in one launch ----
// Per-lattice descriptor, in device memory, written by the host between launches and advanced by
// batch_advance_kernel.  Buffer `cur` holds the current state; `steps` steps were taken since
// initialisation.
struct alignas(128) InstDesc {
    CUtensorMap tm_fg[2], tm_h[2], tm_hist[2];
    Phys p;
    void* pops[2];
    float2* hist[2];
    float2* shist[2];  // mass-flux history (density ratio != 1), else null
    unsigned* status;
    long long steps;
    int cur;
    int first;
};

// Launch s (0-based) of a sequence that started from the descriptors' state; each CTA owns the
// tile tiles[blockIdx.x] = (lattice, tile column | tile row << 16).
struct BatchArgs {
    const InstDesc* __restrict__ descs;
    const uint2* __restrict__ tiles;
    int s;
    // warp-specialised kernel only (ws_ctas > 0): the tile count, the persistent grid, the member
    // count, this launch's tile counter (zero at its start) and the next launch's (zeroed by this one)
    int ntiles, ws_ctas, ndescs;
    unsigned* ctr;
    unsigned* ctr_next;
};

// A bounded wait of the batched warp-specialised kernel gave up: flag every member (the stalled
// tile's lattice is not known to every thread that sees the timeout).
__device__ __forceinline__ void flag_batch_timeout(const BatchArgs& b) {
    for (int k = 0; k < b.ndescs; ++k) atomicOr(b.descs[k].status, kStatusTimeout);
}

template <int ST, bool WALLS, bool LANGMUIR, int FLOW>
__global__ void __launch_bounds__(NT, 4) batch_step_kernel(const __grid_constant__ BatchArgs b) {
    using S = Smem<ST>;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(sm + S::BAR);
    cudaTriggerProgrammaticLaunchCompletion();
    cudaGridDependencySynchronize();  // descriptors and populations of the previous launch
    const uint2 te = b.tiles[blockIdx.x];
    const InstDesc& d = b.descs[te.x];
    const int x0 = (int)(te.y & 0xFFFFu) * TX, y0 = (int)(te.y >> 16) * TY;
    const int cur = (d.cur + b.s) & 1;
    // the lattice's constants in shared memory (made visible by the first barrier of step_tile)
    Phys* sp = reinterpret_cast<Phys*>(sm + S::PHYS);
    static_assert(sizeof(Phys) % 4 == 0, "Phys is copied as words");
    for (int k = threadIdx.x; k < (int)(sizeof(Phys) / 4); k += NT)
        reinterpret_cast<uint32_t*>(sp)[k] = reinterpret_cast<const uint32_t*>(&d.p)[k];
    if (threadIdx.x == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
        issue_tile_loads<ST, FLOW>(sm, &d.tm_fg[cur], &d.tm_h[cur], &d.tm_hist[cur], x0, y0, mbar);
    }
    TileIO io;
    io.src = d.pops[cur];
    io.dst = d.pops[cur ^ 1];
    io.hist_src = d.hist[cur];
    io.hist_dst = d.hist[cur ^ 1];
    io.shist_src = d.shist[cur];
    io.shist_dst = d.shist[cur ^ 1];
    io.status = d.status;
    io.out[0] = io.out[1] = io.out[2] = io.out[3] = io.out[4] = nullptr;
    io.seed = step_seed(d.steps + b.s);
    io.first = d.first && b.s == 0;
    step_tile<ST, WALLS, LANGMUIR, kStep, FLOW>(*sp, io, sm, reinterpret_cast<float2*>(sm + S::PP), mbar, 0, x0, y0);
}

// One step of many lattices by a persistent, warp-specialised grid (the design of step_kernel_pipe).
// The copy lane claims entries of the tile list from this launch's counter; for each it reads the
// lattice's current buffer, stages the lattice's constants (one bulk copy) and the tile's boxes
// (TMA) into a buffer on its full barrier.  It works one tile ahead: the claim, list entry and
// descriptor read of the next tile are in flight while it waits for a buffer, so these dependent
// loads overlap the arithmetic instead of delaying every tile.  Two CTAs per SM (the FP32 buffers
// fill the shared memory of two anyway): at that bound the compiler keeps the cell update in
// registers, where at three it spilled 28-96 B (64-lattice mix: FP32 27.2 -> 28.7 GLUPS, FP16
// 31.7 -> 34.7, FP16_FG 32.2 -> 34.9).
template <int ST, bool WALLS, bool LANGMUIR, int FLOW>
__global__ void __launch_bounds__(NT_PIPE, 2) batch_step_kernel_ws(const __grid_constant__ BatchArgs b) {
    using S = Smem<ST>;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned long long* full = reinterpret_cast<unsigned long long*>(sm + S::PIPE_BAR);
    unsigned long long* empty = full + 2;
    volatile int* slot = reinterpret_cast<volatile int*>(sm + S::BWS_SLOT);  // x0, y0, lattice, cur per buffer
    const unsigned ntiles = (unsigned)b.ntiles;
    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&empty[0], NT / 32);
        mbar_init(&empty[1], NT / 32);
        fence_mbar_init();
    }
    __syncthreads();
    cudaTriggerProgrammaticLaunchCompletion();
    cudaGridDependencySynchronize();  // descriptors and populations of the previous launch

    if (threadIdx.x >= NT) {
        // ---- copy warp ----
        if (threadIdx.x != NT) return;
        if (blockIdx.x == 0) *b.ctr_next = 0u;
        bool pending[2] = {false, false};
        uint32_t issued[2] = {0u, 0u};
        // the tile of the current iteration, claimed and read one iteration ahead
        unsigned k = atomicAdd(b.ctr, 1u);
        uint2 te = make_uint2(0u, 0u);
        int cur = 0;
        if (k < ntiles) {
            te = b.tiles[k];
            cur = (b.descs[te.x].cur + b.s) & 1;
        }
        for (int it = 0;; ++it) {
            const int q = it & 1;
            const unsigned kn = k < ntiles ? atomicAdd(b.ctr, 1u) : ntiles;  // the next claim, early
            if (it >= 2) {
                if (!mbar_wait_bounded(&empty[q], (uint32_t)((it >> 1) - 1) & 1u)) {
                    flag_batch_timeout(b);
                    for (int r = 0; r < 2; ++r)
                        if (pending[r]) mbar_wait_bounded(&full[r], issued[r]);
                    return;
                }
                pending[q] = false;
            }
            if (k >= ntiles) {
                slot[4 * q] = -1;
                mbar_arrive(&full[q]);  // no copy: the compute warps read x0 = -1 and stop
                return;
            }
            const InstDesc* d = &b.descs[te.x];
            const int x0 = (int)(te.y & 0xFFFFu) * TX, y0 = (int)(te.y >> 16) * TY;
            slot[4 * q] = x0;
            slot[4 * q + 1] = y0;
            slot[4 * q + 2] = (int)te.x;
            slot[4 * q + 3] = cur;
            mbar_expect_tx_only(&full[q], (uint32_t)S::PHYS_BYTES);
            bulk_copy_g2s(sm + S::BWS_PHYS + q * S::PHYS_BYTES, &d->p, (uint32_t)S::PHYS_BYTES, &full[q]);
            issue_tile_loads<ST, FLOW>(sm + q * S::STAGE, &d->tm_fg[cur], &d->tm_h[cur], &d->tm_hist[cur], x0, y0, &full[q]);
            pending[q] = true;
            issued[q] = (uint32_t)(it >> 1) & 1u;
            // read the next tile's list entry and buffer now; they arrive while this lane waits
            k = kn;
            if (k < ntiles) {
                te = b.tiles[k];
                cur = (b.descs[te.x].cur + b.s) & 1;
            }
        }
    }

    // ---- compute warps ----
    for (int it = 0;; ++it) {
        const int q = it & 1;
        const uint32_t parity = (uint32_t)(it >> 1) & 1u;
        const bool late = !mbar_wait_bounded(&full[q], parity);
        if (compute_sync_or(late)) {
            if (threadIdx.x == 0) {
                flag_batch_timeout(b);
                mbar_wait_bounded(&full[q], parity);
                mbar_wait_bounded(&full[q ^ 1], (uint32_t)((it + 1) >> 1) & 1u);
            }
            return;
        }
        const int x0 = slot[4 * q], y0 = slot[4 * q + 1];
        if (x0 < 0) return;  // uniform: every compute thread reads the same slot
        const int lat = slot[4 * q + 2], cur = slot[4 * q + 3];
        const InstDesc& d = b.descs[lat];
        TileIO io;
        io.src = d.pops[cur];
        io.dst = d.pops[cur ^ 1];
        io.hist_src = d.hist[cur];
        io.hist_dst = d.hist[cur ^ 1];
        io.shist_src = d.shist[cur];
        io.shist_dst = d.shist[cur ^ 1];
        io.status = d.status;
        io.out[0] = io.out[1] = io.out[2] = io.out[3] = io.out[4] = nullptr;
        io.seed = step_seed(d.steps + b.s);
        io.first = d.first && b.s == 0;
        const Phys& p = *reinterpret_cast<const Phys*>(sm + S::BWS_PHYS + q * S::PHYS_BYTES);
        float2* PP = reinterpret_cast<float2*>(sm + S::PIPE_PP) + q * NE;
        if (step_tile<ST, WALLS, LANGMUIR, kStep, FLOW, true>(p, io, sm + q * S::STAGE, PP, &full[q], parity, x0, y0))
            return;
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[q]);
    }
}

// After a sequence of n launches: advance every descriptor by n steps.
static __global__ void batch_advance_kernel(InstDesc* __restrict__ descs, int count, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count || n <= 0) return;
    descs[k].steps += n;
    descs[k].cur = (descs[k].cur + n) & 1;
    descs[k].first = 0;
}

// ---- initialisation: equilibria of the given fields, written where the first pull reads them ----
struct InitArgs {
    Phys p;
    const double* __restrict__ phi;
    const double* __restrict__ psi;
    const double* __restrict__ ux;
    const double* __restrict__ uy;
    const double* __restrict__ P;
    void* __restrict__ dst;
    float2* __restrict__ hist;    // history buffer of the initial level
    unsigned* __restrict__ status;
    int langmuir;
    int walls;
    int flow;                     // 0: prescribed velocity, no h populations
};

template <int ST>
__global__ void init_kernel(const __grid_constant__ InitArgs a) {
    using T = Traits<ST>;
    using P = typename T::P;
    using Hv = typename T::H;
    const Phys& p = a.p;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const size_t o = (size_t)y * p.nx + x;
    const double phi = a.phi[o], psi = a.psi[o], ux = a.ux[o], uy = a.uy[o], P_ = a.P[o];
    bool bad = !(isfinite(phi) && isfinite(psi) && isfinite(ux) && isfinite(uy) && isfinite(P_));
    if (a.langmuir) bad = bad || !(psi < 1.0);
    if (bad) atomicOr(a.status, kStatusUnstable);
    // local density (the equilibrium is taken without the mass-flux terms, S = 0)
    const double rho = p.var_rho ? (double)p.rhoB + (phi - (double)p.phiB) * (double)p.drho : (double)p.rho;
    const double uu = ux * ux + uy * uy;
    P* fg = static_cast<P*>(a.dst);
    Hv* hp = reinterpret_cast<Hv*>(fg + (size_t)kPairs * p.plane);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const double cu = cx(i) * ux + cy(i) * uy;
        const double w = i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        const double feq = w * phi * (1.0 + 3.0 * cu);
        const double geq = w * psi * (1.0 + 3.0 * cu);
        const double heq = w * (3.0 * P_ + 3.0 * rho * cu + 4.5 * rho * (cu * cu - uu / 3.0));
        // The first pull at x for direction i reads plane i at x - c_i: there, and at every
        // periodic image of that position in the ghost frame, store this cell's equilibrium value.
        // Across a wall x - c_i is in the wall's ghost row, which holds this cell's bounce-back
        // value (its own opposite slot, same weight).
        int sx = x - cx(i), sy = y - cy(i), enc = i;
        const bool wall_ghost = a.walls && (sy < 0 || sy >= p.ny);
        if (wall_ghost) {
            enc = opp(i);
        } else {
            sx = (sx + p.nx) % p.nx;
            sy = (sy + p.ny) % p.ny;
        }
        P vfg;
        if constexpr (!T::kPair16)
            vfg = make_float2((float)feq, (float)geq);
        else
            vfg = pack2<P>(make_float2((float)((feq / w - p.phi_ref) * T::SF), (float)(geq / w * T::SG)));
        Hv vh{};
        if (i > 0 && a.flow) {
            if constexpr (!T::kH16) {
                vh = (Hv)heq;
            } else {
                // stored relative to the storing cell's velocity, as the step will read it back:
                // the source cell for a plain link, this cell (slot opp(i)) across a wall
                const size_t so = wall_ghost ? o : (size_t)sy * p.nx + sx;
                const double sux = (float)a.ux[so], suy = (float)a.uy[so];
                const double vel = 3.0 * rho * (cx(enc) * sux + cy(enc) * suy);
                vh = pack1<Hv>((float)((heq / w - vel) * T::SH));
            }
        }
        auto at = [&](int c, int r) {
            const long long k = p.org + (long long)r * p.pitch + c;
            fg[(long long)i * p.plane + k] = vfg;
            if (i > 0 && a.flow) hp[h_index(i, k, p.plane)] = vh;
        };
        auto row = [&](int c, int r) {
            at(c, r);
            if (c <= 1) at(c + p.nx, r);
            if (c >= p.nx - 2) at(c - p.nx, r);
        };
        row(sx, sy);
        if (!a.walls) {
            if (sy <= 1) row(sx, sy + p.ny);
            if (sy >= p.ny - 2) row(sx, sy - p.ny);
        }
    }
    const float2 u0 = make_float2((float)ux, (float)uy);
    auto hist_at = [&](int c, int r) { a.hist[p.org + (long long)r * p.pitch + c] = u0; };
    auto hist_row = [&](int c, int r) {
        hist_at(c, r);
        if (c <= 1) hist_at(c + p.nx, r);
        if (c >= p.nx - 2) hist_at(c - p.nx, r);
    };
    if constexpr (Smem<ST>::kHalo) {
        // the images exist where the step maintains them (the 16-bit h decode reads them)
        hist_row(x, y);
        if (!a.walls) {
            if (y <= 1) hist_row(x, y + p.ny);
            if (y >= p.ny - 2) hist_row(x, y - p.ny);
        }
    } else {
        hist_at(x, y);
    }
}

// ---- FP64 sums of phi or psi: every population slot is pulled exactly once per step, so the
// total of a field is the plain sum of one lane of the 9 pair planes over the valid cells ----
constexpr int kReduceThreads = 256;
constexpr int kMaxPartials = 1024;

__device__ __forceinline__ double block_sum(double v, double* smem) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    v = 0.0;
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? smem[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// lane 0 sums f (phi), lane 1 sums g (psi); 16-bit storage is decoded to its value first
template <int ST>
__global__ void __launch_bounds__(kReduceThreads) reduce_partial_kernel(const void* __restrict__ pops, int lane,
                                                                        int nx, int ny, int pitch, long long plane,
                                                                        long long org, Phys p,
                                                                        double* __restrict__ partials) {
    using T = Traits<ST>;
    using P = typename T::P;
    __shared__ double smem[32];
    const P* pairs = static_cast<const P*>(pops);
    double acc = 0.0;
    // block b owns rows b, b + gridDim.x, ...; threads stride over (pair plane, x)
    for (int y = blockIdx.x; y < ny; y += gridDim.x) {
        for (int k = threadIdx.x; k < kPairs * nx; k += blockDim.x) {
            const int i = k / nx, x = k - i * nx;
            const float2 v = raw2(pairs[(size_t)i * plane + (size_t)(org + (long long)y * pitch + x)]);
            if constexpr (!T::kPair16) {
                acc += (double)(lane ? v.y : v.x);
            } else {
                const double w = i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
                acc += lane ? w * (double)v.y / T::SG : w * ((double)v.x / T::SF + p.phi_ref);
            }
        }
    }
    acc = block_sum(acc, smem);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Failure-detection self-test: one warp waits, with the bounded wait of the step kernels, on an
// mbarrier whose phase nothing completes; the wait gives up and the status word records it.  It
// exercises the timeout path without a copy in flight, so nothing faults and the context stays
// usable.
static __global__ void selftest_wait_kernel(unsigned* __restrict__ status) {
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // one arrival expected; none comes
        fence_mbar_init();
    }
    __syncthreads();
    const bool done = mbar_wait_bounded(&bar, 0u);
    if (threadIdx.x == 0) *status = done ? 0u : kStatusTimeout;
}

static __global__ void __launch_bounds__(kReduceThreads) reduce_final_kernel(const double* __restrict__ partials, int n,
                                                                      double* __restrict__ out) {
    __shared__ double smem[32];
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) acc += partials[k];
    acc = block_sum(acc, smem);
    if (threadIdx.x == 0) *out = acc;
}

}  // namespace lbm
