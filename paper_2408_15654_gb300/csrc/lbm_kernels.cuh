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
// Cells per thread: FP32 storage updates one cell per thread, (f, g) and (phi, psi) packed as
// FP32x2 pairs.  The 16-bit modes, whose step is bound by instruction issue rather than by HBM,
// update two horizontally adjacent cells per thread: every per-cell quantity is a pair (cell A,
// cell B), so the arithmetic of both cells issues as one packed instruction, their pairs move in
// 64-bit shared-memory loads and global stores, and the per-thread set-up is shared.  All
// arithmetic is written with explicitly rounded operations (one rounding per operation, in the
// order written), so every kernel built from this source rounds alike.
//
// Velocity order (the columns of the printed moment matrix M, Sec. 4):
//   0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1)
#pragma once
#include <cstdint>
#include <type_traits>
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

// Storage traits: element types, compile-time scales, and the x origin of the h boxes in
// (h_i, h_i+1) pairs (TMA x coordinates must be multiples of 16 bytes: 2 pairs of 8 bytes, 4 of
// 4 bytes; box columns x0 - H_X0 + kGX onwards, TX + 2 H_X0 of them).
template <int ST> struct Traits;
template <> struct Traits<kFP32> {
    using P = float2;
    using H = float;
    static constexpr bool kPair16 = false, kH16 = false;
    static constexpr int H_X0 = 2;  // in (h_i, h_i+1) pairs
    static constexpr float SF = 1.f, SG = 1.f, SH = 1.f;
};
template <> struct Traits<kFP16> {
    using P = __half2;
    using H = __half;
    static constexpr bool kPair16 = true, kH16 = true;
    static constexpr int H_X0 = 4;  // in (h_i, h_i+1) pairs
    static constexpr float SF = 1.f, SG = 256.f, SH = 4096.f;  // keep the deviations normal in FP16
};
template <> struct Traits<kBF16> {
    using P = __nv_bfloat162;
    using H = __nv_bfloat16;
    static constexpr bool kPair16 = true, kH16 = true;
    static constexpr int H_X0 = 4;  // in (h_i, h_i+1) pairs
    static constexpr float SF = 1.f, SG = 1.f, SH = 1.f;        // BF16 has the FP32 exponent range
};
template <> struct Traits<kFP16FG> {
    using P = __half2;
    using H = float;
    static constexpr bool kPair16 = true, kH16 = false;
    static constexpr int H_X0 = 2;  // in (h_i, h_i+1) pairs
    static constexpr float SF = 1.f, SG = 256.f, SH = 1.f;
};
template <> struct Traits<kBF16FG> {
    using P = __nv_bfloat162;
    using H = float;
    static constexpr bool kPair16 = true, kH16 = false;
    static constexpr int H_X0 = 2;  // in (h_i, h_i+1) pairs
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
// the x coordinate of every box a multiple of 16 bytes (boxes start 4 or 8 cells left of a tile)
// and every cell of an even column at an even index (pitch is a multiple of 32), so that the two
// cells of a thread move as one aligned vector.
constexpr int kGX = 8, kGY = 2;

// Index, in h values, of link i's slot at cell k of a buffer's h planes (plane stride `plane`
// cells).  h is stored as pairs (h_2j+1, h_2j+2) in plane j, link 2j+1 first, so that a cell's
// eight values leave in four stores (32-bit for 16-bit h, 64-bit for FP32 h) and the flow
// collision's FP32x2 pairs go out as they are.
__host__ __device__ __forceinline__ long long h_index(int i, long long k, long long plane) {
    return (((long long)((i - 1) >> 1) * plane + k) << 1) + ((i - 1) & 1);
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

// Cells per compute thread of storage mode st (see the file comment).
__host__ __device__ constexpr int cpt_of(int st) { return st == kFP32 ? 1 : 2; }

// Tile geometry of CPT cells per thread.  A CTA's NT compute threads own a TX x TY tile, TX / CPT
// threads per tile row, thread t the CPT cells from (x0 + (t % TPR) CPT, y0 + t / TPR).  TMA stages:
//   pair plane i: box of BW x BH pairs,    row r, col c <-> (x0 - 4 + c, y0 - 1 - cy(i) + r)
//   h plane j:    box of TX + 2 H_X0 x (TY + 1) (h_2j+1, h_2j+2) pairs, from row y0 + h_row0(j)
//   u history:    box of TX x TY, or BW x BH (one-cell ring) when h is 16-bit, float2
// so extended-tile cell (ex, ey) (global (x0 - 1 + ex, y0 - 1 + ey)) pulls pair i from
// [ey][ex + 3 - cx(i)], and the own cell (tx, ty)'s unshifted post-collision pair i sits at
// [ty + 1 + cy(i)][tx + 4].  The (phi, psi) exchange tile PP holds extended cell (ex, ey) at
// ey EXP + ex + PPO; with two cells per thread the offset puts a thread's first cell at an even
// index, so its two cells are one 16-byte access.
template <int CPT> struct Geo {
    static constexpr int TX = 32, TY = CPT == 1 ? 8 : 4 * CPT;
    static constexpr int TPR = TX / CPT;        // threads per tile row
    static constexpr int NT = TPR * TY;         // compute threads
    static constexpr int BW = TX + 8, BH = TY + 2;
    static constexpr int FG_BOX = BW * BH;      // pairs per pair-plane box
    static constexpr int EX = TX + 2, EY = TY + 2;
    static constexpr int PPO = CPT == 1 ? 0 : 1;
    static constexpr int EXP = EX + 2 * PPO;
    static constexpr int NE = EXP * EY;
    static constexpr int NRING = 2 * EX + 2 * TY;
    static_assert(NRING <= NT, "one thread per ring cell");
    static_assert(NT % 32 == 0, "whole warps");
};
template <int ST> using GeoOf = Geo<cpt_of(ST)>;

// First row of h box j relative to the tile's first row: the lower source row of its links.
__host__ __device__ constexpr int h_row0(int j) {
    return -(cy(2 * j + 1) > cy(2 * j + 2) ? cy(2 * j + 1) : cy(2 * j + 2));
}

constexpr unsigned kSuspendNs = 200000;    // sleep hint of one wait attempt
constexpr unsigned kWaitLimit = 5000;      // attempts: the wait ends within ~1 s
constexpr unsigned kStatusUnstable = 1u, kStatusTimeout = 2u;

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
    using G = GeoOf<ST>;
    static constexpr bool kHalo = T::kH16;  // the 16-bit h decode needs the source cell's u
    static constexpr int FG_SLOT = round128(G::FG_BOX * (int)sizeof(typename T::P));
    // h boxes: one per plane of pairs (h_2j+1, h_2j+2), spanning the rows of both links (TY + 1)
    static constexpr int H_SLOTS = kHPlanes / 2;
    static constexpr int H_ES = 2 * (int)sizeof(typename T::H);
    static constexpr int H_BW = G::TX + 2 * T::H_X0, H_BH = G::TY + 1;
    static constexpr int H_BOX = H_BW * H_BH;
    static constexpr int H_SLOT = round128(H_BOX * H_ES);
    static constexpr int HIST_W = kHalo ? G::BW : G::TX, HIST_H = kHalo ? G::BH : G::TY;
    static constexpr int HIST_BYTES = HIST_W * HIST_H * 8;
    static constexpr int FG = 0;
    static constexpr int H = FG + kPairs * FG_SLOT;
    static constexpr int HIST = H + H_SLOTS * H_SLOT;
    static constexpr int PP = HIST + round128(HIST_BYTES);
    static constexpr int PP_BYTES = round128(G::NE * 8);
    static constexpr int BAR = PP + PP_BYTES;
    static constexpr int BYTES = BAR + 16;
    // batched kernel: the lattice's constants
    static constexpr int PHYS = BYTES;
    static constexpr int BYTES_BATCH = PHYS + (int)((sizeof(Phys) + 15) / 16 * 16);
    // warp-specialised persistent kernel: two stages of the TMA boxes ([0, PP) each), two
    // (phi, psi) tiles (alternating with the tile count), a full and an empty mbarrier per stage,
    // the tile origin (x0, y0) of each stage
    static constexpr int STAGE = PP;
    static constexpr int PIPE_PP = 2 * STAGE;
    static constexpr int PIPE_BAR = PIPE_PP + 2 * PP_BYTES;
    static constexpr int PIPE_SLOT = PIPE_BAR + 32;
    static constexpr int BYTES_PIPE = PIPE_SLOT + 16;
    // warp-specialised batch kernel: the same buffers and barriers, a 4-word slot per buffer
    // (x0, y0, lattice, current population buffer) and per buffer the lattice's constants
    static constexpr int PHYS_BYTES = (int)sizeof(Phys);
    static constexpr int BWS_SLOT = PIPE_BAR + 32;
    static constexpr int BWS_PHYS = BWS_SLOT + 32;
    static constexpr int BYTES_BWS = BWS_PHYS + 2 * PHYS_BYTES;
    static constexpr unsigned TX_BYTES =
        (unsigned)(kPairs * G::FG_BOX * sizeof(typename T::P) + H_SLOTS * H_BOX * H_ES + HIST_BYTES);
    static constexpr unsigned TX_BYTES_NOH = (unsigned)(kPairs * G::FG_BOX * sizeof(typename T::P) + HIST_BYTES);
};


struct StepArgs {
    CUtensorMap tm_fg;            // {pitch, rows, 9} pairs, box {BW, BH, 1}
    CUtensorMap tm_h;             // {pitch, rows, 4} h pairs, box {H_BW, TY + 1, 1}
    CUtensorMap tm_hist;          // {pitch, rows, 1} float2, box {TX, TY, 1} or {BW, BH, 1}
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

// ---- explicitly rounded arithmetic ----
// C is the per-cell value of a thread's CPT cells (float, or the pair (cell A, cell B)); PV is a
// pair of such values, (f, g), (phi, psi), (x, y) or two links, packed as one float2 for one cell
// and as two cell pairs for two.  Every operation rounds once per lane, so a lane gives the same
// bits whichever packing carries it.
struct PV2 {
    float2 a, b;
};
template <int CPT> struct CellT;
template <> struct CellT<1> {
    using C = float;
    using PV = float2;
};
template <> struct CellT<2> {
    using C = float2;
    using PV = PV2;
};

__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vneg(float2 a) { return __fmul2_rn(a, make_float2(-1.f, -1.f)); }
__device__ __forceinline__ PV2 vadd(PV2 a, PV2 b) { return {vadd(a.a, b.a), vadd(a.b, b.b)}; }
__device__ __forceinline__ PV2 vsub(PV2 a, PV2 b) { return {vsub(a.a, b.a), vsub(a.b, b.b)}; }
__device__ __forceinline__ PV2 vmul(PV2 a, PV2 b) { return {vmul(a.a, b.a), vmul(a.b, b.b)}; }
__device__ __forceinline__ PV2 vfma(PV2 a, PV2 b, PV2 c) { return {vfma(a.a, b.a, c.a), vfma(a.b, b.b, c.b)}; }

// a value for every cell
template <typename C> __device__ __forceinline__ C bcv(float v);
template <> __device__ __forceinline__ float bcv<float>(float v) { return v; }
template <> __device__ __forceinline__ float2 bcv<float2>(float v) { return make_float2(v, v); }
// a pair from its two lanes, and the lanes of a pair
__device__ __forceinline__ float2 mkpv(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ PV2 mkpv(float2 a, float2 b) { return {a, b}; }
__device__ __forceinline__ float la(float2 v) { return v.x; }
__device__ __forceinline__ float lb(float2 v) { return v.y; }
__device__ __forceinline__ float2 la(const PV2& v) { return v.a; }
__device__ __forceinline__ float2 lb(const PV2& v) { return v.b; }
// a pair with the lane values (a, b) for every cell
template <typename PV> __device__ __forceinline__ PV pvk(float a, float b);
template <> __device__ __forceinline__ float2 pvk<float2>(float a, float b) { return make_float2(a, b); }
template <> __device__ __forceinline__ PV2 pvk<PV2>(float a, float b) { return {make_float2(a, a), make_float2(b, b)}; }
// f(v) on every cell's value (library calls that have no packed form)
template <typename F> __device__ __forceinline__ float lanes(float v, F f) { return f(v); }
template <typename F> __device__ __forceinline__ float2 lanes(float2 v, F f) { return make_float2(f(v.x), f(v.y)); }
// the value of cell l
__device__ __forceinline__ float cell_of(float v, int) { return v; }
__device__ __forceinline__ float cell_of(float2 v, int l) { return l ? v.y : v.x; }
// the (lane a, lane b) pair of cell l
__device__ __forceinline__ float2 cell_of(float2 v, int, int) { return v; }
__device__ __forceinline__ float2 cell_of(const PV2& v, int l, int) { return l ? make_float2(v.a.y, v.b.y) : make_float2(v.a.x, v.b.x); }

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
// half `hi` of a 32-bit word holding two 16-bit values, in FP32
template <typename H> __device__ __forceinline__ float half_of(uint32_t w, int hi);
template <> __device__ __forceinline__ float half_of<__half>(uint32_t w, int hi) {
    return __half2float(__ushort_as_half((unsigned short)(hi ? w >> 16 : w & 0xFFFFu)));
}
template <> __device__ __forceinline__ float half_of<__nv_bfloat16>(uint32_t w, int hi) {
    return __uint_as_float(hi ? (w & 0xFFFF0000u) : (w << 16));
}

// Two storage values side by side, aligned for one vector access.
template <typename P> struct alignas(2 * sizeof(P)) Two {
    P v0, v1;
};

// 16-bit storage holds r_i = (f_i / w_i - phi_ref) S_f and g_i / w_i S_g.  The decode constant
// w_i / S is not a binary fraction (w_i = 4/9, 1/9, 1/36), so the stored state is never decoded
// and re-encoded: the step computes its moments from r (each weight class summed raw and scaled
// once; the constant's ~1e-8 relative error then only touches the physics) and writes
// r* = r + (S / w_i) dq_i, the increment of the collision scaled by the exact constant S / w_i.
// A resting bulk, whose increments are below half an FP32 ulp of r, keeps its stored values
// exactly, and the totals of phi and psi carry no coherent decode error.
__host__ __device__ constexpr double wgt_d(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }
// decode constant w_i / S of link i as an (f, g) pair
template <int ST, int I, typename PV> __device__ __forceinline__ PV kdec() {
    using T = Traits<ST>;
    return pvk<PV>((float)(wgt_d(I) / T::SF), (float)(wgt_d(I) / T::SG));
}
// c S / w_i of link i (exact in FP32: 1 / w_i is 9/4, 9 or 36 and S a power of two)
template <int ST, int I, typename PV> __device__ __forceinline__ PV kenc(double c) {
    using T = Traits<ST>;
    return pvk<PV>((float)(c * T::SF / wgt_d(I)), (float)(c * T::SG / wgt_d(I)));
}

// c + h for a 16-bit storage value h: h is widened exactly and the sum rounded once (one
// mixed-precision add, no separate conversion)
__device__ __forceinline__ float addh(float c, __half h) {
    float d;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(__half_as_ushort(h)), "f"(c));
    return d;
}
__device__ __forceinline__ float addh(float c, __nv_bfloat16 h) {
    float d;
    asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(__bfloat16_as_ushort(h)), "f"(c));
    return d;
}
__device__ __forceinline__ __half lo16(__half2 v) { return __low2half(v); }
__device__ __forceinline__ __half hi16(__half2 v) { return __high2half(v); }
__device__ __forceinline__ __nv_bfloat16 lo16(__nv_bfloat162 v) { return __low2bfloat16(v); }
__device__ __forceinline__ __nv_bfloat16 hi16(__nv_bfloat162 v) { return __high2bfloat16(v); }
// ((a + b) + c) + d in FP32 of the f (HI = false) or the g halves (HI = true) of four stored pairs
template <bool HI, typename P> __device__ __forceinline__ float class_sum(P a, P b, P c, P d) {
    if constexpr (HI) return addh(addh(addh(raw1(hi16(a)), hi16(b)), hi16(c)), hi16(d));
    else return addh(addh(addh(raw1(lo16(a)), lo16(b)), lo16(c)), lo16(d));
}
// (phi, psi) of one cell from its nine stored pairs v[i] (link i): FP32 storage sums the values;
// 16-bit storage sums the raw values of each weight class (links 1-4, links 5-8) and scales each
// class sum, and link 0, once by its decode constant
template <int ST> __device__ __forceinline__ float2 pair_sum1(const typename Traits<ST>::P (&v)[9], float2 ref) {
    if constexpr (!Traits<ST>::kPair16) {
        float2 s = ref;
#pragma unroll
        for (int i = 0; i < 9; ++i) s = vadd(s, v[i]);
        return s;
    } else {
        const float2 ax = make_float2(class_sum<false>(v[1], v[3], v[2], v[4]), class_sum<true>(v[1], v[3], v[2], v[4]));
        const float2 dg = make_float2(class_sum<false>(v[5], v[7], v[6], v[8]), class_sum<true>(v[5], v[7], v[6], v[8]));
        return vfma(dg, kdec<ST, 5, float2>(),
                    vfma(ax, kdec<ST, 1, float2>(), vfma(raw2(v[0]), kdec<ST, 0, float2>(), ref)));
    }
}
// The same for the thread's cells, v[i][l] link i of cell l: the lanes of each (phi, psi) pair are
// the cells, with the arithmetic of pair_sum1 per cell
template <int ST>
__device__ __forceinline__ typename CellT<cpt_of(ST)>::PV pair_sum(const typename Traits<ST>::P (&v)[9][cpt_of(ST)],
                                                                   typename CellT<cpt_of(ST)>::PV ref) {
    if constexpr (cpt_of(ST) == 1) {
        float2 s = ref;
#pragma unroll
        for (int i = 0; i < 9; ++i) s = vadd(s, raw2(v[i][0]));
        return s;
    } else {
        auto cls = [&](int a, int b, int c, int d, auto hi) {
            return make_float2(class_sum<decltype(hi)::value>(v[a][0], v[b][0], v[c][0], v[d][0]),
                               class_sum<decltype(hi)::value>(v[a][1], v[b][1], v[c][1], v[d][1]));
        };
        using F = std::false_type;
        using T = std::true_type;
        const PV2 ax{cls(1, 3, 2, 4, F{}), cls(1, 3, 2, 4, T{})}, dg{cls(5, 7, 6, 8, F{}), cls(5, 7, 6, 8, T{})};
        const float2 a0 = raw2(v[0][0]), b0 = raw2(v[0][1]);
        const PV2 r0{make_float2(a0.x, b0.x), make_float2(a0.y, b0.y)};
        return vfma(dg, kdec<ST, 5, PV2>(), vfma(ax, kdec<ST, 1, PV2>(), vfma(r0, kdec<ST, 0, PV2>(), ref)));
    }
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
// a scaled (f_i, g_i) pair r* of one cell to stochastically rounded 16-bit storage
template <int ST> __device__ __forceinline__ typename Traits<ST>::P enc_pair_rs(float2 v, uint32_t key, int i) {
    using T = Traits<ST>;
    const uint32_t bits = cvt_rs2<typename T::P>(v.x, v.y, rbits_of(key, i));
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
// Named barrier 1 of the N compute threads of a warp-specialised CTA (its copy warp never takes
// part); the OR form also tells every thread whether any of them passed true.
template <int N> __device__ __forceinline__ void compute_sync() { asm volatile("bar.sync 1, %0;\n" ::"n"(N) : "memory"); }
template <int N> __device__ __forceinline__ bool compute_sync_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 1, %2, q;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(N)
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

// Moment-space MRT collision of the phase-field and surfactant populations, applied as an
// increment so that FP32 rounding stays at the scale of the departure from equilibrium (in a
// uniform bulk nothing changes):
//   m = M q;  dm_k = -s_k (m_k - m_eq_k) + (1 - s_k/2) m_src_k;  q* = q + M^-1 dm.
// For a scalar s (phi or psi) the equilibrium w_i s (1 + c_i.u/cs2) has moments
// (s, s ux, s uy, s/3, s/3, 0, s ux/3, s uy/3, s/9); the source w_i c_i.V has moments
// (0, cs2 Vx, cs2 Vy, 0, 0, 0, Vx/9, Vy/9, 0) with cs2 V = (vx, vy).  dm_0 = 0.
// q may hold deviations q_i - w_i r (r per lane): the odd moments are unchanged, the even ones
// drop r times (1, 1/3, 1/3, 1/9), so they are compared with sr = s - r.
// The two lanes of every float2 are two independent collisions: LANES = kLanesFG collides (f, g)
// of one cell, kLanesF or kLanesG the f or the g populations of two cells.  nS_k = -s_k and
// K_k = 1 - s_k/2 per lane.
// FP32 storage: q holds the values and becomes q*.  16-bit storage: q holds the raw stored values r
// and becomes r* = r + (S / w_i) (M^-1 dm)_i (the moments come from r, each weight class scaled by
// its decode constant once).
enum Lanes { kLanesF = 0, kLanesG = 1, kLanesFG = 2 };
// per-lane constant of the f and the g population
template <int LANES> __device__ __forceinline__ float2 lane_k(float f, float g) {
    return LANES == kLanesFG ? make_float2(f, g) : (LANES == kLanesF ? make_float2(f, f) : make_float2(g, g));
}
template <int ST, int LANES, int I> __device__ __forceinline__ float2 kdec_l() {
    using T = Traits<ST>;
    return lane_k<LANES>((float)(wgt_d(I) / T::SF), (float)(wgt_d(I) / T::SG));
}
template <int ST, int LANES, int I> __device__ __forceinline__ float2 kenc_l(double c) {
    using T = Traits<ST>;
    return lane_k<LANES>((float)(c * T::SF / wgt_d(I)), (float)(c * T::SG / wgt_d(I)));
}
template <int ST, int LANES>
__device__ __forceinline__ void collide_lanes(float2 q[9], float2 s, float2 sr, float2 ux, float2 uy, float2 vx,
                                              float2 vy, float2 nS1, float2 nS2, float2 nS3, float2 nS4, float2 K1,
                                              float2 K3) {
    constexpr bool raw = Traits<ST>::kPair16;
    const float2 third = make_float2(1.f / 3.f, 1.f / 3.f);
    const float2 a = vadd(q[5], q[7]), b = vadd(q[6], q[8]), c = vsub(q[5], q[7]), d = vsub(q[6], q[8]);
    float2 m1, m2, m3, m4, m5, m6, m7, m8;
    if constexpr (!raw) {
        m5 = vsub(a, b), m8 = vadd(a, b), m6 = vsub(c, d), m7 = vadd(c, d);
        m1 = vadd(vsub(q[1], q[3]), m6), m2 = vadd(vsub(q[2], q[4]), m7);
        m3 = vadd(vadd(q[1], q[3]), m8), m4 = vadd(vadd(q[2], q[4]), m8);
    } else {
        const float2 kax = kdec_l<ST, LANES, 1>(), kdg = kdec_l<ST, LANES, 5>();
        m5 = vmul(kdg, vsub(a, b)), m8 = vmul(kdg, vadd(a, b)), m6 = vmul(kdg, vsub(c, d)), m7 = vmul(kdg, vadd(c, d));
        m1 = vfma(kax, vsub(q[1], q[3]), m6), m2 = vfma(kax, vsub(q[2], q[4]), m7);
        m3 = vfma(kax, vadd(q[1], q[3]), m8), m4 = vfma(kax, vadd(q[2], q[4]), m8);
    }
    const float2 su = vmul(s, ux), sv = vmul(s, uy), s3 = vmul(sr, third);
    const float2 d1 = vfma(nS1, vsub(m1, su), vmul(K1, vx));
    const float2 d2 = vfma(nS1, vsub(m2, sv), vmul(K1, vy));
    const float2 d3 = vmul(nS2, vsub(m3, s3));
    const float2 d4 = vmul(nS2, vsub(m4, s3));
    const float2 d5 = vmul(nS2, m5);
    const float2 mthird = make_float2(-1.f / 3.f, -1.f / 3.f);
    const float2 d6 = vfma(nS3, vfma(su, mthird, m6), vmul(K3, vmul(vx, third)));
    const float2 d7 = vfma(nS3, vfma(sv, mthird, m7), vmul(K3, vmul(vy, third)));
    const float2 d8 = vmul(nS4, vfma(sr, make_float2(-1.f / 9.f, -1.f / 9.f), m8));
    const float2 A = vsub(d1, d6), B = vsub(d3, d8), C_ = vsub(d2, d7), D = vsub(d4, d8);
    const float2 E = vadd(d8, d5), F = vsub(d8, d5), G = vadd(d6, d7), H = vsub(d7, d6);
    if constexpr (!raw) {
        const float2 half = make_float2(0.5f, 0.5f), quarter = make_float2(0.25f, 0.25f);
        q[0] = vadd(q[0], vsub(vsub(d8, d3), d4));
        q[1] = vfma(half, vadd(A, B), q[1]);
        q[3] = vfma(half, vsub(B, A), q[3]);
        q[2] = vfma(half, vadd(C_, D), q[2]);
        q[4] = vfma(half, vsub(D, C_), q[4]);
        q[5] = vfma(quarter, vadd(E, G), q[5]);
        q[7] = vfma(quarter, vsub(E, G), q[7]);
        q[6] = vfma(quarter, vadd(F, H), q[6]);
        q[8] = vfma(quarter, vsub(F, H), q[8]);
    } else {
        q[0] = vfma(kenc_l<ST, LANES, 0>(1.0), vsub(vsub(d8, d3), d4), q[0]);
        q[1] = vfma(kenc_l<ST, LANES, 1>(0.5), vadd(A, B), q[1]);
        q[3] = vfma(kenc_l<ST, LANES, 3>(0.5), vsub(B, A), q[3]);
        q[2] = vfma(kenc_l<ST, LANES, 2>(0.5), vadd(C_, D), q[2]);
        q[4] = vfma(kenc_l<ST, LANES, 4>(0.5), vsub(D, C_), q[4]);
        q[5] = vfma(kenc_l<ST, LANES, 5>(0.25), vadd(E, G), q[5]);
        q[7] = vfma(kenc_l<ST, LANES, 7>(0.25), vsub(E, G), q[7]);
        q[6] = vfma(kenc_l<ST, LANES, 6>(0.25), vadd(F, H), q[6]);
        q[8] = vfma(kenc_l<ST, LANES, 8>(0.25), vsub(F, H), q[8]);
    }
}

// The stored (f, g) pairs of the thread's cells at src (AL: one aligned vector load).
template <int ST>
__device__ __forceinline__ void ld_raw(const typename Traits<ST>::P* src, bool AL, typename Traits<ST>::P (&v)[cpt_of(ST)]) {
    using P = typename Traits<ST>::P;
    if constexpr (cpt_of(ST) == 1) {
        v[0] = *src;
    } else if (AL) {
        const Two<P> w = *reinterpret_cast<const Two<P>*>(src);
        v[0] = w.v0;
        v[1] = w.v1;
    } else {
        v[0] = src[0];
        v[1] = src[1];
    }
}

// Gradients and Laplacian of (phi, psi) at one cell from its 3 x 3 neighbourhood (C the cell):
//   d_a = (1/cs2) sum w_i c_ia q(x+c_i);  lap = (2/cs2) sum_{i>0} w_i (q_i - q)
struct Stencil {
    float2 gX, gY, lap;  // (phi, psi) lanes
};
__device__ __forceinline__ Stencil stencil9(float2 C_, float2 E, float2 W, float2 N, float2 S, float2 NE, float2 NW,
                                            float2 SE, float2 SW) {
    const float2 third = make_float2(1.f / 3.f, 1.f / 3.f), twelfth = make_float2(1.f / 12.f, 1.f / 12.f);
    Stencil s;
    s.gX = vfma(vsub(vadd(NE, SE), vadd(NW, SW)), twelfth, vmul(vsub(E, W), third));
    s.gY = vfma(vsub(vadd(NE, NW), vadd(SE, SW)), twelfth, vmul(vsub(N, S), third));
    const float2 axis = vadd(vadd(E, W), vadd(N, S)), diag = vadd(vadd(NE, NW), vadd(SE, SW));
    s.lap = vmul(vfma(make_float2(4.f, 4.f), axis, vfma(make_float2(-20.f, -20.f), C_, diag)),
                 make_float2(1.f / 6.f, 1.f / 6.f));
    return s;
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

// Flow population I of the thread's cells, pulled from the staged h boxes.  16-bit h: plus the
// first-order velocity part 3 w_I rho_ref c_I.u(x_s) of the cell x_s that stored the slot (the
// source cell x - c_I, whose u is in the history box; across a wall the cell itself, whose
// opposite slot it is, stored with its own u).
template <int ST, int I, typename C>
__device__ __forceinline__ C load_h(const unsigned char* sm, const float2* Hist, const Phys& p, int tx, int ty, bool bb,
                                    C uox, C uoy) {
    using T = Traits<ST>;
    using S = Smem<ST>;
    using G = GeoOf<ST>;
    constexpr int CPT = cpt_of(ST);
    constexpr int j = (I - 1) / 2, half = (I - 1) & 1;   // the box (pair plane) and the half holding link I
    constexpr int dr = -cy(I) - h_row0(j);               // the source row's offset inside it
    const int e = (ty + dr) * S::H_BW + tx + T::H_X0 - cx(I);
    constexpr float dh = (float)(wgt_d(I) / T::SH);      // one decode constant: h has no conserved
                                                         // zeroth moment, and the collision relaxes
                                                         // its ~1e-8 relative error away every step
    const float k = I <= 4 ? p.kh_axis : p.kh_diag;
    const float kx = (float)cx(I) * k, ky = (float)cy(I) * k;
    // 3 w rho c.u of one source cell, or of the own cell's reflection across a wall
    auto vel = [&](float ux, float uy) {
        if constexpr (cx(I) == 0) return vmul(ky, uy);
        else if constexpr (cy(I) == 0) return vmul(kx, ux);
        else return vfma(kx, ux, vmul(ky, uy));
    };
    // the source cells' u in the history box (which has a one-cell ring when h is 16-bit)
    const float2* us = Hist + (ty + 1 - cy(I)) * G::BW + tx + 4 - cx(I);
    if constexpr (CPT == 1) {
        if constexpr (!T::kH16) {
            const float* box = reinterpret_cast<const float*>(sm + S::H + j * S::H_SLOT);
            return box[2 * e + half];
        } else {
            const typename T::H* box = reinterpret_cast<const typename T::H*>(sm + S::H + j * S::H_SLOT);
            const float r = raw1(box[2 * e + half]);
            float v;
            if (bb) {
                v = vel(vneg(uox), vneg(uoy));
            } else {
                const float2 u = us[0];
                v = vel(u.x, u.y);
            }
            return vfma(r, dh, v);
        }
    } else {
        if constexpr (!T::kH16) {
            const float* box = reinterpret_cast<const float*>(sm + S::H + j * S::H_SLOT);
            return make_float2(box[2 * e + half], box[2 * e + 2 + half]);
        } else {
            const uint32_t* box = reinterpret_cast<const uint32_t*>(sm + S::H + j * S::H_SLOT);
            uint32_t w0, w1;
            if constexpr (cx(I) == 0) {
                const uint2 w = *reinterpret_cast<const uint2*>(box + e);
                w0 = w.x;
                w1 = w.y;
            } else {
                w0 = box[e];
                w1 = box[e + 1];
            }
            const float2 r = make_float2(half_of<typename T::H>(w0, half), half_of<typename T::H>(w1, half));
            float2 v;
            if (bb) {
                v = make_float2(vel(-uox.x, -uoy.x), vel(-uox.y, -uoy.y));
            } else if constexpr (cx(I) == 0) {
                const float4 u = *reinterpret_cast<const float4*>(us);
                v = make_float2(vel(u.x, u.y), vel(u.z, u.w));
            } else {
                const float2 u0 = us[0], u1 = us[1];
                v = make_float2(vel(u0.x, u0.y), vel(u1.x, u1.y));
            }
            return vfma(r, make_float2(dh, dh), v);
        }
    }
}

// One fused step (kStep) or the macroscopic fields of the current level (kMoments) for one tile,
// after one thread has issued the tile's TMA loads into `stage` on `mbar`, whose phase of this
// tile has parity `parity`; PP holds the tile's (phi, psi).  Returns true (uniformly) if a copy
// did not arrive within its bounded wait (nothing stored).  The pulled (f, g) of the tile and of
// a one-cell ring give (phi, psi) for the 9-point stencils; the same boxes hold the own cell's
// unshifted post-collision values, whose sums are phi and psi of the previous level
// (m*_0 = phi exactly, Sec. 3.1), so only u of the previous level is stored.
// WS: called by the compute warps of a warp-specialised CTA, which synchronise among themselves
// with named barrier 1 only (the copy warp has staged the tile and waits on its own barriers).
// EDGE = false: the tile is interior (tile_is_interior): every cell and every ring cell lies in
// the grid away from its edges, so no cell writes ghost-frame copies, meets a wall or lies beyond
// the grid, and those tests compile away.  The arithmetic is the same on both paths.
template <int ST, bool WALLS, bool LANGMUIR, int MODE, int FLOW, bool WS = false, bool EDGE = true>
__device__ __forceinline__ bool step_tile(const Phys& p, const TileIO& io, unsigned char* sm, float2* PP,
                                          unsigned long long* mbar, uint32_t parity, int x0, int y0) {
    using T = Traits<ST>;
    using S = Smem<ST>;
    using P = typename T::P;
    constexpr int CPT = cpt_of(ST);
    using G = Geo<CPT>;
    using C = typename CellT<CPT>::C;
    using PV = typename CellT<CPT>::PV;
    constexpr bool var = FLOW == kFlowVarRho;
    static_assert(CPT == 1 || T::kPair16, "two cells per thread only for 16-bit pairs");
    const P* FG = reinterpret_cast<const P*>(sm + S::FG);
    const float2* Hist = reinterpret_cast<const float2*>(sm + S::HIST);
    const int t = threadIdx.x;
    if constexpr (!WS) __syncthreads();
    bool abort = !mbar_wait_bounded(mbar, parity);

    const int tx = (t % G::TPR) * CPT, ty = t / G::TPR;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = !EDGE || ((x < p.nx) && (y < p.ny));
    const bool act1 = CPT == 2 && (!EDGE || (active && x + 1 < p.nx));  // the thread's second cell
    const long long cell = p.org + (long long)y * p.pitch + x;
    // mass flux of the previous step (density ratio != 1 only; the own cells', read early so that
    // its latency overlaps the stencil work)
    C Spx = bcv<C>(0.f), Spy = bcv<C>(0.f);
    if constexpr (var) {
        if (!io.first && active) {
            if constexpr (CPT == 1) {
                const float2 s = io.shist_src[cell];
                Spx = s.x;
                Spy = s.y;
            } else if (act1) {
                const float4 s = *reinterpret_cast<const float4*>(io.shist_src + cell);
                Spx = make_float2(s.x, s.z);
                Spy = make_float2(s.y, s.w);
            } else {
                const float2 s = io.shist_src[cell];
                Spx = make_float2(s.x, 0.f);
                Spy = make_float2(s.y, 0.f);
            }
        }
    }
    // (phi, psi) references of the stored deviations (zero for FP32 storage)
    const PV ref = pvk<PV>(T::kPair16 ? p.phi_ref : 0.f, 0.f);

    // ---- (phi, psi) of the extended tile: the own cells (pulled pairs kept for the collision)
    //      and the ring; cells beyond a wall take the value of the adjacent fluid row ----
    const int eo = (ty + 1) * G::EXP + tx + 1 + G::PPO;
    constexpr int SLOT = S::FG_SLOT / (int)sizeof(P);
    // the pulled pairs: summed here, and loaded again from the staged boxes for the collision, so
    // that they hold no registers through the rest of the cell update
    PV pp;  // (phi, psi)
    const P* pull = FG + ((EDGE && WALLS && y >= p.ny) ? p.ny - y0 : ty + 1) * G::BW + tx + 4;
    {
        P v[9][CPT];
#pragma unroll
        for (int i = 0; i < 9; ++i) ld_raw<ST>(pull + i * SLOT - cx(i), cx(i) == 0, v[i]);
        pp = pair_sum<ST>(v, ref);
        if constexpr (CPT == 1) PP[eo] = pp;
        else *reinterpret_cast<float4*>(PP + eo) = make_float4(pp.a.x, pp.b.x, pp.a.y, pp.b.y);
    }
    if (t < G::NRING) {
        int ex, ey;
        if (t < G::EX) { ex = t; ey = 0; }
        else if (t < 2 * G::EX) { ex = t - G::EX; ey = G::EY - 1; }
        else if (t < 2 * G::EX + G::TY) { ex = 0; ey = 1 + t - 2 * G::EX; }
        else { ex = G::EX - 1; ey = 1 + t - 2 * G::EX - G::TY; }
        int row = ey;
        if (EDGE && WALLS) {
            const int gy = y0 - 1 + ey;
            if (gy < 0) row = 1 - y0;
            else if (gy >= p.ny) row = p.ny - y0;
        }
        const P* base = FG + row * G::BW + ex + 3;
        P r[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) r[i] = base[i * SLOT - cx(i)];
        PP[ey * G::EXP + ex + G::PPO] = pair_sum1<ST>(r, make_float2(T::kPair16 ? p.phi_ref : 0.f, 0.f));
    }
    if (WS ? compute_sync_or<G::NT>(abort) : __syncthreads_or(abort)) {
        // a staging copy did not arrive in time: report it, wait (bounded) for it, store nothing
        if (t == 0) {
            atomicOr(io.status, kStatusTimeout);
            mbar_wait_bounded(mbar, parity);
        }
        if constexpr (WS) compute_sync<G::NT>();
        else __syncthreads();
        return true;
    }
    if (!active) return false;

    const C phi = la(pp), psi = lb(pp);

    // isotropic stencils of (phi, psi), per cell with the two fields packed
    C gpx, gpy, gsx, gsy, lap;
    if constexpr (CPT == 1) {
        const Stencil s = stencil9(pp, PP[eo + 1], PP[eo - 1], PP[eo + G::EXP], PP[eo - G::EXP], PP[eo + G::EXP + 1],
                                   PP[eo + G::EXP - 1], PP[eo - G::EXP + 1], PP[eo - G::EXP - 1]);
        gpx = s.gX.x, gsx = s.gX.y, gpy = s.gY.x, gsy = s.gY.y, lap = s.lap.x;
    } else {
        const float2* rS = PP + eo - G::EXP;
        const float2* rN = PP + eo + G::EXP;
        const float4 s2 = *reinterpret_cast<const float4*>(rS), n2 = *reinterpret_cast<const float4*>(rN),
                     o2 = *reinterpret_cast<const float4*>(PP + eo);
        const float2 sA = make_float2(s2.x, s2.y), sB = make_float2(s2.z, s2.w);
        const float2 nA = make_float2(n2.x, n2.y), nB = make_float2(n2.z, n2.w);
        const float2 oA = make_float2(o2.x, o2.y), oB = make_float2(o2.z, o2.w);
        const float2 sW = rS[-1], sE = rS[2], nW = rN[-1], nE = rN[2], oW = PP[eo - 1], oE = PP[eo + 2];
        const Stencil a = stencil9(oA, oB, oW, nA, sA, nB, nW, sB, sW);
        const Stencil b = stencil9(oB, oE, oA, nB, sB, nE, nA, sE, sA);
        gpx = make_float2(a.gX.x, b.gX.x), gsx = make_float2(a.gX.y, b.gX.y);
        gpy = make_float2(a.gY.x, b.gY.x), gsy = make_float2(a.gY.y, b.gY.y);
        lap = make_float2(a.lap.x, b.lap.x);
    }

    // interface normal and the delta-function terms (Sec. 2.2, Secs. 3.1-3.2)
    const C g2 = vfma(gpx, gpx, vmul(gpy, gpy));
    C nx_, ny_;
    {
        const float eps2 = p.n_eps2;
        const C r = lanes(g2, [eps2](float v) { return v > eps2 ? rsqrtf(v) : 0.f; });
        nx_ = vmul(gpx, r);
        ny_ = vmul(gpy, r);
    }
    const C dA = vsub(bcv<C>(p.phiA), phi), dB = vsub(phi, bcv<C>(p.phiB));
    const C sym = vfma(bcv<C>(-2.f), phi, bcv<C>(__fadd_rn(p.phiA, p.phiB)));
    const C dAB = vmul(dA, dB);
    const C Aterm = vmul(bcv<C>(p.cA), dAB);
    const C Bterm = vmul(vmul(bcv<C>(p.cA), psi), sym);

    // EOS and surface-tension force: capillary + Marangoni, expanded form (Sec. 2.3); F_b = rho g.
    // ndsig = -d sigma / d psi; the gradient of sigma is taken by the chain rule.
    C sigma, ndsig;
    if constexpr (LANGMUIR) {
        const C om = vsub(bcv<C>(1.f), psi);
        sigma = vmul(bcv<C>(p.sigma0), vfma(bcv<C>(p.E0), lanes(om, [](float o) { return __logf(o); }), bcv<C>(1.f)));
        const float kE = __fmul_rn(p.sigma0, p.E0);
        ndsig = lanes(om, [kE](float o) { return __fdividef(kE, o); });
    } else {
        sigma = vmul(bcv<C>(p.sigma0), vfma(bcv<C>(-p.E0), psi, bcv<C>(1.f)));
        ndsig = bcv<C>(__fmul_rn(p.sigma0, p.E0));
    }
    // density (Sec. 2.3): rho(phi), its gradient by the chain rule, and the mass flux S
    C rho_v = bcv<C>(0.f), grx = bcv<C>(0.f), gry = bcv<C>(0.f), Sx = bcv<C>(0.f), Sy = bcv<C>(0.f);
    if constexpr (var) {
        rho_v = vfma(vsub(phi, bcv<C>(p.phiB)), bcv<C>(p.drho), bcv<C>(p.rhoB));
        grx = vmul(bcv<C>(p.drho), gpx);
        gry = vmul(bcv<C>(p.drho), gpy);
        const C nAterm = vmul(bcv<C>(-p.cA), dAB);
        Sx = vmul(bcv<C>(p.sfac), vfma(nAterm, nx_, gpx));
        Sy = vmul(bcv<C>(p.sfac), vfma(nAterm, ny_, gpy));
    }
    // F = cap grad phi + mar_k [|grad phi|^2 grad sigma - (grad sigma . grad phi) grad phi] + rho g
    const C ngsgx = vmul(ndsig, gsx), ngsgy = vmul(ndsig, gsy);  // -grad sigma
    const C nsdg = vfma(ngsgx, gpx, vmul(ngsgy, gpy));           // -(grad sigma . grad phi)
    const C cap = vmul(vmul(bcv<C>(p.cap_k), sigma), vfma(bcv<C>(p.c16W), vmul(dAB, sym), vmul(bcv<C>(-p.W), lap)));
    const C capm = vfma(bcv<C>(p.mar_k), nsdg, cap);
    const C bm = vmul(bcv<C>(-p.mar_k), g2);
    const C rhoF = var ? rho_v : bcv<C>(p.rho);
    const C Fx = vfma(rhoF, bcv<C>(p.gx), vfma(capm, gpx, vmul(bm, ngsgx)));
    const C Fy = vfma(rhoF, bcv<C>(p.gy), vfma(capm, gpy, vmul(bm, ngsgy)));

    // own u of the previous level (also the encoding velocity of the own slots across a wall)
    C uox, uoy;
    {
        const float2* uo = S::kHalo ? Hist + (ty + 1) * G::BW + tx + 4 : Hist + ty * G::TX + tx;
        if constexpr (CPT == 1) {
            const float2 u = *uo;
            uox = u.x;
            uoy = u.y;
        } else {
            const float4 u = *reinterpret_cast<const float4*>(uo);
            uox = make_float2(u.x, u.z);
            uoy = make_float2(u.y, u.w);
        }
    }

    // flow populations pulled from the staged boxes
    C h[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = bcv<C>(0.f);
    if constexpr (FLOW) {
        const bool bb_up = EDGE && WALLS && y == 0;           // links 2, 5, 6 come from below the bottom wall
        const bool bb_dn = EDGE && WALLS && y == p.ny - 1;    // links 4, 7, 8 come from above the top wall
        h[1] = load_h<ST, 1>(sm, Hist, p, tx, ty, false, uox, uoy);
        h[2] = load_h<ST, 2>(sm, Hist, p, tx, ty, bb_up, uox, uoy);
        h[3] = load_h<ST, 3>(sm, Hist, p, tx, ty, false, uox, uoy);
        h[4] = load_h<ST, 4>(sm, Hist, p, tx, ty, bb_dn, uox, uoy);
        h[5] = load_h<ST, 5>(sm, Hist, p, tx, ty, bb_up, uox, uoy);
        h[6] = load_h<ST, 6>(sm, Hist, p, tx, ty, bb_up, uox, uoy);
        h[7] = load_h<ST, 7>(sm, Hist, p, tx, ty, bb_dn, uox, uoy);
        h[8] = load_h<ST, 8>(sm, Hist, p, tx, ty, bb_dn, uox, uoy);
    }

    // velocity: rho u = sum c_i h_i + F/2 (Sec. 3.3), or the imposed velocity (kept in the history);
    // the links paired as (1, 2), (3, 4), (5, 6), (7, 8)
    PV X = mkpv(h[1], h[2]), Y = mkpv(h[3], h[4]), U = mkpv(h[5], h[6]), V = mkpv(h[7], h[8]);
    const PV dXY = vsub(X, Y), dUV = vsub(U, V);  // (h1 - h3, h2 - h4), (h5 - h7, h6 - h8)
    const C h57 = la(dUV), h68 = lb(dUV);
    const C jx = vadd(la(dXY), vsub(h57, h68));
    const C jy = vadd(lb(dXY), vadd(h57, h68));
    const C inv_rho = var ? lanes(rho_v, [](float r) { return __frcp_rn(r); }) : bcv<C>(p.inv_rho);
    C ux, uy;
    if constexpr (FLOW) {
        ux = vmul(vfma(bcv<C>(0.5f), Fx, jx), inv_rho);
        uy = vmul(vfma(bcv<C>(0.5f), Fy, jy), inv_rho);
    } else {
        ux = uox;
        uy = uoy;
    }

    // previous level: (phi, psi) from the own cells' post-collision pairs, u from history
    PV pprev = pp;
    C uxp = ux, uyp = uy;
    if (!io.first) {
        const P* base = FG + (ty + 1) * G::BW + tx + 4;
        P v[9][CPT];
#pragma unroll
        for (int i = 0; i < 9; ++i) ld_raw<ST>(base + i * SLOT + cy(i) * G::BW, true, v[i]);
        pprev = pair_sum<ST>(v, ref);
        uxp = uox;
        uyp = uoy;
    }

    // time derivatives, backward difference over one step: d_t(phi u), d_t(psi u) as pairs, and
    // d_t(rho u u - (S u + u S)/2) (Sec. 3.3)
    const C rho = var ? rho_v : bcv<C>(p.rho);
    const C nuxp = vneg(uxp), nuyp = vneg(uyp);
    const PV dtX = vfma(pp, mkpv(ux, ux), vmul(pprev, mkpv(nuxp, nuxp)));
    const PV dtY = vfma(pp, mkpv(uy, uy), vmul(pprev, mkpv(nuyp, nuyp)));
    C dt_xx, dt_yy, dt_xy, ugr = bcv<C>(0.f);
    // Q = (rho u - S) u of this level (density ratio only): diagonal and symmetrised off-diagonal
    C Jx = bcv<C>(0.f), Jy = bcv<C>(0.f), qxx = bcv<C>(0.f), qyy = bcv<C>(0.f), qxy = bcv<C>(0.f);
    if constexpr (!var) {
        dt_xx = vmul(rho, vfma(ux, ux, vmul(nuxp, uxp)));
        dt_yy = vmul(rho, vfma(uy, uy, vmul(nuyp, uyp)));
        dt_xy = vmul(rho, vfma(ux, uy, vmul(nuxp, uyp)));
    } else {
        const C mhalf = bcv<C>(-0.5f);
        Jx = vmul(rho, ux);
        Jy = vmul(rho, uy);
        qxx = vmul(vsub(Jx, Sx), ux);
        qyy = vmul(vsub(Jy, Sy), uy);
        qxy = vfma(Jx, uy, vmul(mhalf, vfma(Sx, uy, vmul(Sy, ux))));
        const C rp = vfma(vsub(la(pprev), bcv<C>(p.phiB)), bcv<C>(p.drho), bcv<C>(p.rhoB));  // rho of the previous level
        const C Sxp = io.first ? Sx : Spx, Syp = io.first ? Sy : Spy;
        const C Jxp = vmul(rp, uxp), Jyp = vmul(rp, uyp);
        dt_xx = vsub(qxx, vmul(vsub(Jxp, Sxp), uxp));
        dt_yy = vsub(qyy, vmul(vsub(Jyp, Syp), uyp));
        dt_xy = vsub(qxy, vfma(Jxp, uyp, vmul(mhalf, vfma(Sxp, uyp, vmul(Syp, uxp)))));
        ugr = vfma(ux, grx, vmul(uy, gry));
    }

    // pressure (Eq. for P, Sec. 3.3) with K = w0/(c^2 - cs2) = 2/3:
    //   P = 3/5 [sum_{i>0} h_i + u.grad rho / 2 - (2/3) (rho u - S).u + (1/3) d_t(rho u.u - S.u)]
    const PV sXY = vadd(X, Y), sUV = vadd(U, V);  // (h1 + h3, h2 + h4), (h5 + h7, h6 + h8)
    const C hsum = vadd(vadd(la(sXY), lb(sXY)), vadd(la(sUV), lb(sUV)));
    C P_ = bcv<C>(0.f);
    if constexpr (FLOW) {
        const C third = bcv<C>(1.f / 3.f);
        if constexpr (!var)
            P_ = vmul(bcv<C>(0.6f), vfma(third, vadd(dt_xx, dt_yy),
                                         vfma(bcv<C>(__fmul_rn(-2.f / 3.f, p.rho)), vfma(ux, ux, vmul(uy, uy)), hsum)));
        else
            P_ = vmul(bcv<C>(0.6f), vfma(third, vadd(dt_xx, dt_yy),
                                         vfma(bcv<C>(-2.f / 3.f), vadd(qxx, qyy), vfma(bcv<C>(0.5f), ugr, hsum))));
    }

    {
        // |u| >= 0.3, or a non-finite value (NaN fails every comparison; a NaN anywhere in the
        // cell reaches u, phi or psi within a step), or psi >= 1 under the Langmuir EOS
        auto bad_cell = [&](int l) {
            const float ps = cell_of(psi, l);
            bool b = !(fabsf(cell_of(ux, l)) < 0.3f) | !(fabsf(cell_of(uy, l)) < 0.3f) |
                     !(fabsf(cell_of(phi, l)) < 1e30f) | !(fabsf(ps) < 1e30f);
            if (LANGMUIR) b |= !(ps < 1.f);
            return b;
        };
        bool bad = bad_cell(0);
        if (CPT == 2 && act1) bad |= bad_cell(1);
        if (bad) atomicOr(io.status, kStatusUnstable);
    }

    if constexpr (MODE == kMoments) {
#pragma unroll
        for (int l = 0; l < CPT; ++l) {
            if (l == 1 && !act1) break;
            const size_t o = (size_t)y * p.nx + x + l;
            if (io.out[0]) io.out[0][o] = cell_of(phi, l);
            if (io.out[1]) io.out[1][o] = cell_of(psi, l);
            if (io.out[2]) io.out[2][o] = cell_of(ux, l);
            if (io.out[3]) io.out[3][o] = cell_of(uy, l);
            if (io.out[4]) io.out[4][o] = cell_of(P_, l);
        }
    } else {
        using Hv = typename T::H;
        uint32_t key[CPT];
#pragma unroll
        for (int l = 0; l < CPT; ++l) key[l] = T::kPair16 ? cell_key((uint32_t)(cell + l), io.seed) : 0u;
        // ---- destinations: the own cells, their periodic images in the ghost frame, and at a wall
        //      the bounce-back ghosts of the links that cross it.  putv(c) writes all of the
        //      thread's cells at index c (c even with two cells), put1(c, l) cell l alone, and
        //      putbb(d, i, o, l) the opposite slot o of cell l into link i's plane at index d ----
        const bool yl = EDGE && !WALLS && y <= 1, yr = EDGE && !WALLS && y >= p.ny - 2;
        const bool xedge = EDGE && (x <= 1 || x + CPT - 1 >= p.nx - 2);
        const long long DX = p.nx, DY = (long long)p.ny * p.pitch;
        auto each_dest = [&](auto&& putv, auto&& put1, auto&& putbb) {
            putv(cell);
            if (yl) putv(cell + DY);
            if (yr) putv(cell - DY);
            if (xedge) {
#pragma unroll
                for (int l = 0; l < CPT; ++l) {
                    if (l == 1 && !act1) break;
                    const long long c = cell + l;
                    const bool xl = x + l <= 1, xr = x + l >= p.nx - 2;
                    if (xl) put1(c + DX, l);
                    if (xr) put1(c - DX, l);
                    if (yl) {
                        if (xl) put1(c + DY + DX, l);
                        if (xr) put1(c + DY - DX, l);
                    }
                    if (yr) {
                        if (xl) put1(c - DY + DX, l);
                        if (xr) put1(c - DY - DX, l);
                    }
                }
            }
            if (EDGE && WALLS && (y == 0 || y == p.ny - 1)) {
                // the pull of link i across the wall, at (x - c_ix, -1) or (x - c_ix, ny) in plane i,
                // reads this cell's post-collision opposite slot (half-way bounce-back, Sec. 4)
#pragma unroll
                for (int l = 0; l < CPT; ++l) {
                    if (l == 1 && !act1) break;
                    const long long c0 = cell + l;
                    const int xc = x + l;
                    auto bb = [&](int i, int o, int col, long long c) {
                        putbb(c, i, o, l);
                        if (col <= 1) putbb(c + p.nx, i, o, l);
                        if (col >= p.nx - 2) putbb(c - p.nx, i, o, l);
                    };
                    const long long pt = p.pitch;
                    if (y == 0) {
                        bb(2, 4, xc, c0 - pt);
                        bb(5, 7, xc - 1, c0 - pt - 1);
                        bb(6, 8, xc + 1, c0 - pt + 1);
                    } else {
                        bb(4, 2, xc, c0 + pt);
                        bb(7, 5, xc + 1, c0 + pt + 1);
                        bb(8, 6, xc - 1, c0 + pt - 1);
                    }
                }
            }
        };
        P* __restrict__ dfg = static_cast<P*>(io.dst);
        Hv* __restrict__ dh = reinterpret_cast<Hv*>(dfg + (size_t)kPairs * p.plane);
        const long long pl = p.plane;
        // sources of the f and g collisions, cs2 V = d_t(s u) + cs2 (A or B) n, formed before the flow
        // collision; the flow populations are collided and stored first, so that their registers
        // are free before the (f, g) pairs are converted for theirs
        PV vx, vy;
        {
            const C nx3 = vmul(nx_, bcv<C>(1.f / 3.f)), ny3 = vmul(ny_, bcv<C>(1.f / 3.f));
            const PV AB = mkpv(Aterm, Bterm);
            vx = vfma(AB, mkpv(nx3, nx3), dtX);
            vy = vfma(AB, mkpv(ny3, ny3), dtY);
        }
        // ---- flow h (Sec. 3.3); none when the velocity is prescribed ----
        if constexpr (FLOW) {
            C s2, k2, s4, k4;
            if (p.dmu == 0.f && !var) {
                s2 = bcv<C>(p.s2h);
                k2 = bcv<C>(p.k2h);
                s4 = bcv<C>(p.s4h_eff);
                k4 = bcv<C>(p.k4h);
            } else {
                // nu = mu(phi) / rho(phi)
                const C mu = vfma(vmul(vsub(phi, bcv<C>(p.phiB)), bcv<C>(p.inv_dphi)), bcv<C>(p.dmu), bcv<C>(p.muB));
                s2 = lanes(vfma(vmul(bcv<C>(3.f), mu), inv_rho, bcv<C>(0.5f)), [](float v) { return __frcp_rn(v); });
                k2 = vfma(bcv<C>(-0.5f), s2, bcv<C>(1.f));
                s4 = p.tie_s4h ? s2 : bcv<C>(p.s4h);
                k4 = vfma(bcv<C>(-0.5f), s4, bcv<C>(1.f));
            }
            const C s1 = bcv<C>(p.s1h), s3 = bcv<C>(p.s3h), k1 = bcv<C>(p.k1h), k3 = bcv<C>(p.k3h);
            if constexpr (!var) {
                Jx = vmul(rho, ux);
                Jy = vmul(rho, uy);
            }
            // equilibrium moments, Q = (rho u - S) u:
            //   (., Jx, Jy, P + Q_xx, P + Q_yy, (Q_xy + Q_yx)/2, Jx/3, Jy/3, P/3 + (Q_xx + Q_yy)/3)
            // source moments of H, m2H = d_t(rho u u - (S u + u S)/2) + cs2 (u grad rho + grad rho u):
            //   (., Fx, Fy, m2H_xx + u.grad rho/3, m2H_yy + u.grad rho/3, m2H_xy, Fx/3, Fy/3,
            //    (m2H_xx + m2H_yy)/3 + u.grad rho/9)
            // increments dm_k = -s_k (m_k - m_eq_k) + (1 - s_k/2) m_src_k = (1 - s_k/2) m_src_k +
            // s_k (m_eq_k - m_k), then h* = h + M^-1 dm; the x and y moments of each order as one pair
            const C nm5 = vsub(lb(sUV), la(sUV)), m8 = vadd(la(sUV), lb(sUV));  // -m5, m8
            const PV m67 = mkpv(vsub(h57, h68), vadd(h57, h68));                 // (m6, m7)
            const PV m34 = vadd(sXY, mkpv(m8, m8));                               // (m3, m4)
            const PV Fv = mkpv(Fx, Fy), Jv = mkpv(Jx, Jy), uv = mkpv(ux, uy);
            const PV k2v = mkpv(k2, k2), s2v = mkpv(s2, s2);
            const PV third = pvk<PV>(1.f / 3.f, 1.f / 3.f);
            PV d12, d34, d67;
            C d5, d8;
            const PV d12s = vmul(mkpv(s1, s1), vsub(Jv, mkpv(jx, jy)));
            const PV d67s = vmul(mkpv(s3, s3), vfma(pvk<PV>(-3.f, -3.f), m67, Jv));
            d12 = vfma(mkpv(k1, k1), Fv, d12s);
            d67 = vmul(third, vfma(mkpv(k3, k3), Fv, d67s));
            if constexpr (!var) {
                d34 = vfma(k2v, mkpv(dt_xx, dt_yy), vmul(s2v, vsub(vfma(Jv, uv, mkpv(P_, P_)), m34)));
                d5 = vfma(k2, dt_xy, vmul(s2, vfma(Jx, uy, nm5)));
                d8 = vmul(bcv<C>(1.f / 3.f), vfma(k4, vadd(dt_xx, dt_yy),
                                                 vmul(s4, vfma(bcv<C>(-3.f), m8, vadd(P_, vfma(Jx, ux, vmul(Jy, uy)))))));
            } else {
                const C mxx = vfma(bcv<C>(2.f / 3.f), vmul(ux, grx), dt_xx);
                const C myy = vfma(bcv<C>(2.f / 3.f), vmul(uy, gry), dt_yy);
                const C mxy = vfma(bcv<C>(1.f / 3.f), vfma(ux, gry, vmul(uy, grx)), dt_xy);
                const C ug3 = bcv<C>(1.f / 3.f);
                d34 = vfma(k2v, mkpv(vfma(ug3, ugr, mxx), vfma(ug3, ugr, myy)),
                           vmul(s2v, vsub(mkpv(vadd(P_, qxx), vadd(P_, qyy)), m34)));
                d5 = vfma(k2, mxy, vmul(s2, vadd(qxy, nm5)));
                // 3 x the eighth source moment (mxx + myy)/3 + u.grad rho/9
                d8 = vmul(ug3, vfma(k4, vfma(ug3, ugr, vadd(mxx, myy)),
                                    vmul(s4, vfma(bcv<C>(-3.f), m8, vadd(P_, vadd(qxx, qyy))))));
            }
            // (A, C) = (d1 - d6, d2 - d7), (B, D) = (d3 - d8, d4 - d8), (E, F) = (d8 + d5, d8 - d5),
            // (G, H) = (d6 + d7, d7 - d6)
            const PV AC = vsub(d12, d67), BD = vsub(d34, mkpv(d8, d8));
            const PV EF = mkpv(vadd(d8, d5), vsub(d8, d5)), GH = mkpv(vadd(la(d67), lb(d67)), vsub(lb(d67), la(d67)));
            const PV half = pvk<PV>(0.5f, 0.5f), quarter = pvk<PV>(0.25f, 0.25f);
            X = vfma(half, vadd(AC, BD), X);     // h1 += (A + B)/2, h2 += (C + D)/2
            Y = vfma(half, vsub(BD, AC), Y);     // h3 += (B - A)/2, h4 += (D - C)/2
            U = vfma(quarter, vadd(EF, GH), U);  // h5 += (E + G)/4, h6 += (F + H)/4
            V = vfma(quarter, vsub(EF, GH), V);  // h7 += (E - G)/4, h8 += (F - H)/4
            if (EDGE && WALLS) {
                // moving-wall term for the links that leave through a wall, folded in before storing:
                // h_ibar(x_b, t+1) = h*_i(x_b, t) - 2 w_i rho c_i.u_w / cs2
                if (y == 0)
                    V = vsub(V, mkpv(vmul(rho, bcv<C>(6.f * wgt(7) * (-1.f) * p.u_bot)),
                                     vmul(rho, bcv<C>(6.f * wgt(8) * (1.f) * p.u_bot))));
                if (y == p.ny - 1)
                    U = vsub(U, mkpv(vmul(rho, bcv<C>(6.f * wgt(5) * (1.f) * p.u_top)),
                                     vmul(rho, bcv<C>(6.f * wgt(6) * (-1.f) * p.u_top))));
            }
            if constexpr (!T::kH16) {
                // FP32 h: the stored pairs (h_1, h_2), (h_3, h_4), (h_5, h_6), (h_7, h_8)
                float2 outh[4][CPT];
#pragma unroll
                for (int l = 0; l < CPT; ++l) {
                    outh[0][l] = cell_of(X, l, 0);
                    outh[1][l] = cell_of(Y, l, 0);
                    outh[2][l] = cell_of(U, l, 0);
                    outh[3][l] = cell_of(V, l, 0);
                }
                float2* dp = reinterpret_cast<float2*>(dh);
                each_dest(
                    [&](long long c) {
                        if (CPT == 1 || !act1) {
#pragma unroll
                            for (int j = 0; j < 4; ++j) dp[j * pl + c] = outh[j][0];
                        } else {
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                *reinterpret_cast<float4*>(dp + j * pl + c) =
                                    make_float4(outh[j][0].x, outh[j][0].y, outh[j][CPT - 1].x, outh[j][CPT - 1].y);
                        }
                    },
                    [&](long long c, int l) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) dp[j * pl + c] = outh[j][l];
                    },
                    [&](long long d, int i, int o, int l) {
                        const float2 w = outh[(o - 1) >> 1][l];
                        dh[h_index(i, d, pl)] = ((o - 1) & 1) ? w.y : w.x;
                    });
            } else {
                // every slot is stored relative to this cell's new u (what the next step reads back):
                // raw = (h_i / w_i - 3 rho c_i.u) S_h, two links per stochastic conversion
                const float kv = __fmul_rn(p.kh3, T::SH);
                const C vx = vmul(bcv<C>(kv), ux), vy = vmul(bcv<C>(kv), uy);
                const C nvx = vmul(bcv<C>(-kv), ux), nvy = vmul(bcv<C>(-kv), uy);
                constexpr float e1 = (float)(T::SH / wgt_d(1)), e5 = (float)(T::SH / wgt_d(5));  // exact
                const PV r12 = vfma(X, pvk<PV>(e1, e1), mkpv(nvx, nvy));
                const PV r34 = vfma(Y, pvk<PV>(e1, e1), mkpv(vx, vy));
                const PV r56 = vfma(U, pvk<PV>(e5, e5), mkpv(vadd(nvx, nvy), vadd(vx, nvy)));
                const PV r78 = vfma(V, pvk<PV>(e5, e5), mkpv(vadd(vx, vy), vadd(nvx, vy)));
                // the stored pairs (h_1, h_2), (h_3, h_4), (h_5, h_6), (h_7, h_8)
                uint32_t outw[4][CPT];
#pragma unroll
                for (int l = 0; l < CPT; ++l) {
                    const float2 a = cell_of(r12, l, 0), b = cell_of(r34, l, 0), c = cell_of(r56, l, 0),
                                 d = cell_of(r78, l, 0);
                    outw[0][l] = cvt_rs2<typename T::P>(a.x, a.y, rbits_of(key[l], 9));
                    outw[1][l] = cvt_rs2<typename T::P>(b.x, b.y, rbits_of(key[l], 10));
                    outw[2][l] = cvt_rs2<typename T::P>(c.x, c.y, rbits_of(key[l], 11));
                    outw[3][l] = cvt_rs2<typename T::P>(d.x, d.y, rbits_of(key[l], 12));
                }
                uint32_t* dw = reinterpret_cast<uint32_t*>(dh);
                each_dest(
                    [&](long long c) {
                        if (CPT == 1 || !act1) {
#pragma unroll
                            for (int j = 0; j < 4; ++j) dw[j * pl + c] = outw[j][0];
                        } else {
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                *reinterpret_cast<uint2*>(dw + j * pl + c) = make_uint2(outw[j][0], outw[j][CPT - 1]);
                        }
                    },
                    [&](long long c, int l) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) dw[j * pl + c] = outw[j][l];
                    },
                    [&](long long d, int i, int o, int l) {
                        const uint32_t w = outw[(o - 1) >> 1][l];
                        dh[h_index(i, d, pl)] = bits_to<Hv>(((o - 1) & 1) ? (w >> 16) : (w & 0xFFFFu));
                    });
            }
        }
        // ---- f (Sec. 3.1) and g (Sec. 3.2) together ----
        {
            P qs[9][CPT];
            asm volatile("" ::: "memory");  // a fresh load of the staged pairs (see above)
#pragma unroll
            for (int i = 0; i < 9; ++i) ld_raw<ST>(pull + i * SLOT - cx(i), cx(i) == 0, qs[i]);
            P outp[9][CPT];  // the stored (f_i, g_i) of each cell
            if constexpr (CPT == 1) {
                float2 q[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) q[i] = raw2(qs[i][0]);
                collide_lanes<ST, kLanesFG>(q, pp, vsub(pp, ref), make_float2(ux, ux), make_float2(uy, uy), vx, vy,
                                            make_float2(p.nS1[0], p.nS1[1]), make_float2(p.nS2[0], p.nS2[1]),
                                            make_float2(p.nS3[0], p.nS3[1]), make_float2(p.nS4[0], p.nS4[1]),
                                            make_float2(p.K1[0], p.K1[1]), make_float2(p.K3[0], p.K3[1]));
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    if constexpr (!T::kPair16) outp[i][0] = *reinterpret_cast<const P*>(&q[i]);
                    else outp[i][0] = enc_pair_rs<ST>(q[i], key[0], i);
                }
            } else {
                // f of both cells, then g of both cells: one lane per cell, half the live state
                float2 qf[9], qg[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const float2 a0 = raw2(qs[i][0]), a1 = raw2(qs[i][CPT - 1]);
                    qf[i] = make_float2(a0.x, a1.x);
                }
                collide_lanes<ST, kLanesF>(qf, la(pp), vsub(la(pp), bcv<C>(la(ref).x)), ux, uy, la(vx), la(vy),
                                           bcv<C>(p.nS1[0]), bcv<C>(p.nS2[0]), bcv<C>(p.nS3[0]), bcv<C>(p.nS4[0]),
                                           bcv<C>(p.K1[0]), bcv<C>(p.K3[0]));
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const float2 a0 = raw2(qs[i][0]), a1 = raw2(qs[i][CPT - 1]);
                    qg[i] = make_float2(a0.y, a1.y);
                }
                collide_lanes<ST, kLanesG>(qg, lb(pp), lb(pp), ux, uy, lb(vx), lb(vy), bcv<C>(p.nS1[1]),
                                           bcv<C>(p.nS2[1]), bcv<C>(p.nS3[1]), bcv<C>(p.nS4[1]), bcv<C>(p.K1[1]),
                                           bcv<C>(p.K3[1]));
#pragma unroll
                for (int i = 0; i < 9; ++i)
#pragma unroll
                    for (int l = 0; l < CPT; ++l)
                        outp[i][l] = enc_pair_rs<ST>(make_float2(cell_of(qf[i], l), cell_of(qg[i], l)), key[l], i);
            }
            each_dest(
                [&](long long c) {
                    if (CPT == 1 || !act1) {
#pragma unroll
                        for (int i = 0; i < 9; ++i) dfg[i * pl + c] = outp[i][0];
                    } else {
#pragma unroll
                        for (int i = 0; i < 9; ++i)
                            *reinterpret_cast<Two<P>*>(dfg + i * pl + c) = Two<P>{outp[i][0], outp[i][CPT - 1]};
                    }
                },
                [&](long long c, int l) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) dfg[i * pl + c] = outp[i][l];
                },
                [&](long long d, int i, int o, int l) { dfg[i * pl + d] = outp[o][l]; });
        }
        // the u history (and the mass-flux history with a density ratio)
        auto put_hist = [&](float2* dst, C a, C b, long long c) {
            if constexpr (CPT == 1) dst[c] = make_float2(a, b);
            else if (act1) *reinterpret_cast<float4*>(dst + c) = make_float4(a.x, b.x, a.y, b.y);
            else dst[c] = make_float2(a.x, b.x);
        };
        put_hist(io.hist_dst, ux, uy, cell);
        if constexpr (var) put_hist(io.shist_dst, Sx, Sy, cell);
        if constexpr (S::kHalo) {
            // the 16-bit h decode reads the neighbours' u, across periodic edges too
            if (yl) put_hist(io.hist_dst, ux, uy, cell + DY);
            if (yr) put_hist(io.hist_dst, ux, uy, cell - DY);
            if (xedge) {
#pragma unroll
                for (int l = 0; l < CPT; ++l) {
                    if (l == 1 && !act1) break;
                    const long long c = cell + l;
                    const float2 un = make_float2(cell_of(ux, l), cell_of(uy, l));
                    const bool xl = x + l <= 1, xr = x + l >= p.nx - 2;
                    if (xl) io.hist_dst[c + DX] = un;
                    if (xr) io.hist_dst[c - DX] = un;
                    if (yl) {
                        if (xl) io.hist_dst[c + DY + DX] = un;
                        if (xr) io.hist_dst[c + DY - DX] = un;
                    }
                    if (yr) {
                        if (xl) io.hist_dst[c - DY + DX] = un;
                        if (xr) io.hist_dst[c - DY - DX] = un;
                    }
                }
            }
        }
    }
    return false;
}

// A tile whose cells and ring all lie in the grid, at least two cells from every edge: none of its
// cells writes a ghost-frame copy, meets a wall or lies beyond the grid (95 % of the tiles of a
// 2048 x 1024 grid).
template <int ST> __device__ __forceinline__ bool tile_is_interior(const Phys& p, int x0, int y0) {
    using G = GeoOf<ST>;
    return x0 >= 2 && x0 + G::TX + 2 <= p.nx && y0 >= 2 && y0 + G::TY + 2 <= p.ny;
}
// step_tile on the interior or the edge path (the choice is uniform over the tile).
template <int ST, bool WALLS, bool LANGMUIR, int MODE, int FLOW, bool WS = false>
__device__ __forceinline__ bool step_tile_any(const Phys& p, const TileIO& io, unsigned char* sm, float2* PP,
                                              unsigned long long* mbar, uint32_t parity, int x0, int y0) {
    if (tile_is_interior<ST>(p, x0, y0))
        return step_tile<ST, WALLS, LANGMUIR, MODE, FLOW, WS, false>(p, io, sm, PP, mbar, parity, x0, y0);
    return step_tile<ST, WALLS, LANGMUIR, MODE, FLOW, WS, true>(p, io, sm, PP, mbar, parity, x0, y0);
}

// Resident CTAs per SM that the one-tile kernels (step_kernel, and batch_step_kernel but for the
// case below) are compiled for.  FP32 storage: four; with a prescribed velocity (no h) the cell
// update fits 48 registers without spills and the boxes 33 KB, so five (convection test
// 2048 x 1024: 54.3 -> 52.5 us per step).  Two cells per thread (128-thread CTAs): five, at 96
// registers (FP16 at 2048 x 1024: 51.5 us, against 52.3 at six CTAs and 80 registers, where the
// interior path spills); the density-ratio update needs more, so four (128 registers).
template <int ST>
__host__ __device__ constexpr int tile_min_blocks(int flow) {
    return cpt_of(ST) == 2 ? (flow == kFlowVarRho ? 4 : 5) : (flow == kFlowPrescribed ? 5 : 4);
}
// The per-tile batch kernel reads the lattice's constants from shared memory, which takes more
// registers: with FP32 storage and a prescribed velocity, five CTAs per SM would spill 128 B, so four.
template <int ST>
__host__ __device__ constexpr int batch_min_blocks(int flow) {
    return cpt_of(ST) == 1 && flow == kFlowPrescribed ? 4 : tile_min_blocks<ST>(flow);
}
template <int ST, bool WALLS, bool LANGMUIR, int MODE, int FLOW>
__global__ void __launch_bounds__(GeoOf<ST>::NT, tile_min_blocks<ST>(FLOW)) step_kernel(const __grid_constant__ StepArgs a) {
    using G = GeoOf<ST>;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(sm + Smem<ST>::BAR);
    // The first and the last tile row (whose cells also write the ghost frame, and so run longest)
    // are launched first, so that the last wave holds interior tiles only.
    const int ntr = gridDim.y;
    const int tr = blockIdx.y == 0 ? 0 : (blockIdx.y == 1 ? ntr - 1 : (int)blockIdx.y - 1);
    const int x0 = blockIdx.x * G::TX, y0 = tr * G::TY;
    if (threadIdx.x == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
    }
    // Programmatic dependent launch: let the next step's CTAs be scheduled into the slots this
    // grid frees, and wait here until the previous step's writes are complete and visible.
    cudaTriggerProgrammaticLaunchCompletion();
    cudaGridDependencySynchronize();
    if (threadIdx.x == 0) issue_tile_loads<ST, FLOW>(sm, &a.tm_fg, &a.tm_h, &a.tm_hist, x0, y0, mbar);
    step_tile_any<ST, WALLS, LANGMUIR, MODE, FLOW>(a.p, a.io, sm, reinterpret_cast<float2*>(sm + Smem<ST>::PP), mbar, 0,
                                                   x0, y0);
}

// Tile k of a grid of ntx x nty tiles: rows in the order first, last, then the interior (the two
// edge rows, whose cells also write the ghost frame, run first).
template <int ST>
__device__ __forceinline__ void tile_origin(int k, int ntx, int nty, int& x0, int& y0) {
    const int r = k / ntx, c = k - r * ntx;
    const int tr = r == 0 ? 0 : (r == 1 ? nty - 1 : r - 1);
    x0 = c * GeoOf<ST>::TX;
    y0 = tr * GeoOf<ST>::TY;
}

// One step of one lattice by a persistent, warp-specialised grid.  Each CTA has NT compute threads
// (eight warps, as in step_kernel) and one copy warp.  One lane of the copy warp claims tiles
// from an atomic counter (one at a time, which balances the longer edge tiles across the CTAs;
// each claim one iteration ahead, so its latency overlaps the wait for a buffer) and stages each
// into one of two buffers with TMA, on that buffer's "full" mbarrier; the compute warps release a
// buffer on its "empty" mbarrier (one arrival per warp) once the tile is done, so the copy of the
// next tile overlaps the arithmetic of the current one and the copy warp never joins a block-wide
// barrier.  After the last tile the copy lane arrives on a full barrier without a copy; the
// compute warps read the stop mark (x0 = -1) and stop.  Every wait is bounded: a copy lane that
// gives up waits (bounded) for the copies it has in flight.
// Two CTAs per SM: with FP32 storage the two stages fill the shared memory of two, so its bound
// lets the compiler use up to 112 registers (rising bubble, FP32: 81.6 -> 80.6 us); with two cells
// per thread the two cells' update needs them.
// With two cells per thread the register cap is given directly: 96 registers place five warps on an
// SM sub-partition (16 384 registers), four CTAs of five warps per SM; the density-ratio update
// takes 128 (three CTAs), and the batched kernel, which holds the lattice's constants in shared
// memory, 112.
template <int ST> constexpr int nt_pipe() { return GeoOf<ST>::NT + 32; }
constexpr int pipe_regs2(int flow, bool batch = false) { return flow == kFlowVarRho ? 128 : (batch ? 112 : 96); }

template <int ST, bool WALLS, bool LANGMUIR, int FLOW>
__device__ __forceinline__ void step_pipe_body(const StepArgs& a, int ntx, int nty) {
    using S = Smem<ST>;
    using G = GeoOf<ST>;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned long long* full = reinterpret_cast<unsigned long long*>(sm + S::PIPE_BAR);
    unsigned long long* empty = full + 2;
    volatile int* slot = reinterpret_cast<volatile int*>(sm + S::PIPE_SLOT);  // (x0, y0) per buffer
    const unsigned ntiles = (unsigned)(ntx * nty);
    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&empty[0], G::NT / 32);
        mbar_init(&empty[1], G::NT / 32);
        fence_mbar_init();
    }
    __syncthreads();
    cudaTriggerProgrammaticLaunchCompletion();
    cudaGridDependencySynchronize();  // also: the previous launch no longer uses its counter

    if (threadIdx.x >= G::NT) {
        // ---- copy warp ----
        if (threadIdx.x != G::NT) return;
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
            tile_origin<ST>((int)k, ntx, nty, x0, y0);
            slot[2 * b] = x0;
            slot[2 * b + 1] = y0;
            issue_tile_loads<ST, FLOW>(sm + b * S::STAGE, &a.tm_fg, &a.tm_h, &a.tm_hist, x0, y0, &full[b]);
            pending[b] = true;
            issued[b] = (uint32_t)(it >> 1) & 1u;
            k = kn;
        }
    }

    // ---- compute warps ----
    const int lane = (int)threadIdx.x % 32;
    for (int it = 0;; ++it) {
        const int b = it & 1;
        const uint32_t parity = (uint32_t)(it >> 1) & 1u;
        const bool late = !mbar_wait_bounded(&full[b], parity);
        if (compute_sync_or<G::NT>(late)) {  // uniform: a copy (or the stop mark) did not come in time
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
        float2* PP = reinterpret_cast<float2*>(sm + S::PIPE_PP + b * S::PP_BYTES);
        if (step_tile_any<ST, WALLS, LANGMUIR, kStep, FLOW, true>(a.p, a.io, sm + b * S::STAGE, PP, &full[b], parity, x0,
                                                                  y0))
            break;  // uniform (decided by the OR barrier inside)
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);  // this warp is done with buffer b
    }
}
template <int ST, bool WALLS, bool LANGMUIR, int FLOW>
__global__ void __launch_bounds__(nt_pipe<ST>(), 2) step_kernel_pipe(const __grid_constant__ StepArgs a, int ntx, int nty) {
    step_pipe_body<ST, WALLS, LANGMUIR, FLOW>(a, ntx, nty);
}
template <int ST, bool WALLS, bool LANGMUIR, int FLOW>
__global__ void __maxnreg__(pipe_regs2(FLOW)) step_kernel_pipe2(const __grid_constant__ StepArgs a, int ntx, int nty) {
    step_pipe_body<ST, WALLS, LANGMUIR, FLOW>(a, ntx, nty);
}
// The warp-specialised step kernel of storage mode ST.
template <int ST, bool WALLS, bool LANGMUIR, int FLOW> constexpr auto pipe_kernel() {
    if constexpr (cpt_of(ST) == 1) return step_kernel_pipe<ST, WALLS, LANGMUIR, FLOW>;
    else return step_kernel_pipe2<ST, WALLS, LANGMUIR, FLOW>;
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
__global__ void __launch_bounds__(GeoOf<ST>::NT, batch_min_blocks<ST>(FLOW)) batch_step_kernel(const __grid_constant__ BatchArgs b) {
    using S = Smem<ST>;
    using G = GeoOf<ST>;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(sm + S::BAR);
    cudaTriggerProgrammaticLaunchCompletion();
    cudaGridDependencySynchronize();  // descriptors and populations of the previous launch
    const uint2 te = b.tiles[blockIdx.x];
    const InstDesc& d = b.descs[te.x];
    const int x0 = (int)(te.y & 0xFFFFu) * G::TX, y0 = (int)(te.y >> 16) * G::TY;
    const int cur = (d.cur + b.s) & 1;
    // the lattice's constants in shared memory, complete before any thread reads them (the
    // choice of the interior path reads the grid size)
    Phys* sp = reinterpret_cast<Phys*>(sm + S::PHYS);
    static_assert(sizeof(Phys) % 4 == 0, "Phys is copied as words");
    for (int k = threadIdx.x; k < (int)(sizeof(Phys) / 4); k += G::NT)
        reinterpret_cast<uint32_t*>(sp)[k] = reinterpret_cast<const uint32_t*>(&d.p)[k];
    __syncthreads();
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
    step_tile_any<ST, WALLS, LANGMUIR, kStep, FLOW>(*sp, io, sm, reinterpret_cast<float2*>(sm + S::PP), mbar, 0, x0, y0);
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
__device__ __forceinline__ void batch_ws_body(const BatchArgs& b) {
    using S = Smem<ST>;
    using G = GeoOf<ST>;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned long long* full = reinterpret_cast<unsigned long long*>(sm + S::PIPE_BAR);
    unsigned long long* empty = full + 2;
    volatile int* slot = reinterpret_cast<volatile int*>(sm + S::BWS_SLOT);  // x0, y0, lattice, cur per buffer
    const unsigned ntiles = (unsigned)b.ntiles;
    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&empty[0], G::NT / 32);
        mbar_init(&empty[1], G::NT / 32);
        fence_mbar_init();
    }
    __syncthreads();
    cudaTriggerProgrammaticLaunchCompletion();
    cudaGridDependencySynchronize();  // descriptors and populations of the previous launch

    if (threadIdx.x >= G::NT) {
        // ---- copy warp ----
        if (threadIdx.x != G::NT) return;
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
            const int x0 = (int)(te.y & 0xFFFFu) * G::TX, y0 = (int)(te.y >> 16) * G::TY;
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
        if (compute_sync_or<G::NT>(late)) {
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
        float2* PP = reinterpret_cast<float2*>(sm + S::PIPE_PP + q * S::PP_BYTES);
        if (step_tile_any<ST, WALLS, LANGMUIR, kStep, FLOW, true>(p, io, sm + q * S::STAGE, PP, &full[q], parity, x0, y0))
            return;
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[q]);
    }
}
template <int ST, bool WALLS, bool LANGMUIR, int FLOW>
__global__ void __launch_bounds__(nt_pipe<ST>(), 2) batch_step_kernel_ws(const __grid_constant__ BatchArgs b) {
    batch_ws_body<ST, WALLS, LANGMUIR, FLOW>(b);
}
template <int ST, bool WALLS, bool LANGMUIR, int FLOW>
__global__ void __maxnreg__(pipe_regs2(FLOW, true)) batch_step_kernel_ws2(const __grid_constant__ BatchArgs b) {
    batch_ws_body<ST, WALLS, LANGMUIR, FLOW>(b);
}
// The warp-specialised batch kernel of storage mode ST.
template <int ST, bool WALLS, bool LANGMUIR, int FLOW> constexpr auto batch_ws_kernel() {
    if constexpr (cpt_of(ST) == 1) return batch_step_kernel_ws<ST, WALLS, LANGMUIR, FLOW>;
    else return batch_step_kernel_ws2<ST, WALLS, LANGMUIR, FLOW>;
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
    // FP32 storage takes the equilibria in FP32, the precision it stores them in (FP64 arithmetic
    // is slow on this GPU); 16-bit storage rounds them from FP64 through FP32 to 16 bits
    const float phf = (float)phi, psf = (float)psi, uxf = (float)ux, uyf = (float)uy;
    const float rhf = (float)rho, uuf3 = (float)uu * (1.f / 3.f), P3f = 3.f * (float)P_;
    P* fg = static_cast<P*>(a.dst);
    Hv* hp = reinterpret_cast<Hv*>(fg + (size_t)kPairs * p.plane);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
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
        Hv vh{};
        if constexpr (ST == kFP32) {
            const float cu = (float)cx(i) * uxf + (float)cy(i) * uyf;  // sums of +-ux, +-uy: exact
            const float w = (float)wgt_d(i), b = __fmaf_rn(3.f, cu, 1.f);
            vfg = make_float2(w * phf * b, w * psf * b);
            // w (3 P + 3 rho c.u + 4.5 rho ((c.u)^2 - u.u/3))
            if (i > 0 && a.flow)
                vh = (Hv)(w * __fmaf_rn(3.f * rhf, cu, __fmaf_rn(4.5f * rhf, __fmaf_rn(cu, cu, -uuf3), P3f)));
        } else {
            const double cu = cx(i) * ux + cy(i) * uy;
            const double w = wgt_d(i);
            const double feq = w * phi * (1.0 + 3.0 * cu);
            const double geq = w * psi * (1.0 + 3.0 * cu);
            const double heq = w * (3.0 * P_ + 3.0 * rho * cu + 4.5 * rho * (cu * cu - uu / 3.0));
            vfg = pack2<P>(make_float2((float)((feq / w - p.phi_ref) * T::SF), (float)(geq / w * T::SG)));
            if (i > 0 && a.flow) {
                if constexpr (!T::kH16) {
                    vh = (Hv)heq;
                } else {
                    // stored relative to the storing cell's velocity, as the step will read it
                    // back: the source cell for a plain link, this cell (slot opp(i)) across a wall
                    const size_t so = wall_ghost ? o : (size_t)sy * p.nx + sx;
                    const double sux = (float)a.ux[so], suy = (float)a.uy[so];
                    const double vel = 3.0 * rho * (cx(enc) * sux + cy(enc) * suy);
                    vh = pack1<Hv>((float)((heq / w - vel) * T::SH));
                }
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

// ---- FP64 sums of phi or psi.  After a step every cell holds its nine post-collision values in
// its own slots, so the total of a field is the plain sum of one lane of the 9 pair planes over
// the cells.  Before the first step the buffer holds what lbm_init_fields staged for the first
// pull (each cell's equilibrium value of link i at x - c_i, in the wall's ghost row where that
// lies beyond a wall): the sum is then taken over the values each cell pulls ----
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

// lane 0 sums f (phi), lane 1 sums g (psi); 16-bit storage is decoded to its value first;
// pulled: sum the values at x - c_i (the state before the first step) instead of the own slots
template <int ST>
__global__ void __launch_bounds__(kReduceThreads) reduce_partial_kernel(const void* __restrict__ pops, int lane,
                                                                        int pulled, int nx, int ny, int pitch,
                                                                        long long plane,
                                                                        long long org, Phys p,
                                                                        double* __restrict__ partials) {
    using T = Traits<ST>;
    using P = typename T::P;
    __shared__ double smem[32];
    const P* pairs = static_cast<const P*>(pops);
    double acc = 0.0;
    // block b owns rows b, b + gridDim.x, ...; threads stride over (pair plane, x), counted in 64
    // bits (9 nx exceeds the int range for rows wider than 2^31 / 9 cells)
    const long long nk = (long long)kPairs * nx;
    for (int y = blockIdx.x; y < ny; y += gridDim.x) {
        for (long long k = threadIdx.x; k < nk; k += blockDim.x) {
            const int i = (int)(k / nx), x = (int)(k - (long long)i * nx);
            const int sx = pulled ? x - cx(i) : x, sy = pulled ? y - cy(i) : y;
            const float2 v = raw2(pairs[(size_t)i * plane + (size_t)(org + (long long)sy * pitch + sx)]);
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
