// Device code of the fused three-population lattice-Boltzmann step (arXiv 2408.15654).
//
// Data layout in HBM (one population buffer): 26 float planes of ny rows x `pitch` floats,
//   planes 0..8   f_0..f_8   phase field        (Sec. 3.1)
//   planes 9..17  g_0..g_8   surfactant         (Sec. 3.2)
//   planes 18..25 h_1..h_8   flow; h_0 is never stored: column 0 of M^-1 is e_0 and rows 1..8
//                            of M do not see h_0, so h_0 feeds only itself (Sec. 3.3, Sec. 4).
// A buffer holds the post-collision populations of the previous step at the cell that produced
// them; a step pulls f_i(x) = f*_i(x - c_i) ("pull" streaming), so it writes only its own cell
// and two buffers alternate.  At a wall the missing link is the cell's own opposite slot, into
// which the previous step already folded the moving-wall term (half-way bounce-back, Sec. 4).
//
// Velocity order (the columns of the printed moment matrix M, Sec. 4):
//   0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1)
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lbm {

__host__ __device__ constexpr int cx(int i) { return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0); }
__host__ __device__ constexpr int cy(int i) { return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0); }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5); }
__host__ __device__ constexpr float wgt(int i) { return i == 0 ? 4.f / 9.f : (i <= 4 ? 1.f / 9.f : 1.f / 36.f); }

static_assert(opp(1) == 3 && opp(3) == 1 && opp(2) == 4 && opp(4) == 2, "axis opposites");
static_assert(opp(5) == 7 && opp(7) == 5 && opp(6) == 8 && opp(8) == 6, "diagonal opposites");

constexpr int kPlanes = 26;   // f0..f8, g0..g8, h1..h8
constexpr int kPlaneG = 9;
constexpr int kPlaneH = 18;   // plane of h_1

// Physical constants in FP32, precomputed on the host from lbm_params.
struct Phys {
    int nx, ny, pitch, first;
    long long plane;          // floats per plane (ny * pitch)
    float phiA, phiB, inv_dphi;
    float cA;                 // 4 / (W dphi):  A = cA (phiA - phi)(phi - phiB), B = cA psi (phiA + phiB - 2 phi)
    float cap_k, c16W, W;     // capillary: cap_k sigma [c16W (phiA-phi)(phi-phiB)(phiA+phiB-2phi) - W lap phi]
    float mar_k;              // Marangoni: mar_k [|grad phi|^2 grad sigma - (grad sigma . grad phi) grad phi]
    float sigma0, E0;
    float rho, inv_rho;
    float muB, dmu;           // mu(phi) = muB + (phi - phiB)/dphi * dmu
    float gx, gy;
    float s1f, s2f, s3f, s4f;
    float s1g, s2g, s3g, s4g;
    float s1h, s3h, s4h;
    int tie_s4h;              // 1: s4^h = s2^h
    float u_top, u_bot;
    float n_eps2;             // n_eps^2
};

enum Mode { kStep = 0, kMoments = 1 };

struct StepArgs {
    Phys p;
    const float* __restrict__ src;
    float* __restrict__ dst;
    float* __restrict__ hist;     // 2 planes: u_x, u_y of the previous step (in place)
    unsigned* __restrict__ status;
    double* __restrict__ out[5];  // kMoments: phi, psi, ux, uy, P (dense ny x nx), may be null
};

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int EX = TX + 2, EY = TY + 2, NE = EX * EY;

__device__ __forceinline__ int wrap1(int a, int n) {
    a += (a < 0) ? n : 0;
    a -= (a >= n) ? n : 0;
    return min(max(a, 0), n - 1);  // only cells no valid cell reads can still be out of range
}

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Moment-space MRT collision of a scalar-transport population (f or g), applied as an
// increment so that FP32 rounding stays at the scale of the populations' departure from
// equilibrium (in a uniform bulk the increment is zero and the populations are unchanged):
//   m = M q;  dm_k = -s_k (m_k - m_eq_k) + (1 - s_k/2) m_src_k;  q* = q + M^-1 dm.
// Equilibrium w_i s (1 + c_i.u/cs2) has moments (s, s ux, s uy, s/3, s/3, 0, s ux/3, s uy/3, s/9);
// the source w_i c_i.V has moments (0, cs2 Vx, cs2 Vy, 0, 0, 0, Vx/9, Vy/9, 0) with
// cs2 V = (vx, vy) passed in.  dm_0 = 0: the zeroth moment is conserved.
__device__ __forceinline__ void collide_scalar(float q[9], float s, float ux, float uy, float vx, float vy,
                                               float s1, float s2, float s3, float s4) {
    const float third = 1.f / 3.f;
    const float m1 = q[1] - q[3] + q[5] - q[6] - q[7] + q[8];
    const float m2 = q[2] - q[4] + q[5] + q[6] - q[7] - q[8];
    const float m3 = q[1] + q[3] + q[5] + q[6] + q[7] + q[8];
    const float m4 = q[2] + q[4] + q[5] + q[6] + q[7] + q[8];
    const float m5 = q[5] - q[6] + q[7] - q[8];
    const float m6 = q[5] - q[6] - q[7] + q[8];
    const float m7 = q[5] + q[6] - q[7] - q[8];
    const float m8 = q[5] + q[6] + q[7] + q[8];
    const float d1 = -s1 * (m1 - s * ux) + (1.f - 0.5f * s1) * vx;
    const float d2 = -s1 * (m2 - s * uy) + (1.f - 0.5f * s1) * vy;
    const float d3 = -s2 * (m3 - s * third);
    const float d4 = -s2 * (m4 - s * third);
    const float d5 = -s2 * m5;
    const float d6 = -s3 * (m6 - s * ux * third) + (1.f - 0.5f * s3) * vx * third;
    const float d7 = -s3 * (m7 - s * uy * third) + (1.f - 0.5f * s3) * vy * third;
    const float d8 = -s4 * (m8 - s * (1.f / 9.f));
    q[0] += -d3 - d4 + d8;
    q[1] += 0.5f * (d1 + d3 - d6 - d8);
    q[2] += 0.5f * (d2 + d4 - d7 - d8);
    q[3] += 0.5f * (-d1 + d3 + d6 - d8);
    q[4] += 0.5f * (-d2 + d4 + d7 - d8);
    q[5] += 0.25f * (d5 + d6 + d7 + d8);
    q[6] += 0.25f * (-d5 - d6 + d7 + d8);
    q[7] += 0.25f * (d5 - d6 - d7 + d8);
    q[8] += 0.25f * (-d5 + d6 - d7 + d8);
}

// One fused step (kStep) or the macroscopic fields of the current level (kMoments) for a
// TX x TY tile.  The pulled f and g of the tile and of a one-cell ring around it are staged in
// shared memory by cp.async; phi and psi of the ring give the 9-point stencils; the same window
// also holds the own cell's unshifted post-collision values, whose sums are phi and psi of the
// previous level (m*_0 = phi exactly, Sec. 3.1), so only u of the previous level is stored.
template <bool WALLS, bool LANGMUIR, int MODE>
__global__ void __launch_bounds__(NT, 2) step_kernel(const __grid_constant__ StepArgs a) {
    __shared__ float sF[9 * NE];
    __shared__ float sG[9 * NE];
    __shared__ float sPhi[NE];
    __shared__ float sPsi[NE];
    const Phys& p = a.p;
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const float* __restrict__ srcF = a.src;
    const float* __restrict__ srcG = a.src + (size_t)kPlaneG * p.plane;

    // ---- stage 1: pull f and g of the extended tile into shared memory ----
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int e = t + k * NT;
        if (e < NE) {
            const int ey = e / EX, ex = e - ey * EX;
            const int gxx = x0 - 1 + ex, gyy = y0 - 1 + ey;
            const bool row_in = !WALLS || (gyy >= 0 && gyy < p.ny);
            if (row_in) {
                const int cols[3] = {wrap1(gxx - 1, p.nx), wrap1(gxx, p.nx), wrap1(gxx + 1, p.nx)};
                int rows[3];
                bool rin[3];
                if (WALLS) {
                    rows[0] = gyy - 1; rows[1] = gyy; rows[2] = gyy + 1;
                    rin[0] = gyy - 1 >= 0; rin[1] = true; rin[2] = gyy + 1 < p.ny;
                } else {
                    rows[0] = wrap1(gyy - 1, p.ny); rows[1] = wrap1(gyy, p.ny); rows[2] = wrap1(gyy + 1, p.ny);
                    rin[0] = rin[1] = rin[2] = true;
                }
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    // pull source x - c_i; beyond a wall: the own opposite slot
                    int plane = i, r = rows[1 - cy(i)], c = cols[1 - cx(i)];
                    if (WALLS && !rin[1 - cy(i)]) { plane = opp(i); r = rows[1]; c = cols[1]; }
                    const size_t off = (size_t)plane * p.plane + (size_t)r * p.pitch + c;
                    cp_async4(&sF[i * NE + e], srcF + off);
                    cp_async4(&sG[i * NE + e], srcG + off);
                }
            }
        }
    }

    // ---- own cell: h_1..h_8 straight into registers, u of the previous level ----
    const int tx = t % TX, ty = t / TX;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = (x < p.nx) && (y < p.ny);
    float h[9];
    float uxp = 0.f, uyp = 0.f;
    if (active) {
        const int cols[3] = {wrap1(x - 1, p.nx), x, wrap1(x + 1, p.nx)};
        int rows[3];
        bool rin[3];
        if (WALLS) {
            rows[0] = y - 1; rows[1] = y; rows[2] = y + 1;
            rin[0] = y >= 1; rin[1] = true; rin[2] = y + 1 < p.ny;
        } else {
            rows[0] = wrap1(y - 1, p.ny); rows[1] = y; rows[2] = wrap1(y + 1, p.ny);
            rin[0] = rin[1] = rin[2] = true;
        }
        const float* __restrict__ srcH = a.src + (size_t)kPlaneH * p.plane;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            int plane = i, r = rows[1 - cy(i)], c = cols[1 - cx(i)];
            if (WALLS && !rin[1 - cy(i)]) { plane = opp(i); r = y; c = x; }
            h[i] = __ldg(srcH + (size_t)(plane - 1) * p.plane + (size_t)r * p.pitch + c);
        }
        if (!p.first) {
            uxp = __ldg(a.hist + (size_t)y * p.pitch + x);
            uyp = __ldg(a.hist + p.plane + (size_t)y * p.pitch + x);
        }
    }
    cp_async_wait_all();
    __syncthreads();

    // ---- stage 2: phi and psi on the extended tile (cells beyond a wall mirror the fluid row) ----
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int e = t + k * NT;
        if (e < NE) {
            int es = e;
            if (WALLS) {
                const int ey = e / EX, ex = e - ey * EX;
                const int gyy = y0 - 1 + ey;
                if (gyy < 0) es = (1 - y0) * EX + ex;
                else if (gyy >= p.ny) es = (p.ny - y0) * EX + ex;
            }
            float sp = 0.f, ss = 0.f;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                sp += sF[i * NE + es];
                ss += sG[i * NE + es];
            }
            sPhi[e] = sp;
            sPsi[e] = ss;
        }
    }
    __syncthreads();
    if (!active) return;

    // ---- stage 3: the cell ----
    const int eo = (ty + 1) * EX + (tx + 1);
    const float phi = sPhi[eo], psi = sPsi[eo];
    const float third = 1.f / 3.f, twelfth = 1.f / 12.f, sixth = 1.f / 6.f;

    // isotropic stencils: d_a = (1/cs2) sum w_i c_ia q(x+c_i);  lap = (2/cs2) sum_{i>0} w_i (q_i - q)
    float gpx, gpy, lap, gsx, gsy;
    {
        const float E = sPhi[eo + 1], Wn = sPhi[eo - 1], N = sPhi[eo + EX], S = sPhi[eo - EX];
        const float NE_ = sPhi[eo + EX + 1], NW = sPhi[eo + EX - 1], SE = sPhi[eo - EX + 1], SW = sPhi[eo - EX - 1];
        gpx = (E - Wn) * third + (NE_ + SE - NW - SW) * twelfth;
        gpy = (N - S) * third + (NE_ + NW - SE - SW) * twelfth;
        lap = (4.f * (E + Wn + N + S) + (NE_ + NW + SE + SW) - 20.f * phi) * sixth;
    }
    {
        const float E = sPsi[eo + 1], Wn = sPsi[eo - 1], N = sPsi[eo + EX], S = sPsi[eo - EX];
        const float NE_ = sPsi[eo + EX + 1], NW = sPsi[eo + EX - 1], SE = sPsi[eo - EX + 1], SW = sPsi[eo - EX - 1];
        gsx = (E - Wn) * third + (NE_ + SE - NW - SW) * twelfth;
        gsy = (N - S) * third + (NE_ + NW - SE - SW) * twelfth;
    }

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
        sigma = p.sigma0 * (1.f + p.E0 * log1pf(-psi));
        dsig = -p.sigma0 * p.E0 / (1.f - psi);
    } else {
        sigma = p.sigma0 * (1.f - p.E0 * psi);
        dsig = -p.sigma0 * p.E0;
    }
    const float gsgx = dsig * gsx, gsgy = dsig * gsy;
    const float cap = p.cap_k * sigma * (p.c16W * dA * dB * sym - p.W * lap);
    const float sdg = gsgx * gpx + gsgy * gpy;
    const float Fx = cap * gpx + p.mar_k * (g2 * gsgx - sdg * gpx) + p.rho * p.gx;
    const float Fy = cap * gpy + p.mar_k * (g2 * gsgy - sdg * gpy) + p.rho * p.gy;

    // velocity: rho u = sum c_i h_i + F/2 (Sec. 3.3)
    const float jx = h[1] - h[3] + h[5] - h[6] - h[7] + h[8];
    const float jy = h[2] - h[4] + h[5] + h[6] - h[7] - h[8];
    const float ux = (jx + 0.5f * Fx) * p.inv_rho;
    const float uy = (jy + 0.5f * Fy) * p.inv_rho;

    // previous level: phi, psi from the own cell's post-collision populations, u from history
    float phip = phi, psip = psi;
    if (p.first) {
        uxp = ux;
        uyp = uy;
    } else {
        float sp = 0.f, ss = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            int idx = i * NE + eo + cy(i) * EX + cx(i);
            if (WALLS && ((cy(i) == 1 && y == p.ny - 1) || (cy(i) == -1 && y == 0))) idx = opp(i) * NE + eo;
            sp += sF[idx];
            ss += sG[idx];
        }
        phip = sp;
        psip = ss;
    }

    // time derivatives, backward difference over one step
    const float rho = p.rho;
    const float dt_fx = phi * ux - phip * uxp, dt_fy = phi * uy - phip * uyp;
    const float dt_gx = psi * ux - psip * uxp, dt_gy = psi * uy - psip * uyp;
    const float dt_xx = rho * (ux * ux - uxp * uxp);
    const float dt_yy = rho * (uy * uy - uyp * uyp);
    const float dt_xy = rho * (ux * uy - uxp * uyp);

    // pressure (Eq. for P, Sec. 3.3) with K = w0/(c^2 - cs2) = 2/3:
    //   P = 3/5 [sum_{i>0} h_i - (2/3) rho |u|^2 + (1/3) d_t(rho |u|^2)]
    const float hsum = ((h[1] + h[2]) + (h[3] + h[4])) + ((h[5] + h[6]) + (h[7] + h[8]));
    const float P = 0.6f * (hsum - (2.f / 3.f) * rho * (ux * ux + uy * uy) + third * (dt_xx + dt_yy));

    {
        bool bad = !(isfinite(phi) && isfinite(psi) && isfinite(P)) || !(fabsf(ux) < 0.3f && fabsf(uy) < 0.3f);
        if (LANGMUIR) bad = bad || !(psi < 1.f);
        if (bad) atomicOr(a.status, 1u);
    }

    const size_t cell = (size_t)y * p.pitch + x;
    if constexpr (MODE == kMoments) {
        const size_t o = (size_t)y * p.nx + x;
        if (a.out[0]) a.out[0][o] = phi;
        if (a.out[1]) a.out[1][o] = psi;
        if (a.out[2]) a.out[2][o] = ux;
        if (a.out[3]) a.out[3][o] = uy;
        if (a.out[4]) a.out[4][o] = P;
    } else {

    // ---- phase field f (Sec. 3.1): source cs2 V = d_t(phi u) + cs2 A n ----
    {
        float q[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) q[i] = sF[i * NE + eo];
        collide_scalar(q, phi, ux, uy, dt_fx + third * Aterm * nx_, dt_fy + third * Aterm * ny_,
                       p.s1f, p.s2f, p.s3f, p.s4f);
#pragma unroll
        for (int i = 0; i < 9; ++i) a.dst[(size_t)i * p.plane + cell] = q[i];
    }
    // ---- surfactant g (Sec. 3.2): source cs2 V = d_t(psi u) + cs2 B n ----
    {
        float q[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) q[i] = sG[i * NE + eo];
        collide_scalar(q, psi, ux, uy, dt_gx + third * Bterm * nx_, dt_gy + third * Bterm * ny_,
                       p.s1g, p.s2g, p.s3g, p.s4g);
#pragma unroll
        for (int i = 0; i < 9; ++i) a.dst[(size_t)(kPlaneG + i) * p.plane + cell] = q[i];
    }
    // ---- flow h (Sec. 3.3) ----
    {
        const float mu = p.muB + (phi - p.phiB) * p.inv_dphi * p.dmu;
        const float s2 = 1.f / (3.f * mu * p.inv_rho + 0.5f);
        const float s1 = p.s1h, s3 = p.s3h, s4 = p.tie_s4h ? s2 : p.s4h;
        const float Jx = rho * ux, Jy = rho * uy;
        // equilibrium moments: (., Jx, Jy, P + Jx ux, P + Jy uy, Jx uy, Jx/3, Jy/3, P/3 + J.u/3)
        // source moments:      (., Fx, Fy, dt_xx, dt_yy, dt_xy, Fx/3, Fy/3, (dt_xx + dt_yy)/3)
        const float m3 = h[1] + h[3] + h[5] + h[6] + h[7] + h[8];
        const float m4 = h[2] + h[4] + h[5] + h[6] + h[7] + h[8];
        const float m5 = h[5] - h[6] + h[7] - h[8];
        const float m6 = h[5] - h[6] - h[7] + h[8];
        const float m7 = h[5] + h[6] - h[7] - h[8];
        const float m8 = h[5] + h[6] + h[7] + h[8];
        // increments dm_k = -s_k (m_k - m_eq_k) + (1 - s_k/2) m_src_k, then h* = h + M^-1 dm
        const float d1 = -s1 * (jx - Jx) + (1.f - 0.5f * s1) * Fx;
        const float d2 = -s1 * (jy - Jy) + (1.f - 0.5f * s1) * Fy;
        const float d3 = -s2 * (m3 - (P + Jx * ux)) + (1.f - 0.5f * s2) * dt_xx;
        const float d4 = -s2 * (m4 - (P + Jy * uy)) + (1.f - 0.5f * s2) * dt_yy;
        const float d5 = -s2 * (m5 - Jx * uy) + (1.f - 0.5f * s2) * dt_xy;
        const float d6 = -s3 * (m6 - Jx * third) + (1.f - 0.5f * s3) * Fx * third;
        const float d7 = -s3 * (m7 - Jy * third) + (1.f - 0.5f * s3) * Fy * third;
        const float d8 = -s4 * (m8 - third * (P + Jx * ux + Jy * uy)) + (1.f - 0.5f * s4) * third * (dt_xx + dt_yy);
        float q[9];
        q[1] = h[1] + 0.5f * (d1 + d3 - d6 - d8);
        q[2] = h[2] + 0.5f * (d2 + d4 - d7 - d8);
        q[3] = h[3] + 0.5f * (-d1 + d3 + d6 - d8);
        q[4] = h[4] + 0.5f * (-d2 + d4 + d7 - d8);
        q[5] = h[5] + 0.25f * (d5 + d6 + d7 + d8);
        q[6] = h[6] + 0.25f * (-d5 - d6 + d7 + d8);
        q[7] = h[7] + 0.25f * (d5 - d6 - d7 + d8);
        q[8] = h[8] + 0.25f * (-d5 + d6 - d7 + d8);
        if (WALLS) {
            // moving-wall term for the links that leave through a wall, folded in before storing:
            // h_ibar(x_b, t+1) = h*_i(x_b, t) - 2 w_i rho c_i.u_w / cs2
            if (y == 0) {
                q[7] -= 6.f * wgt(7) * rho * (-1.f) * p.u_bot;
                q[8] -= 6.f * wgt(8) * rho * (1.f) * p.u_bot;
            }
            if (y == p.ny - 1) {
                q[5] -= 6.f * wgt(5) * rho * (1.f) * p.u_top;
                q[6] -= 6.f * wgt(6) * rho * (-1.f) * p.u_top;
            }
        }
#pragma unroll
        for (int i = 1; i < 9; ++i) a.dst[(size_t)(kPlaneH + i - 1) * p.plane + cell] = q[i];
    }
    a.hist[cell] = ux;
    a.hist[p.plane + cell] = uy;
    }
}

// ---- initialisation: equilibria of the given fields, written where the first pull reads them ----
struct InitArgs {
    Phys p;
    const double* __restrict__ phi;
    const double* __restrict__ psi;
    const double* __restrict__ ux;
    const double* __restrict__ uy;
    const double* __restrict__ P;
    float* __restrict__ dst;
    float* __restrict__ hist;
    unsigned* __restrict__ status;
    int langmuir;
    int walls;
};

__global__ void init_kernel(const __grid_constant__ InitArgs a) {
    const Phys& p = a.p;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const size_t o = (size_t)y * p.nx + x;
    const double phi = a.phi[o], psi = a.psi[o], ux = a.ux[o], uy = a.uy[o], P = a.P[o];
    bool bad = !(isfinite(phi) && isfinite(psi) && isfinite(ux) && isfinite(uy) && isfinite(P));
    if (a.langmuir) bad = bad || !(psi < 1.0);
    if (bad) atomicOr(a.status, 1u);
    const double rho = p.rho;
    const double uu = ux * ux + uy * uy;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const double cu = cx(i) * ux + cy(i) * uy;
        const double w = i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        const double feq = w * phi * (1.0 + 3.0 * cu);
        const double geq = w * psi * (1.0 + 3.0 * cu);
        const double heq = w * (3.0 * P + 3.0 * rho * cu + 4.5 * rho * (cu * cu - uu / 3.0));
        // the first pull at x for direction i reads slot i of x - c_i, or, across a wall, the
        // opposite slot of x itself
        int tx_ = x - cx(i), ty_ = y - cy(i), plane = i;
        if (a.walls && (ty_ < 0 || ty_ >= p.ny)) {
            tx_ = x; ty_ = y; plane = opp(i);
        } else {
            tx_ = (tx_ + p.nx) % p.nx;
            ty_ = (ty_ + p.ny) % p.ny;
        }
        const size_t cell = (size_t)ty_ * p.pitch + tx_;
        a.dst[(size_t)plane * p.plane + cell] = (float)feq;
        a.dst[(size_t)(kPlaneG + plane) * p.plane + cell] = (float)geq;
        if (plane != 0) a.dst[(size_t)(kPlaneH + plane - 1) * p.plane + cell] = (float)heq;
    }
    const size_t cell = (size_t)y * p.pitch + x;
    a.hist[cell] = (float)ux;
    a.hist[p.plane + cell] = (float)uy;
}

// ---- FP64 sums of phi or psi: every population slot is pulled exactly once per step, so the
// total of a field is the plain sum of its 9 planes over the valid cells ----
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

__global__ void __launch_bounds__(kReduceThreads) reduce_partial_kernel(const float* __restrict__ planes, int nx,
                                                                        int ny, int pitch, long long plane,
                                                                        double* __restrict__ partials) {
    __shared__ double smem[32];
    double acc = 0.0;
    // block b owns rows b, b + gridDim.x, ...; threads stride over (plane, x)
    for (int y = blockIdx.x; y < ny; y += gridDim.x) {
        for (int k = threadIdx.x; k < 9 * nx; k += blockDim.x) {
            const int i = k / nx, x = k - i * nx;
            acc += (double)planes[(size_t)i * plane + (size_t)y * pitch + x];
        }
    }
    acc = block_sum(acc, smem);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kReduceThreads) reduce_final_kernel(const double* __restrict__ partials, int n,
                                                                      double* __restrict__ out) {
    __shared__ double smem[32];
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) acc += partials[k];
    acc = block_sum(acc, smem);
    if (threadIdx.x == 0) *out = acc;
}

}  // namespace lbm
