/*
 * FP64 CPU oracle for the three-population phase-field lattice-Boltzmann step of
 * Zhan, Liang, Chai & Shi, "Phase-field-based lattice Boltzmann method for the transport of
 * insoluble surfactant in two-phase flows" (arXiv 2408.15654).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the CUDA library is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load it; the library never does, and it shares no code with the library.
 *
 * What it computes, in the paper's order (Sec. 3, Sec. 4 preamble):
 *   phase field      f_i -> phi   (Sec. 3.1, Eq. for f_eq / F_i, s_1^f from M_phi)
 *   surfactant       g_i -> psi   (Sec. 3.2, Eq. for g_eq / G_i, Eq. for s_1^g from D)
 *   flow             h_i -> u, P  (Sec. 3.3, h_eq / H_i / m_2H, Eq. for u and P, s_2^h from mu)
 *   coupling         rho(phi), mu(phi), mass flux S, delta-function approximation,
 *                    surface-tension force (capillary + Marangoni, expanded form), EOS
 *                    (Sec. 2.2, Sec. 2.3: Eqs. for rho/mu, S, F_s, Langmuir and linear EOS)
 *   collision        dense 9x9 operators M^-1 S M and M^-1 (I - S/2) M with the natural moment
 *                    matrix M printed in Sec. 4 (M^-1 is obtained here by Gauss-Jordan)
 *   streaming        f_i(x + c_i, t + 1) = f*_i(x, t), periodic in x, periodic in y or
 *                    half-way bounce-back walls (Sec. 4, Ladd's scheme) with a moving-wall term
 *
 * Readings where the paper is silent (each is listed with its reason in the design notes):
 *   - gradients / Laplacian: isotropic D2Q9 stencils
 *       d_a phi = (1/cs2) sum_i w_i c_ia phi(x + c_i),
 *       lap phi = (2/cs2) sum_{i != 0} w_i [phi(x + c_i) - phi(x)];
 *     next to a wall the missing neighbour takes the value of the adjacent fluid cell;
 *   - n = grad phi / |grad phi| when |grad phi| > n_eps, else n = 0;
 *   - time derivatives are backward differences over one step; on the first step after
 *     initialisation they are zero;
 *   - rho u = sum_i c_i h_i + F/2, u = (rho u) / rho;
 *   - grad sigma = sigma'(psi) grad psi;  grad rho = drho/dphi grad phi;
 *   - body force F_b = rho g;
 *   - moving-wall bounce-back for h: h_ibar(x_b, t+1) = h*_i(x_b, t) - 2 w_i rho(x_b, t) c_i.u_w / cs2;
 *     f and g use plain bounce-back (no flux);
 *   - initial populations are the equilibria of the initial fields;
 *   - the free relaxation rates are parameters; a non-positive s4^h stands for s4^h = s2^h.
 *
 * Precision: FP64, round to nearest, compiled without FMA contraction or fast-math.
 *
 * Direct check (tests/test_bruteforce_8x8.py): an independent NumPy statement of the step in
 * distribution space equals every population to 1e-13 after 1 and 10 steps on 8 x 8 grids.
 * Pins (tests/test_oracle_pins.py): the printed M; D2Q9 isotropy; the Appendix A conditions on
 * Lambda, g_eq and G (and the same for f_eq, F); the moments of h_eq and H; recovery of u and P
 * from an equilibrium state; stencils exact on quadratics; the Marangoni integral across a flat
 * interface (linear and Langmuir EOS); vanishing chemical potential on the tanh profile;
 * conservation of sum phi and sum psi; exact rest state; square symmetry; stationary tanh and
 * sech^2 profiles; surfactant swept out of the bulk; surface-diffusion decay exp(-D t/R^2);
 * convection-diffusion of a sine mode; Laplace jump (linear and Langmuir EOS); exact Couette flow;
 * Couette start-up; shear-wave viscous decay; Poiseuille profile under a body force; the closed
 * form of uniformly accelerated flow (pins K); wall channel = mirrored periodic domain.
 * Prescribed-velocity mode (the convection test of Sec. 4): only f and g evolve, u is the imposed
 * field given at initialisation (constant in time, so d_t(phi u) = u d_t phi), there is no h and
 * P is reported as 0.  Pins: with u = 0 it equals the full model at rest with sigma0 = 0; a sine
 * mode of psi is advected and damped as exp(-D k^2 t) sin(k (x - u t)); the centroid of a
 * convected drop moves at u.
 * The terms that act only when rhoA != rhoB (mass flux S, grad rho in H, m2H and P, the S history)
 * have no closed form at a finite interface width; they are pinned by closed forms of the continuum
 * equations that the discrete solution must approach as the interface is resolved: a layered
 * gravity-driven channel (second order), uniform translation of a drop, of a relaxing slab (where S
 * is parallel to u) and of a relaxing drop (which fixes the sign of S), and hydrostatic layers.
 * Dropping S from h_eq, the grad rho part of m2H or u.grad rho from P, flipping the sign of S,
 * taking nu = mu instead of mu / rho, or taking u = sum c h + F/2 without 1/rho, each fails one
 * of them.  The time derivative of S (the S history) is pinned by the same translating relaxing
 * slab refined in the acoustic scaling (velocity, M_phi / W and nu / W fixed in lattice units),
 * where u d_t S is as large as the fluxes it corrects: the deviation from uniform translation
 * falls at about second order, and with the previous S taken equal to the current one it stops
 * falling (a copy of this file with that mistake is built and checked by the tests).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "lbm_oracle.h"

/* ---------------------------------------------------------------------------------------
 * D2Q9 lattice (Sec. 4).  The velocity order is the one fixed by the columns of the printed
 * natural moment matrix M: rest, +x, +y, -x, -y, (+1,+1), (-1,+1), (-1,-1), (+1,-1).
 * Weights are the standard D2Q9 weights; cs2 = c^2 / 3 with c = dx/dt = 1.
 * ------------------------------------------------------------------------------------- */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WGT[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const double CS2 = 1.0 / 3.0;

/* The natural transformation matrix M as printed in Sec. 4 (rows: 1, cx, cy, cx^2, cy^2,
 * cx cy, cx cy^2, cx^2 cy, cx^2 cy^2). */
static const double M_NAT[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 1, 0, 1, 0, 1, 1, 1, 1},
    {0, 0, 1, 0, 1, 1, 1, 1, 1},
    {0, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 1, -1, -1, 1},
    {0, 0, 0, 0, 0, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, 1, 1, 1, 1},
};

static int opposite(int i) {
    for (int j = 0; j < 9; ++j)
        if (CX[j] == -CX[i] && CY[j] == -CY[i]) return j;
    return -1;
}

/* Inverse of M by Gauss-Jordan elimination with partial pivoting. */
static void invert9(const double a_in[9][9], double inv[9][9]) {
    double a[9][18];
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 18; ++c) a[r][c] = c < 9 ? a_in[r][c] : (c - 9 == r ? 1.0 : 0.0);
    for (int col = 0; col < 9; ++col) {
        int piv = col;
        for (int r = col + 1; r < 9; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (piv != col)
            for (int c = 0; c < 18; ++c) {
                double t = a[col][c];
                a[col][c] = a[piv][c];
                a[piv][c] = t;
            }
        double p = a[col][col];
        for (int c = 0; c < 18; ++c) a[col][c] /= p;
        for (int r = 0; r < 9; ++r) {
            if (r == col) continue;
            double m = a[r][col];
            if (m == 0.0) continue;
            for (int c = 0; c < 18; ++c) a[r][c] -= m * a[col][c];
        }
    }
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) inv[r][c] = a[r][c + 9];
}

/* Collision operator Lambda = M^-1 S M and source operator M^-1 (I - S/2) M for the diagonal
 * S = diag(s0, s1, s1, s2, s2, s2, s3, s3, s4) (Sec. 3 evolution equations, Sec. 4). */
static void operators(const double s5[5], double lam[9][9], double src[9][9]) {
    double minv[9][9];
    invert9(M_NAT, minv);
    const double sdiag[9] = {s5[0], s5[1], s5[1], s5[2], s5[2], s5[2], s5[3], s5[3], s5[4]};
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            double l = 0.0, s = 0.0;
            for (int k = 0; k < 9; ++k) {
                l += minv[i][k] * sdiag[k] * M_NAT[k][j];
                s += minv[i][k] * (1.0 - 0.5 * sdiag[k]) * M_NAT[k][j];
            }
            lam[i][j] = l;
            src[i][j] = s;
        }
}

/* ---------------------------------------------------------------------------------------
 * Material laws and equation of state (Sec. 2.2, Sec. 2.3)
 * ------------------------------------------------------------------------------------- */
static double density(const orc_params* p, double phi) {
    return (phi - p->phiB) / (p->phiA - p->phiB) * (p->rhoA - p->rhoB) + p->rhoB;
}
static double viscosity(const orc_params* p, double phi) {
    return (phi - p->phiB) / (p->phiA - p->phiB) * (p->muA - p->muB) + p->muB;
}
/* sigma(psi) and d sigma / d psi: Langmuir (eos = 1) or its linearisation (eos = 0). */
static double surface_tension(const orc_params* p, double psi) {
    if (p->eos == ORC_EOS_LANGMUIR) return p->sigma0 * (1.0 + p->E0 * log(1.0 - psi));
    return p->sigma0 * (1.0 - p->E0 * psi);
}
static double surface_tension_slope(const orc_params* p, double psi) {
    if (p->eos == ORC_EOS_LANGMUIR) return -p->sigma0 * p->E0 / (1.0 - psi);
    return -p->sigma0 * p->E0;
}

/* Relaxation rates: user rates for the free moments, transport rates from Sec. 3:
 *   1/s1^f = M_phi/cs2 + 1/2,  1/s1^g = D/cs2 + 1/2,  1/s2^h = mu/(rho cs2) + 1/2. */
static void rates_f(const orc_params* p, double s[5]) {
    memcpy(s, p->s_f, sizeof(double) * 5);
    s[1] = 1.0 / (p->M_phi / CS2 + 0.5);
}
static void rates_g(const orc_params* p, double s[5]) {
    memcpy(s, p->s_g, sizeof(double) * 5);
    s[1] = 1.0 / (p->D / CS2 + 0.5);
}
static void rates_h(const orc_params* p, double rho, double mu, double s[5]) {
    memcpy(s, p->s_h, sizeof(double) * 5);
    s[2] = 1.0 / (mu / (rho * CS2) + 0.5);
    if (s[4] <= 0.0) s[4] = s[2]; /* a non-positive s4^h means: relax the fourth moment with s2^h */
}

/* ---------------------------------------------------------------------------------------
 * Equilibria and source distributions of one cell (Sec. 3.1-3.3)
 * ------------------------------------------------------------------------------------- */

/* f_eq = w_i phi (1 + c_i.u/cs2);  F_i = w_i c_i.d_t(phi u)/cs2 + w_i c_i.[4(phiA-phi)(phi-phiB)/(W dphi)] n */
static void phase_distributions(const orc_cell_in* c, const orc_params* p, double feq[9], double F[9]) {
    const double dphi = p->phiA - p->phiB;
    const double A = 4.0 * (p->phiA - c->phi) * (c->phi - p->phiB) / (p->W * dphi);
    for (int i = 0; i < 9; ++i) {
        const double cu = CX[i] * c->ux + CY[i] * c->uy;
        feq[i] = WGT[i] * c->phi * (1.0 + cu / CS2);
        F[i] = WGT[i] * (CX[i] * c->dt_phiux + CY[i] * c->dt_phiuy) / CS2 +
               WGT[i] * (CX[i] * A * c->nx + CY[i] * A * c->ny);
    }
}

/* g_eq = w_i psi (1 + c_i.u/cs2);  G_i = w_i c_i.d_t(psi u)/cs2 + w_i c_i.[4 psi (phiA+phiB-2phi)/(W dphi)] n */
static void surfactant_distributions(const orc_cell_in* c, const orc_params* p, double geq[9], double G[9]) {
    const double dphi = p->phiA - p->phiB;
    const double B = 4.0 * c->psi * (p->phiA + p->phiB - 2.0 * c->phi) / (p->W * dphi);
    for (int i = 0; i < 9; ++i) {
        const double cu = CX[i] * c->ux + CY[i] * c->uy;
        geq[i] = WGT[i] * c->psi * (1.0 + cu / CS2);
        G[i] = WGT[i] * (CX[i] * c->dt_psiux + CY[i] * c->dt_psiuy) / CS2 +
               WGT[i] * (CX[i] * B * c->nx + CY[i] * B * c->ny);
    }
}

/* h_eq = lambda_i + w_i [c_i.rho u/cs2 + (rho u - S)u : (c_i c_i - cs2 I)/(2 cs2^2)],
 *   lambda_0 = rho0 + (w0 - 1) P/cs2, lambda_i = w_i P/cs2;
 * H_i = w_i [u.grad rho + c_i.F/cs2 + m2H : (c_i c_i - cs2 I)/(2 cs2^2)],
 *   m2H = d_t(rho u u - (S u + u S)/2) + cs2 (u grad rho + grad rho u). */
static void flow_distributions(const orc_cell_in* c, const orc_params* p, double heq[9], double H[9]) {
    const double u[2] = {c->ux, c->uy};
    const double S[2] = {c->Sx, c->Sy};
    const double gr[2] = {c->drho_x, c->drho_y};
    double Q[2][2], m2H[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            Q[a][b] = (c->rho * u[a] - S[a]) * u[b];
            m2H[a][b] = CS2 * (u[a] * gr[b] + gr[a] * u[b]);
        }
    m2H[0][0] += c->dt_m2_xx;
    m2H[0][1] += c->dt_m2_xy;
    m2H[1][0] += c->dt_m2_xy;
    m2H[1][1] += c->dt_m2_yy;
    const double ugr = u[0] * gr[0] + u[1] * gr[1];
    for (int i = 0; i < 9; ++i) {
        const double ci[2] = {CX[i], CY[i]};
        double qc = 0.0, mc = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                const double t = ci[a] * ci[b] - (a == b ? CS2 : 0.0);
                qc += Q[a][b] * t;
                mc += m2H[a][b] * t;
            }
        const double lambda = (i == 0) ? p->rho0 + (WGT[0] - 1.0) * c->P / CS2 : WGT[i] * c->P / CS2;
        const double cj = ci[0] * c->rho * u[0] + ci[1] * c->rho * u[1];
        heq[i] = lambda + WGT[i] * (cj / CS2 + qc / (2.0 * CS2 * CS2));
        H[i] = WGT[i] * (ugr + (ci[0] * c->Fx + ci[1] * c->Fy) / CS2 + mc / (2.0 * CS2 * CS2));
    }
}

void orc_cell_distributions(const orc_params* p, const orc_cell_in* c, double feq[9], double F[9],
                            double geq[9], double G[9], double heq[9], double H[9]) {
    phase_distributions(c, p, feq, F);
    surfactant_distributions(c, p, geq, G);
    flow_distributions(c, p, heq, H);
}

void orc_operators(const double s5[5], double lam[81], double src[81]) {
    double l[9][9], s[9][9];
    operators(s5, l, s);
    memcpy(lam, l, sizeof(l));
    memcpy(src, s, sizeof(s));
}

void orc_moment_matrix(double m[81]) { memcpy(m, M_NAT, sizeof(M_NAT)); }

void orc_lattice(int cx[9], int cy[9], double w[9]) {
    memcpy(cx, CX, sizeof(CX));
    memcpy(cy, CY, sizeof(CY));
    memcpy(w, WGT, sizeof(WGT));
}

/* ---------------------------------------------------------------------------------------
 * Simulation state
 * ------------------------------------------------------------------------------------- */
struct orc_sim {
    orc_params p;
    long N;
    double *f, *g, *h;             /* pre-collision populations, [9][ny][nx] (h keeps all 9) */
    double *fs, *gs, *hs;          /* post-collision scratch */
    double *phi, *psi;             /* zeroth moments at the current time level */
    double *phi_prev, *psi_prev;   /* history (time level n - 1) */
    double *ux_prev, *uy_prev, *Sx_prev, *Sy_prev;
    double *ux_imp, *uy_imp;       /* imposed velocity (prescribed mode) */
    int first;                     /* 1: no history yet, time derivatives are zero */
    long steps;
    int status;
};

static int wrap(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

/* Value of a cell-centred field at (x, y) with the boundary rules: periodic in x; in y either
 * periodic or, with walls, the adjacent fluid cell's value beyond the wall. */
static double field_at(const orc_sim* s, const double* a, int x, int y) {
    const int nx = s->p.nx, ny = s->p.ny;
    x = wrap(x, nx);
    if (s->p.walls) {
        if (y < 0) y = 0;
        if (y >= ny) y = ny - 1;
    } else {
        y = wrap(y, ny);
    }
    return a[(long)y * nx + x];
}

/* Isotropic stencils for grad and Laplacian of a cell field. */
static void stencils(const orc_sim* s, const double* a, int x, int y, double* gx, double* gy, double* lap) {
    const double a0 = field_at(s, a, x, y);
    double sx = 0.0, sy = 0.0, sl = 0.0;
    for (int i = 0; i < 9; ++i) {
        const double ai = field_at(s, a, x + CX[i], y + CY[i]);
        sx += WGT[i] * CX[i] * ai;
        sy += WGT[i] * CY[i] * ai;
        if (i != 0) sl += WGT[i] * (ai - a0);
    }
    *gx = sx / CS2;
    *gy = sy / CS2;
    if (lap) *lap = 2.0 * sl / CS2;
}

orc_sim* orc_create(const orc_params* p) {
    if (p->nx < 1 || p->ny < 1) return NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->p = *p;
    s->N = (long)p->nx * p->ny;
    const long N = s->N;
    s->f = calloc(9 * N, sizeof(double));
    s->g = calloc(9 * N, sizeof(double));
    s->h = calloc(9 * N, sizeof(double));
    s->fs = calloc(9 * N, sizeof(double));
    s->gs = calloc(9 * N, sizeof(double));
    s->hs = calloc(9 * N, sizeof(double));
    s->phi = calloc(N, sizeof(double));
    s->psi = calloc(N, sizeof(double));
    s->phi_prev = calloc(N, sizeof(double));
    s->psi_prev = calloc(N, sizeof(double));
    s->ux_prev = calloc(N, sizeof(double));
    s->uy_prev = calloc(N, sizeof(double));
    s->Sx_prev = calloc(N, sizeof(double));
    s->Sy_prev = calloc(N, sizeof(double));
    s->ux_imp = calloc(N, sizeof(double));
    s->uy_imp = calloc(N, sizeof(double));
    if (!s->f || !s->g || !s->h || !s->fs || !s->gs || !s->hs || !s->phi || !s->psi || !s->phi_prev ||
        !s->psi_prev || !s->ux_prev || !s->uy_prev || !s->Sx_prev || !s->Sy_prev || !s->ux_imp || !s->uy_imp) {
        orc_destroy(s);
        return NULL;
    }
    s->first = 1;
    return s;
}

void orc_destroy(orc_sim* s) {
    if (!s) return;
    free(s->f); free(s->g); free(s->h);
    free(s->fs); free(s->gs); free(s->hs);
    free(s->phi); free(s->psi);
    free(s->phi_prev); free(s->psi_prev);
    free(s->ux_prev); free(s->uy_prev); free(s->Sx_prev); free(s->Sy_prev);
    free(s->ux_imp); free(s->uy_imp);
    free(s);
}

/* Initial populations = equilibria of the given fields; no history. */
int orc_init(orc_sim* s, const double* phi, const double* psi, const double* ux, const double* uy,
             const double* P) {
    const orc_params* p = &s->p;
    const long N = s->N;
    for (long k = 0; k < N; ++k) {
        orc_cell_in c;
        memset(&c, 0, sizeof(c));
        c.phi = phi[k];
        c.psi = psi[k];
        c.ux = ux[k];
        c.uy = uy[k];
        c.P = P[k];
        c.rho = density(p, phi[k]);
        /* S and grad rho of the initial state only matter for rhoA != rhoB; the initial
         * equilibrium is taken without the mass-flux correction. */
        double feq[9], F[9], geq[9], G[9], heq[9], H[9];
        orc_cell_distributions(p, &c, feq, F, geq, G, heq, H);
        for (int i = 0; i < 9; ++i) {
            s->f[i * N + k] = feq[i];
            s->g[i * N + k] = geq[i];
            s->h[i * N + k] = p->prescribed ? 0.0 : heq[i];
        }
        s->ux_imp[k] = ux[k];
        s->uy_imp[k] = uy[k];
    }
    s->first = 1;
    s->steps = 0;
    s->status = 0;
    return 0;
}

/* Everything a cell needs at time level n: the steps 1-7 of the algorithm.
 * Fills c (inputs to the equilibria / sources) and returns the h relaxation rate via c.s2h. */
typedef struct {
    orc_cell_in c;
    double s2h, mu;
} cell_state;

static void zeroth_moments(orc_sim* s) {
    const long N = s->N;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < N; ++k) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < 9; ++i) {
            a += s->f[i * N + k];
            b += s->g[i * N + k];
        }
        s->phi[k] = a;
        s->psi[k] = b;
    }
}

static void cell_macros(orc_sim* s, int x, int y, cell_state* cs, orc_cell_out* out) {
    const orc_params* p = &s->p;
    const long N = s->N;
    const long k = (long)y * p->nx + x;
    orc_cell_in* c = &cs->c;
    memset(c, 0, sizeof(*c));
    const double dphi = p->phiA - p->phiB;

    /* 1. phi, psi (Sec. 3.1, 3.2) */
    const double phi = s->phi[k], psi = s->psi[k];
    c->phi = phi;
    c->psi = psi;

    /* 2. stencils */
    double gpx, gpy, lap, gsx, gsy;
    stencils(s, s->phi, x, y, &gpx, &gpy, &lap);
    stencils(s, s->psi, x, y, &gsx, &gsy, NULL);

    /* 3. interface normal and delta-function approximations (Sec. 2.2) */
    const double gnorm = sqrt(gpx * gpx + gpy * gpy);
    if (gnorm > p->n_eps) {
        c->nx = gpx / gnorm;
        c->ny = gpy / gnorm;
    } else {
        c->nx = 0.0;
        c->ny = 0.0;
    }
    const double Aterm = 4.0 * (p->phiA - phi) * (phi - p->phiB) / (p->W * dphi);

    /* 4. density, viscosity, relaxation rate of the second-order flow moments */
    const double rho = density(p, phi);
    const double mu = viscosity(p, phi);
    c->rho = rho;
    const double drho = (p->rhoA - p->rhoB) / dphi;
    c->drho_x = drho * gpx;
    c->drho_y = drho * gpy;
    cs->mu = mu;
    cs->s2h = 1.0 / (mu / (rho * CS2) + 0.5);

    /* 5. EOS */
    const double sigma = surface_tension(p, psi);
    const double dsig = surface_tension_slope(p, psi);
    const double gsigx = dsig * gsx, gsigy = dsig * gsy;

    /* 6. surface tension (capillary + Marangoni, expanded form of Sec. 2.3), body force,
     *    mass flux S */
    const double cap = 3.0 * sigma / (2.0 * dphi * dphi) *
                       (16.0 / p->W * (p->phiA - phi) * (phi - p->phiB) * (p->phiA + p->phiB - 2.0 * phi) -
                        p->W * lap);
    const double g2 = gpx * gpx + gpy * gpy;
    const double sdotg = gsigx * gpx + gsigy * gpy;
    const double mar = 3.0 * p->W / (2.0 * dphi * dphi);
    const double Fx = cap * gpx + mar * (g2 * gsigx - sdotg * gpx) + rho * p->gx;
    const double Fy = cap * gpy + mar * (g2 * gsigy - sdotg * gpy) + rho * p->gy;
    c->Fx = Fx;
    c->Fy = Fy;
    const double sfac = p->M_phi * (p->rhoA - p->rhoB) / dphi;
    c->Sx = sfac * (gpx - Aterm * c->nx);
    c->Sy = sfac * (gpy - Aterm * c->ny);

    /* 7. velocity and pressure (Sec. 3.3); in the prescribed mode u is the imposed field */
    double jx = 0.0, jy = 0.0, hsum = 0.0;
    for (int i = 0; i < 9; ++i) {
        const double hi = s->h[i * N + k];
        jx += CX[i] * hi;
        jy += CY[i] * hi;
        if (i != 0) hsum += hi;
    }
    const double ux = p->prescribed ? s->ux_imp[k] : (jx + 0.5 * Fx) / rho;
    const double uy = p->prescribed ? s->uy_imp[k] : (jy + 0.5 * Fy) / rho;
    c->ux = ux;
    c->uy = uy;

    /* time derivatives: backward difference against the stored previous level */
    double phi0 = phi, psi0 = psi, ux0 = ux, uy0 = uy, Sx0 = c->Sx, Sy0 = c->Sy;
    if (!s->first) {
        phi0 = s->phi_prev[k];
        psi0 = s->psi_prev[k];
        ux0 = s->ux_prev[k];
        uy0 = s->uy_prev[k];
        Sx0 = s->Sx_prev[k];
        Sy0 = s->Sy_prev[k];
    }
    const double rho0 = density(p, phi0);
    c->dt_phiux = phi * ux - phi0 * ux0;
    c->dt_phiuy = phi * uy - phi0 * uy0;
    c->dt_psiux = psi * ux - psi0 * ux0;
    c->dt_psiuy = psi * uy - psi0 * uy0;
    c->dt_m2_xx = (rho * ux * ux - c->Sx * ux) - (rho0 * ux0 * ux0 - Sx0 * ux0);
    c->dt_m2_yy = (rho * uy * uy - c->Sy * uy) - (rho0 * uy0 * uy0 - Sy0 * uy0);
    c->dt_m2_xy = (rho * ux * uy - 0.5 * (c->Sx * uy + ux * c->Sy)) -
                  (rho0 * ux0 * uy0 - 0.5 * (Sx0 * uy0 + ux0 * Sy0));
    const double dt_k = (rho * (ux * ux + uy * uy) - (c->Sx * ux + c->Sy * uy)) -
                        (rho0 * (ux0 * ux0 + uy0 * uy0) - (Sx0 * ux0 + Sy0 * uy0));
    const double K = WGT[0] / (1.0 - CS2); /* K = w0 / (c^2 - cs2) with c = 1 */
    const double ugr = ux * c->drho_x + uy * c->drho_y;
    const double jmS_u = (rho * ux - c->Sx) * ux + (rho * uy - c->Sy) * uy;
    c->P = CS2 / (1.0 - WGT[0]) * (hsum + 0.5 * ugr - WGT[0] * jmS_u / (2.0 * CS2) + K * 0.5 * dt_k);
    if (p->prescribed) c->P = 0.0;

    if (out) {
        out->phi = phi;
        out->psi = psi;
        out->ux = ux;
        out->uy = uy;
        out->P = c->P;
        out->gpx = gpx;
        out->gpy = gpy;
        out->lap = lap;
        out->gsx = gsx;
        out->gsy = gsy;
        out->Fx = Fx;
        out->Fy = Fy;
        out->Fmx = mar * (g2 * gsigx - sdotg * gpx);
        out->Fmy = mar * (g2 * gsigy - sdotg * gpy);
    }
}

static void status_check(orc_sim* s, const cell_state* cs) {
    const orc_cell_in* c = &cs->c;
    int bad = !isfinite(c->phi) || !isfinite(c->psi) || !isfinite(c->ux) || !isfinite(c->uy) || !isfinite(c->P);
    if (s->p.eos == ORC_EOS_LANGMUIR && !s->p.prescribed && !(c->psi < 1.0)) bad = 1; /* EOS unused if prescribed */
    if (bad) {
#pragma omp atomic write
        s->status = 1;
    }
}

int orc_step(orc_sim* s, long nsteps) {
    const orc_params* p = &s->p;
    const int nx = p->nx, ny = p->ny;
    const long N = s->N;
    double sf[5], sg[5];
    rates_f(p, sf);
    rates_g(p, sg);
    double lam_f[9][9], src_f[9][9], lam_g[9][9], src_g[9][9];
    operators(sf, lam_f, src_f);
    operators(sg, lam_g, src_g);

    double* rho_now = (double*)malloc(sizeof(double) * N);
    if (!rho_now) return -1;

    for (long step = 0; step < nsteps; ++step) {
        zeroth_moments(s);

        /* collision (Sec. 3 evolution equations, right-hand sides) */
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y) {
            double cached_s2h = -1.0, lam_h[9][9], src_h[9][9];
            for (int x = 0; x < nx; ++x) {
                const long k = (long)y * nx + x;
                cell_state cs;
                cell_macros(s, x, y, &cs, NULL);
                status_check(s, &cs);
                double feq[9], F[9], geq[9], G[9], heq[9], H[9];
                orc_cell_distributions(p, &cs.c, feq, F, geq, G, heq, H);
                if (cs.s2h != cached_s2h) {
                    double sh[5];
                    rates_h(p, cs.c.rho, cs.mu, sh);
                    operators(sh, lam_h, src_h);
                    cached_s2h = cs.s2h;
                }
                for (int i = 0; i < 9; ++i) {
                    double cf = 0.0, cg = 0.0, ch = 0.0;
                    for (int j = 0; j < 9; ++j) {
                        cf += -lam_f[i][j] * (s->f[j * N + k] - feq[j]) + src_f[i][j] * F[j];
                        cg += -lam_g[i][j] * (s->g[j * N + k] - geq[j]) + src_g[i][j] * G[j];
                        ch += -lam_h[i][j] * (s->h[j * N + k] - heq[j]) + src_h[i][j] * H[j];
                    }
                    s->fs[i * N + k] = s->f[i * N + k] + cf;
                    s->gs[i * N + k] = s->g[i * N + k] + cg;
                    s->hs[i * N + k] = p->prescribed ? 0.0 : s->h[i * N + k] + ch;
                }
                rho_now[k] = cs.c.rho;
                /* history for the next step's time derivatives (stored after the sweep) */
                s->ux_prev[k] = cs.c.ux; /* safe: cell_macros of other cells never reads *_prev of k */
                s->uy_prev[k] = cs.c.uy;
                s->Sx_prev[k] = cs.c.Sx;
                s->Sy_prev[k] = cs.c.Sy;
            }
        }
        memcpy(s->phi_prev, s->phi, sizeof(double) * N);
        memcpy(s->psi_prev, s->psi, sizeof(double) * N);
        s->first = 0;

        /* streaming f_i(x + c_i, t + 1) = f*_i(x, t), with half-way bounce-back at walls */
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                const long k = (long)y * nx + x;
                for (int i = 0; i < 9; ++i) {
                    const int xd = wrap(x + CX[i], nx);
                    const int yd_raw = y + CY[i];
                    if (p->walls && (yd_raw < 0 || yd_raw >= ny)) {
                        const int ib = opposite(i);
                        const double uw = yd_raw >= ny ? p->u_top : p->u_bot;
                        s->f[ib * N + k] = s->fs[i * N + k];
                        s->g[ib * N + k] = s->gs[i * N + k];
                        s->h[ib * N + k] =
                            p->prescribed ? 0.0 : s->hs[i * N + k] - 2.0 * WGT[i] * rho_now[k] * (CX[i] * uw) / CS2;
                    } else {
                        const long kd = (long)wrap(yd_raw, ny) * nx + xd;
                        s->f[i * N + kd] = s->fs[i * N + k];
                        s->g[i * N + kd] = s->gs[i * N + k];
                        s->h[i * N + kd] = s->hs[i * N + k];
                    }
                }
            }
        }
        s->steps++;
    }
    free(rho_now);
    return s->status ? 1 : 0;
}

int orc_fields(orc_sim* s, orc_cell_out* out) {
    zeroth_moments(s);
    const int nx = s->p.nx, ny = s->p.ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            cell_state cs;
            cell_macros(s, x, y, &cs, &out[(long)y * nx + x]);
        }
    return 0;
}

int orc_moments(orc_sim* s, double* phi, double* psi, double* ux, double* uy, double* P) {
    const long N = s->N;
    orc_cell_out* out = (orc_cell_out*)malloc(sizeof(orc_cell_out) * N);
    if (!out) return -1;
    orc_fields(s, out);
    for (long k = 0; k < N; ++k) {
        if (phi) phi[k] = out[k].phi;
        if (psi) psi[k] = out[k].psi;
        if (ux) ux[k] = out[k].ux;
        if (uy) uy[k] = out[k].uy;
        if (P) P[k] = out[k].P;
    }
    free(out);
    return 0;
}

double orc_sum(orc_sim* s, int what) {
    zeroth_moments(s);
    const double* a = what == 0 ? s->phi : s->psi;
    double acc = 0.0;
    for (long k = 0; k < s->N; ++k) acc += a[k];
    return acc;
}

void orc_populations(orc_sim* s, double* f, double* g, double* h) {
    const long n = 9 * s->N;
    if (f) memcpy(f, s->f, sizeof(double) * n);
    if (g) memcpy(g, s->g, sizeof(double) * n);
    if (h) memcpy(h, s->h, sizeof(double) * n);
}

int orc_status(const orc_sim* s) { return s->status; }
long orc_steps(const orc_sim* s) { return s->steps; }

int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
