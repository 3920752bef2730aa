/*
 * FP64 CPU oracle for the three-population phase-field lattice-Boltzmann step of arXiv 2408.15654.
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the benchmark).
 * This header belongs to the oracle alone; the CUDA library has its own and includes nothing here.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_EOS_LINEAR 0
#define ORC_EOS_LANGMUIR 1

typedef struct {
    int nx, ny;
    int walls;             /* 0: periodic in y; 1: bounce-back walls below y = 0 and above y = ny - 1 */
    int eos;               /* ORC_EOS_LINEAR or ORC_EOS_LANGMUIR */
    double u_top, u_bot;   /* x velocity of the top / bottom wall */
    double phiA, phiB, rhoA, rhoB, muA, muB;
    double W, M_phi, D, sigma0, E0;
    double gx, gy;         /* body-force acceleration */
    double rho0;           /* constant in lambda_0 of h_eq */
    double n_eps;          /* |grad phi| threshold below which n = 0 */
    double s_f[5], s_g[5], s_h[5]; /* (s0, s1, s2, s3, s4); the transport entries are recomputed */
    int prescribed;        /* 0: u from the flow populations; 1: u imposed (the initial ux, uy), no h */
} orc_params;

/* Everything the equilibria and source distributions of one cell depend on. */
typedef struct {
    double phi, psi, ux, uy, P, rho;
    double nx, ny;                    /* interface normal */
    double Fx, Fy;                    /* total force */
    double Sx, Sy;                    /* mass flux */
    double drho_x, drho_y;            /* grad rho */
    double dt_phiux, dt_phiuy;        /* d_t(phi u) */
    double dt_psiux, dt_psiuy;        /* d_t(psi u) */
    double dt_m2_xx, dt_m2_xy, dt_m2_yy; /* d_t(rho u u - (S u + u S)/2) */
} orc_cell_in;

/* Diagnostic per-cell output at the current time level. */
typedef struct {
    double phi, psi, ux, uy, P;
    double gpx, gpy, lap;     /* grad phi, lap phi */
    double gsx, gsy;          /* grad psi */
    double Fx, Fy;            /* total force */
    double Fmx, Fmy;          /* Marangoni part */
} orc_cell_out;

typedef struct orc_sim orc_sim;

orc_sim* orc_create(const orc_params* p);
void orc_destroy(orc_sim* s);
int orc_init(orc_sim* s, const double* phi, const double* psi, const double* ux, const double* uy,
             const double* P);
int orc_step(orc_sim* s, long nsteps);
int orc_moments(orc_sim* s, double* phi, double* psi, double* ux, double* uy, double* P);
int orc_fields(orc_sim* s, orc_cell_out* out);
double orc_sum(orc_sim* s, int what);
void orc_populations(orc_sim* s, double* f, double* g, double* h);
int orc_status(const orc_sim* s);
long orc_steps(const orc_sim* s);
int orc_set_threads(int n);

void orc_cell_distributions(const orc_params* p, const orc_cell_in* c, double feq[9], double F[9],
                            double geq[9], double G[9], double heq[9], double H[9]);
void orc_operators(const double s5[5], double lam[81], double src[81]);
void orc_moment_matrix(double m[81]);
void orc_lattice(int cx[9], int cy[9], double w[9]);

#ifdef __cplusplus
}
#endif
#endif
