/*
 * lbo.h -- plain FP64 CPU oracle of the coupled lattice Boltzmann step for
 * N-phase flows with liquid-solid phase change (Huang, Zhan, Chai, Huang, Liu,
 * "A diffuse-interface model for N-phase flows with liquid-solid phase change",
 * arXiv 2603.22902, Sections 2 and 3).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously-correct reference
 * that the CUDA path is checked against.  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no source,
 * header, table or helper with the CUDA library.
 *
 * Lattice: D2Q9, c_s^2 = 1/3, dx = dt = 1.  Fields are row-major [ny][nx]
 * (x fastest).  Sides are indexed 0 = x-min, 1 = x-max, 2 = y-min, 3 = y-max.
 */
#ifndef LBO_H
#define LBO_H

#ifdef __cplusplus
extern "C" {
#endif

#define LBO_MAXN 4

enum { LBO_PERIODIC = 0, LBO_WALL = 1, LBO_OUTFLOW = 2 };
enum { LBO_ADIABATIC = 0, LBO_DIRICHLET = 1 };

typedef struct {
    int nx, ny, N;
    /* per-phase liquid / solid properties (eq. 2 of Section 2) */
    double rho_l[LBO_MAXN], rho_s[LBO_MAXN];
    double mu_l[LBO_MAXN], mu_s[LBO_MAXN];
    double lam_l[LBO_MAXN], lam_s[LBO_MAXN];
    double cp_l[LBO_MAXN], cp_s[LBO_MAXN];
    double latent[LBO_MAXN];          /* specific latent heat L_p; 0 = never changes phase */
    double sigma[LBO_MAXN * LBO_MAXN]; /* pairwise surface tension, symmetric, zero diagonal */
    double eps;                        /* interface width epsilon */
    double mobility;                   /* M = c_s^2 (tau_g - 1/2) */
    double T_sol, T_liq;               /* solidus / liquidus temperatures (eq. H) */
    double rho_ref, cp_ref;            /* reference density and heat capacity of the enthalpy LBE */
    double u_solid[2];                 /* solid velocity u_s of the penalty force */
    double accel[2];                   /* body acceleration; G = rho * accel */
    int bc[4];                         /* LBO_PERIODIC / LBO_WALL / LBO_OUTFLOW per side */
    int tbc[4];                        /* LBO_ADIABATIC / LBO_DIRICHLET per side (walls only) */
    double T_wall[4];                  /* Dirichlet wall temperature per side */
    double wet_cos[4][LBO_MAXN * LBO_MAXN]; /* cos(theta_pq) per wall side, antisymmetric */
    int two_phase_textbook;            /* N = 2 only: textbook two-phase interface terms (pin) */
    int penalty_literal;               /* pin only: penalty weight f_s instead of f_s * sum of
                                          the phase-changing phi_p (shows that the frozen-layer
                                          pin tells the two readings apart) */
} lbo_params;

typedef struct lbo_state lbo_state;

/* Build the state from initial fields phi[N][ny][nx], T, ux, uy (t = 0):
 * rho*H from the inverse of eq. H, p = 0, all populations at equilibrium.
 * Returns NULL on invalid parameters. */
lbo_state* lbo_create(const lbo_params* P, const double* phi, const double* T,
                      const double* ux, const double* uy);
void lbo_destroy(lbo_state* s);

/* Advance nsteps time steps. */
void lbo_step(lbo_state* s, long nsteps);
long lbo_steps(const lbo_state* s);

/* Macroscopic fields of the current state (NULL = skip):
 * phi[N][ny][nx], T, specific enthalpy H = (rho H)/rho, liquid fraction f_l,
 * velocity u, pressure p, mixture density rho, volumetric enthalpy rho*H. */
void lbo_fields(lbo_state* s, double* phi, double* T, double* H, double* fl,
                double* ux, double* uy, double* p, double* rho, double* rhoH);

/* Raw populations (pre-collision, post-streaming) f[9], g[N][9], h[9] planes. */
void lbo_populations(const lbo_state* s, double* f, double* g, double* h);

/* Cell-local pieces exposed for the pins. */
void lbo_enthalpy_map(const lbo_params* P, const double* phi, double rhoH,
                      double* fl, double* T, double* rho, double* psi, double* chi);
double lbo_inverse_map(const lbo_params* P, const double* phi, double T);

/* Isotropic gradient / Laplacian of one scalar field with the boundary
 * rules of the step (zero-gradient ghosts at walls and outflows). */
void lbo_stencil(const lbo_params* P, const double* field, double* gx, double* gy, double* lap);

#ifdef __cplusplus
}
#endif
#endif
