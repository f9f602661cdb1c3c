/*
 * lbo.c -- plain FP64 CPU oracle of the coupled lattice Boltzmann time step
 * of arXiv 2603.22902 ("A diffuse-interface model for N-phase flows with
 * liquid-solid phase change").
 *
 * TEST INFRASTRUCTURE ONLY: slow, obviously correct, never used by the product
 * path.  Built with -O2 -ffp-contract=off so every product and sum is rounded
 * exactly as written.
 *
 * One step follows the paper in this order, one full-field pass per stage:
 *   A  moments         phi_p = sum_i g_ip / (1 - mdot'/2)        (Sec. 3, phi recovery)
 *                      rhoH  = sum_i h_i + Q'/2                  (Sec. 3, H recovery)
 *   B  mixture + map   eq. 2 mixtures, eq. H -> (f_l, T), f_s = 1 - f_l
 *   C  stencils        isotropic gradients / Laplacians of phi_p, rho, psi
 *   D  interface       pairwise normals n_pq, R_p, chemical potential mu_p,
 *                      surface force F_s = sum_p mu_p grad phi_p   (Sec. 2)
 *   E  flow            u*, penalty f, u, mdot, S, Lambda, p      (Sec. 3, flow LBE)
 *   F  collisions      f (flow), g_p (phase field), h (enthalpy) (Sec. 3)
 *   G  lagged fields   mdot', Q' = rho c_p T mdot, psi', (phi_p u)'
 *   H  streaming       with bounce-back walls, outflow copy, periodic wrap,
 *                      non-equilibrium extrapolation for Dirichlet temperature
 * A primed quantity (') is the value stored by the previous step.
 * The readings of passages the paper leaves open are listed in the design notes;
 * the ones that change arithmetic are named where they are used below.
 *
 * Parity unpinned (no test ties these to anything but the code itself):
 *   (none left: the pairwise wetting ghost of N > 2 is pinned by the Janus drop's
 *   wetting lengths of Table 2, and the penalty weight in mixed cells by the frozen
 *   layer under a driven channel of ambient fluid)
 */
#include "lbo.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 (Section 3 uses c_s = c / sqrt(3)). */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
#define CS2 (1.0 / 3.0)

/* Thresholds of the two guards in the pairwise normal (stage D). */
#define PAIR_SUM_MIN 1e-12
#define NORMAL_MIN 1e-12

struct lbo_state {
    lbo_params P;
    int nx, ny, N, nc;
    long steps;
    double *f, *g, *h;    /* pre-collision populations [9][nc], [N][9][nc], [9][nc] */
    double *fp, *gp, *hp; /* post-collision populations, same layout */
    double *mdot_m, *Q_m, *psi_m, *phiu_m; /* lagged: [nc], [nc], [nc], [N][2][nc] */
    double *wall_h;                        /* NEE ghosts: [2 y-sides][9][nx] */
    /* work fields of the current state */
    double *phi, *rhoH, *fl, *T, *rho, *mu, *lam, *cp, *psi, *chi; /* phi: [N][nc] */
    double *gphi, *lphi, *grho, *gpsi; /* [N][2][nc], [N][nc], [2][nc], [2][nc] */
    double *ux, *uy, *p, *mdot;
};

/* ------------------------------------------------------------------------ */
/* Section 2, eq. 2 and eq. H                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
    double rs, rl;   /* solid / liquid mixture density   sum_p phi_p rho_p^{s,l} */
    double cs, cl;   /* solid / liquid mixture heat capacity                     */
    double ms, ml;   /* solid / liquid mixture viscosity                         */
    double ks, kl;   /* solid / liquid mixture conductivity                      */
    double Lv;       /* latent heat per volume sum_p phi_p rho_p^l L_p           */
    double drho;     /* sum_p (rho_p^s - rho_p^l) phi_p                          */
    double pcm;      /* sum of phi_p over the phases that change phase (L_p > 0) */
} mixture_t;

static mixture_t mixture(const lbo_params* P, const double* phi)
{
    mixture_t m;
    memset(&m, 0, sizeof m);
    for (int p = 0; p < P->N; ++p) {
        m.rs += phi[p] * P->rho_s[p];
        m.rl += phi[p] * P->rho_l[p];
        m.cs += phi[p] * P->cp_s[p];
        m.cl += phi[p] * P->cp_l[p];
        m.ms += phi[p] * P->mu_s[p];
        m.ml += phi[p] * P->mu_l[p];
        m.ks += phi[p] * P->lam_s[p];
        m.kl += phi[p] * P->lam_l[p];
        m.Lv += phi[p] * P->rho_l[p] * P->latent[p];
        m.drho += (P->rho_s[p] - P->rho_l[p]) * phi[p];
        if (P->latent[p] > 0.0) m.pcm += phi[p];
    }
    return m;
}

/* eq. H: liquid fraction and temperature from the volumetric enthalpy.
 * rho_s H_s = rs cs T_s and rho_l H_l = rl cl T_l + Lv.  A cell without any
 * phase-changing material (Lv <= 0) is liquid: the ambient fluid has f_s = 0
 * (Fig. 1 caption). */
static void enthalpy_map(const lbo_params* P, const mixture_t* m, double rhoH, double* fl, double* T)
{
    const double As = m->rs * m->cs * P->T_sol;
    const double Al = m->rl * m->cl * P->T_liq + m->Lv;
    if (!(m->Lv > 0.0)) {
        *fl = 1.0;
        *T = P->T_liq + (rhoH - Al) / (m->rl * m->cl);
    } else if (rhoH < As) {
        *fl = 0.0;
        *T = rhoH / (m->rs * m->cs);
    } else if (rhoH > Al) {
        *fl = 1.0;
        *T = P->T_liq + (rhoH - Al) / (m->rl * m->cl);
    } else if (Al - As > 0.0) {
        *fl = (rhoH - As) / (Al - As);
        *T = P->T_sol + (*fl) * (P->T_liq - P->T_sol);
    } else {
        *fl = 1.0;
        *T = P->T_liq;
    }
}

/* Inverse of eq. H used at t = 0: a cell at or above the liquidus is liquid. */
static double inverse_map(const lbo_params* P, const mixture_t* m, double T)
{
    const double As = m->rs * m->cs * P->T_sol;
    const double Al = m->rl * m->cl * P->T_liq + m->Lv;
    if (!(m->Lv > 0.0)) return Al + m->rl * m->cl * (T - P->T_liq);
    if (T < P->T_sol) return m->rs * m->cs * T;
    if (T >= P->T_liq) return Al + m->rl * m->cl * (T - P->T_liq);
    return As + (T - P->T_sol) / (P->T_liq - P->T_sol) * (Al - As);
}

void lbo_enthalpy_map(const lbo_params* P, const double* phi, double rhoH, double* fl,
                      double* T, double* rho, double* psi, double* chi)
{
    mixture_t m = mixture(P, phi);
    double l, t;
    enthalpy_map(P, &m, rhoH, &l, &t);
    const double fs = 1.0 - l;
    if (fl) *fl = l;
    if (T) *T = t;
    if (rho) *rho = fs * m.rs + l * m.rl;
    if (psi) *psi = fs * m.drho;
    if (chi) *chi = fs * m.pcm;
}

double lbo_inverse_map(const lbo_params* P, const double* phi, double T)
{
    mixture_t m = mixture(P, phi);
    return inverse_map(P, &m, T);
}

/* ------------------------------------------------------------------------ */
/* Stencils with the boundary ghost rules                                    */
/* ------------------------------------------------------------------------ */

/* Cell index of neighbour x + c_i.  Periodic sides wrap; any other side clamps
 * to the boundary node (zero-gradient ghost).  *wx / *wy receive the wall side
 * crossed in x / y, or -1. */
static int neighbour(const lbo_params* P, int x, int y, int i, int* wx, int* wy)
{
    int X = x + CX[i], Y = y + CY[i];
    *wx = -1;
    *wy = -1;
    if (X < 0 || X >= P->nx) {
        const int side = X < 0 ? 0 : 1;
        if (P->bc[side] == LBO_PERIODIC) {
            X = (X + P->nx) % P->nx;
        } else {
            if (P->bc[side] == LBO_WALL) *wx = side;
            X = X < 0 ? 0 : P->nx - 1;
        }
    }
    if (Y < 0 || Y >= P->ny) {
        const int side = Y < 0 ? 2 : 3;
        if (P->bc[side] == LBO_PERIODIC) {
            Y = (Y + P->ny) % P->ny;
        } else {
            if (P->bc[side] == LBO_WALL) *wy = side;
            Y = Y < 0 ? 0 : P->ny - 1;
        }
    }
    return Y * P->nx + X;
}

/* Isotropic second-order stencils:
 *   grad chi = sum_i w_i c_i chi(x + c_i) / c_s^2
 *   lap  chi = sum_{i != 0} 2 w_i (chi(x + c_i) - chi(x)) / c_s^2            */
static void scalar_stencil(const lbo_params* P, const double* a, int x, int y, double* gx,
                           double* gy, double* lap)
{
    double v[9];
    for (int i = 0; i < 9; ++i) {
        int wx, wy;
        v[i] = a[neighbour(P, x, y, i, &wx, &wy)];
    }
    double sx = 0.0, sy = 0.0, sl = 0.0;
    for (int i = 0; i < 9; ++i) {
        sx += W[i] * CX[i] * v[i];
        sy += W[i] * CY[i] * v[i];
    }
    for (int i = 1; i < 9; ++i) sl += 2.0 * W[i] * (v[i] - v[0]);
    *gx = sx / CS2;
    *gy = sy / CS2;
    *lap = sl / CS2;
}

void lbo_stencil(const lbo_params* P, const double* field, double* gx, double* gy, double* lap)
{
    for (int y = 0; y < P->ny; ++y)
        for (int x = 0; x < P->nx; ++x) {
            const int c = y * P->nx + x;
            scalar_stencil(P, field, x, y, &gx[c], &gy[c], &lap[c]);
        }
}

/* Order parameters at neighbour x + c_i.  At a wall the ghost value carries
 * the wetting condition n_w . grad phi_p = -(4/eps) sum_q cos(theta_pq) phi_p phi_q
 * (central difference across the half-way wall), from the boundary node. */
static void phi_neighbour(const lbo_state* s, int x, int y, int i, double* out)
{
    const lbo_params* P = &s->P;
    int wx, wy;
    const int c = neighbour(P, x, y, i, &wx, &wy);
    double ph[LBO_MAXN];
    for (int p = 0; p < s->N; ++p) ph[p] = s->phi[p * s->nc + c];
    for (int p = 0; p < s->N; ++p) {
        double corr = 0.0;
        for (int q = 0; q < s->N; ++q) {
            if (q == p) continue;
            double cosv = 0.0;
            if (wx >= 0) cosv += P->wet_cos[wx][p * LBO_MAXN + q];
            if (wy >= 0) cosv += P->wet_cos[wy][p * LBO_MAXN + q];
            corr += cosv * ph[p] * ph[q];
        }
        out[p] = ph[p] + 4.0 / P->eps * corr;
    }
}

/* ------------------------------------------------------------------------ */
/* Stages A, B, C                                                            */
/* ------------------------------------------------------------------------ */

/* The per-cell loops below carry `omp parallel for`: every cell of a stage writes only
 * its own outputs and reads the previous stage's, so a build with -fopenmp (the
 * multi-threaded timing of the benchmark) gives bitwise the same results; the default
 * build ignores the pragmas. */
static void stage_A(lbo_state* s)
{
#pragma omp parallel for schedule(static)
    for (int c = 0; c < s->nc; ++c) {
        for (int p = 0; p < s->N; ++p) {
            double sum = 0.0;
            for (int i = 0; i < 9; ++i) sum += s->g[(p * 9 + i) * s->nc + c];
            s->phi[p * s->nc + c] = sum / (1.0 - 0.5 * s->mdot_m[c]);
        }
        double sh = 0.0;
        for (int i = 0; i < 9; ++i) sh += s->h[i * s->nc + c];
        s->rhoH[c] = sh + 0.5 * s->Q_m[c];
    }
}

static void stage_B(lbo_state* s)
{
#pragma omp parallel for schedule(static)
    for (int c = 0; c < s->nc; ++c) {
        double ph[LBO_MAXN];
        for (int p = 0; p < s->N; ++p) ph[p] = s->phi[p * s->nc + c];
        mixture_t m = mixture(&s->P, ph);
        double l, t;
        enthalpy_map(&s->P, &m, s->rhoH[c], &l, &t);
        const double fs = 1.0 - l;
        s->fl[c] = l;
        s->T[c] = t;
        s->rho[c] = fs * m.rs + l * m.rl;
        s->mu[c] = fs * m.ms + l * m.ml;
        s->lam[c] = fs * m.ks + l * m.kl;
        s->cp[c] = fs * m.cs + l * m.cl;
        s->psi[c] = fs * m.drho;
        /* penalty weight: the solid volume fraction f_s * sum of the phase-changing phi_p
         * (reading of the penalty force in cells that also hold ambient fluid) */
        s->chi[c] = s->P.penalty_literal ? fs : fs * m.pcm;
    }
}

static void stage_C(lbo_state* s)
{
    const int nc = s->nc, N = s->N;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < s->ny; ++y)
        for (int x = 0; x < s->nx; ++x) {
            const int c = y * s->nx + x;
            double v[9][LBO_MAXN];
            for (int i = 0; i < 9; ++i) phi_neighbour(s, x, y, i, v[i]);
            for (int p = 0; p < N; ++p) {
                double sx = 0.0, sy = 0.0, sl = 0.0;
                for (int i = 0; i < 9; ++i) {
                    sx += W[i] * CX[i] * v[i][p];
                    sy += W[i] * CY[i] * v[i][p];
                }
                for (int i = 1; i < 9; ++i) sl += 2.0 * W[i] * (v[i][p] - v[0][p]);
                s->gphi[(p * 2 + 0) * nc + c] = sx / CS2;
                s->gphi[(p * 2 + 1) * nc + c] = sy / CS2;
                s->lphi[p * nc + c] = sl / CS2;
            }
            double lap;
            scalar_stencil(&s->P, s->rho, x, y, &s->grho[c], &s->grho[nc + c], &lap);
            scalar_stencil(&s->P, s->psi, x, y, &s->gpsi[c], &s->gpsi[nc + c], &lap);
        }
}

/* ------------------------------------------------------------------------ */
/* Equilibria and source terms (Section 3)                                   */
/* ------------------------------------------------------------------------ */

/* s_i(u) = w_i [ c_i.u / c_s^2 + (c_i.u)^2 / (2 c_s^4) - u.u / (2 c_s^2) ] */
static double s_i(int i, double ux, double uy)
{
    const double cu = CX[i] * ux + CY[i] * uy;
    return W[i] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - (ux * ux + uy * uy) / (2.0 * CS2));
}

/* pressure-based flow equilibrium */
static double f_eq(int i, double p, double rho, double ux, double uy)
{
    const double pw = (i == 0) ? p / CS2 * (W[0] - 1.0) : p / CS2 * W[i];
    return pw + rho * s_i(i, ux, uy);
}

/* F_i = w_i [ S + c_i.(F + rho f) / c_s^2 + (c_i c_i - c_s^2 I) : Lambda / (2 c_s^4) ] */
static double force_i(int i, double S, double Fx, double Fy, double Lxx, double Lxy, double Lyy)
{
    const double cf = CX[i] * Fx + CY[i] * Fy;
    const double q = (CX[i] * CX[i] - CS2) * Lxx + 2.0 * CX[i] * CY[i] * Lxy + (CY[i] * CY[i] - CS2) * Lyy;
    return W[i] * (S + cf / CS2 + q / (2.0 * CS2 * CS2));
}

/* enthalpy equilibrium with the isotropic part carried by rho_ref c_p,ref T */
static double h_eq(const lbo_params* P, int i, double rhoH, double T, double rho, double cp,
                   double ux, double uy)
{
    const double E = P->rho_ref * P->cp_ref * T;
    const double uu = ux * ux + uy * uy;
    if (i == 0) return rhoH - E + W[0] * (E - rho * cp * T * uu / (2.0 * CS2));
    const double cu = CX[i] * ux + CY[i] * uy;
    const double q = cu * cu - CS2 * uu;
    return W[i] * (E + rho * cp * T * (cu / CS2 + q / (2.0 * CS2 * CS2)));
}

/* g'(x) for g(x) = x^2 (1 - x)^2 */
static double gprime(double x) { return 2.0 * x * (1.0 - x) * (1.0 - 2.0 * x); }

/* ------------------------------------------------------------------------ */
/* Stages D-G for one cell                                                   */
/* ------------------------------------------------------------------------ */

static void cell_update(lbo_state* s, int x, int y, int collide)
{
    const lbo_params* P = &s->P;
    const int nc = s->nc, N = s->N;
    const int c = y * s->nx + x;
    double ph[LBO_MAXN], gx[LBO_MAXN], gy[LBO_MAXN], lp[LBO_MAXN];
    for (int p = 0; p < N; ++p) {
        ph[p] = s->phi[p * nc + c];
        gx[p] = s->gphi[(p * 2 + 0) * nc + c];
        gy[p] = s->gphi[(p * 2 + 1) * nc + c];
        lp[p] = s->lphi[p * nc + c];
    }
    const double rho = s->rho[c];

    /* D: R_p = sum_{q != p} 4 phi_p phi_q / eps n_pq,  n_pq = grad phi_pq / |grad phi_pq|,
     *    phi_pq = phi_p / (phi_p + phi_q);
     *    mu_p = sum_{q != p} 2 beta_pq [g'(phi_p) - g'(phi_p + phi_q)] - k_pq lap phi_q,
     *    beta_pq = 3 sigma_pq / eps,  k_pq = -3 eps sigma_pq / 4;  F_s = sum_p mu_p grad phi_p */
    double Rx[LBO_MAXN], Ry[LBO_MAXN], mu_phi[LBO_MAXN];
    double Fsx = 0.0, Fsy = 0.0;
    if (!P->two_phase_textbook) {
        for (int p = 0; p < N; ++p) {
            Rx[p] = 0.0;
            Ry[p] = 0.0;
            mu_phi[p] = 0.0;
            for (int q = 0; q < N; ++q) {
                if (q == p) continue;
                const double sum = ph[p] + ph[q];
                double nx = 0.0, ny = 0.0;
                if (sum > PAIR_SUM_MIN) {
                    /* quotient rule: grad phi_pq = (phi_q grad phi_p - phi_p grad phi_q) / (phi_p + phi_q)^2 */
                    const double Gx = (ph[q] * gx[p] - ph[p] * gx[q]) / (sum * sum);
                    const double Gy = (ph[q] * gy[p] - ph[p] * gy[q]) / (sum * sum);
                    const double Gn = sqrt(Gx * Gx + Gy * Gy);
                    if (Gn > NORMAL_MIN) {
                        nx = Gx / Gn;
                        ny = Gy / Gn;
                    }
                }
                Rx[p] += 4.0 * ph[p] * ph[q] / P->eps * nx;
                Ry[p] += 4.0 * ph[p] * ph[q] / P->eps * ny;
                const double sig = P->sigma[p * LBO_MAXN + q];
                const double beta = 3.0 / P->eps * sig;
                const double kap = -3.0 * P->eps / 4.0 * sig;
                mu_phi[p] += 2.0 * beta * (gprime(ph[p]) - gprime(ph[p] + ph[q])) - kap * lp[q];
            }
        }
        for (int p = 0; p < N; ++p) {
            Fsx += mu_phi[p] * gx[p];
            Fsy += mu_phi[p] * gy[p];
        }
    } else {
        /* two-phase conservative Allen-Cahn with the standard free energy:
         * R = 4 phi (1 - phi) / eps n,  mu = (12 sigma / eps) g'(phi) - (3 sigma eps / 2) lap phi,
         * F_s = mu grad phi, all from phi = phi_1 alone */
        const double phi = ph[0];
        const double gn = sqrt(gx[0] * gx[0] + gy[0] * gy[0]);
        double nx = 0.0, ny = 0.0;
        if (gn > NORMAL_MIN) {
            nx = gx[0] / gn;
            ny = gy[0] / gn;
        }
        Rx[0] = 4.0 * phi * (1.0 - phi) / P->eps * nx;
        Ry[0] = 4.0 * phi * (1.0 - phi) / P->eps * ny;
        Rx[1] = -Rx[0];
        Ry[1] = -Ry[0];
        const double sig = P->sigma[0 * LBO_MAXN + 1];
        const double mu = 12.0 * sig / P->eps * gprime(phi) - 3.0 * sig * P->eps / 2.0 * lp[0];
        Fsx = mu * gx[0];
        Fsy = mu * gy[0];
    }
    const double Fx = Fsx + rho * P->accel[0]; /* F = F_s + G */
    const double Fy = Fsy + rho * P->accel[1];

    /* E: rho u* = sum c_i f_i + F/2,  f = f_s^v (u_s - u*),  u = u* + f/2 */
    double jx = 0.0, jy = 0.0, sum_f_not0 = 0.0;
    double fi[9];
    for (int i = 0; i < 9; ++i) {
        fi[i] = s->f[i * nc + c];
        jx += CX[i] * fi[i];
        jy += CY[i] * fi[i];
        if (i != 0) sum_f_not0 += fi[i];
    }
    const double usx = (jx + 0.5 * Fx) / rho;
    const double usy = (jy + 0.5 * Fy) / rho;
    const double fpx = s->chi[c] * (P->u_solid[0] - usx);
    const double fpy = s->chi[c] * (P->u_solid[1] - usy);
    const double ux = usx + 0.5 * fpx;
    const double uy = usy + 0.5 * fpy;

    /* mdot = -(1/rho) D psi / Dt, backward difference in time */
    const double gpsx = s->gpsi[c], gpsy = s->gpsi[nc + c];
    const double mdot = -((s->psi[c] - s->psi_m[c]) + (ux * gpsx + uy * gpsy)) / rho;
    /* S = rho mdot + u . grad rho */
    const double S = rho * mdot + (ux * s->grho[c] + uy * s->grho[nc + c]);
    /* Lambda = uF + Fu + c_s^2 S I */
    const double Lxx = 2.0 * ux * Fx + CS2 * S;
    const double Lyy = 2.0 * uy * Fy + CS2 * S;
    const double Lxy = ux * Fy + uy * Fx;
    const double tau_f = s->mu[c] / (rho * CS2) + 0.5;
    const double F0 = force_i(0, S, Fx + rho * fpx, Fy + rho * fpy, Lxx, Lxy, Lyy);
    const double p = CS2 / (1.0 - W[0]) * (sum_f_not0 + 0.5 * S + (tau_f - 0.5) * F0 + rho * s_i(0, ux, uy));

    s->ux[c] = ux;
    s->uy[c] = uy;
    s->p[c] = p;
    s->mdot[c] = mdot;
    if (!collide) return;

    /* F: flow collision */
    for (int i = 0; i < 9; ++i) {
        const double feq = f_eq(i, p, rho, ux, uy);
        const double Fi = force_i(i, S, Fx + rho * fpx, Fy + rho * fpy, Lxx, Lxy, Lyy);
        s->fp[i * nc + c] = fi[i] - (fi[i] - feq) / tau_f + (1.0 - 1.0 / (2.0 * tau_f)) * Fi;
    }
    /* phase-field collisions: g_eq = w_i phi_p (1 + c_i.u / c_s^2),
     * G = w_i [c_i . d_t(phi_p u) / c_s^2 + c_i . R_p] + w_i phi_p mdot */
    const double tau_g = P->mobility / CS2 + 0.5;
    for (int p = 0; p < N; ++p) {
        const double dtx = ph[p] * ux - s->phiu_m[(p * 2 + 0) * nc + c];
        const double dty = ph[p] * uy - s->phiu_m[(p * 2 + 1) * nc + c];
        for (int i = 0; i < 9; ++i) {
            const double gi = s->g[(p * 9 + i) * nc + c];
            const double geq = W[i] * ph[p] * (1.0 + (CX[i] * ux + CY[i] * uy) / CS2);
            const double Gi = W[i] * ((CX[i] * dtx + CY[i] * dty) / CS2 + (CX[i] * Rx[p] + CY[i] * Ry[p])) +
                              W[i] * ph[p] * mdot;
            s->gp[(p * 9 + i) * nc + c] = gi - (gi - geq) / tau_g + (1.0 - 1.0 / (2.0 * tau_g)) * Gi;
        }
    }
    /* enthalpy collision: tau_h = lambda / (rho_ref c_p,ref c_s^2) + 1/2, H_i = w_i rho c_p T mdot */
    const double T = s->T[c], cp = s->cp[c], rhoH = s->rhoH[c];
    const double tau_h = s->lam[c] / (P->rho_ref * P->cp_ref * CS2) + 0.5;
    double heq[9];
    for (int i = 0; i < 9; ++i) {
        const double hi = s->h[i * nc + c];
        heq[i] = h_eq(P, i, rhoH, T, rho, cp, ux, uy);
        const double Hi = W[i] * rho * cp * T * mdot;
        s->hp[i * nc + c] = hi - (hi - heq[i]) / tau_h + (1.0 - 1.0 / (2.0 * tau_h)) * Hi;
    }
    /* Dirichlet temperature by non-equilibrium extrapolation: the ghost node behind
     * the half-way wall has T_g = 2 T_w - T and u = 0; its post-collision population
     * is h_eq(ghost) + (1 - 1/tau_h) (h_i - h_eq_i) of this boundary node. */
    for (int side = 2; side < 4; ++side) {
        const int row = side == 2 ? 0 : s->ny - 1;
        if (y != row || P->bc[side] != LBO_WALL || P->tbc[side] != LBO_DIRICHLET) continue;
        const double Tg = 2.0 * P->T_wall[side] - T;
        for (int i = 0; i < 9; ++i) {
            const int inward = side == 2 ? (CY[i] > 0) : (CY[i] < 0);
            if (!inward) continue;
            const double ghost_eq = h_eq(P, i, 0.0, Tg, rho, cp, 0.0, 0.0);
            s->wall_h[((side - 2) * 9 + i) * s->nx + x] =
                ghost_eq + (1.0 - 1.0 / tau_h) * (s->h[i * nc + c] - heq[i]);
        }
    }

    /* G: lagged fields for the next step */
    s->mdot_m[c] = mdot;
    s->Q_m[c] = rho * cp * T * mdot;
    s->psi_m[c] = s->psi[c];
    for (int p = 0; p < N; ++p) {
        s->phiu_m[(p * 2 + 0) * nc + c] = ph[p] * ux;
        s->phiu_m[(p * 2 + 1) * nc + c] = ph[p] * uy;
    }
}

/* ------------------------------------------------------------------------ */
/* Stage H: streaming with boundary rules                                    */
/* ------------------------------------------------------------------------ */

/* Post-streaming value of population i at (x, y) of one species plane set.
 * The upstream node x - c_i: periodic sides wrap; an x-wall reflects (half-way
 * bounce-back) before anything else; an outflow side copies from the same
 * boundary row/column; a y-wall reflects, or takes the NEE ghost for the
 * enthalpy populations at a Dirichlet wall. */
static double pulled(const lbo_state* s, const double* post, int x, int y, int i, int is_h)
{
    const lbo_params* P = &s->P;
    int X = x - CX[i], Y = y - CY[i];
    if (X < 0 || X >= s->nx) {
        const int side = X < 0 ? 0 : 1;
        if (P->bc[side] == LBO_PERIODIC) X = (X + s->nx) % s->nx;
        else if (P->bc[side] == LBO_OUTFLOW) X = x;
        else return post[OPP[i] * s->nc + y * s->nx + x];
    }
    if (Y < 0 || Y >= s->ny) {
        const int side = Y < 0 ? 2 : 3;
        if (P->bc[side] == LBO_PERIODIC) Y = (Y + s->ny) % s->ny;
        else if (P->bc[side] == LBO_OUTFLOW) Y = y;
        else if (is_h && P->tbc[side] == LBO_DIRICHLET) return s->wall_h[((side - 2) * 9 + i) * s->nx + X];
        else return post[OPP[i] * s->nc + y * s->nx + x];
    }
    return post[i * s->nc + Y * s->nx + X];
}

static void stage_H(lbo_state* s)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < s->ny; ++y)
        for (int x = 0; x < s->nx; ++x) {
            const int c = y * s->nx + x;
            for (int i = 0; i < 9; ++i) {
                s->f[i * s->nc + c] = pulled(s, s->fp, x, y, i, 0);
                s->h[i * s->nc + c] = pulled(s, s->hp, x, y, i, 1);
                for (int p = 0; p < s->N; ++p)
                    s->g[(p * 9 + i) * s->nc + c] = pulled(s, s->gp + (size_t)p * 9 * s->nc, x, y, i, 0);
            }
        }
}

/* ------------------------------------------------------------------------ */
/* Public entry points                                                       */
/* ------------------------------------------------------------------------ */

static int valid(const lbo_params* P)
{
    if (P->nx < 3 || P->ny < 3 || P->N < 2 || P->N > LBO_MAXN) return 0;
    if (!(P->eps > 0.0) || !(P->mobility > 0.0) || !(P->rho_ref > 0.0) || !(P->cp_ref >= 0.0)) return 0;
    if (!(P->T_sol <= P->T_liq)) return 0;
    if (P->two_phase_textbook && P->N != 2) return 0;
    for (int p = 0; p < P->N; ++p) {
        if (!(P->rho_l[p] > 0.0) || !(P->rho_s[p] > 0.0) || !(P->cp_l[p] > 0.0) || !(P->cp_s[p] > 0.0)) return 0;
        if (!(P->mu_l[p] >= 0.0) || !(P->mu_s[p] >= 0.0) || !(P->lam_l[p] > 0.0) || !(P->lam_s[p] > 0.0)) return 0;
        if (!(P->latent[p] >= 0.0)) return 0;
        for (int q = 0; q < P->N; ++q) {
            if (P->sigma[p * LBO_MAXN + q] != P->sigma[q * LBO_MAXN + p]) return 0;
            if (p == q && P->sigma[p * LBO_MAXN + q] != 0.0) return 0;
        }
    }
    for (int side = 0; side < 4; ++side) {
        if (P->bc[side] < 0 || P->bc[side] > 2) return 0;
        if (P->tbc[side] == LBO_DIRICHLET && P->bc[side] != LBO_WALL) return 0;
        if (P->tbc[side] == LBO_DIRICHLET && side < 2) return 0;
    }
    if ((P->bc[0] == LBO_PERIODIC) != (P->bc[1] == LBO_PERIODIC)) return 0;
    if ((P->bc[2] == LBO_PERIODIC) != (P->bc[3] == LBO_PERIODIC)) return 0;
    return 1;
}

static double* zalloc(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

lbo_state* lbo_create(const lbo_params* Pin, const double* phi0, const double* T0, const double* ux0,
                      const double* uy0)
{
    if (!valid(Pin)) return NULL;
    lbo_state* s = (lbo_state*)calloc(1, sizeof *s);
    s->P = *Pin;
    lbo_params* P = &s->P;
    /* reference heat capacity c_p,ref = 2 c_p,s c_p,l / (c_p,s + c_p,l) (Section 3) of the
     * first phase unless the caller gives one */
    if (P->cp_ref == 0.0) P->cp_ref = 2.0 * P->cp_s[0] * P->cp_l[0] / (P->cp_s[0] + P->cp_l[0]);
    s->nx = P->nx;
    s->ny = P->ny;
    s->N = P->N;
    s->nc = P->nx * P->ny;
    const size_t nc = (size_t)s->nc, N = (size_t)s->N;
    s->f = zalloc(9 * nc);
    s->g = zalloc(9 * N * nc);
    s->h = zalloc(9 * nc);
    s->fp = zalloc(9 * nc);
    s->gp = zalloc(9 * N * nc);
    s->hp = zalloc(9 * nc);
    s->mdot_m = zalloc(nc);
    s->Q_m = zalloc(nc);
    s->psi_m = zalloc(nc);
    s->phiu_m = zalloc(2 * N * nc);
    s->wall_h = zalloc(2 * 9 * (size_t)s->nx);
    s->phi = zalloc(N * nc);
    s->rhoH = zalloc(nc);
    s->fl = zalloc(nc);
    s->T = zalloc(nc);
    s->rho = zalloc(nc);
    s->mu = zalloc(nc);
    s->lam = zalloc(nc);
    s->cp = zalloc(nc);
    s->psi = zalloc(nc);
    s->chi = zalloc(nc);
    s->gphi = zalloc(2 * N * nc);
    s->lphi = zalloc(N * nc);
    s->grho = zalloc(2 * nc);
    s->gpsi = zalloc(2 * nc);
    s->ux = zalloc(nc);
    s->uy = zalloc(nc);
    s->p = zalloc(nc);
    s->mdot = zalloc(nc);

    /* t = 0: rho H from the inverse of eq. H, then eq. H forward for f_l and T,
     * p = 0, populations at equilibrium, mdot' = Q' = 0, psi' = psi, (phi u)' = phi u */
    for (size_t c = 0; c < nc; ++c) {
        double ph[LBO_MAXN];
        for (size_t p = 0; p < N; ++p) ph[p] = phi0[p * nc + c];
        mixture_t m = mixture(P, ph);
        const double rhoH = inverse_map(P, &m, T0[c]);
        double l, t;
        enthalpy_map(P, &m, rhoH, &l, &t);
        const double fs = 1.0 - l;
        const double rho = fs * m.rs + l * m.rl;
        const double cp = fs * m.cs + l * m.cl;
        const double ux = ux0 ? ux0[c] : 0.0, uy = uy0 ? uy0[c] : 0.0;
        for (int i = 0; i < 9; ++i) {
            s->f[i * nc + c] = f_eq(i, 0.0, rho, ux, uy);
            s->h[i * nc + c] = h_eq(P, i, rhoH, t, rho, cp, ux, uy);
            for (size_t p = 0; p < N; ++p)
                s->g[(p * 9 + i) * nc + c] = W[i] * ph[p] * (1.0 + (CX[i] * ux + CY[i] * uy) / CS2);
        }
        s->mdot_m[c] = 0.0;
        s->Q_m[c] = 0.0;
        s->psi_m[c] = fs * m.drho;
        for (size_t p = 0; p < N; ++p) {
            s->phiu_m[(p * 2 + 0) * nc + c] = ph[p] * ux;
            s->phiu_m[(p * 2 + 1) * nc + c] = ph[p] * uy;
        }
    }
    return s;
}

void lbo_destroy(lbo_state* s)
{
    if (!s) return;
    double* bufs[] = {s->f,    s->g,     s->h,   s->fp,   s->gp,   s->hp,   s->mdot_m, s->Q_m,
                      s->psi_m, s->phiu_m, s->wall_h, s->phi, s->rhoH, s->fl, s->T,      s->rho,
                      s->mu,   s->lam,   s->cp,  s->psi,  s->chi,  s->gphi, s->lphi,   s->grho,
                      s->gpsi, s->ux,    s->uy,  s->p,    s->mdot};
    for (size_t k = 0; k < sizeof bufs / sizeof bufs[0]; ++k) free(bufs[k]);
    free(s);
}

void lbo_step(lbo_state* s, long nsteps)
{
    for (long n = 0; n < nsteps; ++n) {
        stage_A(s);
        stage_B(s);
        stage_C(s);
#pragma omp parallel for schedule(static)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) cell_update(s, x, y, 1);
        stage_H(s);
        s->steps++;
    }
}

long lbo_steps(const lbo_state* s) { return s->steps; }

void lbo_fields(lbo_state* s, double* phi, double* T, double* H, double* fl, double* ux, double* uy,
                double* p, double* rho, double* rhoH)
{
    /* stages A-E on the current state, without collision; the lagged fields are
     * left untouched because cell_update returns before stage G */
    stage_A(s);
    stage_B(s);
    stage_C(s);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < s->ny; ++y)
        for (int x = 0; x < s->nx; ++x) cell_update(s, x, y, 0);
    const size_t nc = (size_t)s->nc;
    for (size_t c = 0; c < nc; ++c) {
        if (phi)
            for (int q = 0; q < s->N; ++q) phi[q * nc + c] = s->phi[q * nc + c];
        if (T) T[c] = s->T[c];
        if (H) H[c] = s->rhoH[c] / s->rho[c];
        if (fl) fl[c] = s->fl[c];
        if (ux) ux[c] = s->ux[c];
        if (uy) uy[c] = s->uy[c];
        if (p) p[c] = s->p[c];
        if (rho) rho[c] = s->rho[c];
        if (rhoH) rhoH[c] = s->rhoH[c];
    }
}

void lbo_populations(const lbo_state* s, double* f, double* g, double* h)
{
    const size_t nc = (size_t)s->nc;
    if (f) memcpy(f, s->f, 9 * nc * sizeof(double));
    if (g) memcpy(g, s->g, 9 * (size_t)s->N * nc * sizeof(double));
    if (h) memcpy(h, s->h, 9 * nc * sizeof(double));
}
