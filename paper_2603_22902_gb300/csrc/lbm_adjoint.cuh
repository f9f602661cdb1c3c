// lbm_adjoint.cuh -- hand-written reverse (adjoint) of the FP64 fused step, for
// gradients of a loss of the final state with respect to the run's parameters.
//
// One step maps set A (populations f, g_p, h and the lagged planes) to set B.  Its
// adjoint maps the adjoint of set B (A-bar_{n+1}) to that of set A (A-bar_n), and adds
// the step's share of the parameter gradients.  It runs in three kernels:
//   1. mac_kernel: phi_p, rho, psi of every cell of A (the stencil inputs), FP64 planes;
//   2. adj_cell_kernel: per cell x, the step of x recomputed, then reversed from the
//      adjoints of everything x wrote (its pushed populations, gathered from A-bar_{n+1}
//      through the same boundary rules, and its lagged outputs).  It writes the adjoint
//      of x's own populations and lagged inputs as used directly, the adjoint of x's own
//      phi_p and rho H as used by x, and, per stencil point k, the adjoint of the
//      stencil inputs phi_p, rho, psi of cell x + c_k (ghost values beyond a wall are
//      folded onto the cell they copy);
//   3. adj_moments_kernel: per cell y, the adjoints of phi_p(y), rho(y), psi(y) summed
//      from every cell whose stencil used y, reversed through y's eq. H map and eq. 2
//      sums and through the moments phi_p = sum g / (1 - mdot'/2), rho H = sum h + Q'/2.
// Kinks of eq. H (the branches at f_l = 0 and 1) take the derivative of the branch the
// forward step took, as do the guards of the pairwise normals (a zero normal has zero
// derivative).  Apart from ill-conditioned normals in the far tails of nearly absent
// phases (ADJ_NORMAL_COND below), the result is the exact derivative of the discrete step.
//
// Parameter gradients accumulate per cell in FP64 planes (slot layout below) and are
// reduced once at the end, in a fixed order.
#pragma once

#include "lbm_device.cuh"
#include "lbm_launch.cuh"
#include "lbm_prec.cuh"
#include "lbm_step.cuh"

namespace lbm {

// Flat index of population i of species s at cell c in a FP64 population set.
__device__ __forceinline__ long long pidx(const KParams& P, int s, int i, long long c)
{
    return i == 0 ? (long long)s * P.S + c : P.rest_elems + (long long)(s * 8 + i - 1) * P.S + c;
}

__device__ __forceinline__ int dir_of(int dx, int dy)
{
    for (int k = 0; k < 9; ++k)
        if (cx(k) == dx && cy(k) == dy) return k;
    return 0;
}

// Target slot of the push of q_J from (x, y) (the rules of push()): false when dropped.
template <int KIND>
__device__ __forceinline__ bool push_target(const KParams& P, int J, int x, int y, long long& cell, int& slot)
{
    int tx = x + cx(J), ty = y + cy(J);
    bool xo = false, yo = false;
    if (cx(J) != 0 && (unsigned)tx >= (unsigned)P.nx) {
        if (P.bc[0] == PERIODIC) tx = tx < 0 ? tx + P.nx : tx - P.nx;
        else xo = true;
    }
    if (cy(J) != 0 && (unsigned)ty >= (unsigned)P.ny) {
        if (P.bc[2] == PERIODIC) ty = ty < 0 ? ty + P.ny : ty - P.ny;
        else yo = true;
    }
    const long long own = (long long)y * P.nx + x;
    if (!xo && !yo) {
        cell = (long long)ty * P.nx + tx;
        slot = J;
        return true;
    }
    if (xo) {
        cell = own;
        slot = opp(J);
        return true;
    }
    const int side = ty < 0 ? 2 : 3;
    if (P.bc[side] == WALL && !(KIND == KIND_H && P.tbc[side] == DIRICHLET)) {
        cell = own;
        slot = opp(J);
        return true;
    }
    return false;
}

// Target of a boundary-row write (push_row): slot J of (x + c_J, y); false beyond an x wall.
__device__ __forceinline__ bool row_target(const KParams& P, int J, int x, int y, long long& cell)
{
    int tx = x + cx(J);
    if (cx(J) != 0 && (unsigned)tx >= (unsigned)P.nx) {
        if (P.bc[0] != PERIODIC) return false;
        tx = tx < 0 ? tx + P.nx : tx - P.nx;
    }
    cell = (long long)y * P.nx + tx;
    return true;
}

// Adjoint of everything cell (x, y) wrote for species s (KIND) from its nine pushes
// (plus the outflow row copies of the same values).
template <int KIND>
__device__ __forceinline__ void gather_species(const KParams& P, const double* bpop, int s, int x, int y,
                                               double (&qb)[9])
{
    for (int j = 0; j < 9; ++j) {
        long long cell;
        int slot;
        qb[j] = push_target<KIND>(P, j, x, y, cell, slot) ? bpop[pidx(P, s, slot, cell)] : 0.0;
    }
    if (y == 0 && P.bc[2] == OUTFLOW) {
        const int js[3] = {2, 5, 6};
        for (int m = 0; m < 3; ++m) {
            long long cell;
            if (row_target(P, js[m], x, y, cell)) qb[js[m]] += bpop[pidx(P, s, js[m], cell)];
        }
    }
    if (y == P.ny - 1 && P.bc[3] == OUTFLOW) {
        const int js[3] = {4, 7, 8};
        for (int m = 0; m < 3; ++m) {
            long long cell;
            if (row_target(P, js[m], x, y, cell)) qb[js[m]] += bpop[pidx(P, s, js[m], cell)];
        }
    }
}

// Reverse of eq. H: adjoints (fl_b, T_b) of the outputs -> adjoints of the mixture sums
// and of rho H, along the branch the forward map takes.
template <int N>
__device__ __forceinline__ void map_reverse(const KParams& P, const Mix<N>& m, double rhoH, double fl_b, double T_b,
                                            double& rs_b, double& rl_b, double& cs_b, double& cl_b, double& Lv_b,
                                            double& rhoH_b)
{
    const double rcs = m.rs * m.cs, rcl = m.rl * m.cl;
    const double As = rcs * P.T_sol;
    const double Al = fma(rcl, P.T_liq, m.Lv);
    double rcs_b = 0.0, rcl_b = 0.0, As_b = 0.0, Al_b = 0.0;
    if (!(m.Lv > 0.0) || (!(rhoH < As) && rhoH > Al)) {
        // liquid: f_l = 1, T = T_liq + (rhoH - Al) / rcl
        rhoH_b += T_b / rcl;
        Al_b -= T_b / rcl;
        rcl_b -= (rhoH - Al) / (rcl * rcl) * T_b;
    } else if (rhoH < As) {
        // solid: f_l = 0, T = rhoH / rcs
        rhoH_b += T_b / rcs;
        rcs_b -= rhoH / (rcs * rcs) * T_b;
    } else if (Al - As > 0.0) {
        // mushy: f_l = (rhoH - As) / (Al - As), T = T_sol + f_l (T_liq - T_sol)
        const double d = Al - As;
        const double fl = (rhoH - As) / d;
        const double flb = fl_b + T_b * (P.T_liq - P.T_sol);
        rhoH_b += flb / d;
        As_b += flb * (fl - 1.0) / d;
        Al_b -= flb * fl / d;
    }
    rcs_b += P.T_sol * As_b;
    rcl_b += P.T_liq * Al_b;
    Lv_b += Al_b;
    rs_b += m.cs * rcs_b;
    cs_b += m.rs * rcs_b;
    rl_b += m.cl * rcl_b;
    cl_b += m.rl * rcl_b;
}

// The pairwise normal is held fixed (its derivative dropped) where it is ill-conditioned:
// |a| / |G| > ADJ_NORMAL_COND, a = (4/eps) phi_p phi_q the weight of the normal in R_p.
// Across an equilibrium interface of the pair, phi_p / (phi_p + phi_q) follows the tanh
// profile and |a| / |G| = 1 exactly.  Values far above 1 occur only where the pairwise
// fraction is much flatter than an interface: in the far tails of nearly absent phases,
// where the direction is set by rounding-level structure and the term a n is below
// ~1e-6.  There the linearisation of n grows without bound over many steps while the
// loss itself does not change, so the derivative through n is not followed.
constexpr double ADJ_NORMAL_COND = 10.0;

// g'(x) and g''(x) of g(x) = x^2 (1 - x)^2.
__device__ __forceinline__ double gp1(double x) { return 2.0 * x * (1.0 - x) * (1.0 - 2.0 * x); }
__device__ __forceinline__ double gp2(double x) { return 2.0 - 12.0 * x + 12.0 * x * x; }

// phi_p, rho, psi of every cell of set A (the inputs of the stencils).
template <int N>
__global__ void mac_kernel(const KParams P, const double* __restrict__ pin, const double* __restrict__ ain,
                           double* __restrict__ mac)
{
    const PopView<PrecFP64> pv = pop_view<PrecFP64>(P, pin);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < P.S;
         c += (long long)gridDim.x * blockDim.x) {
        double ph[N], r, ps;
        halo_moments<N, PrecFP64>(P, pv, ain, c, ph, r, ps);
        for (int p = 0; p < N; ++p) mac[p * P.S + c] = ph[p];
        mac[N * P.S + c] = r;
        mac[(N + 1) * P.S + c] = ps;
    }
}

// Stencil point k of cell (x, y): the in-domain cell supplying it (periodic sides wrap;
// beyond a wall or outflow the ghost copies the clamped cell), its direction from
// (x, y), and the wetting coefficient sides (-1 = none).
__device__ __forceinline__ void stencil_source(const KParams& P, int x, int y, int k, long long& cell, int& ksrc,
                                               int& wx, int& wy)
{
    const bool xper = P.bc[0] == PERIODIC, yper = P.bc[2] == PERIODIC;
    int gx = x + cx(k), gy = y + cy(k);
    const bool xo = !xper && (gx < 0 || gx >= P.nx);
    const bool yo = !yper && (gy < 0 || gy >= P.ny);
    int dx = cx(k), dy = cy(k);
    wx = -1;
    wy = -1;
    if (xo) {
        wx = gx < 0 ? 0 : 1;
        gx = min(max(gx, 0), P.nx - 1);
        dx = gx - x;
    } else if (gx < 0 || gx >= P.nx) {
        gx = wrap_index(gx, P.nx);
    }
    if (yo) {
        wy = gy < 0 ? 2 : 3;
        gy = min(max(gy, 0), P.ny - 1);
        dy = gy - y;
    } else if (gy < 0 || gy >= P.ny) {
        gy = wrap_index(gy, P.ny);
    }
    cell = (long long)gy * P.nx + gx;
    ksrc = dir_of(dx, dy);
}

// The adjoint of one cell's step (see the file comment).
template <int N>
__global__ void __launch_bounds__(128) adj_cell_kernel(const KParams P, const AdjBufs B)
{
    const long long S = P.S;
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= S) return;
    const int x = (int)(c % P.nx), y = (int)(c / P.nx);
    const Coef<double>& C = P.d;

    // ================= forward recompute (the FP64 step of cell c) =================
    double f[9], g[N][9], h[9];
    for (int i = 0; i < 9; ++i) {
        f[i] = B.pin[pidx(P, 0, i, c)];
        h[i] = B.pin[pidx(P, N + 1, i, c)];
        for (int p = 0; p < N; ++p) g[p][i] = B.pin[pidx(P, 1 + p, i, c)];
    }
    const double mdm = B.ain[aux_mdot() * S + c], Qm = B.ain[aux_Q() * S + c];
    const double psim = B.ain[aux_psi() * S + c];
    const double iden = 1.0 / (1.0 - 0.5 * mdm);
    double phi[N];
    for (int p = 0; p < N; ++p) {
        double sg = 0.0;
        for (int i = 0; i < 9; ++i) sg += g[p][i];
        phi[p] = sg * iden;
    }
    double sh = 0.0;
    for (int i = 0; i < 9; ++i) sh += h[i];
    const double rhoH = fma(0.5, Qm, sh);
    const Mix<N> m = mixture_map<N>(P, phi);
    double fl, T;
    enthalpy_map<N, true>(P, m, rhoH, fl, T);
    const double fs = 1.0 - fl;
    const double Rs = mix_sum<N, double>(phi, C.rho_s), Rl = mix_sum<N, double>(phi, C.rho_l);
    const double Ms = mix_sum<N, double>(phi, C.mu_s), Ml = mix_sum<N, double>(phi, C.mu_l);
    const double Ks = mix_sum<N, double>(phi, C.lam_s), Kl = mix_sum<N, double>(phi, C.lam_l);
    const double Cs = mix_sum<N, double>(phi, C.cp_s), Cl = mix_sum<N, double>(phi, C.cp_l);
    const double Dr = mix_sum<N, double>(phi, C.drho), Pc = mix_sum<N, double>(phi, C.pcm);
    const double rho = fma(fs, Rs, fl * Rl), mu = fma(fs, Ms, fl * Ml);
    const double lam = fma(fs, Ks, fl * Kl), cp = fma(fs, Cs, fl * Cl);
    const double psi = fs * Dr, chi = fs * Pc;

    // stencil values (ghosts beyond walls / outflows as in the forward step)
    double vphi[9][N], vrho[9], vpsi[9];
    int ksrc[9], wxk[9], wyk[9];
    for (int k = 0; k < 9; ++k) {
        long long sc;
        stencil_source(P, x, y, k, sc, ksrc[k], wxk[k], wyk[k]);
        double ph[N];
        for (int p = 0; p < N; ++p) ph[p] = B.mac[p * S + sc];
        for (int p = 0; p < N; ++p) {
            double corr = 0.0;
            if (wxk[k] >= 0 || wyk[k] >= 0)
                for (int q = 0; q < N; ++q) {
                    if (q == p) continue;
                    double cw = 0.0;
                    if (wxk[k] >= 0) cw += C.wet[wxk[k]][p][q];
                    if (wyk[k] >= 0) cw += C.wet[wyk[k]][p][q];
                    corr = fma(cw * ph[p], ph[q], corr);
                }
            vphi[k][p] = ph[p] + corr;
        }
        vrho[k] = B.mac[N * S + sc];
        vpsi[k] = B.mac[(N + 1) * S + sc];
    }
    // the own cell's stencil centre is its own value (it is the same computation)
    auto gradv = [&](const double* v, double& gx_, double& gy_) {
        gx_ = (v[1] - v[3]) * (1.0 / 3.0) + ((v[5] - v[6]) + (v[8] - v[7])) * (1.0 / 12.0);
        gy_ = (v[2] - v[4]) * (1.0 / 3.0) + ((v[5] - v[8]) + (v[6] - v[7])) * (1.0 / 12.0);
    };
    double gpx[N], gpy[N], lap[N];
    for (int p = 0; p < N; ++p) {
        double v[9];
        for (int k = 0; k < 9; ++k) v[k] = vphi[k][p];
        gradv(v, gpx[p], gpy[p]);
        lap[p] = ((v[1] + v[3]) + (v[2] + v[4])) * (2.0 / 3.0) + ((v[5] + v[6]) + (v[8] + v[7])) * (1.0 / 6.0) -
                 v[0] * (10.0 / 3.0);
    }
    double grx, gry, gsx, gsy;
    gradv(vrho, grx, gry);
    gradv(vpsi, gsx, gsy);

    // stage D
    constexpr int NP = N * (N - 1) / 2;
    double pGx[NP], pGy[NP], pr[NP], pnx[NP], pny[NP];
    bool pok[NP];
    double Rx[N], Ry[N], mup[N], gpv[N];
    for (int p = 0; p < N; ++p) {
        Rx[p] = Ry[p] = mup[p] = 0.0;
        gpv[p] = 2.0 * phi[p] * (1.0 - phi[p]) * (1.0 - 2.0 * phi[p]);
    }
    {
        int k = 0;
        for (int p = 0; p < N; ++p)
            for (int q = p + 1; q < N; ++q, ++k) {
                const double s = phi[p] + phi[q];
                double nxv = 0.0, nyv = 0.0;
                pok[k] = false;
                pGx[k] = pGy[k] = pr[k] = 0.0;
                if (s > 1e-12) {
                    const double Gx = phi[q] * gpx[p] - phi[p] * gpx[q];
                    const double Gy = phi[q] * gpy[p] - phi[p] * gpy[q];
                    const double G2 = Gx * Gx + Gy * Gy;
                    const double s2 = s * s;
                    if (G2 > PrecFP64::NABS2 * (s2 * s2)) {
                        const double r = rsqrt(G2);
                        nxv = Gx * r;
                        nyv = Gy * r;
                        pok[k] = true;
                        pGx[k] = Gx;
                        pGy[k] = Gy;
                        pr[k] = r;
                    }
                }
                pnx[k] = nxv;
                pny[k] = nyv;
                const double a = C.four_eps * phi[p] * phi[q];
                Rx[p] = fma(a, nxv, Rx[p]);
                Ry[p] = fma(a, nyv, Ry[p]);
                Rx[q] = fma(-a, nxv, Rx[q]);
                Ry[q] = fma(-a, nyv, Ry[q]);
                const double gs = 2.0 * s * (1.0 - s) * (1.0 - 2.0 * s);
                mup[p] += fma(C.b2[p][q], gpv[p] - gs, C.kk[p][q] * lap[q]);
                mup[q] += fma(C.b2[q][p], gpv[q] - gs, C.kk[q][p] * lap[p]);
            }
    }
    double Fx = rho * C.accel[0], Fy = rho * C.accel[1];
    for (int p = 0; p < N; ++p) {
        Fx = fma(mup[p], gpx[p], Fx);
        Fy = fma(mup[p], gpy[p], Fy);
    }
    // stage E
    const double jx = ((f[1] - f[3]) + (f[5] - f[7])) + (f[8] - f[6]);
    const double jy = ((f[2] - f[4]) + (f[5] - f[7])) + (f[6] - f[8]);
    const double sum_f = ((f[1] + f[2]) + (f[3] + f[4])) + ((f[5] + f[6]) + (f[7] + f[8]));
    const double Af = fma(3.0, mu, 0.5 * rho);
    const double Bh = fma(lam, C.tau_h_scale, 0.5);
    const double irho = 1.0 / rho, om = rho / Af, oh = 1.0 / Bh;
    const double usx = fma(0.5, Fx, jx) * irho, usy = fma(0.5, Fy, jy) * irho;
    const double fpx = chi * (C.us[0] - usx), fpy = chi * (C.us[1] - usy);
    const double ux = fma(0.5, fpx, usx), uy = fma(0.5, fpy, usy);
    const double Mm = (psi - psim) + (ux * gsx + uy * gsy);
    const double mdot = -Mm * irho;
    const double Ssrc = fma(rho, mdot, ux * grx + uy * gry);
    const double Lxx = fma(2.0 * ux, Fx, Ssrc * (1.0 / 3.0));
    const double Lyy = fma(2.0 * uy, Fy, Ssrc * (1.0 / 3.0));
    const double Lxy = fma(ux, Fy, uy * Fx);
    const double tmh = 3.0 * mu * irho;
    const double w0 = wgt(0);
    const double F0 = w0 * fma(-1.5, Lxx + Lyy, Ssrc);
    const double uu = fma(ux, ux, uy * uy);
    const double prs = 0.6 * (((sum_f + 0.5 * Ssrc) + tmh * F0) - rho * w0 * 1.5 * uu);
    // stage F (values the reverse needs)
    const double kf = fma(-0.5, om, 1.0), om1 = 1.0 - om;
    const double Fex = fma(rho, fpx, Fx), Fey = fma(rho, fpy, Fy);
    const double rom = om * rho;
    const double og = C.omega_g, kg = C.kg, og1 = 1.0 - og;
    const double Z = rho * cp * T, E = C.E_ref * T;
    const double kh = fma(-0.5, oh, 1.0), oh1 = 1.0 - oh;
    const double Zm = Z * mdot;
    const double ohZ = oh * Z;

    // ======================= reverse =======================
    double f_b[9], g_b[N][9], h_b[9];
    for (int i = 0; i < 9; ++i) {
        f_b[i] = h_b[i] = 0.0;
        for (int p = 0; p < N; ++p) g_b[p][i] = 0.0;
    }
    double phi_b[N], Rx_b[N], Ry_b[N], mup_b[N], gpx_b[N], gpy_b[N], lap_b[N], gpv_b[N];
    for (int p = 0; p < N; ++p) phi_b[p] = Rx_b[p] = Ry_b[p] = mup_b[p] = gpx_b[p] = gpy_b[p] = lap_b[p] = gpv_b[p] = 0.0;
    double rho_b = 0, mu_b = 0, lam_b = 0, cp_b = 0, psi_b = 0, chi_b = 0, T_b = 0, rhoH_b = 0;
    double ux_b = 0, uy_b = 0, uu_b = 0, mdot_b = 0, S_b = 0, Lxx_b = 0, Lyy_b = 0, Lxy_b = 0, p_b = 0;
    double om_b = 0, oh_b = 0, irho_b = 0, Fx_b = 0, Fy_b = 0, fpx_b = 0, fpy_b = 0;
    double grx_b = 0, gry_b = 0, gsx_b = 0, gsy_b = 0, psim_b = 0;

    // lagged outputs of this step (inputs of the next): mdot, Q = Zm, psi, phi_p u
    mdot_b += B.baux[aux_mdot() * S + c];
    double Zm_b = B.baux[aux_Q() * S + c];
    psi_b += B.baux[aux_psi() * S + c];

    // ---- enthalpy collision ----
    {
        double qb[9];
        gather_species<KIND_H>(P, B.bpop, N + 1, x, y, qb);
        double Z_b = 0, E_b = 0, kh_b = 0, oh1_b = 0, ohZ_b = 0;
        // Dirichlet rows: v_j = oh1 (h_j - heq_j) + w_j Eg, Eg = E_ref (2 T_w - T)
        auto dirichlet = [&](int side, int j0, int j1, int j2) {
            const int js[3] = {j0, j1, j2};
            double Eg_b = 0.0;
            for (int mm = 0; mm < 3; ++mm) {
                const int j = js[mm];
                long long cell;
                if (!row_target(P, j, x, y, cell)) continue;
                const double vb = B.bpop[pidx(P, N + 1, j, cell)];
                const double cu = cx(j) * ux + cy(j) * uy;
                const double Pj = fma(4.5 * cu, cu, fma(3.0, cu, -1.5 * uu));
                const double heq = wgt(j) * fma(Z, Pj, E);
                oh1_b += vb * (h[j] - heq);
                h_b[j] += vb * oh1;
                const double heq_b = -vb * oh1;
                Eg_b += vb * wgt(j);
                E_b += heq_b * wgt(j);
                Z_b += heq_b * wgt(j) * Pj;
                const double Pj_b = heq_b * wgt(j) * Z;
                const double cu_b = Pj_b * (3.0 + 9.0 * cu);
                uu_b += -1.5 * Pj_b;
                ux_b += cu_b * cx(j);
                uy_b += cu_b * cy(j);
            }
            B.grad[(GS_TW + side) * S + c] += 2.0 * C.E_ref * Eg_b;
            T_b -= C.E_ref * Eg_b;
        };
        if (y == 0 && P.bc[2] == WALL && P.tbc[2] == DIRICHLET) dirichlet(2, 2, 5, 6);
        if (y == P.ny - 1 && P.bc[3] == WALL && P.tbc[3] == DIRICHLET) dirichlet(3, 4, 7, 8);
        // q_0 = oh heq0 + kh w0 Zm + oh1 h0
        const double heq0 = (rhoH - E) + w0 * fma(-1.5 * Z, uu, E);
        oh_b += qb[0] * heq0;
        const double heq0_b = qb[0] * oh;
        kh_b += qb[0] * w0 * Zm;
        Zm_b += qb[0] * kh * w0;
        oh1_b += qb[0] * h[0];
        h_b[0] += qb[0] * oh1;
        double Bb[9];
        for (int i = 1; i < 9; ++i) {
            Bb[i] = qb[i] * wgt(i);
            oh1_b += qb[i] * h[i];
            h_b[i] += qb[i] * oh1;
        }
        const double bx_b = Bb[1] + Bb[3], by_b = Bb[2] + Bb[4];
        const double t1 = Bb[5] + Bb[7], t2 = Bb[6] + Bb[8];
        const double bd_b = t1 + t2, cxy_b = t1 - t2;
        const double sxy = Bb[5] - Bb[7], syx = Bb[6] - Bb[8];
        const double cxv_b = (Bb[1] - Bb[3]) + sxy - syx;
        const double cyv_b = (Bb[2] - Bb[4]) + sxy + syx;
        const double c0_b = bx_b + by_b + bd_b;
        const double cxx_b = bx_b + bd_b, cyy_b = by_b + bd_b;
        // heq0 = (rhoH - E) + w0 (E - 1.5 Z uu)
        rhoH_b += heq0_b;
        E_b += heq0_b * (w0 - 1.0);
        Z_b += heq0_b * w0 * (-1.5 * uu);
        uu_b += heq0_b * w0 * (-1.5 * Z);
        // c0 = oh (E - 1.5 Z uu) + kh Zm
        oh_b += c0_b * fma(-1.5 * Z, uu, E);
        E_b += c0_b * oh;
        Z_b += c0_b * oh * (-1.5 * uu);
        uu_b += c0_b * oh * (-1.5 * Z);
        kh_b += c0_b * Zm;
        Zm_b += c0_b * kh;
        // moments of the equilibrium
        ohZ_b += 3.0 * ux * cxv_b + 3.0 * uy * cyv_b + 4.5 * ux * ux * cxx_b + 4.5 * uy * uy * cyy_b +
                 9.0 * ux * uy * cxy_b;
        ux_b += 3.0 * ohZ * cxv_b + 9.0 * ohZ * ux * cxx_b + 9.0 * ohZ * uy * cxy_b;
        uy_b += 3.0 * ohZ * cyv_b + 9.0 * ohZ * uy * cyy_b + 9.0 * ohZ * ux * cxy_b;
        oh_b += ohZ_b * Z;
        Z_b += ohZ_b * oh;
        oh_b += -0.5 * kh_b - oh1_b;
        Z_b += Zm_b * mdot;
        mdot_b += Zm_b * Z;
        T_b += C.E_ref * E_b;
        rho_b += Z_b * cp * T;
        cp_b += Z_b * rho * T;
        T_b += Z_b * rho * cp;
    }

    // ---- phase-field collisions ----
    for (int pp = 0; pp < N; ++pp) {
        double qb[9];
        gather_species<KIND_G>(P, B.bpop, 1 + pp, x, y, qb);
        for (int i = 0; i < 9; ++i) g_b[pp][i] += og1 * qb[i];
        double wq[9];
        for (int i = 0; i < 9; ++i) wq[i] = wgt(i) * qb[i];
        const double b0_b = wq[0] + wq[1] + wq[2] + wq[3] + wq[4] + wq[5] + wq[6] + wq[7] + wq[8];
        const double bxv_b = wq[1] - wq[3] + wq[5] - wq[7] - wq[6] + wq[8];
        const double byv_b = wq[2] - wq[4] + wq[5] - wq[7] + wq[6] - wq[8];
        const double ph = phi[pp];
        // b0 = og phi + kg phi mdot
        phi_b[pp] += b0_b * (og + kg * mdot);
        mdot_b += b0_b * kg * ph;
        // bxv = 3 og phi ux + kg (3 Dx + Rx), Dx = phi ux - (phi u)'_x
        const double Dx_b = 3.0 * kg * bxv_b, Dy_b = 3.0 * kg * byv_b;
        phi_b[pp] += bxv_b * 3.0 * og * ux + byv_b * 3.0 * og * uy;
        ux_b += bxv_b * 3.0 * og * ph;
        uy_b += byv_b * 3.0 * og * ph;
        Rx_b[pp] += kg * bxv_b;
        Ry_b[pp] += kg * byv_b;
        // the lagged output (phi u) of this step and the input (phi u)' of the previous
        const double Px_b = Dx_b + B.baux[aux_phiux(pp) * S + c];
        const double Py_b = Dy_b + B.baux[aux_phiuy(N, pp) * S + c];
        phi_b[pp] += Px_b * ux + Py_b * uy;
        ux_b += Px_b * ph;
        uy_b += Py_b * ph;
        B.aaux[aux_phiux(pp) * S + c] = -Dx_b;
        B.aaux[aux_phiuy(N, pp) * S + c] = -Dy_b;
    }

    // ---- flow collision ----
    {
        double qb[9];
        gather_species<KIND_F>(P, B.bpop, 0, x, y, qb);
        double Xb[9], om1_b = 0.0;
        for (int i = 0; i < 9; ++i) {
            f_b[i] += om1 * qb[i];
            om1_b += qb[i] * f[i];
            Xb[i] = wgt(i) * qb[i];
        }
        // X_0 = a0 - 6.75 om p
        om_b += Xb[0] * (-6.75 * prs);
        p_b += Xb[0] * (-6.75 * om);
        double a0_b = Xb[0];
        const double bx_b = Xb[1] + Xb[3], by_b = Xb[2] + Xb[4];
        const double t1 = Xb[5] + Xb[7], t2 = Xb[6] + Xb[8];
        const double bd_b = t1 + t2, axy_b = t1 - t2;
        const double sxy = Xb[5] - Xb[7], syx = Xb[6] - Xb[8];
        const double ax_b = (Xb[1] - Xb[3]) + sxy - syx;
        const double ay_b = (Xb[2] - Xb[4]) + sxy + syx;
        a0_b += bx_b + by_b + bd_b;
        const double axx_b = bx_b + bd_b, ayy_b = by_b + bd_b;
        double k_b = 0.0, rom_b = 0.0, Fex_b = 0.0, Fey_b = 0.0;
        // a0 = om (3p - 1.5 rho uu) + k (S - 1.5 (Lxx + Lyy))
        om_b += a0_b * fma(-1.5 * rho, uu, 3.0 * prs);
        p_b += a0_b * 3.0 * om;
        rho_b += a0_b * (-1.5 * om * uu);
        uu_b += a0_b * (-1.5 * om * rho);
        k_b += a0_b * fma(-1.5, Lxx + Lyy, Ssrc);
        S_b += a0_b * kf;
        Lxx_b += a0_b * (-1.5 * kf);
        Lyy_b += a0_b * (-1.5 * kf);
        // ax = 3 (rom ux + k Fex), ay likewise
        rom_b += 3.0 * (ux * ax_b + uy * ay_b);
        ux_b += 3.0 * rom * ax_b;
        uy_b += 3.0 * rom * ay_b;
        k_b += 3.0 * (Fex * ax_b + Fey * ay_b);
        Fex_b += 3.0 * kf * ax_b;
        Fey_b += 3.0 * kf * ay_b;
        // axx = 4.5 (rom ux ux + k Lxx), ayy, axy = 9 (rom ux uy + k Lxy)
        rom_b += 4.5 * ux * ux * axx_b + 4.5 * uy * uy * ayy_b + 9.0 * ux * uy * axy_b;
        ux_b += 9.0 * rom * ux * axx_b + 9.0 * rom * uy * axy_b;
        uy_b += 9.0 * rom * uy * ayy_b + 9.0 * rom * ux * axy_b;
        k_b += 4.5 * Lxx * axx_b + 4.5 * Lyy * ayy_b + 9.0 * Lxy * axy_b;
        Lxx_b += 4.5 * kf * axx_b;
        Lyy_b += 4.5 * kf * ayy_b;
        Lxy_b += 9.0 * kf * axy_b;
        // rom = om rho; Fe = F + rho fpen; k = 1 - om/2; om1 = 1 - om
        om_b += rom_b * rho;
        rho_b += rom_b * om;
        Fx_b += Fex_b;
        Fy_b += Fey_b;
        rho_b += Fex_b * fpx + Fey_b * fpy;
        fpx_b += Fex_b * rho;
        fpy_b += Fey_b * rho;
        om_b += -0.5 * k_b - om1_b;
    }

    // ---- stage E ----
    {
        // p = 0.6 ((sum_f + S/2) + tmh F0 - 1.5 w0 rho uu)
        const double sum_f_b = 0.6 * p_b;
        S_b += 0.3 * p_b;
        const double tmh_b = 0.6 * F0 * p_b;
        const double F0_b = 0.6 * tmh * p_b;
        rho_b += -0.9 * w0 * uu * p_b;
        uu_b += -0.9 * w0 * rho * p_b;
        for (int i = 1; i < 9; ++i) f_b[i] += sum_f_b;
        // uu = ux^2 + uy^2
        ux_b += 2.0 * ux * uu_b;
        uy_b += 2.0 * uy * uu_b;
        // F0 = w0 (S - 1.5 (Lxx + Lyy))
        S_b += w0 * F0_b;
        Lxx_b += -1.5 * w0 * F0_b;
        Lyy_b += -1.5 * w0 * F0_b;
        // tmh = 3 mu / rho
        mu_b += 3.0 * irho * tmh_b;
        irho_b += 3.0 * mu * tmh_b;
        // Lxy = ux Fy + uy Fx; Lxx = 2 ux Fx + S/3; Lyy = 2 uy Fy + S/3
        ux_b += Fy * Lxy_b + 2.0 * Fx * Lxx_b;
        uy_b += Fx * Lxy_b + 2.0 * Fy * Lyy_b;
        Fx_b += uy * Lxy_b + 2.0 * ux * Lxx_b;
        Fy_b += ux * Lxy_b + 2.0 * uy * Lyy_b;
        S_b += (Lxx_b + Lyy_b) * (1.0 / 3.0);
        // S = rho mdot + u . grad rho
        rho_b += mdot * S_b;
        mdot_b += rho * S_b;
        ux_b += grx * S_b;
        uy_b += gry * S_b;
        grx_b += ux * S_b;
        gry_b += uy * S_b;
        // mdot = -M / rho, M = (psi - psi') + u . grad psi
        const double M_b = -irho * mdot_b;
        irho_b += -Mm * mdot_b;
        psi_b += M_b;
        psim_b -= M_b;
        ux_b += gsx * M_b;
        uy_b += gsy * M_b;
        gsx_b += ux * M_b;
        gsy_b += uy * M_b;
        // u = u* + fpen / 2; fpen = chi (u_s - u*); u* = (j + F/2) / rho
        double usx_b = ux_b, usy_b = uy_b;
        fpx_b += 0.5 * ux_b;
        fpy_b += 0.5 * uy_b;
        chi_b += (C.us[0] - usx) * fpx_b + (C.us[1] - usy) * fpy_b;
        usx_b -= chi * fpx_b;
        usy_b -= chi * fpy_b;
        const double jx_b = irho * usx_b, jy_b = irho * usy_b;
        Fx_b += 0.5 * irho * usx_b;
        Fy_b += 0.5 * irho * usy_b;
        irho_b += fma(0.5, Fx, jx) * usx_b + fma(0.5, Fy, jy) * usy_b;
        f_b[1] += jx_b;
        f_b[3] -= jx_b;
        f_b[5] += jx_b + jy_b;
        f_b[7] -= jx_b + jy_b;
        f_b[8] += jx_b - jy_b;
        f_b[6] += jy_b - jx_b;
        f_b[2] += jy_b;
        f_b[4] -= jy_b;
        // irho = 1/rho, om = rho / Af, oh = 1 / Bh; Af = 3 mu + rho/2, Bh = lam tau_s + 1/2
        rho_b += -irho * irho * irho_b;
        const double iAf = 1.0 / Af;
        rho_b += om_b * iAf;
        const double Af_b = -om * iAf * om_b;
        const double Bh_b = -oh * oh * oh_b;
        mu_b += 3.0 * Af_b;
        rho_b += 0.5 * Af_b;
        lam_b += C.tau_h_scale * Bh_b;
    }

    // ---- stage D ----
    {
        // F = rho g + sum_p mu_p grad phi_p
        rho_b += C.accel[0] * Fx_b + C.accel[1] * Fy_b;
        for (int p = 0; p < N; ++p) {
            mup_b[p] += gpx[p] * Fx_b + gpy[p] * Fy_b;
            gpx_b[p] += mup[p] * Fx_b;
            gpy_b[p] += mup[p] * Fy_b;
        }
        int k = 0;
        for (int p = 0; p < N; ++p)
            for (int q = p + 1; q < N; ++q, ++k) {
                const double s = phi[p] + phi[q];
                // mu_p += b2_pq (g'(phi_p) - g'(s)) + kk_pq lap_q; mu_q likewise
                gpv_b[p] += C.b2[p][q] * mup_b[p];
                gpv_b[q] += C.b2[q][p] * mup_b[q];
                const double gs_b = -C.b2[p][q] * mup_b[p] - C.b2[q][p] * mup_b[q];
                lap_b[q] += C.kk[p][q] * mup_b[p];
                lap_b[p] += C.kk[q][p] * mup_b[q];
                double s_b = gp2(s) * gs_b;
                // R_p += a n, R_q -= a n, a = (4/eps) phi_p phi_q
                const double dRx = Rx_b[p] - Rx_b[q], dRy = Ry_b[p] - Ry_b[q];
                const double a = C.four_eps * phi[p] * phi[q];
                const double a_b = dRx * pnx[k] + dRy * pny[k];
                phi_b[p] += C.four_eps * phi[q] * a_b;
                phi_b[q] += C.four_eps * phi[p] * a_b;
                if (pok[k] && fabs(a) * pr[k] <= ADJ_NORMAL_COND) {
                    // n = G / |G|: G-bar = (n-bar - n (n . n-bar)) / |G|
                    const double nxb = a * dRx, nyb = a * dRy;
                    const double nd = pnx[k] * nxb + pny[k] * nyb;
                    const double Gx_b = pr[k] * (nxb - pnx[k] * nd);
                    const double Gy_b = pr[k] * (nyb - pny[k] * nd);
                    // G = phi_q grad phi_p - phi_p grad phi_q
                    phi_b[q] += gpx[p] * Gx_b + gpy[p] * Gy_b;
                    phi_b[p] -= gpx[q] * Gx_b + gpy[q] * Gy_b;
                    gpx_b[p] += phi[q] * Gx_b;
                    gpy_b[p] += phi[q] * Gy_b;
                    gpx_b[q] -= phi[p] * Gx_b;
                    gpy_b[q] -= phi[p] * Gy_b;
                }
                phi_b[p] += s_b;
                phi_b[q] += s_b;
            }
        for (int p = 0; p < N; ++p) phi_b[p] += gp2(phi[p]) * gpv_b[p];
    }

    // ---- stage C: stencil adjoints per point, ghosts folded onto their source ----
    {
        double sb[9][N + 2];
        for (int k = 0; k < 9; ++k)
            for (int f2 = 0; f2 < N + 2; ++f2) sb[k][f2] = 0.0;
        // point adjoints before folding: vb[k][field]
        double vb[9][N + 2];
        for (int k = 0; k < 9; ++k)
            for (int f2 = 0; f2 < N + 2; ++f2) vb[k][f2] = 0.0;
        auto grad_rev = [&](int fld, double gx_b, double gy_b) {
            vb[1][fld] += gx_b * (1.0 / 3.0);
            vb[3][fld] -= gx_b * (1.0 / 3.0);
            vb[5][fld] += gx_b * (1.0 / 12.0) + gy_b * (1.0 / 12.0);
            vb[6][fld] += -gx_b * (1.0 / 12.0) + gy_b * (1.0 / 12.0);
            vb[8][fld] += gx_b * (1.0 / 12.0) - gy_b * (1.0 / 12.0);
            vb[7][fld] += -gx_b * (1.0 / 12.0) - gy_b * (1.0 / 12.0);
            vb[2][fld] += gy_b * (1.0 / 3.0);
            vb[4][fld] -= gy_b * (1.0 / 3.0);
        };
        for (int p = 0; p < N; ++p) {
            grad_rev(p, gpx_b[p], gpy_b[p]);
            for (int k = 1; k < 5; ++k) vb[k][p] += lap_b[p] * (2.0 / 3.0);
            for (int k = 5; k < 9; ++k) vb[k][p] += lap_b[p] * (1.0 / 6.0);
            vb[0][p] += lap_b[p] * (-10.0 / 3.0);
        }
        grad_rev(N, grx_b, gry_b);
        grad_rev(N + 1, gsx_b, gsy_b);
        for (int k = 0; k < 9; ++k) {
            const int ks = ksrc[k];
            sb[ks][N] += vb[k][N];
            sb[ks][N + 1] += vb[k][N + 1];
            if (wxk[k] < 0 && wyk[k] < 0) {
                for (int p = 0; p < N; ++p) sb[ks][p] += vb[k][p];
            } else {
                // ghost phi_p = phi_p(s) + sum_{q != p} cw_pq phi_p(s) phi_q(s)
                long long sc;
                int kk2, a1, a2;
                stencil_source(P, x, y, k, sc, kk2, a1, a2);
                double ph[N];
                for (int p = 0; p < N; ++p) ph[p] = B.mac[p * S + sc];
                for (int p = 0; p < N; ++p) {
                    sb[ks][p] += vb[k][p];
                    for (int q = 0; q < N; ++q) {
                        if (q == p) continue;
                        double cw = 0.0;
                        if (wxk[k] >= 0) cw += C.wet[wxk[k]][p][q];
                        if (wyk[k] >= 0) cw += C.wet[wyk[k]][p][q];
                        sb[ks][p] += vb[k][p] * cw * ph[q];
                        sb[ks][q] += vb[k][p] * cw * ph[p];
                    }
                }
            }
        }
        for (int k = 0; k < 9; ++k)
            for (int f2 = 0; f2 < N + 2; ++f2) B.sb[((long long)k * (N + 2) + f2) * S + c] = sb[k][f2];
    }

    // ---- own stage A + B: eq. 2 sums and eq. H of the cell's own use ----
    {
        const double fs_b = rho_b * Rs + mu_b * Ms + lam_b * Ks + cp_b * Cs + psi_b * Dr + chi_b * Pc;
        const double fl_b = rho_b * Rl + mu_b * Ml + lam_b * Kl + cp_b * Cl - fs_b;
        const double Rs_b = rho_b * fs, Rl_b = rho_b * fl, Ms_b = mu_b * fs, Ml_b = mu_b * fl;
        const double Ks_b = lam_b * fs, Kl_b = lam_b * fl, Cs_b = cp_b * fs, Cl_b = cp_b * fl;
        const double Dr_b = psi_b * fs, Pc_b = chi_b * fs;
        double rs_b = 0, rl_b = 0, cs_b = 0, cl_b = 0, Lv_b = 0;
        map_reverse<N>(P, m, rhoH, fl_b, T_b, rs_b, rl_b, cs_b, cl_b, Lv_b, rhoH_b);
        for (int p = 0; p < N; ++p) {
            phi_b[p] += Rs_b * C.rho_s[p] + Rl_b * C.rho_l[p] + Ms_b * C.mu_s[p] + Ml_b * C.mu_l[p] +
                        Ks_b * C.lam_s[p] + Kl_b * C.lam_l[p] + Cs_b * C.cp_s[p] + Cl_b * C.cp_l[p] +
                        Dr_b * C.drho[p] + Pc_b * C.pcm[p];
            phi_b[p] += rs_b * P.d.rho_s[p] + rl_b * P.d.rho_l[p] + cs_b * P.d.cp_s[p] + cl_b * P.d.cp_l[p] +
                        Lv_b * P.rhoL[p];
            B.grad[(GS_RHOL + p) * S + c] += Lv_b * phi[p];
            B.grad[(GS_LAMS + p) * S + c] += Ks_b * phi[p];
            B.grad[(GS_LAML + p) * S + c] += Kl_b * phi[p];
        }
        for (int p = 0; p < N; ++p) B.own[p * S + c] = phi_b[p];
        B.own[N * S + c] = rhoH_b;
    }

    // direct adjoints of the cell's own populations and lagged inputs
    for (int i = 0; i < 9; ++i) {
        B.apop[pidx(P, 0, i, c)] = f_b[i];
        B.apop[pidx(P, N + 1, i, c)] = h_b[i];
        for (int p = 0; p < N; ++p) B.apop[pidx(P, 1 + p, i, c)] = g_b[p][i];
    }
    B.aaux[aux_mdot() * S + c] = 0.0;
    B.aaux[aux_Q() * S + c] = 0.0;
    B.aaux[aux_psi() * S + c] = psim_b;
}

// Stencil adjoints of cell y gathered from its users, reversed through y's own eq. H,
// eq. 2 sums and moments.  SEED: no users; instead the adjoint of the loss
// sum_x w (phi_pcm f_l - f_target)^2, and the loss per cell into its plane.  (f_l alone
// is ill-conditioned where little phase-changing material is present: the mushy band
// of eq. H is Lv wide, and Lv -> 0 there; weighted by phi_pcm it is not.)
template <int N, bool SEED>
__global__ void __launch_bounds__(128) adj_moments_kernel(const KParams P, const AdjBufs B)
{
    const long long S = P.S;
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= S) return;
    const int x = (int)(c % P.nx), y = (int)(c / P.nx);
    const Coef<double>& C = P.d;
    const bool xper = P.bc[0] == PERIODIC, yper = P.bc[2] == PERIODIC;
    double phi_b[N], rho_b = 0.0, psi_b = 0.0, rhoH_b = 0.0;
    for (int p = 0; p < N; ++p) phi_b[p] = 0.0;
    if (!SEED) {
        for (int p = 0; p < N; ++p) phi_b[p] = B.own[p * S + c];
        rhoH_b = B.own[N * S + c];
        for (int k = 0; k < 9; ++k) {
            // the user x = y - c_k used y as its stencil point k
            int ux_ = x - cx(k), uy_ = y - cy(k);
            if (ux_ < 0 || ux_ >= P.nx) {
                if (!xper) continue;
                ux_ = wrap_index(ux_, P.nx);
            }
            if (uy_ < 0 || uy_ >= P.ny) {
                if (!yper) continue;
                uy_ = wrap_index(uy_, P.ny);
            }
            const long long uc = (long long)uy_ * P.nx + ux_;
            for (int p = 0; p < N; ++p) phi_b[p] += B.sb[((long long)k * (N + 2) + p) * S + uc];
            rho_b += B.sb[((long long)k * (N + 2) + N) * S + uc];
            psi_b += B.sb[((long long)k * (N + 2) + N + 1) * S + uc];
        }
    }
    // recompute the moments and eq. H of y
    double g[N][9], h[9];
    for (int i = 0; i < 9; ++i) {
        h[i] = B.pin[pidx(P, N + 1, i, c)];
        for (int p = 0; p < N; ++p) g[p][i] = B.pin[pidx(P, 1 + p, i, c)];
    }
    const double mdm = B.ain[aux_mdot() * S + c], Qm = B.ain[aux_Q() * S + c];
    const double iden = 1.0 / (1.0 - 0.5 * mdm);
    double phi[N];
    for (int p = 0; p < N; ++p) {
        double sg = 0.0;
        for (int i = 0; i < 9; ++i) sg += g[p][i];
        phi[p] = sg * iden;
    }
    double sh = 0.0;
    for (int i = 0; i < 9; ++i) sh += h[i];
    const double rhoH = fma(0.5, Qm, sh);
    const Mix<N> m = mixture_map<N>(P, phi);
    double fl, T;
    enthalpy_map<N, false>(P, m, rhoH, fl, T);
    const double fs = 1.0 - fl;
    const double Rs = mix_sum<N, double>(phi, C.rho_s), Rl = mix_sum<N, double>(phi, C.rho_l);
    const double Dr = mix_sum<N, double>(phi, C.drho);
    double fl_b = 0.0;
    if (SEED) {
        // q = phi_pcm f_l, the liquid fraction of the phase-changing material
        // (phi_pcm = sum_p phi_p over the phases with L_p > 0)
        const double Pc = mix_sum<N, double>(phi, C.pcm);
        const double w = B.weight ? B.weight[c] : 1.0;
        const double d = Pc * fl - B.fl_target[c];
        const double q_b = 2.0 * w * d;
        fl_b = q_b * Pc;
        for (int p = 0; p < N; ++p) phi_b[p] += q_b * fl * C.pcm[p];
        B.grad[(long long)GS_LOSS * S + c] = w * d * d;
    }
    // rho = fs Rs + fl Rl, psi = fs Dr
    const double fs_b = rho_b * Rs + psi_b * Dr;
    fl_b += rho_b * Rl - fs_b;
    const double Rs_b = rho_b * fs, Rl_b = rho_b * fl, Dr_b = psi_b * fs;
    double rs_b = 0, rl_b = 0, cs_b = 0, cl_b = 0, Lv_b = 0;
    map_reverse<N>(P, m, rhoH, fl_b, 0.0, rs_b, rl_b, cs_b, cl_b, Lv_b, rhoH_b);
    double mdm_b = 0.0;
    for (int p = 0; p < N; ++p) {
        phi_b[p] += Rs_b * C.rho_s[p] + Rl_b * C.rho_l[p] + Dr_b * C.drho[p];
        phi_b[p] += rs_b * P.d.rho_s[p] + rl_b * P.d.rho_l[p] + cs_b * P.d.cp_s[p] + cl_b * P.d.cp_l[p] +
                    Lv_b * P.rhoL[p];
        B.grad[(GS_RHOL + p) * S + c] += Lv_b * phi[p];
        // phi_p = (sum_i g_ip) / (1 - mdot'/2)
        const double gb = phi_b[p] * iden;
        for (int i = 0; i < 9; ++i) {
            const long long k = pidx(P, 1 + p, i, c);
            B.apop[k] = SEED ? gb : B.apop[k] + gb;
        }
        mdm_b += phi_b[p] * phi[p] * 0.5 * iden;
    }
    // rho H = sum_i h_i + Q'/2
    for (int i = 0; i < 9; ++i) {
        const long long k = pidx(P, N + 1, i, c);
        B.apop[k] = SEED ? rhoH_b : B.apop[k] + rhoH_b;
    }
    if (SEED) {
        for (int i = 0; i < 9; ++i) B.apop[pidx(P, 0, i, c)] = 0.0;
        for (int k = 0; k < 3 + 2 * N; ++k) B.aaux[k * S + c] = 0.0;
        B.aaux[aux_mdot() * S + c] = mdm_b;
        B.aaux[aux_Q() * S + c] = 0.5 * rhoH_b;
    } else {
        B.aaux[aux_mdot() * S + c] += mdm_b;
        B.aaux[aux_Q() * S + c] += 0.5 * rhoH_b;
    }
}

// The initial state's dependence on the parameters: rho H(t = 0) comes from the inverse
// of eq. H, which holds the latent heat per volume Lv = sum_p phi_p rho_l^p L_p (liquid:
// d rhoH / d Lv = 1; solid: 0; mushy: (T - T_sol) / (T_liq - T_sol)); it enters h_0 only
// (h_0 = rho H - E + ...), whose adjoint is that of the first set.  (A mushy start would
// also move f_l and with it rho and c_p; starts at T != T_m have none.)
template <int N>
__global__ void adj_init_kernel(const KParams P, const double* __restrict__ phi0, const double* __restrict__ T0,
                                const double* __restrict__ apop, double* __restrict__ grad)
{
    const long long S = P.S;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < S; c += (long long)gridDim.x * blockDim.x) {
        double phi[N];
        for (int p = 0; p < N; ++p) phi[p] = phi0[p * S + c];
        const Mix<N> m = mixture_map<N>(P, phi);
        const double T = T0[c];
        double dLv;
        if (!(m.Lv > 0.0) || T >= P.T_liq) dLv = 1.0;
        else if (T < P.T_sol) dLv = 0.0;
        else dLv = (T - P.T_sol) / (P.T_liq - P.T_sol);
        const double hb0 = apop[pidx(P, N + 1, 0, c)];
        for (int p = 0; p < N; ++p) grad[(GS_RHOL + p) * S + c] += hb0 * dLv * phi[p];
    }
}

}  // namespace lbm
