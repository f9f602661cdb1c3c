// lbm_step.cuh -- the fused FP64 time step of the coupled LB scheme
// (arXiv 2603.22902, Section 3), one kernel launch per step.
//
// State between launches: pre-collision (post-streaming) populations
// f[9], g_p[9] (p < N), h[9] as structure-of-arrays planes, and the lagged planes
// mdot', Q' = rho c_p T mdot, psi', (phi_p u)'.  One launch reads set A and writes
// set B (ping-pong), so it is race-free across blocks.
//
// Per block (a TX x TY tile, one thread per cell):
//   1. each thread loads its cell's populations into registers and evaluates the
//      moments (phi_p = sum g / (1 - mdot'/2), rho H = sum h + Q'/2), the mixture
//      rule (eq. 2) and the enthalpy map (eq. H);
//   2. the 1-cell halo ring recomputes phi_p, rho, psi of the neighbour cells from
//      their own populations (no second kernel, no extra HBM field), and ghost
//      values beyond walls/outflows are filled (zero gradient; wetting for phi_p);
//   3. the isotropic 9-point gradients / Laplacians of phi_p, rho, psi come from
//      shared memory; then the pairwise normals n_pq, R_p, mu_p, F_s (Section 2),
//      u*, the penalty force, u, mdot, S, Lambda, p (Section 3), and the three BGK
//      collisions with their source terms;
//   4. post-collision populations are pushed to the neighbours' slots of set B with
//      the boundary rules (bounce-back, outflow copy, non-equilibrium extrapolation
//      of the Dirichlet temperature), and the lagged planes are written.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

struct ExportPtrs {
    double *phi, *T, *H, *fl, *ux, *uy, *p;
};

// v mod n in [0, n) for any int v (n > 0).
__device__ __forceinline__ int wrap_index(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// Stage A + B for a halo cell: phi_p, rho and psi only.
template <int N>
__device__ __forceinline__ void halo_moments(const KParams& P, const double* __restrict__ pin,
                                             const double* __restrict__ ain, long long c,
                                             double (&phi)[N], double& rho, double& psi)
{
    const long long S = P.S;
    const double mdm = LBM_LD(P, ain, aux_mdot() * S + c, P.aux_elems, 1);
    const double Qm = LBM_LD(P, ain, aux_Q() * S + c, P.aux_elems, 2);
    const double den = 1.0 - 0.5 * mdm;
#pragma unroll
    for (int p = 0; p < N; ++p) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) s += LBM_LD(P, pin, plane_g(p, i) * S + c, P.pop_elems, 3);
        phi[p] = s / den;
    }
    double sh = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) sh += LBM_LD(P, pin, plane_h(N, i) * S + c, P.pop_elems, 4);
    const double rhoH = fma(0.5, Qm, sh);
    const Mix<N> m = mixture_core<N>(P, phi);
    double fl, T;
    enthalpy_map<N, false>(P, m, rhoH, fl, T);
    const double fs = 1.0 - fl;
    rho = fma(fs, m.rs, fl * m.rl);
    psi = fs * m.dr;
}

// Push one post-collision population q_j of node (x, y) into set B.
// Periodic sides wrap; a population leaving through an x wall is reflected into the
// node's own opposite slot (half-way bounce-back); through a y wall likewise, except
// the enthalpy populations at a Dirichlet wall (their incoming slots are filled by the
// ghost rule); through an outflow side it is dropped.
template <int J, bool IS_H>
__device__ __forceinline__ void push(const KParams& P, double* __restrict__ pout, int plane, int plane_opp,
                                     int x, int y, double q)
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
    if (!xo && !yo) {
        LBM_ST(P, pout, plane * P.S + (long long)ty * P.nx + tx, P.pop_elems, 10, q);
    } else if (xo) {
        LBM_ST(P, pout, plane_opp * P.S + (long long)y * P.nx + x, P.pop_elems, 11, q);
    } else {
        const int side = ty < 0 ? 2 : 3;
        if (P.bc[side] == WALL && !(IS_H && P.tbc[side] == DIRICHLET))
            LBM_ST(P, pout, plane_opp * P.S + (long long)y * P.nx + x, P.pop_elems, 12, q);
    }
}

// Extra write of a boundary-row rule: value v into slot J of node (x + c_J, y),
// same row; skipped when that node is beyond an x wall.
template <int J>
__device__ __forceinline__ void push_row(const KParams& P, double* __restrict__ pout, int plane, int x, int y, double v)
{
    int tx = x + cx(J);
    if (cx(J) != 0 && (unsigned)tx >= (unsigned)P.nx) {
        if (P.bc[0] != PERIODIC) return;
        tx = tx < 0 ? tx + P.nx : tx - P.nx;
    }
    LBM_ST(P, pout, plane * P.S + (long long)y * P.nx + tx, P.pop_elems, 13, v);
}

template <int N, int TX, int TY, bool COLLIDE>
__global__ void __launch_bounds__(TX * TY)
fused_step_kernel(const KParams P, const double* __restrict__ pin, double* __restrict__ pout,
                  const double* __restrict__ ain, double* __restrict__ aout, ExportPtrs ex)
{
    constexpr int W = TX + 2, H = TY + 2, NT = TX * TY, NRING = 2 * W + 2 * TY;
    __shared__ double s_phi[N][H][W];
    __shared__ double s_rho[H][W];
    __shared__ double s_psi[H][W];

    const int nx = P.nx, ny = P.ny;
    const long long S = P.S;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool owned = x < nx && y < ny;
    const bool xper = P.bc[0] == PERIODIC, yper = P.bc[2] == PERIODIC;

    // halo position (lx, ly) of the tile: recompute the neighbour's moments
    // The cell coordinates are brought into range before anything else (periodic:
    // full modulo, since a tile may be wider / taller than the domain; otherwise:
    // clamped), so no address outside the planes is ever formed, even for a position
    // whose value the ghost rule supplies later.
    auto halo_at = [&](int lx, int ly) {
        int gx = x0 + lx - 1, gy = y0 + ly - 1;
        bool beyond = false;
        if (gx < 0 || gx >= nx) {
            if (xper) gx = wrap_index(gx, nx);
            else { beyond = true; gx = min(max(gx, 0), nx - 1); }
        }
        if (gy < 0 || gy >= ny) {
            if (yper) gy = wrap_index(gy, ny);
            else { beyond = true; gy = min(max(gy, 0), ny - 1); }
        }
        if (beyond) return;
        double ph[N], r, ps;
        halo_moments<N>(P, pin, ain, (long long)gy * nx + gx, ph, r, ps);
#pragma unroll
        for (int p = 0; p < N; ++p) s_phi[p][ly][lx] = ph[p];
        s_rho[ly][lx] = r;
        s_psi[ly][lx] = ps;
    };

    // ---- stage A + B of the own cell --------------------------------------
    double f[9], g[N][9], h[9];
    double phi[N], rhoH = 0.0, fl = 1.0, T = 0.0, rho = 1.0, mu = 0.0, lam = 0.0, cp = 1.0, psi = 0.0, chi = 0.0;
    // every thread keeps an in-range cell index: loads under `if (owned)` may be
    // issued speculatively, so a thread outside the domain must not form an address
    // past the end of the planes
    const long long c = owned ? (long long)y * nx + x : 0;
    if (owned) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = LBM_LD(P, pin, plane_f(i) * S + c, P.pop_elems, 5);
#pragma unroll
        for (int p = 0; p < N; ++p)
#pragma unroll
            for (int i = 0; i < 9; ++i) g[p][i] = LBM_LD(P, pin, plane_g(p, i) * S + c, P.pop_elems, 6);
#pragma unroll
        for (int i = 0; i < 9; ++i) h[i] = LBM_LD(P, pin, plane_h(N, i) * S + c, P.pop_elems, 7);
        const double mdm = LBM_LD(P, ain, aux_mdot() * S + c, P.aux_elems, 8);
        const double Qm = LBM_LD(P, ain, aux_Q() * S + c, P.aux_elems, 9);
        const double den = 1.0 - 0.5 * mdm;
#pragma unroll
        for (int p = 0; p < N; ++p) {
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < 9; ++i) s += g[p][i];
            phi[p] = s / den;
        }
        double sh = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) sh += h[i];
        rhoH = fma(0.5, Qm, sh);
        const Mix<N> m = mixture_core<N>(P, phi);
        enthalpy_map<N, true>(P, m, rhoH, fl, T);
        const double fs = 1.0 - fl;
        double ms = 0.0, ml = 0.0, ks = 0.0, kl = 0.0;
#pragma unroll
        for (int p = 0; p < N; ++p) {
            ms = fma(phi[p], P.mu_s[p], ms);
            ml = fma(phi[p], P.mu_l[p], ml);
            ks = fma(phi[p], P.lam_s[p], ks);
            kl = fma(phi[p], P.lam_l[p], kl);
        }
        rho = fma(fs, m.rs, fl * m.rl);
        mu = fma(fs, ms, fl * ml);
        lam = fma(fs, ks, fl * kl);
        cp = fma(fs, m.cs, fl * m.cl);
        psi = fs * m.dr;
        chi = fs * m.pcm;
#pragma unroll
        for (int p = 0; p < N; ++p) s_phi[p][ty + 1][tx + 1] = phi[p];
        s_rho[ty + 1][tx + 1] = rho;
        s_psi[ty + 1][tx + 1] = psi;
    } else {
        halo_at(tx + 1, ty + 1);
    }
    // ---- halo ring ---------------------------------------------------------
    for (int k = tid; k < NRING; k += NT) {
        int lx, ly;
        if (k < W) { lx = k; ly = 0; }
        else if (k < 2 * W) { lx = k - W; ly = H - 1; }
        else if (k < 2 * W + TY) { lx = 0; ly = k - 2 * W + 1; }
        else { lx = W - 1; ly = k - 2 * W - TY + 1; }
        halo_at(lx, ly);
    }
    __syncthreads();
    // ---- ghosts beyond walls / outflows ------------------------------------
    for (int k = tid; k < W * H; k += NT) {
        const int lx = k % W, ly = k / W;
        const int gx = x0 + lx - 1, gy = y0 + ly - 1;
        const bool xo = !xper && (gx < 0 || gx >= nx);
        const bool yo = !yper && (gy < 0 || gy >= ny);
        if (!xo && !yo) continue;
        const int sx = xo ? min(max(gx, 0), nx - 1) - x0 + 1 : lx;
        const int sy = yo ? min(max(gy, 0), ny - 1) - y0 + 1 : ly;
        const int wx = xo ? (gx < 0 ? 0 : 1) : -1;
        const int wy = yo ? (gy < 0 ? 2 : 3) : -1;
        double ph[N];
#pragma unroll
        for (int p = 0; p < N; ++p) ph[p] = s_phi[p][sy][sx];
#pragma unroll
        for (int p = 0; p < N; ++p) {
            double corr = 0.0;
#pragma unroll
            for (int q = 0; q < N; ++q) {
                if (q == p) continue;
                double cw = 0.0;
                if (wx >= 0) cw += P.wet[wx][p][q];
                if (wy >= 0) cw += P.wet[wy][p][q];
                corr = fma(cw * ph[p], ph[q], corr);
            }
            s_phi[p][ly][lx] = ph[p] + corr;
        }
        s_rho[ly][lx] = s_rho[sy][sx];
        s_psi[ly][lx] = s_psi[sy][sx];
    }
    __syncthreads();
    if (!owned) return;

    // ---- stage C: isotropic stencils ---------------------------------------
    const int lx = tx + 1, ly = ty + 1;
    double gpx[N], gpy[N], lap[N];
    auto grad = [&](double (*a)[W], double& gx_, double& gy_) {
        const double e = a[ly][lx + 1], w = a[ly][lx - 1], n = a[ly + 1][lx], s = a[ly - 1][lx];
        const double ne = a[ly + 1][lx + 1], nw = a[ly + 1][lx - 1], se = a[ly - 1][lx + 1], sw = a[ly - 1][lx - 1];
        gx_ = (e - w) * (1.0 / 3.0) + ((ne - nw) + (se - sw)) * (1.0 / 12.0);
        gy_ = (n - s) * (1.0 / 3.0) + ((ne - se) + (nw - sw)) * (1.0 / 12.0);
    };
#pragma unroll
    for (int p = 0; p < N; ++p) {
        double (*a)[W] = s_phi[p];
        grad(a, gpx[p], gpy[p]);
        const double v0 = a[ly][lx];
        const double ax = (a[ly][lx + 1] + a[ly][lx - 1]) + (a[ly + 1][lx] + a[ly - 1][lx]);
        const double dg = (a[ly + 1][lx + 1] + a[ly + 1][lx - 1]) + (a[ly - 1][lx + 1] + a[ly - 1][lx - 1]);
        lap[p] = ax * (2.0 / 3.0) + dg * (1.0 / 6.0) - v0 * (10.0 / 3.0);
    }
    double grx, gry, gsx, gsy;
    grad(s_rho, grx, gry);
    grad(s_psi, gsx, gsy);

    // ---- stage D: pairwise normals, R_p, chemical potentials, F_s -----------
    double Rx[N], Ry[N], mup[N], gpv[N];
#pragma unroll
    for (int p = 0; p < N; ++p) {
        Rx[p] = 0.0;
        Ry[p] = 0.0;
        mup[p] = 0.0;
        gpv[p] = gprime(phi[p]);
    }
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
        for (int q = p + 1; q < N; ++q) {
            const double s = phi[p] + phi[q];
            double nxv = 0.0, nyv = 0.0;
            if (s > 1e-12) {
                const double is2 = 1.0 / (s * s);
                const double Gx = (phi[q] * gpx[p] - phi[p] * gpx[q]) * is2;
                const double Gy = (phi[q] * gpy[p] - phi[p] * gpy[q]) * is2;
                const double G2 = Gx * Gx + Gy * Gy;
                if (G2 > 1e-24) {
                    const double r = rsqrt(G2);
                    nxv = Gx * r;
                    nyv = Gy * r;
                }
            }
            const double a = P.four_eps * phi[p] * phi[q];
            Rx[p] = fma(a, nxv, Rx[p]);
            Ry[p] = fma(a, nyv, Ry[p]);
            Rx[q] = fma(-a, nxv, Rx[q]);
            Ry[q] = fma(-a, nyv, Ry[q]);
            const double gs = gprime(s);
            mup[p] += fma(P.b2[p][q], gpv[p] - gs, P.kk[p][q] * lap[q]);
            mup[q] += fma(P.b2[q][p], gpv[q] - gs, P.kk[q][p] * lap[p]);
        }
    double Fx = rho * P.accel[0], Fy = rho * P.accel[1];
#pragma unroll
    for (int p = 0; p < N; ++p) {
        Fx = fma(mup[p], gpx[p], Fx);
        Fy = fma(mup[p], gpy[p], Fy);
    }

    // ---- stage E: flow macroscopics ----------------------------------------
    const double jx = ((f[1] - f[3]) + (f[5] - f[7])) + (f[8] - f[6]);
    const double jy = ((f[2] - f[4]) + (f[5] - f[7])) + (f[6] - f[8]);
    const double sum_f = ((f[1] + f[2]) + (f[3] + f[4])) + ((f[5] + f[6]) + (f[7] + f[8]));
    const double irho = 1.0 / rho;
    const double usx = fma(0.5, Fx, jx) * irho, usy = fma(0.5, Fy, jy) * irho;
    const double fpx = chi * (P.us[0] - usx), fpy = chi * (P.us[1] - usy);
    const double ux = fma(0.5, fpx, usx), uy = fma(0.5, fpy, usy);
    const double psim = LBM_LD(P, ain, aux_psi() * S + c, P.aux_elems, 14);
    const double mdot = -((psi - psim) + (ux * gsx + uy * gsy)) * irho;
    const double Ssrc = fma(rho, mdot, ux * grx + uy * gry);
    const double Lxx = fma(2.0 * ux, Fx, Ssrc * (1.0 / 3.0));
    const double Lyy = fma(2.0 * uy, Fy, Ssrc * (1.0 / 3.0));
    const double Lxy = fma(ux, Fy, uy * Fx);
    const double tau_f = fma(3.0 * mu, irho, 0.5);
    const double F0 = wgt(0) * fma(-1.5, Lxx + Lyy, Ssrc);
    const double uu = fma(ux, ux, uy * uy);
    const double p = 0.6 * (((sum_f + 0.5 * Ssrc) + (tau_f - 0.5) * F0) - rho * wgt(0) * 1.5 * uu);

    if (!COLLIDE) {
#pragma unroll
        for (int q = 0; q < N; ++q)
            if (ex.phi) LBM_ST(P, ex.phi, q * S + c, N * S, 20, phi[q]);
        if (ex.T) LBM_ST(P, ex.T, c, S, 21, T);
        if (ex.H) LBM_ST(P, ex.H, c, S, 22, rhoH * irho);
        if (ex.fl) LBM_ST(P, ex.fl, c, S, 23, fl);
        if (ex.ux) LBM_ST(P, ex.ux, c, S, 24, ux);
        if (ex.uy) LBM_ST(P, ex.uy, c, S, 25, uy);
        if (ex.p) LBM_ST(P, ex.p, c, S, 26, p);
        return;
    }

    // ---- stage F: flow collision -------------------------------------------
    {
        const double om = 1.0 / tau_f, k = fma(-0.5, om, 1.0), om1 = 1.0 - om;
        const double Fex = fma(rho, fpx, Fx), Fey = fma(rho, fpy, Fy);
        const double rom = om * rho;
        const double a0 = om * fma(-1.5 * rho, uu, 3.0 * p) + k * fma(-1.5, Lxx + Lyy, Ssrc);
        const double ax = 3.0 * fma(rom, ux, k * Fex);
        const double ay = 3.0 * fma(rom, uy, k * Fey);
        const double axx = 4.5 * fma(rom * ux, ux, k * Lxx);
        const double ayy = 4.5 * fma(rom * uy, uy, k * Lyy);
        const double axy = 9.0 * fma(rom * ux, uy, k * Lxy);
        const double bx = a0 + axx, by = a0 + ayy, bd = a0 + axx + ayy;
        double X[9];
        X[0] = fma(-6.75 * om, p, a0);
        X[1] = bx + ax;
        X[3] = bx - ax;
        X[2] = by + ay;
        X[4] = by - ay;
        X[5] = (bd + axy) + (ax + ay);
        X[7] = (bd + axy) - (ax + ay);
        X[6] = (bd - axy) + (ay - ax);
        X[8] = (bd - axy) - (ay - ax);
        double q[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) q[i] = fma(wgt(i), X[i], om1 * f[i]);
#define LBM_PUSH_F(J) push<J, false>(P, pout, plane_f(J), plane_f(opp(J)), x, y, q[J]);
        LBM_PUSH_F(0) LBM_PUSH_F(1) LBM_PUSH_F(2) LBM_PUSH_F(3) LBM_PUSH_F(4)
        LBM_PUSH_F(5) LBM_PUSH_F(6) LBM_PUSH_F(7) LBM_PUSH_F(8)
#undef LBM_PUSH_F
        if (y == 0 && P.bc[2] == OUTFLOW) {
            push_row<2>(P, pout, plane_f(2), x, y, q[2]);
            push_row<5>(P, pout, plane_f(5), x, y, q[5]);
            push_row<6>(P, pout, plane_f(6), x, y, q[6]);
        }
        if (y == ny - 1 && P.bc[3] == OUTFLOW) {
            push_row<4>(P, pout, plane_f(4), x, y, q[4]);
            push_row<7>(P, pout, plane_f(7), x, y, q[7]);
            push_row<8>(P, pout, plane_f(8), x, y, q[8]);
        }
    }

    // ---- stage F: phase-field collisions -------------------------------------
    {
        const double og = P.omega_g, kg = P.kg, og1 = 1.0 - og;
#pragma unroll
        for (int pp = 0; pp < N; ++pp) {
            const double Dx = phi[pp] * ux - LBM_LD(P, ain, aux_phiux(pp) * S + c, P.aux_elems, 15);
            const double Dy = phi[pp] * uy - LBM_LD(P, ain, aux_phiuy(N, pp) * S + c, P.aux_elems, 16);
            const double b0 = og * phi[pp] + kg * phi[pp] * mdot;
            const double bxv = 3.0 * og * phi[pp] * ux + kg * fma(3.0, Dx, Rx[pp]);
            const double byv = 3.0 * og * phi[pp] * uy + kg * fma(3.0, Dy, Ry[pp]);
            double q[9];
            q[0] = fma(wgt(0), b0, og1 * g[pp][0]);
            q[1] = fma(wgt(1), b0 + bxv, og1 * g[pp][1]);
            q[3] = fma(wgt(3), b0 - bxv, og1 * g[pp][3]);
            q[2] = fma(wgt(2), b0 + byv, og1 * g[pp][2]);
            q[4] = fma(wgt(4), b0 - byv, og1 * g[pp][4]);
            q[5] = fma(wgt(5), b0 + (bxv + byv), og1 * g[pp][5]);
            q[7] = fma(wgt(7), b0 - (bxv + byv), og1 * g[pp][7]);
            q[6] = fma(wgt(6), b0 + (byv - bxv), og1 * g[pp][6]);
            q[8] = fma(wgt(8), b0 - (byv - bxv), og1 * g[pp][8]);
#define LBM_PUSH_G(J) push<J, false>(P, pout, plane_g(pp, J), plane_g(pp, opp(J)), x, y, q[J]);
            LBM_PUSH_G(0) LBM_PUSH_G(1) LBM_PUSH_G(2) LBM_PUSH_G(3) LBM_PUSH_G(4)
            LBM_PUSH_G(5) LBM_PUSH_G(6) LBM_PUSH_G(7) LBM_PUSH_G(8)
#undef LBM_PUSH_G
            if (y == 0 && P.bc[2] == OUTFLOW) {
                push_row<2>(P, pout, plane_g(pp, 2), x, y, q[2]);
                push_row<5>(P, pout, plane_g(pp, 5), x, y, q[5]);
                push_row<6>(P, pout, plane_g(pp, 6), x, y, q[6]);
            }
            if (y == ny - 1 && P.bc[3] == OUTFLOW) {
                push_row<4>(P, pout, plane_g(pp, 4), x, y, q[4]);
                push_row<7>(P, pout, plane_g(pp, 7), x, y, q[7]);
                push_row<8>(P, pout, plane_g(pp, 8), x, y, q[8]);
            }
            LBM_ST(P, aout, aux_phiux(pp) * S + c, P.aux_elems, 30, phi[pp] * ux);
            LBM_ST(P, aout, aux_phiuy(N, pp) * S + c, P.aux_elems, 31, phi[pp] * uy);
        }
    }

    // ---- stage F: enthalpy collision + Dirichlet ghosts ---------------------
    {
        const double Z = rho * cp * T, E = P.E_ref * T;
        const double oh = 1.0 / fma(lam, P.tau_h_scale, 0.5), kh = fma(-0.5, oh, 1.0), oh1 = 1.0 - oh;
        const double Zm = Z * mdot;
        const double c0 = oh * fma(-1.5 * Z, uu, E) + kh * Zm;
        const double ohZ = oh * Z;
        const double cxv = 3.0 * ohZ * ux, cyv = 3.0 * ohZ * uy;
        const double cxx = 4.5 * ohZ * ux * ux, cyy = 4.5 * ohZ * uy * uy, cxy = 9.0 * ohZ * ux * uy;
        const double heq0 = (rhoH - E) + wgt(0) * fma(-1.5 * Z, uu, E);
        const double bx = c0 + cxx, by = c0 + cyy, bd = c0 + cxx + cyy;
        double q[9];
        q[0] = fma(oh, heq0, fma(kh * wgt(0), Zm, oh1 * h[0]));
        q[1] = fma(wgt(1), bx + cxv, oh1 * h[1]);
        q[3] = fma(wgt(3), bx - cxv, oh1 * h[3]);
        q[2] = fma(wgt(2), by + cyv, oh1 * h[2]);
        q[4] = fma(wgt(4), by - cyv, oh1 * h[4]);
        q[5] = fma(wgt(5), (bd + cxy) + (cxv + cyv), oh1 * h[5]);
        q[7] = fma(wgt(7), (bd + cxy) - (cxv + cyv), oh1 * h[7]);
        q[6] = fma(wgt(6), (bd - cxy) + (cyv - cxv), oh1 * h[6]);
        q[8] = fma(wgt(8), (bd - cxy) - (cyv - cxv), oh1 * h[8]);
#define LBM_PUSH_H(J) push<J, true>(P, pout, plane_h(N, J), plane_h(N, opp(J)), x, y, q[J]);
        LBM_PUSH_H(0) LBM_PUSH_H(1) LBM_PUSH_H(2) LBM_PUSH_H(3) LBM_PUSH_H(4)
        LBM_PUSH_H(5) LBM_PUSH_H(6) LBM_PUSH_H(7) LBM_PUSH_H(8)
#undef LBM_PUSH_H
        // equilibrium of direction j != 0 (for the ghost rule)
        auto heq = [&](int j) {
            const double cu = cx(j) * ux + cy(j) * uy;
            return wgt(j) * fma(Z, fma(4.5 * cu, cu, fma(3.0, cu, -1.5 * uu)), E);
        };
        // Dirichlet wall: ghost behind the half-way wall with T_g = 2 T_w - T, u = 0;
        // its post-collision population is h_eq(ghost) + (1 - 1/tau_h)(h_j - h_eq_j).
        if (y == 0 && P.bc[2] == WALL && P.tbc[2] == DIRICHLET) {
            const double Eg = P.E_ref * (2.0 * P.Tw[2] - T);
            push_row<2>(P, pout, plane_h(N, 2), x, y, fma(oh1, h[2] - heq(2), wgt(2) * Eg));
            push_row<5>(P, pout, plane_h(N, 5), x, y, fma(oh1, h[5] - heq(5), wgt(5) * Eg));
            push_row<6>(P, pout, plane_h(N, 6), x, y, fma(oh1, h[6] - heq(6), wgt(6) * Eg));
        } else if (y == 0 && P.bc[2] == OUTFLOW) {
            push_row<2>(P, pout, plane_h(N, 2), x, y, q[2]);
            push_row<5>(P, pout, plane_h(N, 5), x, y, q[5]);
            push_row<6>(P, pout, plane_h(N, 6), x, y, q[6]);
        }
        if (y == ny - 1 && P.bc[3] == WALL && P.tbc[3] == DIRICHLET) {
            const double Eg = P.E_ref * (2.0 * P.Tw[3] - T);
            push_row<4>(P, pout, plane_h(N, 4), x, y, fma(oh1, h[4] - heq(4), wgt(4) * Eg));
            push_row<7>(P, pout, plane_h(N, 7), x, y, fma(oh1, h[7] - heq(7), wgt(7) * Eg));
            push_row<8>(P, pout, plane_h(N, 8), x, y, fma(oh1, h[8] - heq(8), wgt(8) * Eg));
        } else if (y == ny - 1 && P.bc[3] == OUTFLOW) {
            push_row<4>(P, pout, plane_h(N, 4), x, y, q[4]);
            push_row<7>(P, pout, plane_h(N, 7), x, y, q[7]);
            push_row<8>(P, pout, plane_h(N, 8), x, y, q[8]);
        }

        // ---- stage G: lagged planes ------------------------------------------
        LBM_ST(P, aout, aux_mdot() * S + c, P.aux_elems, 32, mdot);
        LBM_ST(P, aout, aux_Q() * S + c, P.aux_elems, 33, Zm);
        LBM_ST(P, aout, aux_psi() * S + c, P.aux_elems, 34, psi);
    }
}

}  // namespace lbm
