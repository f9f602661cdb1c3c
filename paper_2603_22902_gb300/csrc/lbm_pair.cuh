// lbm_pair.cuh -- the fused time step with two cells per thread, for the policies that
// compute in FP32 (FP32, FP16 and BF16 storage).
//
// A thread owns the cells (x, y) and (x, y + 1) of a TX x TY tile (TX x TY/2 threads per
// block).  The arithmetic of the step, which is the same for both cells, runs on packed
// FP32 pairs (add / sub / mul / fma .rn.f32x2: one instruction for the two cells), and the
// two cells share their stencil loads (a 3 x 4 window of shared memory for two 3 x 3
// stencils), their address arithmetic and their loop overhead.  With half the threads, a
// lattice of 512 x 512 fills the GPU in fewer waves, and every thread has twice the
// independent loads in flight.  Everything that branches per cell (the FP32 screen and
// FP64 fallback of eq. H, the guards of the pairwise normal, the divisions, the boundary
// rules of the pushes) runs per cell, as in the one-cell step (lbm_step.cuh), whose
// per-cell functions are reused; the ring of the tile is recomputed one cell per thread
// as there.  The order of operations is that of the one-cell step, so the two forms agree
// to the rounding of contractions (an FMA formed in one and not the other).
#pragma once

#include "lbm_step.cuh"

namespace lbm {

// Two FP32 values, one per cell of the pair, with packed arithmetic.
struct __align__(8) f2 {
    float a, b;
    f2() = default;
    __device__ __forceinline__ constexpr f2(float x, float y) : a(x), b(y) {}
    __device__ __forceinline__ explicit constexpr f2(float x) : a(x), b(x) {}
};

__device__ __forceinline__ unsigned long long f2_bits(f2 v)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.a), "f"(v.b));
    return r;
}
__device__ __forceinline__ f2 f2_from(unsigned long long r)
{
    f2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.a), "=f"(v.b) : "l"(r));
    return v;
}
__device__ __forceinline__ f2 operator+(f2 x, f2 y)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(x)), "l"(f2_bits(y)));
    return f2_from(r);
}
__device__ __forceinline__ f2 operator-(f2 x, f2 y)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(x)), "l"(f2_bits(y)));
    return f2_from(r);
}
__device__ __forceinline__ f2 operator*(f2 x, f2 y)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(x)), "l"(f2_bits(y)));
    return f2_from(r);
}
__device__ __forceinline__ f2 operator-(f2 x) { return f2(-x.a, -x.b); }
__device__ __forceinline__ f2 operator*(f2 x, float s) { return x * f2(s); }
__device__ __forceinline__ f2 operator*(float s, f2 x) { return f2(s) * x; }
__device__ __forceinline__ f2& operator+=(f2& x, f2 y) { return x = x + y; }
// a b + c with one rounding per cell
__device__ __forceinline__ f2 rfma(f2 a, f2 b, f2 c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
    return f2_from(r);
}
__device__ __forceinline__ f2 rfma(float a, f2 b, f2 c) { return rfma(f2(a), b, c); }
__device__ __forceinline__ f2 rfma(f2 a, float b, f2 c) { return rfma(a, f2(b), c); }

// A lagged value of one cell, as float.
template <class Pr>
__device__ __forceinline__ float ld_aux(const KParams& P, const typename Pr::TA* __restrict__ a, long long idx, int site)
{
    return (float)LBM_LDX(Pr::COH, P, a, idx, P.aux_elems, site);
}

template <int N>
__device__ __forceinline__ f2 mix_sum2(const f2 (&phi)[N], const float (&a)[MAXN])
{
    f2 v = f2(0.0f);
#pragma unroll
    for (int p = 0; p < N; ++p) v = rfma(phi[p], f2(a[p]), v);
    return v;
}

// Population i of species s at the cells c and c + nx (dequantised).
template <class Pr, int KIND>
__device__ __forceinline__ f2 ld_pop2(const KParams& P, const PopView<Pr>& v, int s, int i, long long c0, long long c1,
                                      bool late)
{
    if (late) return f2(ld_pop_late<Pr, KIND>(P, v, s, i, c0, 5), ld_pop_late<Pr, KIND>(P, v, s, i, c1, 5));
    return f2(ld_pop<Pr, KIND>(P, v, s, i, c0, 3), ld_pop<Pr, KIND>(P, v, s, i, c1, 3));
}

// One TX x TY tile of one time step with two cells per thread: TX x TY/2 threads, thread
// (tx, tp) owns the cells (x0 + tx, y0 + 2 tp) and (x0 + tx, y0 + 2 tp + 1).
template <int N, int TX, int TY, bool COLLIDE, class Pr>
__device__ __forceinline__ void step_tile_pair(const KParams& P, const void* __restrict__ pin_base,
                                               void* __restrict__ pout_base, const typename Pr::TA* __restrict__ ain,
                                               typename Pr::TA* __restrict__ aout, const ExportPtrs& ex, int bx,
                                               int by, float* smem)
{
    static_assert(std::is_same<typename Pr::R, float>::value, "the pair step computes in FP32");
    static_assert(TY % 2 == 0, "pairs of rows");
    using R = float;
    using TA = typename Pr::TA;
    constexpr int W = TX + 2, H = TY + 2, NT = TX * TY / 2;
    R (*s_phi)[H][W] = reinterpret_cast<R (*)[H][W]>(smem);
    R (*s_rho)[W] = reinterpret_cast<R (*)[W]>(smem + N * H * W);
    R (*s_psi)[W] = reinterpret_cast<R (*)[W]>(smem + (N + 1) * H * W);

    const int nx = P.nx, ny = P.ny;
    const long long S = P.S;
    const int tid = threadIdx.x;
    const int tx = tid % TX, tp = tid / TX;
    const int x0 = bx * TX, y0 = by * TY;
    const int x = x0 + tx, y = y0 + 2 * tp;
    const bool own0 = x < nx && y < ny, own1 = x < nx && y + 1 < ny;
    const bool xper = P.bc[0] == PERIODIC, yper = P.bc[2] == PERIODIC;
    const PopView<Pr> pin = pop_view<Pr>(P, pin_base);
    const Coef<float>& C = P.f;

    auto locate = [&](int lx, int ly, long long& cell) {
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
        cell = (long long)gy * nx + gx;
        return !beyond;
    };
    auto halo_at = [&](int lx, int ly) {
        long long cell;
        if (!locate(lx, ly, cell)) return;
        R ph[N], r, ps;
        halo_moments<N, Pr>(P, pin, ain, cell, ph, r, ps);
#pragma unroll
        for (int p = 0; p < N; ++p) s_phi[p][ly][lx] = ph[p];
        s_rho[ly][lx] = r;
        s_psi[ly][lx] = ps;
    };

    // cells of the pair; an unowned second cell (odd ny in the last tile row) reads the
    // first cell's values and writes nothing
    const long long c0 = (long long)min(y, ny - 1) * nx + min(x, nx - 1);
    const long long c1 = own1 ? c0 + nx : c0;
    const int lx = tx + 1, ly = 2 * tp + 1;

    // ---- stages A + B: the pair's moments, packed; eq. H per cell ---------------------
    f2 phi[N], rhoH, fl, T, rho, psi, mu, lam, cp, chi;
    if (own0) {
        const f2 mdm(ld_aux<Pr>(P, ain, aux_mdot() * S + c0, 1), ld_aux<Pr>(P, ain, aux_mdot() * S + c1, 1));
        const f2 Qm(ld_aux<Pr>(P, ain, aux_Q() * S + c0, 2), ld_aux<Pr>(P, ain, aux_Q() * S + c1, 2));
        const f2 den = f2(1.0f) - f2(0.5f) * mdm;
        const f2 iden(1.0f / den.a, 1.0f / den.b);
#pragma unroll
        for (int p = 0; p < N; ++p) {
            f2 s = f2(0.0f);
#pragma unroll
            for (int i = 0; i < 9; ++i) s += ld_pop2<Pr, KIND_G>(P, pin, 1 + p, i, c0, c1, false);
            phi[p] = s * iden;
        }
        f2 sh = f2(0.0f);
#pragma unroll
        for (int i = 0; i < 9; ++i) sh += ld_pop2<Pr, KIND_H>(P, pin, N + 1, i, c0, c1, false);
        rhoH = rfma(f2(0.5f), Qm, sh);
        R pa[N], pb[N];
#pragma unroll
        for (int p = 0; p < N; ++p) {
            pa[p] = phi[p].a;
            pb[p] = phi[p].b;
        }
        map_cell<N, Pr, true>(P, pa, rhoH.a, fl.a, T.a);
        map_cell<N, Pr, true>(P, pb, rhoH.b, fl.b, T.b);
        const f2 fs = f2(1.0f) - fl;
        rho = rfma(fs, mix_sum2<N>(phi, C.rho_s), fl * mix_sum2<N>(phi, C.rho_l));
        psi = fs * mix_sum2<N>(phi, C.drho);
        mu = rfma(fs, mix_sum2<N>(phi, C.mu_s), fl * mix_sum2<N>(phi, C.mu_l));
        lam = rfma(fs, mix_sum2<N>(phi, C.lam_s), fl * mix_sum2<N>(phi, C.lam_l));
        cp = rfma(fs, mix_sum2<N>(phi, C.cp_s), fl * mix_sum2<N>(phi, C.cp_l));
        chi = fs * mix_sum2<N>(phi, C.pcm);
#pragma unroll
        for (int p = 0; p < N; ++p) {
            s_phi[p][ly][lx] = phi[p].a;
            if (own1) s_phi[p][ly + 1][lx] = phi[p].b;
        }
        s_rho[ly][lx] = rho.a;
        s_psi[ly][lx] = psi.a;
        if (own1) {
            s_rho[ly + 1][lx] = rho.b;
            s_psi[ly + 1][lx] = psi.b;
        }
    }
    // positions of the tile that no thread owns (beyond the lattice on a periodic axis
    // that is narrower or shorter than the tile) and the ring: one cell per thread
    if (!own0) halo_at(lx, ly);
    if (!own1) halo_at(lx, ly + 1);
    constexpr int NRING = 2 * W + 2 * TY;
    for (int k = tid; k < NRING; k += NT) {
        int rx, ry;
        if (k < W) { rx = k; ry = 0; }
        else if (k < 2 * W) { rx = k - W; ry = H - 1; }
        else if (k < 2 * W + TY) { rx = 0; ry = k - 2 * W + 1; }
        else { rx = W - 1; ry = k - 2 * W - TY + 1; }
        halo_at(rx, ry);
    }
    __syncthreads();
    // ---- ghosts beyond walls / outflows (as the one-cell step) -------------------------
    const bool ghosts = (!xper && (x0 < 1 || x0 + TX > nx - 1)) || (!yper && (y0 < 1 || y0 + TY > ny - 1));
    if (ghosts) {
        for (int k = tid; k < W * H; k += NT) {
            const int gx_ = k % W, gy_ = k / W;
            const int gx = x0 + gx_ - 1, gy = y0 + gy_ - 1;
            const bool xo = !xper && (gx < 0 || gx >= nx);
            const bool yo = !yper && (gy < 0 || gy >= ny);
            if (!xo && !yo) continue;
            const int sx = xo ? min(max(gx, 0), nx - 1) - x0 + 1 : gx_;
            const int sy = yo ? min(max(gy, 0), ny - 1) - y0 + 1 : gy_;
            const int wx = xo ? (gx < 0 ? 0 : 1) : -1;
            const int wy = yo ? (gy < 0 ? 2 : 3) : -1;
            R ph[N];
#pragma unroll
            for (int p = 0; p < N; ++p) ph[p] = s_phi[p][sy][sx];
#pragma unroll
            for (int p = 0; p < N; ++p) {
                R corr = 0.0f;
#pragma unroll
                for (int q = 0; q < N; ++q) {
                    if (q == p) continue;
                    R cw = 0.0f;
                    if (wx >= 0) cw += C.wet[wx][p][q];
                    if (wy >= 0) cw += C.wet[wy][p][q];
                    corr = fmaf(cw * ph[p], ph[q], corr);
                }
                s_phi[p][gy_][gx_] = ph[p] + corr;
            }
            s_rho[gy_][gx_] = s_rho[sy][sx];
            s_psi[gy_][gx_] = s_psi[sy][sx];
        }
        __syncthreads();
    }
    if (!own0) return;

    // ---- stage C: stencils of both cells from a 3 x 4 window -------------------------
    f2 gpx[N + 2], gpy[N + 2], lap[N];
#pragma unroll
    for (int fi = 0; fi < N + 2; ++fi) {
        R (*a)[W] = reinterpret_cast<R (*)[W]>(smem + fi * H * W);
        // rows ly - 1 .. ly + 2 of columns lx - 1, lx, lx + 1
        const R w0 = a[ly - 1][lx - 1], m0 = a[ly - 1][lx], e0 = a[ly - 1][lx + 1];
        const R w1 = a[ly][lx - 1], m1 = a[ly][lx], e1 = a[ly][lx + 1];
        const R w2 = a[ly + 1][lx - 1], m2 = a[ly + 1][lx], e2 = a[ly + 1][lx + 1];
        const R w3 = a[ly + 2][lx - 1], m3 = a[ly + 2][lx], e3 = a[ly + 2][lx + 1];
        // for the cell of row r: e, w (same row), n, s (rows r + 1, r - 1), ne .. sw
        const f2 e(e1, e2), w(w1, w2), n(m2, m3), s(m0, m1);
        const f2 ne(e2, e3), nw(w2, w3), se(e0, e1), sw(w0, w1);
        gpx[fi] = (e - w) * (1.0f / 3.0f) + ((ne - nw) + (se - sw)) * (1.0f / 12.0f);
        gpy[fi] = (n - s) * (1.0f / 3.0f) + ((ne - se) + (nw - sw)) * (1.0f / 12.0f);
        if (fi < N) {
            const f2 v0(m1, m2);
            const f2 ax = (e + w) + (n + s);
            const f2 dg = (ne + nw) + (se + sw);
            lap[fi] = ax * (2.0f / 3.0f) + dg * (1.0f / 6.0f) - v0 * (10.0f / 3.0f);
        }
    }
    const f2 grx = gpx[N], gry = gpy[N], gsx = gpx[N + 1], gsy = gpy[N + 1];

    // ---- stage D: pairwise normals (guards per cell), R_p, mu_p, F_s -----------------
    f2 Rx[N], Ry[N], mup[N], gpv[N];
#pragma unroll
    for (int p = 0; p < N; ++p) {
        Rx[p] = f2(0.0f);
        Ry[p] = f2(0.0f);
        mup[p] = f2(0.0f);
        gpv[p] = f2(2.0f) * phi[p] * (f2(1.0f) - phi[p]) * (f2(1.0f) - f2(2.0f) * phi[p]);
    }
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
        for (int q = p + 1; q < N; ++q) {
            const f2 s = phi[p] + phi[q];
            const f2 Gx = phi[q] * gpx[p] - phi[p] * gpx[q];
            const f2 Gy = phi[q] * gpy[p] - phi[p] * gpy[q];
            const f2 G2 = Gx * Gx + Gy * Gy;
            const f2 s2 = s * s;
            const f2 lim = f2((float)Pr::NABS2) * (s2 * s2);
            bool oka = s.a > 1e-12f && G2.a > lim.a, okb = s.b > 1e-12f && G2.b > lim.b;
            if constexpr (Pr::NGUARD > 0.0f) {
                const f2 ref = phi[q] * phi[q] * (gpx[p] * gpx[p] + gpy[p] * gpy[p]) +
                               phi[p] * phi[p] * (gpx[q] * gpx[q] + gpy[q] * gpy[q]);
                const f2 gl = f2(Pr::NGUARD * Pr::NGUARD) * ref;
                oka = oka && G2.a > gl.a;
                okb = okb && G2.b > gl.b;
            }
            const f2 r(oka ? rsqrtf(G2.a) : 0.0f, okb ? rsqrtf(G2.b) : 0.0f);
            const f2 nxv = Gx * r, nyv = Gy * r;
            const f2 a = f2(C.four_eps) * phi[p] * phi[q];
            Rx[p] = rfma(a, nxv, Rx[p]);
            Ry[p] = rfma(a, nyv, Ry[p]);
            Rx[q] = rfma(-a, nxv, Rx[q]);
            Ry[q] = rfma(-a, nyv, Ry[q]);
            const f2 gs = f2(2.0f) * s * (f2(1.0f) - s) * (f2(1.0f) - f2(2.0f) * s);
            mup[p] += rfma(f2(C.b2[p][q]), gpv[p] - gs, f2(C.kk[p][q]) * lap[q]);
            mup[q] += rfma(f2(C.b2[q][p]), gpv[q] - gs, f2(C.kk[q][p]) * lap[p]);
        }
    f2 Fx = rho * C.accel[0], Fy = rho * C.accel[1];
#pragma unroll
    for (int p = 0; p < N; ++p) {
        Fx = rfma(mup[p], gpx[p], Fx);
        Fy = rfma(mup[p], gpy[p], Fy);
    }

    // ---- stage E: flow macroscopics ----------------------------------------------------
    f2 f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = ld_pop2<Pr, KIND_F>(P, pin, 0, i, c0, c1, true);
    const f2 jx = ((f[1] - f[3]) + (f[5] - f[7])) + (f[8] - f[6]);
    const f2 jy = ((f[2] - f[4]) + (f[5] - f[7])) + (f[6] - f[8]);
    const f2 sum_f = ((f[1] + f[2]) + (f[3] + f[4])) + ((f[5] + f[6]) + (f[7] + f[8]));
    const f2 Af = rfma(f2(3.0f), mu, f2(0.5f) * rho);
    const f2 Bh = rfma(lam, f2(C.tau_h_scale), f2(0.5f));
    const f2 dAB = rho * Af * Bh;
    const f2 rAB(1.0f / dAB.a, 1.0f / dAB.b);
    const f2 irho = (Af * Bh) * rAB;
    const f2 om = (rho * rho) * (Bh * rAB);
    const f2 oh = (rho * Af) * rAB;
    const f2 usx = rfma(f2(0.5f), Fx, jx) * irho, usy = rfma(f2(0.5f), Fy, jy) * irho;
    const f2 fpx = chi * (f2(C.us[0]) - usx), fpy = chi * (f2(C.us[1]) - usy);
    const f2 ux = rfma(f2(0.5f), fpx, usx), uy = rfma(f2(0.5f), fpy, usy);
    const f2 psim(ld_aux<Pr>(P, ain, aux_psi() * S + c0, 14), ld_aux<Pr>(P, ain, aux_psi() * S + c1, 14));
    const f2 mdot = -((psi - psim) + (ux * gsx + uy * gsy)) * irho;
    const f2 Ssrc = rfma(rho, mdot, ux * grx + uy * gry);
    const f2 Lxx = rfma(f2(2.0f) * ux, Fx, Ssrc * (1.0f / 3.0f));
    const f2 Lyy = rfma(f2(2.0f) * uy, Fy, Ssrc * (1.0f / 3.0f));
    const f2 Lxy = rfma(ux, Fy, uy * Fx);
    const f2 tmh = f2(3.0f) * mu * irho;
    const float w0 = wgt_r<float>(0);
    const f2 F0 = f2(w0) * rfma(f2(-1.5f), Lxx + Lyy, Ssrc);
    const f2 uu = rfma(ux, ux, uy * uy);
    const f2 p = f2(0.6f) * (((sum_f + f2(0.5f) * Ssrc) + tmh * F0) - rho * f2(w0) * f2(1.5f) * uu);

    if (!COLLIDE) {
        const long long cc[2] = {c0, c1};
        const bool oo[2] = {true, own1};
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (!oo[k]) continue;
            const long long c = cc[k];
            auto pick = [&](f2 v) { return (double)(k == 0 ? v.a : v.b); };
#pragma unroll
            for (int q = 0; q < N; ++q)
                if (ex.phi) LBM_ST(P, ex.phi, q * S + c, N * S, 20, pick(phi[q]));
            if (ex.T) LBM_ST(P, ex.T, c, S, 21, pick(T));
            if (ex.H) LBM_ST(P, ex.H, c, S, 22, pick(rhoH * irho));
            if (ex.fl) LBM_ST(P, ex.fl, c, S, 23, pick(fl));
            if (ex.ux) LBM_ST(P, ex.ux, c, S, 24, pick(ux));
            if (ex.uy) LBM_ST(P, ex.uy, c, S, 25, pick(uy));
            if (ex.p) LBM_ST(P, ex.p, c, S, 26, pick(p));
        }
        return;
    }
    const PopView<Pr> pout = pop_view<Pr>(P, pout_base);
    const bool interior = x0 >= 1 && x0 + TX <= nx - 1 && y0 >= 1 && y0 + TY <= ny - 1;
    auto push2 = [&](int KINDS, int s, const f2 (&q)[9]) {
        R qa[9], qb[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            qa[i] = q[i].a;
            qb[i] = q[i].b;
        }
        if (KINDS == KIND_F) {
            push_species<KIND_F, Pr>(P, pout, s, x, y, interior, qa);
            if (own1) push_species<KIND_F, Pr>(P, pout, s, x, y + 1, interior, qb);
        } else if (KINDS == KIND_G) {
            push_species<KIND_G, Pr>(P, pout, s, x, y, interior, qa);
            if (own1) push_species<KIND_G, Pr>(P, pout, s, x, y + 1, interior, qb);
        } else {
            push_species<KIND_H, Pr>(P, pout, s, x, y, interior, qa);
            if (own1) push_species<KIND_H, Pr>(P, pout, s, x, y + 1, interior, qb);
        }
    };

    // ---- stage F: flow collision -------------------------------------------------------
    {
        const f2 k = rfma(f2(-0.5f), om, f2(1.0f)), om1 = f2(1.0f) - om;
        const f2 Fex = rfma(rho, fpx, Fx), Fey = rfma(rho, fpy, Fy);
        const f2 rom = om * rho;
        const f2 a0 = om * rfma(f2(-1.5f) * rho, uu, f2(3.0f) * p) + k * rfma(f2(-1.5f), Lxx + Lyy, Ssrc);
        const f2 ax = f2(3.0f) * rfma(rom, ux, k * Fex);
        const f2 ay = f2(3.0f) * rfma(rom, uy, k * Fey);
        const f2 axx = f2(4.5f) * rfma(rom * ux, ux, k * Lxx);
        const f2 ayy = f2(4.5f) * rfma(rom * uy, uy, k * Lyy);
        const f2 axy = f2(9.0f) * rfma(rom * ux, uy, k * Lxy);
        const f2 bx_ = a0 + axx, by_ = a0 + ayy, bd = a0 + axx + ayy;
        f2 X[9];
        X[0] = rfma(f2(-6.75f) * om, p, a0);
        X[1] = bx_ + ax;
        X[3] = bx_ - ax;
        X[2] = by_ + ay;
        X[4] = by_ - ay;
        X[5] = (bd + axy) + (ax + ay);
        X[7] = (bd + axy) - (ax + ay);
        X[6] = (bd - axy) + (ay - ax);
        X[8] = (bd - axy) - (ay - ax);
        f2 q[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) q[i] = rfma(f2(wgt_r<float>(i)), X[i], om1 * f[i]);
        push2(KIND_F, 0, q);
    }

    // ---- stage F: phase-field collisions -----------------------------------------------
    {
        const f2 og(C.omega_g), kg(C.kg), og1 = f2(1.0f) - og;
#pragma unroll
        for (int pp = 0; pp < N; ++pp) {
            f2 gq[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) gq[i] = ld_pop2<Pr, KIND_G>(P, pin, 1 + pp, i, c0, c1, true);
            const f2 ux_m(ld_aux<Pr>(P, ain, aux_phiux(pp) * S + c0, 15), ld_aux<Pr>(P, ain, aux_phiux(pp) * S + c1, 15));
            const f2 uy_m(ld_aux<Pr>(P, ain, aux_phiuy(N, pp) * S + c0, 16),
                          ld_aux<Pr>(P, ain, aux_phiuy(N, pp) * S + c1, 16));
            const f2 Dx = phi[pp] * ux - ux_m;
            const f2 Dy = phi[pp] * uy - uy_m;
            const f2 b0 = og * phi[pp] + kg * phi[pp] * mdot;
            const f2 bxv = f2(3.0f) * og * phi[pp] * ux + kg * rfma(f2(3.0f), Dx, Rx[pp]);
            const f2 byv = f2(3.0f) * og * phi[pp] * uy + kg * rfma(f2(3.0f), Dy, Ry[pp]);
            f2 q[9];
            q[0] = rfma(f2(wgt_r<float>(0)), b0, og1 * gq[0]);
            q[1] = rfma(f2(wgt_r<float>(1)), b0 + bxv, og1 * gq[1]);
            q[3] = rfma(f2(wgt_r<float>(3)), b0 - bxv, og1 * gq[3]);
            q[2] = rfma(f2(wgt_r<float>(2)), b0 + byv, og1 * gq[2]);
            q[4] = rfma(f2(wgt_r<float>(4)), b0 - byv, og1 * gq[4]);
            q[5] = rfma(f2(wgt_r<float>(5)), b0 + (bxv + byv), og1 * gq[5]);
            q[7] = rfma(f2(wgt_r<float>(7)), b0 - (bxv + byv), og1 * gq[7]);
            q[6] = rfma(f2(wgt_r<float>(6)), b0 + (byv - bxv), og1 * gq[6]);
            q[8] = rfma(f2(wgt_r<float>(8)), b0 - (byv - bxv), og1 * gq[8]);
            push2(KIND_G, 1 + pp, q);
            const f2 pux = phi[pp] * ux, puy = phi[pp] * uy;
            LBM_ST(P, aout, aux_phiux(pp) * S + c0, P.aux_elems, 30, (TA)pux.a);
            LBM_ST(P, aout, aux_phiuy(N, pp) * S + c0, P.aux_elems, 31, (TA)puy.a);
            if (own1) {
                LBM_ST(P, aout, aux_phiux(pp) * S + c1, P.aux_elems, 30, (TA)pux.b);
                LBM_ST(P, aout, aux_phiuy(N, pp) * S + c1, P.aux_elems, 31, (TA)puy.b);
            }
        }
    }

    // ---- stage F: enthalpy collision, Dirichlet ghosts; stage G --------------------------
    {
        f2 h[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) h[i] = ld_pop2<Pr, KIND_H>(P, pin, N + 1, i, c0, c1, true);
        const f2 Z = rho * cp * T, E = f2(C.E_ref) * T;
        const f2 kh = rfma(f2(-0.5f), oh, f2(1.0f)), oh1 = f2(1.0f) - oh;
        const f2 Zm = Z * mdot;
        const f2 c0_ = oh * rfma(f2(-1.5f) * Z, uu, E) + kh * Zm;
        const f2 ohZ = oh * Z;
        const f2 cxv = f2(3.0f) * ohZ * ux, cyv = f2(3.0f) * ohZ * uy;
        const f2 cxx = f2(4.5f) * ohZ * ux * ux, cyy = f2(4.5f) * ohZ * uy * uy, cxy = f2(9.0f) * ohZ * ux * uy;
        const f2 heq0 = (rhoH - E) + f2(wgt_r<float>(0)) * rfma(f2(-1.5f) * Z, uu, E);
        const f2 bx_ = c0_ + cxx, by_ = c0_ + cyy, bd = c0_ + cxx + cyy;
        f2 q[9];
        q[0] = rfma(oh, heq0, rfma(kh * f2(wgt_r<float>(0)), Zm, oh1 * h[0]));
        q[1] = rfma(f2(wgt_r<float>(1)), bx_ + cxv, oh1 * h[1]);
        q[3] = rfma(f2(wgt_r<float>(3)), bx_ - cxv, oh1 * h[3]);
        q[2] = rfma(f2(wgt_r<float>(2)), by_ + cyv, oh1 * h[2]);
        q[4] = rfma(f2(wgt_r<float>(4)), by_ - cyv, oh1 * h[4]);
        q[5] = rfma(f2(wgt_r<float>(5)), (bd + cxy) + (cxv + cyv), oh1 * h[5]);
        q[7] = rfma(f2(wgt_r<float>(7)), (bd + cxy) - (cxv + cyv), oh1 * h[7]);
        q[6] = rfma(f2(wgt_r<float>(6)), (bd - cxy) + (cyv - cxv), oh1 * h[6]);
        q[8] = rfma(f2(wgt_r<float>(8)), (bd - cxy) - (cyv - cxv), oh1 * h[8]);
        push2(KIND_H, N + 1, q);
        // Dirichlet wall rows (per cell, as the one-cell step)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int yy = y + k;
            if (k == 1 && !own1) break;
            const int dside = (yy == 0 && P.bc[2] == WALL && P.tbc[2] == DIRICHLET)        ? 2
                              : (yy == ny - 1 && P.bc[3] == WALL && P.tbc[3] == DIRICHLET) ? 3
                                                                                            : -1;
            if (dside < 0) continue;
            auto pick = [&](f2 v) { return k == 0 ? v.a : v.b; };
            const bool top = dside == 3;
            const R uyk = pick(uy), uxk = pick(ux), Zk = pick(Z), Ek = pick(E), uuk = pick(uu), oh1k = pick(oh1);
            const R vy = top ? -uyk : uyk;
            const R Eg = C.E_ref * (2.0f * C.Tw[dside] - pick(T));
            auto heq = [&](R w, R cu) { return w * fmaf(Zk, fmaf(4.5f * cu, cu, fmaf(3.0f, cu, -1.5f * uuk)), Ek); };
            const R wa = wgt_r<float>(2), wd = wgt_r<float>(5);
            push_row_at<KIND_H, Pr>(P, pout, N + 1, top ? 4 : 2, 0, x, yy,
                                    fmaf(oh1k, pick(top ? h[4] : h[2]) - heq(wa, vy), wa * Eg));
            push_row_at<KIND_H, Pr>(P, pout, N + 1, top ? 8 : 5, 1, x, yy,
                                    fmaf(oh1k, pick(top ? h[8] : h[5]) - heq(wd, uxk + vy), wd * Eg));
            push_row_at<KIND_H, Pr>(P, pout, N + 1, top ? 7 : 6, -1, x, yy,
                                    fmaf(oh1k, pick(top ? h[7] : h[6]) - heq(wd, vy - uxk), wd * Eg));
        }
        LBM_ST(P, aout, aux_mdot() * S + c0, P.aux_elems, 32, (TA)mdot.a);
        LBM_ST(P, aout, aux_Q() * S + c0, P.aux_elems, 33, (TA)Zm.a);
        LBM_ST(P, aout, aux_psi() * S + c0, P.aux_elems, 34, (TA)psi.a);
        if (own1) {
            LBM_ST(P, aout, aux_mdot() * S + c1, P.aux_elems, 32, (TA)mdot.b);
            LBM_ST(P, aout, aux_Q() * S + c1, P.aux_elems, 33, (TA)Zm.b);
            LBM_ST(P, aout, aux_psi() * S + c1, P.aux_elems, 34, (TA)psi.b);
        }
    }
}

// Resident threads per SM that the register allocation of the two-cells-per-thread step
// must allow (each thread carries two cells).
#ifndef LBM_PAIR_OCC
#define LBM_PAIR_OCC 512
#endif

// One launch = one time step of one lattice with two cells per thread.
template <int N, int TX, int TY, bool COLLIDE, class Pr>
__global__ void __launch_bounds__(TX * TY / 2, (LBM_PAIR_OCC + TX * TY / 2 - 1) / (TX * TY / 2))
fused_pair_kernel(const KParams P, const void* __restrict__ pin_base, void* __restrict__ pout_base,
                  const typename Pr::TA* __restrict__ ain, typename Pr::TA* __restrict__ aout, ExportPtrs ex)
{
    __shared__ float smem[(N + 2) * (TX + 2) * (TY + 2)];
    step_tile_pair<N, TX, TY, COLLIDE, Pr>(P, pin_base, pout_base, ain, aout, ex, blockIdx.x, blockIdx.y, smem);
}

}  // namespace lbm
