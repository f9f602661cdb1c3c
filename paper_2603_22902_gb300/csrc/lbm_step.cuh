// lbm_step.cuh -- the fused time step of the coupled LB scheme (arXiv 2603.22902,
// Section 3), one kernel launch per step, generic over the storage / arithmetic
// precision policy (lbm_prec.cuh).
//
// State between launches: pre-collision (post-streaming) populations f, g_p (p < N),
// h as structure-of-arrays planes (rest block + moving block), and the lagged planes
// mdot', Q' = rho c_p T mdot, psi', (phi_p u)'.  One launch reads set A and writes
// set B (ping-pong), so it is race-free across blocks.
//
// Per block (a TX x TY tile, one thread per cell):
//   1. the moments of every cell of the tile and of its 1-cell ring (phi_p = sum g /
//      (1 - mdot'/2), rho H = sum h + Q'/2), the mixture rule (eq. 2) and the enthalpy
//      map (eq. H): the ring cells recompute phi_p, rho, psi from their own populations
//      (no second kernel, no extra HBM field).  FP64 / FP32 / 16-bit policies evaluate the
//      own cell in registers and share the ring out; the compact (double-word) policy runs
//      one loop over all positions so that this code exists once.  f_l is always the FP64
//      map's; the FP32-arithmetic and double-word policies screen eq. H in FP32 first and
//      run the FP64 map only where the screen cannot decide f_l (map_cell);
//   2. ghost values beyond walls/outflows are filled (zero gradient; wetting for phi_p),
//      skipped by tiles that have none;
//   3. the isotropic 9-point gradients / Laplacians of phi_p, rho, psi come from
//      shared memory; then the pairwise normals n_pq, R_p, mu_p, F_s (Section 2),
//      u*, the penalty force, u, mdot, S, Lambda, p (Section 3), and the three BGK
//      collisions with their source terms;
//   4. post-collision populations are pushed to the neighbours' slots of set B with
//      the boundary rules (bounce-back, outflow copy, non-equilibrium extrapolation
//      of the Dirichlet temperature; rows that are neither the lattice's first nor its
//      last skip the checks, see push_species), and the lagged planes are written.
// No address outside the planes is ever formed, not even for a value that is then
// not used: the compiler may issue loads ahead of the branch that guards them.
#pragma once

#include "lbm_device.cuh"
#include "lbm_prec.cuh"

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

// Species kinds of the moving planes (their 16-bit encodings differ).
constexpr int KIND_F = 0, KIND_G = 1, KIND_H = 2;

// Views of one population set: rest block (N + 2 planes) and moving block (8 (N + 2)).
template <class Pr>
struct PopView {
    typename Pr::TR* rest;
    typename Pr::TM* move;
};
template <class Pr>
__device__ __forceinline__ PopView<Pr> pop_view(const KParams& P, const void* base)
{
    char* b = (char*)base;
    return PopView<Pr>{(typename Pr::TR*)b, (typename Pr::TM*)(b + P.rest_elems * (long long)sizeof(typename Pr::TR))};
}

// A stored moving population (direction i >= 1) as a value of the arithmetic type R.
template <class Pr, int KIND>
__device__ __forceinline__ typename Pr::R dequant(const KParams& P, typename Pr::TM q, int i)
{
    using R = typename Pr::R;
    if constexpr (!Pr::QUANT) {
        return (R)q;
    } else {
        const float w = (float)wgt(i);
        const float qf = to_f(q);
        if (KIND == KIND_F) return qf * (w * F_SCALE);
        if (KIND == KIND_G) return qf * w;
        return qf * (w * P.f.E_ref);
    }
}

// Load population i of species s at cell c (dequantised to R).
template <class Pr, int KIND>
__device__ __forceinline__ typename Pr::R ld_pop(const KParams& P, const PopView<Pr>& v, int s, int i, long long c, int site)
{
    using R = typename Pr::R;
    if (i == 0) return (R)LBM_LDX(Pr::COH, P, v.rest, (long long)s * P.S + c, P.rest_elems, site);
    const auto q = LBM_LDX(Pr::COH, P, v.move, (long long)(s * 8 + i - 1) * P.S + c, P.move_elems, site);
    return dequant<Pr, KIND>(P, q, i);
}

// The same load for a second read of a population in one step: through the cached
// (L1) path instead of the read-only one, so that the compiler does not merge it with
// the first read and keep the value in a register meanwhile.
template <class Pr, int KIND>
__device__ __forceinline__ typename Pr::R ld_pop_late(const KParams& P, const PopView<Pr>& v, int s, int i, long long c,
                                                      int site)
{
    using R = typename Pr::R;
    const long long idx = i == 0 ? (long long)s * P.S + c : (long long)(s * 8 + i - 1) * P.S + c;
#ifdef LBM_CHECK_BOUNDS
    if (!lbm_in_bounds(P.dbg, idx, i == 0 ? P.rest_elems : P.move_elems, site)) return R(0);
#else
    (void)site;
#endif
    if (i == 0) return (R)lbm_ld_l1<Pr::COH>(v.rest + idx);
    return dequant<Pr, KIND>(P, lbm_ld_l1<Pr::COH>(v.move + idx), i);
}

// Store population i of species s at cell c (quantised from R).
template <class Pr, int KIND>
__device__ __forceinline__ void st_pop(const KParams& P, const PopView<Pr>& v, int s, int i, long long c,
                                       typename Pr::R val, int site)
{
    using TM = typename Pr::TM;
    if (i == 0) {
        LBM_ST(P, v.rest, (long long)s * P.S + c, P.rest_elems, site, (typename Pr::TR)val);
        return;
    }
    const long long idx = (long long)(s * 8 + i - 1) * P.S + c;
    if constexpr (!Pr::QUANT) {
        LBM_ST(P, v.move, idx, P.move_elems, site, (TM)val);
    } else {
        const float w = (float)wgt(i);
        float q;
        if (KIND == KIND_F) q = (float)val * (1.0f / (w * F_SCALE));
        else if (KIND == KIND_G) q = (float)val * (1.0f / w);
        else q = (float)val * (1.0f / w) * P.f.inv_E_ref;
        LBM_ST(P, v.move, idx, P.move_elems, site, from_f<TM>(q));
    }
}

// Where a step reads its inputs.  A loader addresses a cell of the tile-with-ring by a
// Cell value and gives its populations (dequantised) and lagged values.
//   GlobalLoader: the population and lagged sets in global memory, cells by their index in
//     the lattice (step_tile_l maps a position of the tile-with-ring to it).
//   StagedLoader: the same inputs of one tile copied into shared memory by the
//     tensor-memory accelerator (lbm_staged.cuh); cells by their position in the tile.
template <class Pr>
struct GlobalLoader {
    using R = typename Pr::R;
    using Cell = long long;
    static constexpr bool GLOBAL = true;   // step_tile_l locates the cells itself
    const KParams& P;
    PopView<Pr> pin;
    const typename Pr::TA* __restrict__ ain;
    long long S;
    int nx;
    __device__ __forceinline__ Cell own(int x, int y, int, int) const { return (long long)y * nx + x; }
    template <int KIND>
    __device__ __forceinline__ R pop(int s, int i, Cell c, int site) const
    {
        return ld_pop<Pr, KIND>(P, pin, s, i, c, site);
    }
    template <int KIND>
    __device__ __forceinline__ R pop_late(int s, int i, Cell c, int site) const
    {
        return ld_pop_late<Pr, KIND>(P, pin, s, i, c, site);
    }
    __device__ __forceinline__ R aux(int a, Cell c, int site) const
    {
        return (R)LBM_LDX(Pr::COH, P, ain, a * S + c, P.aux_elems, site);
    }
};

// eq. H for one cell: f_l (and T when WANT_T) from rho H and phi_p, in FP64.  Policies
// that compute in FP32 screen the cell in FP32 first: where rho H lies above the
// liquidus value Al, or (with phase-changing material present) below the solidus value
// As, by more than 1e-5 of the magnitudes involved (25 times the FP32 rounding bound of
// As and Al), the FP64 map would return f_l = 1 or 0 as well, and T is then taken from
// the same branch formula in FP32.  Only the other cells (the mushy band, values near a
// threshold, phase-changing material below FP32 range) run the FP64 map, so f_l is the
// FP64 map's value in every cell.  The double-word policy screens its high words the same
// way and takes T of a decided cell in double-word arithmetic.
template <int N, class Pr, bool WANT_T>
__device__ __forceinline__ void map_cell(const KParams& P, const typename Pr::R (&phi)[N], typename Pr::R rhoH,
                                         typename Pr::R& fl, typename Pr::R& T)
{
    using R = typename Pr::R;
    if constexpr (std::is_same<R, float>::value) {
        const Coef<float>& C = P.f;
        float rs = 0.0f, rl = 0.0f, cs = 0.0f, cl = 0.0f, Lv = 0.0f;
#pragma unroll
        for (int p = 0; p < N; ++p) {
            rs = fmaf(phi[p], C.rho_s[p], rs);
            rl = fmaf(phi[p], C.rho_l[p], rl);
            cs = fmaf(phi[p], C.cp_s[p], cs);
            cl = fmaf(phi[p], C.cp_l[p], cl);
            Lv = fmaf(phi[p], C.rhoL[p], Lv);
        }
        const float rcs = rs * cs, rcl = rl * cl;
        const float As = rcs * C.T_sol, Al = fmaf(rcl, C.T_liq, Lv);
        const float tol = 1e-5f * (fabsf(As) + fabsf(rcl * C.T_liq) + fabsf(Lv) + fabsf(rhoH)) + 1e-30f;
        if (rhoH > Al + tol) {
            fl = 1.0f;
            if (WANT_T) T = C.T_liq + (rhoH - Al) / rcl;
            return;
        }
        if (Lv > 0.0f && rhoH < As - tol) {
            fl = 0.0f;
            if (WANT_T) T = rhoH / rcs;
            return;
        }
    } else if constexpr (std::is_same<R, df64>::value) {
        // the same screen on the high words (within 2^-24 of the double words); T of a
        // decided cell from the branch formula in double-word arithmetic
        const Coef<float>& Cf = P.f;
        float rs = 0.0f, rl = 0.0f, cs = 0.0f, cl = 0.0f, Lv = 0.0f;
#pragma unroll
        for (int p = 0; p < N; ++p) {
            rs = fmaf(phi[p].hi, Cf.rho_s[p], rs);
            rl = fmaf(phi[p].hi, Cf.rho_l[p], rl);
            cs = fmaf(phi[p].hi, Cf.cp_s[p], cs);
            cl = fmaf(phi[p].hi, Cf.cp_l[p], cl);
            Lv = fmaf(phi[p].hi, Cf.rhoL[p], Lv);
        }
        const float rcs = rs * cs, rcl = rl * cl, h = rhoH.hi;
        const float As = rcs * Cf.T_sol, Al = fmaf(rcl, Cf.T_liq, Lv);
        const float tol = 1e-5f * (fabsf(As) + fabsf(rcl * Cf.T_liq) + fabsf(Lv) + fabsf(h)) + 1e-30f;
        const Coef<df64>& C = P.x;
        if (h > Al + tol) {
            fl = R(1);
            if (WANT_T) {
                const R rcl_d = mix_sum<N, R>(phi, C.rho_l) * mix_sum<N, R>(phi, C.cp_l);
                const R Al_d = rfma(rcl_d, C.T_liq, mix_sum<N, R>(phi, C.rhoL));
                T = C.T_liq + (rhoH - Al_d) / rcl_d;
            }
            return;
        }
        if (Lv > 0.0f && h < As - tol) {
            fl = R(0);
            if (WANT_T) T = rhoH / (mix_sum<N, R>(phi, C.rho_s) * mix_sum<N, R>(phi, C.cp_s));
            return;
        }
    }
    double phd[N];
#pragma unroll
    for (int p = 0; p < N; ++p) phd[p] = (double)phi[p];
    const Mix<N> m = mixture_map<N>(P, phd);
    double fld, Td = 0.0;
    enthalpy_map<N, WANT_T>(P, m, (double)rhoH, fld, Td);
    fl = (R)fld;
    if (WANT_T) T = (R)Td;
}

// Stage A + B for a halo cell: phi_p, rho and psi only (the map in FP64).
template <int N, class Pr, class L>
__device__ __forceinline__ void halo_moments_l(const KParams& P, const L& ld, typename L::Cell c,
                                               typename Pr::R (&phi)[N], typename Pr::R& rho, typename Pr::R& psi)
{
    using R = typename Pr::R;
    const R mdm = ld.aux(aux_mdot(), c, 1);
    const R Qm = ld.aux(aux_Q(), c, 2);
    const R iden = R(1) / (R(1) - R(0.5) * mdm);
#pragma unroll
    for (int p = 0; p < N; ++p) {
        R s = R(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) s += ld.template pop<KIND_G>(1 + p, i, c, 3);
        phi[p] = s * iden;
    }
    R sh = R(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) sh += ld.template pop<KIND_H>(N + 1, i, c, 4);
    const R rhoH = rfma(R(0.5), Qm, sh);
    // eq. H (f_l as the FP64 map gives it); the rest of eq. 2 in R
    R fl, T;
    map_cell<N, Pr, false>(P, phi, rhoH, fl, T);
    const Coef<R>& C = coef<R>(P);
    const R fs = R(1) - fl;
    rho = rfma(fs, mix_sum<N, R>(phi, C.rho_s), fl * mix_sum<N, R>(phi, C.rho_l));
    psi = fs * mix_sum<N, R>(phi, C.drho);
}
template <int N, class Pr>
__device__ __forceinline__ void halo_moments(const KParams& P, const PopView<Pr>& pin,
                                             const typename Pr::TA* __restrict__ ain, long long c,
                                             typename Pr::R (&phi)[N], typename Pr::R& rho, typename Pr::R& psi)
{
    const GlobalLoader<Pr> ld{P, pin, ain, P.S, P.nx};
    halo_moments_l<N, Pr>(P, ld, c, phi, rho, psi);
}

// Stage A + B of one cell of the tile or its ring: phi_p, rho H, f_l, T, rho and psi.
// f_l is the FP64 map's (map_cell), the rest of eq. 2 runs in R.  T is needed only for the tile's own
// cells, but almost every warp holds both kinds, so it is computed for all (a branch on
// the kind would run both versions of the map).
template <int N, class Pr, class L>
__device__ __forceinline__ void cell_moments_l(const KParams& P, const L& ld, typename L::Cell c,
                                               typename Pr::R (&phi)[N], typename Pr::R& rhoH, typename Pr::R& fl,
                                               typename Pr::R& T, typename Pr::R& rho, typename Pr::R& psi)
{
    using R = typename Pr::R;
    using K = exact_t<R>;
    const R mdm = ld.aux(aux_mdot(), c, 1);
    const R Qm = ld.aux(aux_Q(), c, 2);
    const R iden = R(1) / (R(1) - K(0.5) * mdm);
#pragma unroll
    for (int p = 0; p < N; ++p) {
        R s = R(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) s += ld.template pop<KIND_G>(1 + p, i, c, 3);
        phi[p] = s * iden;
    }
    R sh = R(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) sh += ld.template pop<KIND_H>(N + 1, i, c, 4);
    rhoH = rfma(K(0.5), Qm, sh);
    map_cell<N, Pr, true>(P, phi, rhoH, fl, T);
    const Coef<R>& C = coef<R>(P);
    const R fs = R(1) - fl;
    rho = rfma(fs, mix_sum<N, R>(phi, C.rho_s), fl * mix_sum<N, R>(phi, C.rho_l));
    psi = fs * mix_sum<N, R>(phi, C.drho);
}

// Push one post-collision population q_j of species s at node (x, y) into set B.
// Periodic sides wrap; a population leaving through an x wall is reflected into the
// node's own opposite slot (half-way bounce-back); through a y wall likewise, except
// the enthalpy populations at a Dirichlet wall (their incoming slots are filled by the
// ghost rule); through an outflow side it is dropped.
template <int J, int KIND, class Pr>
__device__ __forceinline__ void push(const KParams& P, const PopView<Pr>& out, int s, int x, int y, typename Pr::R q)
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
        st_pop<Pr, KIND>(P, out, s, J, (long long)ty * P.nx + tx, q, 10);
    } else if (xo) {
        st_pop<Pr, KIND>(P, out, s, opp(J), own, q, 11);
    } else {
        const int side = ty < 0 ? 2 : 3;
        if (P.bc[side] == WALL && !(KIND == KIND_H && P.tbc[side] == DIRICHLET))
            st_pop<Pr, KIND>(P, out, s, opp(J), own, q, 12);
    }
}

// Extra write of a boundary-row rule: value v into slot J of node (x + c_J, y),
// same row; skipped when that node is beyond an x wall.
template <int J, int KIND, class Pr>
__device__ __forceinline__ void push_row(const KParams& P, const PopView<Pr>& out, int s, int x, int y,
                                         typename Pr::R v)
{
    int tx = x + cx(J);
    if (cx(J) != 0 && (unsigned)tx >= (unsigned)P.nx) {
        if (P.bc[0] != PERIODIC) return;
        tx = tx < 0 ? tx + P.nx : tx - P.nx;
    }
    st_pop<Pr, KIND>(P, out, s, J, (long long)y * P.nx + tx, v, 13);
}

// push_row for a direction j known at run time, whose x component is dx.
template <int KIND, class Pr>
__device__ __forceinline__ void push_row_at(const KParams& P, const PopView<Pr>& out, int s, int j, int dx, int x,
                                            int y, typename Pr::R v)
{
    int tx = x + dx;
    if (dx != 0 && (unsigned)tx >= (unsigned)P.nx) {
        if (P.bc[0] != PERIODIC) return;
        tx = tx < 0 ? tx + P.nx : tx - P.nx;
    }
    st_pop<Pr, KIND>(P, out, s, j, (long long)y * P.nx + tx, v, 13);
}

// All nine pushes of one species, plus the outflow copies of the boundary rows.  Three
// paths, chosen per cell by the caller:
//   PUSH_INTERIOR: the cell's row is neither the lattice's first nor its last, and its
//     tile's columns and their ring lie inside the lattice: every population lands in the
//     neighbour c + c_J, no wrap and no boundary rule;
//   PUSH_XWRAP: the cell's row is neither the first nor the last, and x is periodic: the
//     neighbour c + c_J with its x taken modulo nx, no boundary rule;
//   PUSH_GENERAL: the checks of push() for every population.
constexpr int PUSH_GENERAL = 0, PUSH_INTERIOR = 1, PUSH_XWRAP = 2;
template <int KIND, class Pr>
__device__ __forceinline__ void push_species(const KParams& P, const PopView<Pr>& out, int s, int x, int y,
                                             int path, const typename Pr::R (&q)[9])
{
    if (path == PUSH_INTERIOR) {
        const long long c = (long long)y * P.nx + x;
        st_pop<Pr, KIND>(P, out, s, 0, c, q[0], 10);
#pragma unroll
        for (int j = 1; j < 9; ++j) st_pop<Pr, KIND>(P, out, s, j, c + (cy(j) * P.nx + cx(j)), q[j], 10);
        return;
    }
    if (path == PUSH_XWRAP) {
        const long long row = (long long)y * P.nx;
        const int xm = x == 0 ? P.nx - 1 : x - 1, xp = x == P.nx - 1 ? 0 : x + 1;
        st_pop<Pr, KIND>(P, out, s, 0, row + x, q[0], 10);
#pragma unroll
        for (int j = 1; j < 9; ++j)
            st_pop<Pr, KIND>(P, out, s, j, row + cy(j) * P.nx + (cx(j) < 0 ? xm : (cx(j) > 0 ? xp : x)), q[j], 10);
        return;
    }
    push<0, KIND, Pr>(P, out, s, x, y, q[0]);
    push<1, KIND, Pr>(P, out, s, x, y, q[1]);
    push<2, KIND, Pr>(P, out, s, x, y, q[2]);
    push<3, KIND, Pr>(P, out, s, x, y, q[3]);
    push<4, KIND, Pr>(P, out, s, x, y, q[4]);
    push<5, KIND, Pr>(P, out, s, x, y, q[5]);
    push<6, KIND, Pr>(P, out, s, x, y, q[6]);
    push<7, KIND, Pr>(P, out, s, x, y, q[7]);
    push<8, KIND, Pr>(P, out, s, x, y, q[8]);
    if (y == 0 && P.bc[2] == OUTFLOW) {
        push_row<2, KIND, Pr>(P, out, s, x, y, q[2]);
        push_row<5, KIND, Pr>(P, out, s, x, y, q[5]);
        push_row<6, KIND, Pr>(P, out, s, x, y, q[6]);
    }
    if (y == P.ny - 1 && P.bc[3] == OUTFLOW) {
        push_row<4, KIND, Pr>(P, out, s, x, y, q[4]);
        push_row<7, KIND, Pr>(P, out, s, x, y, q[7]);
        push_row<8, KIND, Pr>(P, out, s, x, y, q[8]);
    }
}

// Resident threads per SM the register allocation must allow (launch bounds): the
// policy's choice, or LBM_OCC_THREADS when a build overrides it for tuning.
#ifdef LBM_OCC_THREADS
#define LBM_OCC(Pr) (LBM_OCC_THREADS)
#else
#define LBM_OCC(Pr) (Pr::OCC_THREADS)
#endif
// Shared-memory elements of type R that step_tile needs: phi_p, rho and psi on the
// tile and its one-cell ring, and (COMPACT policies) rho H, f_l, T of the tile's cells.
template <int N, int TX, int TY, class Pr>
__host__ __device__ constexpr int tile_smem_elems()
{
    return (N + 2) * (TX + 2) * (TY + 2) + (Pr::COMPACT ? 3 * TX * TY : 0);
}

// One TX x TY tile (tile column bx, row by) of one time step, run by a block of
// TX * TY threads; smem holds tile_smem_elems<N, TX, TY, Pr>() elements of shared memory.
// Every thread of the block must call it (it holds two block barriers); the caller
// places a block barrier before smem is used again.
template <int N, int TX, int TY, bool COLLIDE, class Pr, class L>
__device__ __forceinline__ void step_tile_l(const KParams& P, const L& ld, void* __restrict__ pout_base,
                                            typename Pr::TA* __restrict__ aout, const ExportPtrs& ex, int bx, int by,
                                            typename Pr::R* smem)
{
    using R = typename Pr::R;
    using K = exact_t<R>;
    using TA = typename Pr::TA;
    constexpr int W = TX + 2, H = TY + 2, NT = TX * TY;
    R (*s_phi)[H][W] = reinterpret_cast<R (*)[H][W]>(smem);          // [N][H][W]
    R (*s_rho)[W] = reinterpret_cast<R (*)[W]>(smem + N * H * W);    // [H][W]
    R (*s_psi)[W] = reinterpret_cast<R (*)[W]>(smem + (N + 1) * H * W);
    R (*s_own)[NT] = reinterpret_cast<R (*)[NT]>(smem + (N + 2) * H * W);  // COMPACT: rho H, f_l, T of own cells

    const int nx = P.nx, ny = P.ny;
    const long long S = P.S;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = bx * TX, y0 = by * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool owned = x < nx && y < ny;
    const bool xper = P.bc[0] == PERIODIC, yper = P.bc[2] == PERIODIC;
    const Coef<R>& C = coef<R>(P);
    using Cell = typename L::Cell;

    // Position (lx, ly) of the tile-with-ring as a cell of the loader.  In global memory the
    // coordinates are brought into range before anything else (periodic: full modulo, since
    // a tile may be wider / taller than the domain; otherwise clamped, and the position is
    // reported as beyond the domain, to be filled by the ghost rule), so no address outside
    // the planes is ever formed; a staged tile has its ring inside the lattice.
    auto locate = [&](int lx, int ly, Cell& cell) {
        if constexpr (L::GLOBAL) {
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
        } else {
            return ld.locate(lx, ly, cell);
        }
    };
    R phi[N], rhoH, fl, T, rho, psi, mu, lam, cp, chi;
    if constexpr (Pr::COMPACT) {
        // ---- stages A + B: one code path for all (TX + 2)(TY + 2) positions, so that
        // the moments are compiled once; the own cells' rho H, f_l, T go to shared memory
#pragma unroll 1
        for (int k = tid; k < W * H; k += NT) {
            const int lx = k % W, ly = k / W;
            Cell cell;
            if (!locate(lx, ly, cell)) continue;
            R ph[N], rH, flv, Tv, r, ps;
            cell_moments_l<N, Pr>(P, ld, cell, ph, rH, flv, Tv, r, ps);
#pragma unroll
            for (int p = 0; p < N; ++p) s_phi[p][ly][lx] = ph[p];
            s_rho[ly][lx] = r;
            s_psi[ly][lx] = ps;
            const int ox = lx - 1, oy = ly - 1;
            if ((unsigned)ox < (unsigned)TX && (unsigned)oy < (unsigned)TY) {
                const int o = oy * TX + ox;
                s_own[0][o] = rH;
                s_own[1][o] = flv;
                s_own[2][o] = Tv;
            }
        }
    } else {
        // ---- stages A + B: the own cell in registers (the rest of eq. 2 as well),
        // then the ring, phi_p, rho and psi only -----------------------------------
        auto halo_at = [&](int lx, int ly) {
            Cell cell;
            if (!locate(lx, ly, cell)) return;
            R ph[N], r, ps;
            halo_moments_l<N, Pr>(P, ld, cell, ph, r, ps);
#pragma unroll
            for (int p = 0; p < N; ++p) s_phi[p][ly][lx] = ph[p];
            s_rho[ly][lx] = r;
            s_psi[ly][lx] = ps;
        };
        if (owned) {
            cell_moments_l<N, Pr>(P, ld, ld.own(x, y, tx, ty), phi, rhoH, fl, T, rho, psi);
            const R fs = R(1) - fl;
            mu = rfma(fs, mix_sum<N, R>(phi, C.mu_s), fl * mix_sum<N, R>(phi, C.mu_l));
            lam = rfma(fs, mix_sum<N, R>(phi, C.lam_s), fl * mix_sum<N, R>(phi, C.lam_l));
            cp = rfma(fs, mix_sum<N, R>(phi, C.cp_s), fl * mix_sum<N, R>(phi, C.cp_l));
            chi = fs * mix_sum<N, R>(phi, C.pcm);
#pragma unroll
            for (int p = 0; p < N; ++p) s_phi[p][ty + 1][tx + 1] = phi[p];
            s_rho[ty + 1][tx + 1] = rho;
            s_psi[ty + 1][tx + 1] = psi;
        } else {
            halo_at(tx + 1, ty + 1);
        }
        constexpr int NRING = 2 * W + 2 * TY;
        for (int k = tid; k < NRING; k += NT) {
            int lx, ly;
            if (k < W) { lx = k; ly = 0; }
            else if (k < 2 * W) { lx = k - W; ly = H - 1; }
            else if (k < 2 * W + TY) { lx = 0; ly = k - 2 * W + 1; }
            else { lx = W - 1; ly = k - 2 * W - TY + 1; }
            halo_at(lx, ly);
        }
    }
    __syncthreads();
    // ---- ghosts beyond walls / outflows ------------------------------------
    // (none when the ring lies inside the lattice along every non-periodic axis: then
    // the pass and its barrier are skipped by the whole block)
    const bool ghosts = (!xper && (x0 < 1 || x0 + TX > nx - 1)) || (!yper && (y0 < 1 || y0 + TY > ny - 1));
    if (ghosts) {
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
            R ph[N];
    #pragma unroll
            for (int p = 0; p < N; ++p) ph[p] = s_phi[p][sy][sx];
    #pragma unroll
            for (int p = 0; p < N; ++p) {
                R corr = R(0);
    #pragma unroll
                for (int q = 0; q < N; ++q) {
                    if (q == p) continue;
                    R cw = R(0);
                    if (wx >= 0) cw += C.wet[wx][p][q];
                    if (wy >= 0) cw += C.wet[wy][p][q];
                    corr = rfma(cw * ph[p], ph[q], corr);
                }
                s_phi[p][ly][lx] = ph[p] + corr;
            }
            s_rho[ly][lx] = s_rho[sy][sx];
            s_psi[ly][lx] = s_psi[sy][sx];
        }
        __syncthreads();
    }
    if (!owned) return;

    const int lx = tx + 1, ly = ty + 1;
    const long long c = (long long)y * nx + x;   // stores: lattice index
    const Cell oc = ld.own(x, y, tx, ty);        // loads of the own cell
    if constexpr (Pr::COMPACT) {
        // ---- own cell: the rest of eq. 2 ---------------------------------------
#pragma unroll
        for (int p = 0; p < N; ++p) phi[p] = s_phi[p][ly][lx];
        rhoH = s_own[0][tid];
        fl = s_own[1][tid];
        T = s_own[2][tid];
        rho = s_rho[ly][lx];
        psi = s_psi[ly][lx];
        const R fs = R(1) - fl;
        mu = rfma(fs, mix_sum<N, R>(phi, C.mu_s), fl * mix_sum<N, R>(phi, C.mu_l));
        lam = rfma(fs, mix_sum<N, R>(phi, C.lam_s), fl * mix_sum<N, R>(phi, C.lam_l));
        cp = rfma(fs, mix_sum<N, R>(phi, C.cp_s), fl * mix_sum<N, R>(phi, C.cp_l));
        chi = fs * mix_sum<N, R>(phi, C.pcm);
    }

    // ---- stage C: isotropic stencils ---------------------------------------
    // gradients of phi_p (fields 0..N-1), rho (N) and psi (N+1), Laplacians of phi_p; the
    // fields are consecutive planes of shared memory (one rolled loop in COMPACT builds)
    R gpx[N + 2], gpy[N + 2], lap[N];
#pragma unroll(Pr::COMPACT ? 1 : N + 2)
    for (int fi = 0; fi < N + 2; ++fi) {
        R (*a)[W] = reinterpret_cast<R (*)[W]>(smem + fi * H * W);
        const R e = a[ly][lx + 1], w = a[ly][lx - 1], n = a[ly + 1][lx], s = a[ly - 1][lx];
        const R ne = a[ly + 1][lx + 1], nw = a[ly + 1][lx - 1], se = a[ly - 1][lx + 1], sw = a[ly - 1][lx - 1];
        gpx[fi] = (e - w) * R(1.0 / 3.0) + ((ne - nw) + (se - sw)) * R(1.0 / 12.0);
        gpy[fi] = (n - s) * R(1.0 / 3.0) + ((ne - se) + (nw - sw)) * R(1.0 / 12.0);
        if (fi < N) {
            const R v0 = a[ly][lx];
            const R ax = (e + w) + (n + s);
            const R dg = (ne + nw) + (se + sw);
            lap[fi] = ax * R(2.0 / 3.0) + dg * R(1.0 / 6.0) - v0 * R(10.0 / 3.0);
        }
    }
    const R grx = gpx[N], gry = gpy[N], gsx = gpx[N + 1], gsy = gpy[N + 1];

    // ---- stage D: pairwise normals, R_p, chemical potentials, F_s -----------
    R Rx[N], Ry[N], mup[N], gpv[N];
#pragma unroll
    for (int p = 0; p < N; ++p) {
        Rx[p] = R(0);
        Ry[p] = R(0);
        mup[p] = R(0);
        gpv[p] = K(2) * phi[p] * (R(1) - phi[p]) * (R(1) - K(2) * phi[p]);  // g'(phi), g = phi^2 (1 - phi)^2
    }
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
        for (int q = p + 1; q < N; ++q) {
            const R s = phi[p] + phi[q];
            R nxv = R(0), nyv = R(0);
            if (s > R(1e-12)) {
                // n_pq = grad(phi_p / s) / |grad(phi_p / s)|, s = phi_p + phi_q; the quotient
                // rule gives grad(phi_p / s) = G / s^2 with G below, so n_pq = G / |G| and the
                // guard |grad(phi_p / s)| > threshold reads |G|^2 > threshold^2 s^4
                const R Gx = phi[q] * gpx[p] - phi[p] * gpx[q];
                const R Gy = phi[q] * gpy[p] - phi[p] * gpy[q];
                const R G2 = Gx * Gx + Gy * Gy;
                const R s2 = s * s;
                bool ok = G2 > R(Pr::NABS2) * (s2 * s2);
                if constexpr (Pr::NGUARD > 0.0f) {
                    const R ref = phi[q] * phi[q] * (gpx[p] * gpx[p] + gpy[p] * gpy[p]) +
                                  phi[p] * phi[p] * (gpx[q] * gpx[q] + gpy[q] * gpy[q]);
                    ok = ok && G2 > R(Pr::NGUARD * Pr::NGUARD) * ref;
                }
                if (ok) {
                    const R r = rrsqrt(G2);
                    nxv = Gx * r;
                    nyv = Gy * r;
                }
            }
            const R a = C.four_eps * phi[p] * phi[q];
            Rx[p] = rfma(a, nxv, Rx[p]);
            Ry[p] = rfma(a, nyv, Ry[p]);
            Rx[q] = rfma(-a, nxv, Rx[q]);
            Ry[q] = rfma(-a, nyv, Ry[q]);
            const R gs = K(2) * s * (R(1) - s) * (R(1) - K(2) * s);
            mup[p] += rfma(C.b2[p][q], gpv[p] - gs, C.kk[p][q] * lap[q]);
            mup[q] += rfma(C.b2[q][p], gpv[q] - gs, C.kk[q][p] * lap[p]);
        }
    R Fx = rho * C.accel[0], Fy = rho * C.accel[1];
#pragma unroll
    for (int p = 0; p < N; ++p) {
        Fx = rfma(mup[p], gpx[p], Fx);
        Fy = rfma(mup[p], gpy[p], Fy);
    }

    // ---- stage E: flow macroscopics ----------------------------------------
    R f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = ld.template pop_late<KIND_F>(0, i, oc, 5);
    const R jx = ((f[1] - f[3]) + (f[5] - f[7])) + (f[8] - f[6]);
    const R jy = ((f[2] - f[4]) + (f[5] - f[7])) + (f[6] - f[8]);
    const R sum_f = ((f[1] + f[2]) + (f[3] + f[4])) + ((f[5] + f[6]) + (f[7] + f[8]));
    // 1 / rho, omega_f = 1 / tau_f = rho / A and omega_h = 1 / tau_h = 1 / B from one
    // division: tau_f = A / rho, A = 3 mu + rho / 2 (tau_f = mu / (rho c_s^2) + 1/2) and
    // tau_h = B = lambda / (rho_ref c_p,ref c_s^2) + 1/2
    const R Af = rfma(K(3), mu, K(0.5) * rho);
    const R Bh = rfma(lam, C.tau_h_scale, K(0.5));
    const R rAB = R(1) / (rho * Af * Bh);
    const R irho = (Af * Bh) * rAB;
    const R om = (rho * rho) * (Bh * rAB);
    const R oh = (rho * Af) * rAB;
    const R usx = rfma(K(0.5), Fx, jx) * irho, usy = rfma(K(0.5), Fy, jy) * irho;
    const R fpx = chi * (C.us[0] - usx), fpy = chi * (C.us[1] - usy);
    const R ux = rfma(K(0.5), fpx, usx), uy = rfma(K(0.5), fpy, usy);
    const R psim = ld.aux(aux_psi(), oc, 14);
    const R mdot = -((psi - psim) + (ux * gsx + uy * gsy)) * irho;
    const R Ssrc = rfma(rho, mdot, ux * grx + uy * gry);
    const R Lxx = rfma(K(2) * ux, Fx, Ssrc * R(1.0 / 3.0));
    const R Lyy = rfma(K(2) * uy, Fy, Ssrc * R(1.0 / 3.0));
    const R Lxy = rfma(ux, Fy, uy * Fx);
    const R tmh = K(3) * mu * irho;  // tau_f - 1/2
    const R F0 = wgt_r<R>(0) * rfma(K(-1.5), Lxx + Lyy, Ssrc);
    const R uu = rfma(ux, ux, uy * uy);
    const R p = R(0.6) * (((sum_f + K(0.5) * Ssrc) + tmh * F0) - rho * wgt_r<R>(0) * K(1.5) * uu);

    if (!COLLIDE) {
#pragma unroll
        for (int q = 0; q < N; ++q)
            if (ex.phi) LBM_ST(P, ex.phi, q * S + c, N * S, 20, (double)phi[q]);
        if (ex.T) LBM_ST(P, ex.T, c, S, 21, (double)T);
        if (ex.H) LBM_ST(P, ex.H, c, S, 22, (double)(rhoH * irho));
        if (ex.fl) LBM_ST(P, ex.fl, c, S, 23, (double)fl);
        if (ex.ux) LBM_ST(P, ex.ux, c, S, 24, (double)ux);
        if (ex.uy) LBM_ST(P, ex.uy, c, S, 25, (double)uy);
        if (ex.p) LBM_ST(P, ex.p, c, S, 26, (double)p);
        return;
    }
    const PopView<Pr> pout = pop_view<Pr>(P, pout_base);
    // the push path of this cell (push_species): the same for a row of the tile, so for a
    // warp of a 32-wide tile; only the lattice's first and last rows, and columns at a
    // side that is not periodic, take the general path
    const bool row_inside = y >= 1 && y <= ny - 2;
    const int path = row_inside && x0 >= 1 && x0 + TX <= nx - 1 ? PUSH_INTERIOR
                     : row_inside && xper                         ? PUSH_XWRAP
                                                                  : PUSH_GENERAL;

    // ---- stage F: flow collision -------------------------------------------
    {
        const R k = rfma(K(-0.5), om, R(1)), om1 = R(1) - om;
        const R Fex = rfma(rho, fpx, Fx), Fey = rfma(rho, fpy, Fy);
        const R rom = om * rho;
        const R a0 = om * rfma(K(-1.5) * rho, uu, K(3) * p) + k * rfma(K(-1.5), Lxx + Lyy, Ssrc);
        const R ax = K(3) * rfma(rom, ux, k * Fex);
        const R ay = K(3) * rfma(rom, uy, k * Fey);
        const R axx = K(4.5) * rfma(rom * ux, ux, k * Lxx);
        const R ayy = K(4.5) * rfma(rom * uy, uy, k * Lyy);
        const R axy = K(9) * rfma(rom * ux, uy, k * Lxy);
        const R bx = a0 + axx, by = a0 + ayy, bd = a0 + axx + ayy;
        R X[9];
        X[0] = rfma(K(-6.75) * om, p, a0);
        X[1] = bx + ax;
        X[3] = bx - ax;
        X[2] = by + ay;
        X[4] = by - ay;
        X[5] = (bd + axy) + (ax + ay);
        X[7] = (bd + axy) - (ax + ay);
        X[6] = (bd - axy) + (ay - ax);
        X[8] = (bd - axy) - (ay - ax);
        R q[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) q[i] = rfma(wgt_r<R>(i), X[i], om1 * f[i]);
        push_species<KIND_F, Pr>(P, pout, 0, x, y, path, q);
    }

    // ---- stage F: phase-field collisions -------------------------------------
    {
        const R og = C.omega_g, kg = C.kg, og1 = R(1) - og;
#pragma unroll(Pr::COMPACT ? 1 : N)
        for (int pp = 0; pp < N; ++pp) {
            R gq[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) gq[i] = ld.template pop_late<KIND_G>(1 + pp, i, oc, 6);
            const R Dx = phi[pp] * ux - ld.aux(aux_phiux(pp), oc, 15);
            const R Dy = phi[pp] * uy - ld.aux(aux_phiuy(N, pp), oc, 16);
            const R b0 = og * phi[pp] + kg * phi[pp] * mdot;
            const R bxv = K(3) * og * phi[pp] * ux + kg * rfma(K(3), Dx, Rx[pp]);
            const R byv = K(3) * og * phi[pp] * uy + kg * rfma(K(3), Dy, Ry[pp]);
            R q[9];
            q[0] = rfma(wgt_r<R>(0), b0, og1 * gq[0]);
            q[1] = rfma(wgt_r<R>(1), b0 + bxv, og1 * gq[1]);
            q[3] = rfma(wgt_r<R>(3), b0 - bxv, og1 * gq[3]);
            q[2] = rfma(wgt_r<R>(2), b0 + byv, og1 * gq[2]);
            q[4] = rfma(wgt_r<R>(4), b0 - byv, og1 * gq[4]);
            q[5] = rfma(wgt_r<R>(5), b0 + (bxv + byv), og1 * gq[5]);
            q[7] = rfma(wgt_r<R>(7), b0 - (bxv + byv), og1 * gq[7]);
            q[6] = rfma(wgt_r<R>(6), b0 + (byv - bxv), og1 * gq[6]);
            q[8] = rfma(wgt_r<R>(8), b0 - (byv - bxv), og1 * gq[8]);
            push_species<KIND_G, Pr>(P, pout, 1 + pp, x, y, path, q);
            LBM_ST(P, aout, aux_phiux(pp) * S + c, P.aux_elems, 30, (TA)(phi[pp] * ux));
            LBM_ST(P, aout, aux_phiuy(N, pp) * S + c, P.aux_elems, 31, (TA)(phi[pp] * uy));
        }
    }

    // ---- stage F: enthalpy collision + Dirichlet ghosts ---------------------
    {
        R h[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) h[i] = ld.template pop_late<KIND_H>(N + 1, i, oc, 7);
        const R Z = rho * cp * T, E = C.E_ref * T;
        const R kh = rfma(K(-0.5), oh, R(1)), oh1 = R(1) - oh;
        const R Zm = Z * mdot;
        const R c0 = oh * rfma(K(-1.5) * Z, uu, E) + kh * Zm;
        const R ohZ = oh * Z;
        const R cxv = K(3) * ohZ * ux, cyv = K(3) * ohZ * uy;
        const R cxx = K(4.5) * ohZ * ux * ux, cyy = K(4.5) * ohZ * uy * uy, cxy = K(9) * ohZ * ux * uy;
        const R heq0 = (rhoH - E) + wgt_r<R>(0) * rfma(K(-1.5) * Z, uu, E);
        const R bx = c0 + cxx, by = c0 + cyy, bd = c0 + cxx + cyy;
        R q[9];
        q[0] = rfma(oh, heq0, rfma(kh * wgt_r<R>(0), Zm, oh1 * h[0]));
        q[1] = rfma(wgt_r<R>(1), bx + cxv, oh1 * h[1]);
        q[3] = rfma(wgt_r<R>(3), bx - cxv, oh1 * h[3]);
        q[2] = rfma(wgt_r<R>(2), by + cyv, oh1 * h[2]);
        q[4] = rfma(wgt_r<R>(4), by - cyv, oh1 * h[4]);
        q[5] = rfma(wgt_r<R>(5), (bd + cxy) + (cxv + cyv), oh1 * h[5]);
        q[7] = rfma(wgt_r<R>(7), (bd + cxy) - (cxv + cyv), oh1 * h[7]);
        q[6] = rfma(wgt_r<R>(6), (bd - cxy) + (cyv - cxv), oh1 * h[6]);
        q[8] = rfma(wgt_r<R>(8), (bd - cxy) - (cyv - cxv), oh1 * h[8]);
        // outflow rows are copied inside push_species; Dirichlet rows get their
        // incoming populations from the ghost rule below
        push_species<KIND_H, Pr>(P, pout, N + 1, x, y, path, q);
        // Dirichlet wall: ghost behind the half-way wall with T_g = 2 T_w - T, u = 0; its
        // post-collision population is h_eq(ghost) + (1 - 1/tau_h)(h_j - h_eq_j) for the
        // three directions j that enter the boundary row (one code path for both walls:
        // directions (0, sy), (1, sy), (-1, sy), sy = +1 at the bottom, -1 at the top).
        const int dside = (y == 0 && P.bc[2] == WALL && P.tbc[2] == DIRICHLET)        ? 2
                          : (y == ny - 1 && P.bc[3] == WALL && P.tbc[3] == DIRICHLET) ? 3
                                                                                       : -1;
        if (dside >= 0) {
            const bool top = dside == 3;
            const R vy = top ? -uy : uy;
            const R Eg = C.E_ref * (K(2) * C.Tw[dside] - T);
            // equilibrium of a moving direction with weight w and c_j . u = cu
            auto heq = [&](R w, R cu) { return w * rfma(Z, rfma(K(4.5) * cu, cu, rfma(K(3), cu, K(-1.5) * uu)), E); };
            const R wa = wgt_r<R>(2), wd = wgt_r<R>(5);
            push_row_at<KIND_H, Pr>(P, pout, N + 1, top ? 4 : 2, 0, x, y,
                                    rfma(oh1, (top ? h[4] : h[2]) - heq(wa, vy), wa * Eg));
            push_row_at<KIND_H, Pr>(P, pout, N + 1, top ? 8 : 5, 1, x, y,
                                    rfma(oh1, (top ? h[8] : h[5]) - heq(wd, ux + vy), wd * Eg));
            push_row_at<KIND_H, Pr>(P, pout, N + 1, top ? 7 : 6, -1, x, y,
                                    rfma(oh1, (top ? h[7] : h[6]) - heq(wd, vy - ux), wd * Eg));
        }

        // ---- stage G: lagged planes ------------------------------------------
        LBM_ST(P, aout, aux_mdot() * S + c, P.aux_elems, 32, (TA)mdot);
        LBM_ST(P, aout, aux_Q() * S + c, P.aux_elems, 33, (TA)Zm);
        LBM_ST(P, aout, aux_psi() * S + c, P.aux_elems, 34, (TA)psi);
    }
}

// One TX x TY tile read from global memory (the loader of the one-cell step).
template <int N, int TX, int TY, bool COLLIDE, class Pr>
__device__ __forceinline__ void step_tile(const KParams& P, const void* __restrict__ pin_base,
                                          void* __restrict__ pout_base, const typename Pr::TA* __restrict__ ain,
                                          typename Pr::TA* __restrict__ aout, const ExportPtrs& ex, int bx, int by,
                                          typename Pr::R* smem)
{
    const GlobalLoader<Pr> ld{P, pop_view<Pr>(P, pin_base), ain, P.S, P.nx};
    step_tile_l<N, TX, TY, COLLIDE, Pr>(P, ld, pout_base, aout, ex, bx, by, smem);
}

// Tile (bx, by) of block b of a one-dimensional grid of tx * ty tiles.  The tiles on the
// outer ring of the tile grid (those at a side of the lattice: ghost pass, pushes with
// the boundary rules, wrapped reads; about twice the time of an interior tile) take the
// lowest block indices, so that they start in the first wave and overlap the interior
// tiles of later waves instead of finishing last.  Grids of fewer than three tiles along
// an axis are taken in order.
__device__ __forceinline__ void ring_first_tile(int b, int tx, int ty, int& bx, int& by)
{
    if (tx < 3 || ty < 3) {
        bx = b % tx;
        by = b / tx;
        return;
    }
    if (b < 2 * tx) {                       // bottom row, then top row
        bx = b % tx;
        by = b < tx ? 0 : ty - 1;
        return;
    }
    const int k = b - 2 * tx;
    if (k < 2 * (ty - 2)) {                 // left and right columns
        bx = (k & 1) ? tx - 1 : 0;
        by = 1 + (k >> 1);
        return;
    }
    const int m = k - 2 * (ty - 2);         // interior tiles, row by row
    bx = 1 + m % (tx - 2);
    by = 1 + m / (tx - 2);
}

// Tile (bx, by) of block b of a launch over the tile rows `rows` of a tx x ty tile grid:
// all rows in the order of ring_first_tile, or the inner / edge rows in row order.
__device__ __forceinline__ void tile_of_block(int b, int tx, int ty, const TileRows& rows, int& bx, int& by)
{
    if (rows.part == ROWS_ALL) {
        ring_first_tile(b, tx, ty, bx, by);
        return;
    }
    bx = b % tx;
    const int k = b / tx;
    by = rows.part == ROWS_INNER ? rows.lo + k : (k < rows.lo ? k : rows.hi + (k - rows.lo));
}

// One launch = one time step of one lattice (or of some of its tile rows, `rows`), one
// block per tile (a one-dimensional grid, the tiles at the sides first).
template <int N, int TX, int TY, bool COLLIDE, class Pr>
__global__ void __launch_bounds__(TX * TY, (LBM_OCC(Pr) + TX * TY - 1) / (TX * TY))
fused_step_kernel(const KParams P, const void* __restrict__ pin_base, void* __restrict__ pout_base,
                  const typename Pr::TA* __restrict__ ain, typename Pr::TA* __restrict__ aout, ExportPtrs ex,
                  TileRows rows)
{
    __shared__ typename Pr::R smem[tile_smem_elems<N, TX, TY, Pr>()];
    int bx, by;
    tile_of_block(blockIdx.x, (P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY, rows, bx, by);
    step_tile<N, TX, TY, COLLIDE, Pr>(P, pin_base, pout_base, ain, aout, ex, bx, by, smem);
}

}  // namespace lbm
