// lbm_device.cuh -- device-side constants, parameter block and cell-local
// physics of the coupled LB step (arXiv 2603.22902, Sections 2-3).
#pragma once

#include <cstdint>
#include <type_traits>

#include "lbm_df64.cuh"
#include "lbm_lattice.cuh"

namespace lbm {

constexpr int MAXN = 4;
constexpr int PERIODIC = 0, WALL = 1, OUTFLOW = 2;
constexpr int ADIABATIC = 0, DIRICHLET = 1;

// Which tile rows of the lattice a step launch covers: all of them (ROWS_ALL), the rows
// [lo, hi) (ROWS_INNER), or the others (ROWS_EDGE).  A slab handle steps its inner tile
// rows, whose cells and one-cell ring stay clear of the rows its halo exchange writes,
// while the exchange of the previous step is in flight, and the edge rows after it.
constexpr int ROWS_ALL = 0, ROWS_INNER = 1, ROWS_EDGE = 2;
struct TileRows {
    int part, lo, hi;
};
// Tile rows a launch covers, of ty in the lattice.
__host__ __device__ inline int tile_rows_count(int ty, const TileRows& r)
{
    return r.part == ROWS_INNER ? r.hi - r.lo : r.part == ROWS_EDGE ? ty - (r.hi - r.lo) : ty;
}

// Arithmetic helpers for the compute type R of a precision policy.
__device__ __forceinline__ double rfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double rrsqrt(double a) { return rsqrt(a); }
__device__ __forceinline__ float rrsqrt(float a) { return rsqrtf(a); }
// Type of a constant that FP32 holds exactly (2, 3, 0.5, 4.5, ...) in arithmetic of
// type R: R itself, except float for double words (a product with a float costs 5 FP32
// instructions instead of 8).  FP64 arithmetic is unchanged by it.
template <class R>
using exact_t = typename std::conditional<std::is_same<R, df64>::value, float, R>::type;

// Per-run coefficients used by the arithmetic of the step, in type T.  The host fills
// a double, a float and a double-word copy, so a policy computing in FP32 or in
// double-word arithmetic reads its own constants and converts nothing per cell
// (FP64 <-> FP32 conversions share the FP64 unit).
template <class T>
struct Coef {
    // eq. 2 mixture coefficients per phase
    T rho_l[MAXN], rho_s[MAXN], mu_l[MAXN], mu_s[MAXN];
    T lam_l[MAXN], lam_s[MAXN], cp_l[MAXN], cp_s[MAXN];
    T drho[MAXN];                 // rho_s^p - rho_l^p
    T pcm[MAXN];                  // 1 where L_p > 0 (the phase changes phase), else 0
    // Section 2 free energy: 2 beta_pq = 6 sigma_pq / eps and -k_pq = 3 eps sigma_pq / 4
    T b2[MAXN][MAXN], kk[MAXN][MAXN];
    T four_eps;                   // 4 / eps
    T wet[4][MAXN][MAXN];         // (4 / eps) cos(theta_pq) per wall side (0 elsewhere)
    T E_ref;                      // rho_ref c_p,ref
    T inv_E_ref;                  // 1 / (rho_ref c_p,ref)
    T tau_h_scale;                // 1 / (rho_ref c_p,ref c_s^2)
    T us[2], accel[2];
    T omega_g, kg;                // 1 / tau_g and 1 - 1/(2 tau_g), tau_g = M / c_s^2 + 1/2
    T Tw[4];                      // Dirichlet wall temperature
    T rhoL[MAXN];                 // rho_l^p L_p (the FP64 map reads KParams::rhoL)
    T T_sol, T_liq;               // (the FP64 map reads KParams::T_sol, T_liq)
};

// Parameter block passed by value to every kernel (lives in the constant bank).
// Everything derivable once per run is derived on the host.
struct KParams {
    int nx, ny, N;
    long long S;                  // plane stride in elements (nx * ny)
    int bc[4], tbc[4];            // side kinds, sides 0 x-min, 1 x-max, 2 y-min, 3 y-max
    Coef<double> d;               // coefficients, FP64
    Coef<float> f;                // the same, rounded to FP32
    Coef<df64> x;                 // the same, as double words (hi + lo)
    double rhoL[MAXN];            // rho_l^p L_p: latent heat per volume of pure phase p
    double T_sol, T_liq;
    long long rest_elems, move_elems; // elements of the rest / moving block of one population set
    long long aux_elems;          // elements of one lagged set
    unsigned long long* dbg;      // LBM_CHECK_BOUNDS builds: {violations, first site, first index}
};

template <class R>
__device__ __forceinline__ const Coef<R>& coef(const KParams& P)
{
    if constexpr (std::is_same<R, double>::value) return P.d;
    else if constexpr (std::is_same<R, df64>::value) return P.x;
    else return P.f;
}

// Global loads.  Data that the same launch never writes goes through the read-only
// (non-coherent) path; a persistent launch that runs several steps reads what other
// blocks wrote in its previous step, so its loads bypass L1 (cache-global).
template <bool COH, class T>
__device__ __forceinline__ T lbm_ld(const T* p)
{
    if constexpr (std::is_same<T, df64>::value) {
        const float2 v = COH ? __ldcg(reinterpret_cast<const float2*>(p)) : __ldg(reinterpret_cast<const float2*>(p));
        return df64(v.x, v.y);
    } else if constexpr (COH) {
        return __ldcg(p);
    } else {
        return __ldg(p);
    }
}
// The same through L1 (ld.ca) where the launch never writes the data, else
// cache-global: a second read of a value in one step that the compiler must not merge
// with the first read.
template <bool COH, class T>
__device__ __forceinline__ T lbm_ld_l1(const T* p)
{
    if constexpr (std::is_same<T, df64>::value) {
        const float2 v = COH ? __ldcg(reinterpret_cast<const float2*>(p)) : __ldca(reinterpret_cast<const float2*>(p));
        return df64(v.x, v.y);
    } else if constexpr (COH) {
        return __ldcg(p);
    } else {
        return __ldca(p);
    }
}

// Global-memory access with an optional bounds check.  In LBM_CHECK_BOUNDS builds an
// out-of-range index is recorded in P.dbg (count, site code, index) and the access is
// skipped (a load returns 0); nothing traps.  Normal builds compile to the plain access.
#ifdef LBM_CHECK_BOUNDS
__device__ __forceinline__ bool lbm_in_bounds(unsigned long long* dbg, long long idx, long long lim, int site)
{
    if (idx >= 0 && idx < lim) return true;
    if (dbg && atomicAdd(dbg, 1ull) == 0ull) {
        dbg[1] = (unsigned long long)site;
        dbg[2] = (unsigned long long)idx;
    }
    return false;
}
template <class T>
__device__ __forceinline__ T lbm_zero_like(const T*)
{
    return static_cast<T>(0.0f);
}
#define LBM_LDX(COH, P_, ptr, idx, lim, site) \
    (lbm_in_bounds((P_).dbg, (idx), (lim), (site)) ? lbm_ld<COH>((ptr) + (idx)) : lbm_zero_like(ptr))
#define LBM_ST(P_, ptr, idx, lim, site, val)                                  \
    do {                                                                      \
        if (lbm_in_bounds((P_).dbg, (idx), (lim), (site))) (ptr)[idx] = (val); \
    } while (0)
#else
#define LBM_LDX(COH, P_, ptr, idx, lim, site) lbm_ld<COH>((ptr) + (idx))
#define LBM_ST(P_, ptr, idx, lim, site, val) ((ptr)[idx] = (val))
#endif
#define LBM_LD(P_, ptr, idx, lim, site) LBM_LDX(false, P_, ptr, idx, lim, site)

// Plane layout of one population set: f[0..8], g_0[0..8] .. g_{N-1}[0..8], h[0..8].
__host__ __device__ constexpr int plane_f(int i) { return i; }
__host__ __device__ constexpr int plane_g(int p, int i) { return 9 + 9 * p + i; }
__host__ __device__ constexpr int plane_h(int N, int i) { return 9 + 9 * N + i; }
__host__ __device__ constexpr int npop_planes(int N) { return 9 * (N + 2); }
// Lagged planes: mdot', Q', psi', (phi_p u)' x N, (phi_p u)' y N.
__host__ __device__ constexpr int aux_mdot() { return 0; }
__host__ __device__ constexpr int aux_Q() { return 1; }
__host__ __device__ constexpr int aux_psi() { return 2; }
__host__ __device__ constexpr int aux_phiux(int p) { return 3 + p; }
__host__ __device__ constexpr int aux_phiuy(int N, int p) { return 3 + N + p; }
__host__ __device__ constexpr int naux_planes(int N) { return 3 + 2 * N; }

// Mixture (eq. 2) sums over the phases, FP64 (initial state and the map).
template <int N>
struct Mix {
    double rs, rl, cs, cl, Lv, dr, pcm;
};

template <int N>
__device__ __forceinline__ Mix<N> mixture_core(const KParams& P, const double (&phi)[N])
{
    Mix<N> m{0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int p = 0; p < N; ++p) {
        m.rs = fma(phi[p], P.d.rho_s[p], m.rs);
        m.rl = fma(phi[p], P.d.rho_l[p], m.rl);
        m.cs = fma(phi[p], P.d.cp_s[p], m.cs);
        m.cl = fma(phi[p], P.d.cp_l[p], m.cl);
        m.Lv = fma(phi[p], P.rhoL[p], m.Lv);
        m.dr = fma(phi[p], P.d.drho[p], m.dr);
        m.pcm = fma(phi[p], P.d.pcm[p], m.pcm);
    }
    return m;
}

// The part of the mixture that eq. H needs (FP64 in every precision): rs, rl, cs, cl, Lv.
template <int N>
__device__ __forceinline__ Mix<N> mixture_map(const KParams& P, const double (&phi)[N])
{
    Mix<N> m{0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int p = 0; p < N; ++p) {
        m.rs = fma(phi[p], P.d.rho_s[p], m.rs);
        m.rl = fma(phi[p], P.d.rho_l[p], m.rl);
        m.cs = fma(phi[p], P.d.cp_s[p], m.cs);
        m.cl = fma(phi[p], P.d.cp_l[p], m.cl);
        m.Lv = fma(phi[p], P.rhoL[p], m.Lv);
    }
    return m;
}

// sum_p phi_p a_p in the arithmetic type R (same order of operations as mixture_core).
template <int N, class R>
__device__ __forceinline__ R mix_sum(const R (&phi)[N], const R (&a)[MAXN])
{
    R v = R(0);
#pragma unroll
    for (int p = 0; p < N; ++p) v = rfma(phi[p], a[p], v);
    return v;
}

// eq. H: liquid fraction (and, with WANT_T, temperature) from rho H.
// rho_s H_s = rs cs T_sol, rho_l H_l = rl cl T_liq + Lv; a cell without phase-changing
// material (Lv <= 0) is liquid (the ambient fluid has f_s = 0).
template <int N, bool WANT_T>
__device__ __forceinline__ void enthalpy_map(const KParams& P, const Mix<N>& m, double rhoH, double& fl, double& T)
{
    const double rcs = m.rs * m.cs, rcl = m.rl * m.cl;
    const double As = rcs * P.T_sol;
    const double Al = fma(rcl, P.T_liq, m.Lv);
    if (!(m.Lv > 0.0)) {
        fl = 1.0;
        if (WANT_T) T = P.T_liq + (rhoH - Al) / rcl;
    } else if (rhoH < As) {
        fl = 0.0;
        if (WANT_T) T = rhoH / rcs;
    } else if (rhoH > Al) {
        fl = 1.0;
        if (WANT_T) T = P.T_liq + (rhoH - Al) / rcl;
    } else if (Al - As > 0.0) {
        fl = (rhoH - As) / (Al - As);
        if (WANT_T) T = fma(fl, P.T_liq - P.T_sol, P.T_sol);
    } else {
        fl = 1.0;
        if (WANT_T) T = P.T_liq;
    }
}

// Inverse of eq. H at t = 0 (a cell at or above the liquidus is liquid).
template <int N>
__device__ __forceinline__ double inverse_map(const KParams& P, const Mix<N>& m, double T)
{
    const double rcs = m.rs * m.cs, rcl = m.rl * m.cl;
    const double As = rcs * P.T_sol;
    const double Al = fma(rcl, P.T_liq, m.Lv);
    if (!(m.Lv > 0.0)) return Al + rcl * (T - P.T_liq);
    if (T < P.T_sol) return rcs * T;
    if (T >= P.T_liq) return Al + rcl * (T - P.T_liq);
    return As + (T - P.T_sol) / (P.T_liq - P.T_sol) * (Al - As);
}

// g'(x) for g(x) = x^2 (1 - x)^2
__device__ __forceinline__ double gprime(double x) { return 2.0 * x * (1.0 - x) * (1.0 - 2.0 * x); }

}  // namespace lbm
