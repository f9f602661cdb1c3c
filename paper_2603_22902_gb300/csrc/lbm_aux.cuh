// lbm_aux.cuh -- initial state and diagnostics kernels, generic over the precision
// policy (lbm_prec.cuh).  Both evaluate in FP64 and (de)quantise at the store / load.
#pragma once

#include "lbm_device.cuh"
#include "lbm_prec.cuh"
#include "lbm_step.cuh"

namespace lbm {

// t = 0 (Section 3 equilibria, Section 2 eq. H inverted): from phi_p, T, u build
// rho H, then f_l, T, rho, c_p by eq. H / eq. 2; populations at equilibrium with
// p = 0; mdot' = Q' = 0, psi' = psi, (phi_p u)' = phi_p u.
template <int N, class Pr>
__global__ void init_kernel(const KParams P, const double* __restrict__ phi_in, const double* __restrict__ T_in,
                            const double* __restrict__ ux_in, const double* __restrict__ uy_in,
                            void* __restrict__ pop_base, typename Pr::TA* __restrict__ aux)
{
    using R = typename Pr::R;
    using TA = typename Pr::TA;
    const long long S = P.S;
    const PopView<Pr> pop = pop_view<Pr>(P, pop_base);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < S; c += (long long)gridDim.x * blockDim.x) {
        double phi[N];
#pragma unroll
        for (int p = 0; p < N; ++p) phi[p] = LBM_LD(P, phi_in, p * S + c, N * S, 40);
        const double ux = ux_in ? LBM_LD(P, ux_in, c, S, 41) : 0.0, uy = uy_in ? LBM_LD(P, uy_in, c, S, 42) : 0.0;
        const Mix<N> m = mixture_core<N>(P, phi);
        const double rhoH = inverse_map<N>(P, m, LBM_LD(P, T_in, c, S, 43));
        double fl, T;
        enthalpy_map<N, true>(P, m, rhoH, fl, T);
        const double fs = 1.0 - fl;
        const double rho = fma(fs, m.rs, fl * m.rl);
        const double cp = fma(fs, m.cs, fl * m.cl);
        const double uu = ux * ux + uy * uy;
        const double E = P.d.E_ref * T, Z = rho * cp * T;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double cu = cx(i) * ux + cy(i) * uy;
            const double si = wgt(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            st_pop<Pr, KIND_F>(P, pop, 0, i, c, (R)(rho * si), 44);
            double he;
            if (i == 0) he = rhoH - E + wgt(0) * (E - 1.5 * Z * uu);
            else he = wgt(i) * (E + Z * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
            st_pop<Pr, KIND_H>(P, pop, N + 1, i, c, (R)he, 45);
#pragma unroll
            for (int p = 0; p < N; ++p)
                st_pop<Pr, KIND_G>(P, pop, 1 + p, i, c, (R)(wgt(i) * phi[p] * (1.0 + 3.0 * cu)), 46);
        }
        LBM_ST(P, aux, aux_mdot() * S + c, P.aux_elems, 47, (TA)0.0);
        LBM_ST(P, aux, aux_Q() * S + c, P.aux_elems, 47, (TA)0.0);
        LBM_ST(P, aux, aux_psi() * S + c, P.aux_elems, 47, (TA)(fs * m.dr));
#pragma unroll
        for (int p = 0; p < N; ++p) {
            LBM_ST(P, aux, aux_phiux(p) * S + c, P.aux_elems, 48, (TA)(phi[p] * ux));
            LBM_ST(P, aux, aux_phiuy(N, p) * S + c, P.aux_elems, 48, (TA)(phi[p] * uy));
        }
    }
}

// Diagnostics, pass 1: per-block partial sums (fixed order inside the block) in FP64
// of sum phi_p, sum f_s phi_p, max |sum_p phi_p - 1| and the count of non-finite cells,
// over the cells c0 .. c0 + cells - 1 (the whole lattice, or the own rows of a slab).
// partial[b * (2N + 2) + k]; pass 2 adds the blocks in index order.
template <int N, int NT, class Pr>
__global__ void __launch_bounds__(NT) diag_partial_kernel(const KParams P, const void* __restrict__ pop_base,
                                                          const typename Pr::TA* __restrict__ aux,
                                                          double* __restrict__ partial, long long c0,
                                                          long long cells)
{
    constexpr int K = 2 * N + 2;
    __shared__ double red[K][NT];
    const long long S = P.S;
    const PopView<Pr> pop = pop_view<Pr>(P, pop_base);
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (long long k = blockIdx.x * (long long)NT + threadIdx.x; k < cells; k += (long long)gridDim.x * NT) {
        const long long c = c0 + k;
        const double den = 1.0 - 0.5 * (double)LBM_LD(P, aux, aux_mdot() * S + c, P.aux_elems, 50);
        double phi[N], sum = 0.0;
#pragma unroll
        for (int p = 0; p < N; ++p) {
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < 9; ++i) s += (double)ld_pop<Pr, KIND_G>(P, pop, 1 + p, i, c, 51);
            phi[p] = s / den;
            sum += phi[p];
        }
        double sh = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) sh += (double)ld_pop<Pr, KIND_H>(P, pop, N + 1, i, c, 52);
        double f0 = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) f0 += (double)ld_pop<Pr, KIND_F>(P, pop, 0, i, c, 53);
        const double rhoH = fma(0.5, (double)LBM_LD(P, aux, aux_Q() * S + c, P.aux_elems, 54), sh);
        const Mix<N> m = mixture_core<N>(P, phi);
        double fl, T;
        enthalpy_map<N, false>(P, m, rhoH, fl, T);
        const double fs = 1.0 - fl;
        const bool bad = !isfinite(sum) || !isfinite(rhoH) || !isfinite(f0);
#pragma unroll
        for (int p = 0; p < N; ++p) {
            acc[p] += phi[p];
            acc[N + p] += fs * phi[p];
        }
        acc[2 * N] = fmax(acc[2 * N], fabs(sum - 1.0));
        acc[2 * N + 1] += bad ? 1.0 : 0.0;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (k == 2 * N) red[k][threadIdx.x] = fmax(red[k][threadIdx.x], red[k][threadIdx.x + s]);
                else red[k][threadIdx.x] += red[k][threadIdx.x + s];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) partial[blockIdx.x * K + k] = red[k][0];
}

// Diagnostics, pass 2: one warp adds the block partials in a fixed order
// (lane-strided, then a shuffle tree), so the result does not depend on timing.
template <int N>
__global__ void diag_final_kernel(const double* __restrict__ partial, int nblocks, double* __restrict__ out)
{
    constexpr int K = 2 * N + 2;
    const int lane = threadIdx.x;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double v = 0.0;
        for (int b = lane; b < nblocks; b += 32) {
            const double w = partial[b * K + k];
            v = (k == 2 * N) ? fmax(v, w) : v + w;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double o = __shfl_down_sync(0xffffffffu, v, off);
            v = (k == 2 * N) ? fmax(v, o) : v + o;
        }
        if (lane == 0) out[k] = v;
    }
}

}  // namespace lbm
