// lbm_kernels_impl.cuh -- definitions of the launchers; included by one .cu per N.
#pragma once

#include "lbm_aux.cuh"
#include "lbm_launch.cuh"
#include "lbm_step.cuh"

namespace lbm {

template <int N, int TX, int TY, bool COLLIDE>
static cudaError_t launch_fused_t(const KParams& P, const double* pin, double* pout, const double* ain,
                                  double* aout, ExportPtrs ex, cudaStream_t st)
{
    dim3 grid((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY);
    fused_step_kernel<N, TX, TY, COLLIDE><<<grid, TX * TY, 0, st>>>(P, pin, pout, ain, aout, ex);
    return cudaGetLastError();
}

template <int N, bool COLLIDE>
static cudaError_t launch_fused(const KParams& P, const double* pin, double* pout, const double* ain, double* aout,
                                ExportPtrs ex, int tile, cudaStream_t st)
{
    switch (tile) {
        case TILE_32x4: return launch_fused_t<N, 32, 4, COLLIDE>(P, pin, pout, ain, aout, ex, st);
        case TILE_64x4: return launch_fused_t<N, 64, 4, COLLIDE>(P, pin, pout, ain, aout, ex, st);
        case TILE_16x16: return launch_fused_t<N, 16, 16, COLLIDE>(P, pin, pout, ain, aout, ex, st);
        default: return launch_fused_t<N, 32, 8, COLLIDE>(P, pin, pout, ain, aout, ex, st);
    }
}

template <int N>
cudaError_t launch_step(const KParams& P, const double* pin, double* pout, const double* ain, double* aout,
                        int tile, cudaStream_t st)
{
    return launch_fused<N, true>(P, pin, pout, ain, aout, ExportPtrs{}, tile, st);
}

template <int N>
cudaError_t launch_export(const KParams& P, const double* pin, const double* ain, double* phi, double* T,
                          double* H, double* fl, double* ux, double* uy, double* p, cudaStream_t st)
{
    return launch_fused<N, false>(P, pin, nullptr, ain, nullptr, ExportPtrs{phi, T, H, fl, ux, uy, p}, TILE_32x8, st);
}

template <int N>
cudaError_t launch_init(const KParams& P, const double* phi, const double* T, const double* ux, const double* uy,
                        double* pop, double* aux, cudaStream_t st)
{
    long long blocks = (P.S + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    init_kernel<N><<<(int)blocks, 256, 0, st>>>(P, phi, T, ux, uy, pop, aux);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_diag(const KParams& P, const double* pop, const double* aux, double* partial, double* out,
                        cudaStream_t st)
{
    const int nb = diag_blocks(P.S);
    diag_partial_kernel<N, DIAG_NT><<<nb, DIAG_NT, 0, st>>>(P, pop, aux, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final_kernel<N><<<1, 32, 0, st>>>(partial, nb, out);
    return cudaGetLastError();
}

#define LBM_INSTANTIATE(N)                                                                                         \
    template cudaError_t launch_step<N>(const KParams&, const double*, double*, const double*, double*, int,       \
                                        cudaStream_t);                                                             \
    template cudaError_t launch_export<N>(const KParams&, const double*, const double*, double*, double*, double*, \
                                          double*, double*, double*, double*, cudaStream_t);                       \
    template cudaError_t launch_init<N>(const KParams&, const double*, const double*, const double*, const double*, \
                                        double*, double*, cudaStream_t);                                           \
    template cudaError_t launch_diag<N>(const KParams&, const double*, const double*, double*, double*, cudaStream_t);

}  // namespace lbm
