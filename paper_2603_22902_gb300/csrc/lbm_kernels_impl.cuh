// lbm_kernels_impl.cuh -- definitions of the launchers; included by one .cu per
// (N, precision) pair so that the instantiations compile in parallel.
#pragma once

#include <algorithm>

#include "lbm_adjoint.cuh"
#include "lbm_aux.cuh"
#include "lbm_batch.cuh"
#include "lbm_launch.cuh"
#include "lbm_staged.cuh"
#include "lbm_step.cuh"

namespace lbm {

template <int N, int TX, int TY, bool COLLIDE, class Pr>
static cudaError_t launch_fused_t(const KParams& P, const void* pin, void* pout, const void* ain, void* aout,
                                  ExportPtrs ex, cudaStream_t st, TileRows rows)
{
    using TA = typename Pr::TA;
    const int tiles = ((P.nx + TX - 1) / TX) * tile_rows_count((P.ny + TY - 1) / TY, rows);
    if (tiles == 0) return cudaSuccess;
    fused_step_kernel<N, TX, TY, COLLIDE, Pr><<<tiles, TX * TY, 0, st>>>(P, pin, pout, (const TA*)ain, (TA*)aout, ex,
                                                                         rows);
    return cudaGetLastError();
}

// The double-word policy is compiled for the 32 x 8 tile only (each shape of its kernel
// adds much code); lbm_set_tile and the batch plans refuse other shapes for it.
template <class Pr>
constexpr bool single_shape() { return std::is_same<Pr, PrecDF64>::value; }

template <int N, bool COLLIDE, class Pr>
static cudaError_t launch_fused(const KParams& P, const void* pin, void* pout, const void* ain, void* aout,
                                ExportPtrs ex, int tile, cudaStream_t st, TileRows rows = TileRows{ROWS_ALL, 0, 0})
{
    if constexpr (single_shape<Pr>()) {
        return launch_fused_t<N, 32, 8, COLLIDE, Pr>(P, pin, pout, ain, aout, ex, st, rows);
    } else {
        switch (tile) {
            case TILE_32x4: return launch_fused_t<N, 32, 4, COLLIDE, Pr>(P, pin, pout, ain, aout, ex, st, rows);
            case TILE_64x4: return launch_fused_t<N, 64, 4, COLLIDE, Pr>(P, pin, pout, ain, aout, ex, st, rows);
            case TILE_16x16: return launch_fused_t<N, 16, 16, COLLIDE, Pr>(P, pin, pout, ain, aout, ex, st, rows);
            default: return launch_fused_t<N, 32, 8, COLLIDE, Pr>(P, pin, pout, ain, aout, ex, st, rows);
        }
    }
}

template <int N, class Pr>
cudaError_t launch_step(const KParams& P, const void* pin, void* pout, const void* ain, void* aout, int tile,
                        cudaStream_t st, TileRows rows)
{
    return launch_fused<N, true, Pr>(P, pin, pout, ain, aout, ExportPtrs{}, tile, st, rows);
}

template <int N, class Pr>
cudaError_t launch_export(const KParams& P, const void* pin, const void* ain, double* phi, double* T, double* H,
                          double* fl, double* ux, double* uy, double* p, cudaStream_t st)
{
    return launch_fused<N, false, Pr>(P, pin, nullptr, ain, nullptr, ExportPtrs{phi, T, H, fl, ux, uy, p}, TILE_32x8,
                                      st);
}

template <int N, class Pr>
cudaError_t launch_staged(const KParams& P, const StageMaps& maps, const void* pin, void* pout, const void* ain,
                          void* aout, int* status, cudaStream_t st, TileRows rows)
{
    if constexpr (staged_policy<Pr>() && (N == 2 || N == 3)) {
        using Lay = StageLayout<N, Pr>;
        using TA = typename Pr::TA;
        const int tiles_x = (P.nx + STAGE_TX - 1) / STAGE_TX, tiles_y = (P.ny + STAGE_TY - 1) / STAGE_TY;
        cudaError_t e = cudaFuncSetAttribute(staged_tile_kernel<N, Pr>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Lay::TOTAL);
        if (e != cudaSuccess) return e;
        const int tiles = tiles_x * tile_rows_count(tiles_y, rows);
        if (tiles == 0) return cudaSuccess;
        staged_tile_kernel<N, Pr><<<tiles, STAGE_NT, Lay::TOTAL, st>>>(P, maps, pin, pout, (const TA*)ain, (TA*)aout,
                                                                        status, rows);
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

template <int N, class Pr>
cudaError_t launch_init(const KParams& P, const double* phi, const double* T, const double* ux, const double* uy,
                        void* pop, void* aux, cudaStream_t st)
{
    long long blocks = (P.S + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    init_kernel<N, Pr><<<(int)blocks, 256, 0, st>>>(P, phi, T, ux, uy, pop, (typename Pr::TA*)aux);
    return cudaGetLastError();
}

template <int N, class Pr>
cudaError_t launch_diag(const KParams& P, const void* pop, const void* aux, double* partial, double* out,
                        cudaStream_t st, long long c0, long long cells)
{
    if (cells < 0) cells = P.S - c0;
    const int nb = diag_blocks(cells);
    diag_partial_kernel<N, DIAG_NT, Pr><<<nb, DIAG_NT, 0, st>>>(P, pop, (const typename Pr::TA*)aux, partial, c0,
                                                                cells);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final_kernel<N><<<1, 32, 0, st>>>(partial, nb, out);
    return cudaGetLastError();
}

template <int N, int TX, int TY, class Pr>
static cudaError_t launch_batch_persistent_t(const BatchTable& T, int nsteps, int blocks, cudaStream_t st)
{
    BatchTable t = T;
    int n = nsteps;
    void* args[] = {(void*)&t, (void*)&n};
    return cudaLaunchCooperativeKernel((const void*)batch_persistent_kernel<N, TX, TY, Pr>, dim3(blocks),
                                       dim3(BATCH_NT), args, 0, st);
}

template <int N, class Pr>
cudaError_t launch_batch_persistent(const BatchTable& T, int kind, int nsteps, int blocks, cudaStream_t st)
{
    if constexpr (single_shape<Pr>()) {
        if (kind != TILE_32x8) return cudaErrorNotSupported;
        return launch_batch_persistent_t<N, 32, 8, Pr>(T, nsteps, blocks, st);
    } else {
        switch (kind) {
            case TILE_64x4: return launch_batch_persistent_t<N, 64, 4, Pr>(T, nsteps, blocks, st);
            case TILE_16x16: return launch_batch_persistent_t<N, 16, 16, Pr>(T, nsteps, blocks, st);
            default: return launch_batch_persistent_t<N, 32, 8, Pr>(T, nsteps, blocks, st);
        }
    }
}

template <int N, class Pr>
cudaError_t batch_blocks_per_sm(int kind, int* out)
{
    if constexpr (single_shape<Pr>()) {
        if (kind != TILE_32x8) return cudaErrorNotSupported;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, batch_persistent_kernel<N, 32, 8, Pr>, BATCH_NT, 0);
    } else {
        switch (kind) {
            case TILE_64x4:
                return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, batch_persistent_kernel<N, 64, 4, Pr>, BATCH_NT, 0);
            case TILE_16x16:
                return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, batch_persistent_kernel<N, 16, 16, Pr>, BATCH_NT,
                                                                     0);
            default:
                return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, batch_persistent_kernel<N, 32, 8, Pr>, BATCH_NT, 0);
        }
    }
}

template <int N, class Pr>
cudaError_t launch_batch_step(const BatchTable& T, int kind, int s, cudaStream_t st)
{
    if constexpr (single_shape<Pr>()) {
        if (kind != TILE_32x8) return cudaErrorNotSupported;
        batch_step_kernel<N, 32, 8, Pr><<<T.total_tiles, BATCH_NT, 0, st>>>(T, s);
        return cudaGetLastError();
    } else {
        switch (kind) {
            case TILE_64x4: batch_step_kernel<N, 64, 4, Pr><<<T.total_tiles, BATCH_NT, 0, st>>>(T, s); break;
            case TILE_16x16: batch_step_kernel<N, 16, 16, Pr><<<T.total_tiles, BATCH_NT, 0, st>>>(T, s); break;
            default: batch_step_kernel<N, 32, 8, Pr><<<T.total_tiles, BATCH_NT, 0, st>>>(T, s); break;
        }
        return cudaGetLastError();
    }
}

template <int N, class Pr>
cudaError_t launch_batch_staged(const BatchTable& T, const StageMaps* maps, int s, cudaStream_t st)
{
    if constexpr (staged_policy<Pr>() && (N == 2 || N == 3)) {
        using Lay = StageLayout<N, Pr>;
        cudaError_t e = cudaFuncSetAttribute(batch_staged_kernel<N, Pr>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Lay::TOTAL);
        if (e != cudaSuccess) return e;
        batch_staged_kernel<N, Pr><<<T.total_tiles, STAGE_NT, Lay::TOTAL, st>>>(T, maps, s);
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

template <int N>
cudaError_t launch_adj_mac(const KParams& P, const double* pin, const double* ain, double* mac, cudaStream_t st)
{
    const long long blocks = std::min<long long>((P.S + 255) / 256, 65535);
    mac_kernel<N><<<(int)blocks, 256, 0, st>>>(P, pin, ain, mac);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_adj_cell(const KParams& P, const AdjBufs& B, cudaStream_t st)
{
    adj_cell_kernel<N><<<(unsigned)((P.S + 127) / 128), 128, 0, st>>>(P, B);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_adj_moments(const KParams& P, const AdjBufs& B, bool seed, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((P.S + 127) / 128);
    if (seed) adj_moments_kernel<N, true><<<blocks, 128, 0, st>>>(P, B);
    else adj_moments_kernel<N, false><<<blocks, 128, 0, st>>>(P, B);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_adj_init(const KParams& P, const double* phi0, const double* T0, const double* apop, double* grad,
                            cudaStream_t st)
{
    const long long blocks = std::min<long long>((P.S + 255) / 256, 65535);
    adj_init_kernel<N><<<(int)blocks, 256, 0, st>>>(P, phi0, T0, apop, grad);
    return cudaGetLastError();
}

#define LBM_INSTANTIATE_ADJ(N)                                                                                    \
    template cudaError_t launch_adj_mac<N>(const KParams&, const double*, const double*, double*, cudaStream_t); \
    template cudaError_t launch_adj_cell<N>(const KParams&, const AdjBufs&, cudaStream_t);                         \
    template cudaError_t launch_adj_moments<N>(const KParams&, const AdjBufs&, bool, cudaStream_t);                \
    template cudaError_t launch_adj_init<N>(const KParams&, const double*, const double*, const double*, double*,  \
                                            cudaStream_t);

#define LBM_INSTANTIATE(N, PR)                                                                                      \
    template cudaError_t launch_step<N, PR>(const KParams&, const void*, void*, const void*, void*, int,           \
                                            cudaStream_t, TileRows);                                                \
    template cudaError_t launch_staged<N, PR>(const KParams&, const StageMaps&, const void*, void*, const void*,   \
                                              void*, int*, cudaStream_t, TileRows);                                 \
    template cudaError_t launch_export<N, PR>(const KParams&, const void*, const void*, double*, double*, double*, \
                                              double*, double*, double*, double*, cudaStream_t);                    \
    template cudaError_t launch_init<N, PR>(const KParams&, const double*, const double*, const double*,           \
                                            const double*, void*, void*, cudaStream_t);                             \
    template cudaError_t launch_diag<N, PR>(const KParams&, const void*, const void*, double*, double*, cudaStream_t, \
                                            long long, long long);                                                  \
    template cudaError_t launch_batch_persistent<N, PR>(const BatchTable&, int, int, int, cudaStream_t);            \
    template cudaError_t batch_blocks_per_sm<N, PR>(int, int*);                                                     \
    template cudaError_t launch_batch_step<N, PR>(const BatchTable&, int, int, cudaStream_t);                       \
    template cudaError_t launch_batch_staged<N, PR>(const BatchTable&, const StageMaps*, int, cudaStream_t);

}  // namespace lbm
