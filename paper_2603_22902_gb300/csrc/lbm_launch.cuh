// lbm_launch.cuh -- host-side launchers of the device kernels, one explicit
// instantiation set per phase count N and precision policy (lbm_kernels_*.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "lbm_device.cuh"
#include "lbm_prec.cuh"

namespace lbm {

// Compiled tile shapes of the fused step kernel (TX x TY threads, one cell each).
enum TileId { TILE_32x8 = 0, TILE_32x4 = 1, TILE_64x4 = 2, TILE_16x16 = 3, TILE_COUNT = 4 };
inline bool tile_dims(int id, int& tx, int& ty)
{
    switch (id) {
        case TILE_32x8: tx = 32; ty = 8; return true;
        case TILE_32x4: tx = 32; ty = 4; return true;
        case TILE_64x4: tx = 64; ty = 4; return true;
        case TILE_16x16: tx = 16; ty = 16; return true;
        default: return false;
    }
}

template <int N, class Pr>
cudaError_t launch_step(const KParams& P, const void* pin, void* pout, const void* ain, void* aout, int tile,
                        cudaStream_t st, TileRows rows = TileRows{ROWS_ALL, 0, 0});
template <int N, class Pr>
cudaError_t launch_export(const KParams& P, const void* pin, const void* ain, double* phi, double* T, double* H,
                          double* fl, double* ux, double* uy, double* p, cudaStream_t st);
template <int N, class Pr>
cudaError_t launch_init(const KParams& P, const double* phi, const double* T, const double* ux, const double* uy,
                        void* pop, void* aux, cudaStream_t st);
// The step with its inputs staged by the TMA (lbm_staged.cuh): policies with 16-bit moving
// populations, N = 2 or 3, one block per tile.  maps are the six tensor maps of the input set;
// status receives 1 when an mbarrier wait gave up.  cudaErrorNotSupported for other policies.
struct StageMaps {
    CUtensorMap m[6];   // boxes A..F of lbm_staged.cuh
};
template <int N, class Pr>
cudaError_t launch_staged(const KParams& P, const StageMaps& maps, const void* pin, void* pout, const void* ain,
                          void* aout, int* status, cudaStream_t st, TileRows rows = TileRows{ROWS_ALL, 0, 0});
template <class Pr>
constexpr bool staged_policy()
{
    return Pr::QUANT;
}
// Two-pass deterministic reduction; partial must hold diag_blocks() * (2N + 2) doubles,
// out 2N + 2 doubles (mass[N], solid[N], max |sum phi - 1|, non-finite count).
constexpr int DIAG_NT = 256;
inline int diag_blocks(long long cells)
{
    long long b = (cells + DIAG_NT - 1) / DIAG_NT;
    if (b > 4 * 152) b = 4 * 152;  // a few blocks per SM of a GB300 is enough
    return (int)(b < 1 ? 1 : b);
}
// Over the cells c0 .. c0 + cells - 1 (cells < 0: to the end of the lattice).
template <int N, class Pr>
cudaError_t launch_diag(const KParams& P, const void* pop, const void* aux, double* partial, double* out,
                        cudaStream_t st, long long c0 = 0, long long cells = -1);

// ---- batches of independent cases (lbm_batch.cuh) -----------------------------------
constexpr int BATCH_NT = 256;   // threads of every batch block (all batch tile shapes)

struct BatchCase {
    const void* pop[2];
    void* aux[2];
    int tiles_x, tiles_y;
    int tile_kind;          // TILE_32x8, TILE_64x4 or TILE_16x16
    int first_tile;         // index of the case's first tile in the flat list
};

struct BatchTable {            // one group of cases sharing a tile shape
    int total_tiles;
    const BatchCase* cases;     // [all cases of the batch]
    const KParams* params;      // [all cases of the batch]
    const int* tile_case;       // [total_tiles] case of each tile of the group, cases in order
    unsigned char* parity;      // the set holding the current state of the group's cases
    unsigned int* bar;          // grid barrier: {arrivals, generation}; arrivals 0 before a launch
    int* status;                // 0, or 1 when a barrier wait gave up
    long long spin_limit;       // polls of a barrier wait before it gives up
};

// One cooperative launch running nsteps steps of the group (tile shape `kind`); blocks
// must not exceed the resident limit (batch_blocks_per_sm x SMs).
template <int N, class Pr>
cudaError_t launch_batch_persistent(const BatchTable& T, int kind, int nsteps, int blocks, cudaStream_t st);
template <int N, class Pr>
cudaError_t batch_blocks_per_sm(int kind, int* out);
// One launch of step s of the group, one block per tile.
template <int N, class Pr>
cudaError_t launch_batch_step(const BatchTable& T, int kind, int s, cudaStream_t st);
// One launch of step s of a group of 32x8 tiles in the staged form (16-bit storage, N = 2 or 3;
// cudaErrorNotSupported otherwise); maps[2 c + k]: case c, population and lagged set k.
template <int N, class Pr>
cudaError_t launch_batch_staged(const BatchTable& T, const StageMaps* maps, int s, cudaStream_t st);

// ---- adjoint of the FP64 step (lbm_adjoint.cuh) ------------------------------------
// Gradient slots (planes of the gradient buffer).
constexpr int GS_TW = 0;                   // T_wall[side], 4 slots
constexpr int GS_RHOL = 4;                 // rho_l^p L_p (latent heat per volume), MAXN slots
constexpr int GS_LAMS = 4 + MAXN;          // lambda_s^p
constexpr int GS_LAML = 4 + 2 * MAXN;      // lambda_l^p
constexpr int GS_COUNT = 4 + 3 * MAXN;

struct AdjBufs {
    const double* pin;     // set A populations (FP64 policy layout)
    const double* ain;     // set A lagged planes
    const double* bpop;    // adjoint of set B populations
    const double* baux;    // adjoint of set B lagged planes
    double* apop;          // adjoint of set A populations (written)
    double* aaux;          // adjoint of set A lagged planes (written)
    const double* mac;     // phi_p (N planes), rho, psi of set A
    double* own;           // phi_p-bar (N planes) and rhoH-bar of each cell's own use
    double* sb;            // stencil adjoints [k][N + 2][S]
    double* grad;          // gradient planes [GS_COUNT][S], accumulated
    const double* fl_target;  // loss seed: target f_l plane (adj_moments_kernel<N, true>)
    const double* weight;     // loss seed: weight plane, or NULL (weight 1)
};

// Loss plane after the gradient planes: sum_x w (f_l - f_target)^2 per cell.
constexpr int GS_LOSS = GS_COUNT;

template <int N>
cudaError_t launch_adj_mac(const KParams& P, const double* pin, const double* ain, double* mac, cudaStream_t st);
template <int N>
cudaError_t launch_adj_cell(const KParams& P, const AdjBufs& B, cudaStream_t st);
// seed = true: the loss seed at the final state instead of the users' stencil adjoints
template <int N>
cudaError_t launch_adj_moments(const KParams& P, const AdjBufs& B, bool seed, cudaStream_t st);
template <int N>
cudaError_t launch_adj_init(const KParams& P, const double* phi0, const double* T0, const double* apop, double* grad,
                            cudaStream_t st);
// Sums of nplanes planes of S doubles in a fixed order: partial needs nplanes * 256
// doubles, out nplanes.
cudaError_t launch_plane_sums(const double* planes, int nplanes, long long S, double* partial, double* out,
                              cudaStream_t st);

// Call f(std::integral_constant<int, N>{}, Prec{}) for the runtime phase count and
// precision id (LBM_FP64 / FP32 / FP16S / BF16S / DF64 = 0..4).
template <class F>
auto dispatch(int N, int prec, F&& f)
{
    auto byN = [&](auto pr) {
        if (N == 2) return f(std::integral_constant<int, 2>{}, pr);
        if (N == 3) return f(std::integral_constant<int, 3>{}, pr);
        return f(std::integral_constant<int, 4>{}, pr);
    };
    switch (prec) {
        case 1: return byN(PrecFP32{});
        case 2: return byN(PrecFP16S{});
        case 3: return byN(PrecBF16S{});
        case 4: return byN(PrecDF64{});
        default: return byN(PrecFP64{});
    }
}

}  // namespace lbm
