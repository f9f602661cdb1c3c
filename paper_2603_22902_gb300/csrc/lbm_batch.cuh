// lbm_batch.cuh -- many independent lattices (cases) advanced together: every tile of
// every case is one work item of a flat list, so cases of uneven sizes fill the GPU.
//
// Cases are grouped by tile shape (32x8, 64x4 or 16x16, all 256 threads); each group
// has its own flat tile list and is launched on its own, since the groups never
// exchange data.  Two launch forms run the same per-tile step (step_tile in
// lbm_step.cuh):
//   * persistent: one cooperative launch runs nsteps steps; its blocks stride over
//     the tile list and meet at a grid barrier after every step (the next step of a
//     case reads what the neighbouring tiles wrote).  Loads bypass L1 (Coherent<Pr>),
//     since the blocks read data that other blocks wrote during the same launch.
//   * per step: one launch per step, one block per tile, read-only-path loads;
//   * staged (16-bit storage, N = 2 or 3, 32x8 tiles): the per-step form with each tile
//     computed from a TMA-staged copy of its inputs (staged_tile_issue / _finish,
//     lbm_staged.cuh), through six tensor maps per case and set kept in global memory;
//     the copies are in flight while the block loads the case's parameter block.
//
// Ping-pong: for case c, set pop[k] holds the state when k == parity, a device byte of
// the group.  The persistent kernel flips it itself when it has run an odd number of
// steps, so a captured graph of that launch can be replayed as it is.
#pragma once

#include "lbm_device.cuh"
#include "lbm_launch.cuh"
#include "lbm_prec.cuh"
#include "lbm_staged.cuh"
#include "lbm_step.cuh"

namespace lbm {

// Grid-wide barrier of a cooperative launch (all blocks resident).  Block-level
// barrier, then thread 0 fences, arrives and waits for the generation to change; the
// last block to arrive resets the count and bumps the generation.  The wait gives up
// after spin_limit polls, records status 1 and returns false.
__device__ __forceinline__ bool grid_barrier(const BatchTable& T)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* gen = T.bar + 1;
        const unsigned int g = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(T.bar, 1u) == gridDim.x - 1) {
            atomicExch(T.bar, 0u);
            __threadfence();
            atomicAdd(T.bar + 1, 1u);
        } else {
            long long n = 0;
            while (*gen == g) {
                if (++n > T.spin_limit || *(volatile int*)T.status != 0) {
                    atomicExch(T.status, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Copy the parameter block of case c into shared memory (all threads of the block).
__device__ __forceinline__ void load_params(KParams& dst, const KParams* src)
{
    static_assert(sizeof(KParams) % sizeof(long long) == 0, "KParams copied as 8-byte words");
    const long long* s = reinterpret_cast<const long long*>(src);
    long long* d = reinterpret_cast<long long*>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(KParams) / sizeof(long long)); k += blockDim.x) d[k] = __ldg(s + k);
}

// Persistent form: nsteps steps of every case of one tile shape in one cooperative
// launch.  Blocks stride over the flat tile list; consecutive tiles of a block often
// belong to the same case, whose parameter block then stays in shared memory.
template <int N, int TX, int TY, class Pr>
__global__ void __launch_bounds__(BATCH_NT, (LBM_OCC(Pr) + BATCH_NT - 1) / BATCH_NT)
batch_persistent_kernel(const BatchTable T, int nsteps)
{
    static_assert(TX * TY == BATCH_NT, "batch tiles have BATCH_NT cells");
    using PC = Coherent<Pr>;
    using TA = typename Pr::TA;
    __shared__ KParams sP;
    __shared__ typename Pr::R smem[tile_smem_elems<N, TX, TY, Pr>()];
    const int a0 = *(volatile unsigned char*)T.parity;
    int loaded = -1;
    for (int s = 0; s < nsteps; ++s) {
        const int a = a0 ^ (s & 1);
        for (int t = blockIdx.x; t < T.total_tiles; t += gridDim.x) {
            const int c = __ldg(T.tile_case + t);
            __syncthreads();  // the previous tile is done with sP and smem
            if (c != loaded) {
                load_params(sP, T.params + c);
                loaded = c;
                __syncthreads();
            }
            const BatchCase& C = T.cases[c];
            const int local = t - C.first_tile;
            step_tile<N, TX, TY, true, PC>(sP, C.pop[a], const_cast<void*>(C.pop[a ^ 1]), (const TA*)C.aux[a],
                                           (TA*)C.aux[a ^ 1], ExportPtrs{}, local % C.tiles_x, local / C.tiles_x,
                                           smem);
        }
        if (!grid_barrier(T)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (nsteps & 1)) *T.parity = (unsigned char)(a0 ^ 1);
}

// Per-step form: one block per tile of the flat list, step s of the call.
template <int N, int TX, int TY, class Pr>
__global__ void __launch_bounds__(BATCH_NT, (LBM_OCC(Pr) + BATCH_NT - 1) / BATCH_NT)
batch_step_kernel(const BatchTable T, int s)
{
    static_assert(TX * TY == BATCH_NT, "batch tiles have BATCH_NT cells");
    using TA = typename Pr::TA;
    __shared__ KParams sP;
    __shared__ typename Pr::R smem[tile_smem_elems<N, TX, TY, Pr>()];
    const int t = blockIdx.x;
    const int c = __ldg(T.tile_case + t);
    load_params(sP, T.params + c);
    __syncthreads();
    const int a = (*(volatile unsigned char*)T.parity) ^ (s & 1);
    const BatchCase& C = T.cases[c];
    const int local = t - C.first_tile;
    step_tile<N, TX, TY, true, Pr>(sP, C.pop[a], const_cast<void*>(C.pop[a ^ 1]), (const TA*)C.aux[a],
                                   (TA*)C.aux[a ^ 1], ExportPtrs{}, local % C.tiles_x, local / C.tiles_x, smem);
}

// Staged form: one block per tile of the flat list (32x8 tiles), step s of the call;
// maps[2 c + k] are the tensor maps of case c's population and lagged set k.
template <int N, class Pr>
__global__ void __launch_bounds__(STAGE_NT, stage_blocks_per_sm<N>())
batch_staged_kernel(const BatchTable T, const StageMaps* __restrict__ maps, int s)
{
    extern __shared__ __align__(128) unsigned char dyn_raw[];
    using TA = typename Pr::TA;
    __shared__ KParams sP;
    const int t = blockIdx.x;
    const int c = __ldg(T.tile_case + t);
    const int a = (*(volatile unsigned char*)T.parity) ^ (s & 1);
    const BatchCase& C = T.cases[c];
    const int local = t - C.first_tile;
    const int bx = local % C.tiles_x, by = local / C.tiles_x;
    staged_tile_issue<N, Pr>(maps[2 * c + a], bx, by, dyn_raw);
    load_params(sP, T.params + c);   // while the copies are in flight
    __syncthreads();                 // staged_tile_finish reads sP from its first line
    staged_tile_finish<N, Pr>(sP, C.pop[a], const_cast<void*>(C.pop[a ^ 1]), (const TA*)C.aux[a], (TA*)C.aux[a ^ 1],
                              T.status, bx, by, dyn_raw);
}

}  // namespace lbm
