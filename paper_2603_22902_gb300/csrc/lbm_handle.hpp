// lbm_handle.hpp -- the handle behind lbm_handle* (internal to the library: the C ABI
// in lbm_capi.cu and the batches in lbm_batch_capi.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/lbm.h"
#include "lbm_launch.cuh"

struct lbm_handle {
    int device = 0;
    int N = 0, nx = 0, ny = 0;
    int precision = LBM_FP64;
    int diag_every = 0;
    int tile = lbm::TILE_32x8;
    lbm::KParams P{};
    void* pop[2] = {nullptr, nullptr};    // one population set each (rest + moving block)
    void* aux[2] = {nullptr, nullptr};    // 3 + 2N lagged planes each
    size_t pop_bytes = 0, aux_bytes = 0;
    double* io = nullptr;                 // N + 6 planes: staging for host I/O
    double* diag_partial = nullptr;
    double* diag_out = nullptr;
    unsigned long long* dbg = nullptr;    // bounds-check record (LBM_CHECK_BOUNDS builds)
    int cur = 0;
    bool ready = false;
    long long steps = 0;
    cudaStream_t stream = nullptr;
    // TMA-staged step (lbm_set_staging): tensor maps of both population sets, status word
    bool staged = false;
    lbm::StageMaps stage_maps[2];
    int* stage_status = nullptr;
    // y slab (lbm_slab_create): ghost rows below / above the band, first global row
    bool slab = false;
    int slab_ghost[2] = {0, 0};
    int slab_y0 = 0;
    bool slab_inner_pending = false;      // lbm_slab_step_part: inner rows stepped, edge rows not yet
    std::string err;
};

// The six tensor maps of the staged step (boxes A..F of lbm_staged.cuh) over a population
// set `pop` and a lagged set `aux` laid out like the handle's (16-bit storage, N = 2,
// nx a multiple of 8); false when the driver cannot encode them.  Defined in lbm_capi.cu,
// used by the handle's own staged step and by the staged batch form.
bool lbm_encode_stage_maps(const lbm_handle* h, const void* pop, const void* aux, lbm::StageMaps* M);
