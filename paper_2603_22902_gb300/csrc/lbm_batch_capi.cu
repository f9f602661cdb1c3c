// lbm_batch_capi.cu -- batches of independent cases (the lbm_batch_* calls of
// include/lbm.h): work-list tables, ping-pong bookkeeping of the member handles,
// graph capture of the launches of a call (either form), and the plan autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_handle.hpp"
#include "lbm_trace.hpp"
#include "lbm_launch.cuh"

using namespace lbm;

namespace {

constexpr int NKIND = 3;                                          // batch tile shapes
constexpr int KIND_TILE[NKIND] = {TILE_32x8, TILE_64x4, TILE_16x16};
constexpr int KIND_TX[NKIND] = {32, 64, 16}, KIND_TY[NKIND] = {8, 4, 16};
// Polls of a grid-barrier wait before it gives up.  Each poll is a global load plus a
// 128 ns sleep (the sleep is a hint, so the bound is on polls): 2^21 polls take at least
// 0.27 s and about a second in practice, against a step time of milliseconds.  Groups
// so large that a step could approach that get proportionally more (one poll per 8
// cells, i.e. >= 16 ns per cell, a hundred times the step cost of a cell).
constexpr long long SPIN_MIN = 1LL << 21;

int size_class(long long cells)
{
    if (cells <= 128LL * 128) return 0;
    if (cells <= 256LL * 256) return 1;
    if (cells <= 384LL * 384) return 2;
    return 3;
}

int kind_of_shape(int bx, int by)
{
    for (int k = 0; k < NKIND; ++k)
        if (KIND_TX[k] == bx && KIND_TY[k] == by) return k;
    return -1;
}

thread_local std::string g_batch_create_error;

}  // namespace

struct lbm_batch {
    int device = 0, N = 0, precision = 0, ncases = 0, sms = 0;
    std::vector<lbm_handle*> h;
    int mode = LBM_BATCH_PERSISTENT;
    int blocks_per_sm = 0;
    long long wait_limit = 0;               // polls of a barrier wait; 0 = the size-based default
    int class_kind[LBM_BATCH_CLASSES] = {0, 0, 0, 0};
    // tables: host mirrors and device copies
    std::vector<BatchCase> cases;
    std::vector<int> group;                 // group (tile kind) of each case
    int group_tiles[NKIND] = {0, 0, 0}, group_first[NKIND] = {0, 0, 0};
    long long group_cells[NKIND] = {0, 0, 0};
    unsigned char parity[NKIND] = {0, 0, 0};
    BatchCase* d_cases = nullptr;
    KParams* d_params = nullptr;
    int* d_tile_case = nullptr;
    unsigned char* d_parity = nullptr;     // [NKIND]
    unsigned int* d_bar = nullptr;         // [NKIND][2]
    int* d_status = nullptr;
    // staged form: tensor maps of every case's two sets (maps[2 c + k] over pop[k], aux[k]
    // of the case table), and the groups whose cases all have them
    std::vector<StageMaps> maps;
    StageMaps* d_maps = nullptr;
    bool group_stageable[NKIND] = {false, false, false};
    // graph of the launches of one call length, for the mode it was captured in
    cudaGraphExec_t exec = nullptr;
    long graph_steps = -1;
    int graph_mode = -1;
    bool graph_ok = true;          // persistent form (a cooperative launch may refuse capture)
    bool graph_ok_step = true;     // per-step form
    cudaStream_t stream = nullptr, capture = nullptr;
    std::string err;
};

static int bfail(lbm_batch* b, int code, const std::string& msg)
{
    if (b) b->err = msg;
    else g_batch_create_error = msg;
    return code;
}

static int bcuda(lbm_batch* b, cudaError_t e, const char* where)
{
    cudaGetLastError();
    return bfail(b, LBM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define BATCH_TRY(b, call)                               \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return bcuda(b, e_, #call); \
    } while (0)

static void drop_graph(lbm_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_steps = -1;
    b->graph_mode = -1;
}

static void free_tables(lbm_batch* b)
{
    cudaFree(b->d_cases);
    cudaFree(b->d_params);
    cudaFree(b->d_tile_case);
    cudaFree(b->d_maps);
    b->d_cases = nullptr;
    b->d_params = nullptr;
    b->d_tile_case = nullptr;
    b->d_maps = nullptr;
}

// Tensor maps of case c's two sets as the case table holds them; false where the case
// cannot be staged (policy, N, nx) or the driver cannot encode them.
static bool encode_case_maps(lbm_batch* b, int c)
{
    const lbm_handle* h = b->h[c];
    const BatchCase& C = b->cases[c];
    return lbm_encode_stage_maps(h, C.pop[0], C.aux[0], &b->maps[2 * c]) &&
           lbm_encode_stage_maps(h, C.pop[1], C.aux[1], &b->maps[2 * c + 1]);
}

// Group membership, tile lists and the case table for the current plan; the sets of
// each case are laid out so that pop[parity of its group] is the handle's current set.
static int build_tables(lbm_batch* b)
{
    drop_graph(b);
    free_tables(b);
    const int nc = b->ncases;
    b->cases.assign(nc, BatchCase{});
    b->group.assign(nc, 0);
    std::vector<int> tiles[NKIND];
    for (int g = 0; g < NKIND; ++g) {
        b->group_tiles[g] = 0;
        b->group_cells[g] = 0;
    }
    for (int c = 0; c < nc; ++c) {
        const lbm_handle* h = b->h[c];
        const int g = b->class_kind[size_class((long long)h->nx * h->ny)];
        b->group[c] = g;
        BatchCase& C = b->cases[c];
        C.tiles_x = (h->nx + KIND_TX[g] - 1) / KIND_TX[g];
        C.tiles_y = (h->ny + KIND_TY[g] - 1) / KIND_TY[g];
        C.tile_kind = KIND_TILE[g];
        C.first_tile = b->group_tiles[g];
        const long long n = (long long)C.tiles_x * C.tiles_y;
        if ((long long)b->group_tiles[g] + n > (1LL << 30))
            return bfail(b, LBM_EINVAL, "a batch group exceeds 2^30 tiles");
        for (long long k = 0; k < n; ++k) tiles[g].push_back(c);
        b->group_tiles[g] += (int)n;
        b->group_cells[g] += (long long)h->nx * h->ny;
        const int p = b->parity[g];
        C.pop[p] = h->pop[h->cur];
        C.pop[p ^ 1] = h->pop[h->cur ^ 1];
        C.aux[p] = h->aux[h->cur];
        C.aux[p ^ 1] = h->aux[h->cur ^ 1];
    }
    std::vector<int> flat;
    for (int g = 0; g < NKIND; ++g) {
        b->group_first[g] = (int)flat.size();
        flat.insert(flat.end(), tiles[g].begin(), tiles[g].end());
    }
    std::vector<KParams> params(nc);
    for (int c = 0; c < nc; ++c) params[c] = b->h[c]->P;
    // the staged form: groups of 32x8 tiles whose every case has its tensor maps
    b->maps.assign(2 * (size_t)nc, StageMaps{});
    const bool stage_policy = (b->precision == LBM_FP16S || b->precision == LBM_BF16S) && (b->N == 2 || b->N == 3);
    for (int g = 0; g < NKIND; ++g) b->group_stageable[g] = stage_policy && KIND_TILE[g] == TILE_32x8 && b->group_tiles[g] > 0;
    for (int c = 0; c < nc; ++c)
        if (b->group_stageable[b->group[c]] && !encode_case_maps(b, c)) b->group_stageable[b->group[c]] = false;
    BATCH_TRY(b, cudaSetDevice(b->device));
    BATCH_TRY(b, cudaMalloc(&b->d_cases, nc * sizeof(BatchCase)));
    BATCH_TRY(b, cudaMalloc(&b->d_params, nc * sizeof(KParams)));
    BATCH_TRY(b, cudaMalloc(&b->d_tile_case, std::max<size_t>(flat.size(), 1) * sizeof(int)));
    BATCH_TRY(b, cudaMemcpy(b->d_cases, b->cases.data(), nc * sizeof(BatchCase), cudaMemcpyHostToDevice));
    BATCH_TRY(b, cudaMemcpy(b->d_params, params.data(), nc * sizeof(KParams), cudaMemcpyHostToDevice));
    if (!flat.empty())
        BATCH_TRY(b, cudaMemcpy(b->d_tile_case, flat.data(), flat.size() * sizeof(int), cudaMemcpyHostToDevice));
    BATCH_TRY(b, cudaMalloc(&b->d_maps, b->maps.size() * sizeof(StageMaps)));
    BATCH_TRY(b, cudaMemcpy(b->d_maps, b->maps.data(), b->maps.size() * sizeof(StageMaps), cudaMemcpyHostToDevice));
    return LBM_OK;
}

static BatchTable group_table(const lbm_batch* b, int g)
{
    BatchTable T{};
    T.total_tiles = b->group_tiles[g];
    T.cases = b->d_cases;
    T.params = b->d_params;
    T.tile_case = b->d_tile_case + b->group_first[g];
    T.parity = b->d_parity + g;
    T.bar = b->d_bar + 2 * g;
    T.status = b->d_status;
    T.spin_limit = b->wait_limit > 0 ? b->wait_limit : std::max(SPIN_MIN, b->group_cells[g] / 8);
    return T;
}

// A member handle stepped on its own (or given new fields) since the table was built:
// re-point its sets (and their tensor maps).  Returns true when the device tables must be
// refreshed.
static bool resync_cases(lbm_batch* b)
{
    bool dirty = false;
    for (int c = 0; c < b->ncases; ++c) {
        lbm_handle* h = b->h[c];
        BatchCase& C = b->cases[c];
        const int p = b->parity[b->group[c]];
        if (C.pop[p] != h->pop[h->cur]) {
            C.pop[p] = h->pop[h->cur];
            C.pop[p ^ 1] = h->pop[h->cur ^ 1];
            C.aux[p] = h->aux[h->cur];
            C.aux[p ^ 1] = h->aux[h->cur ^ 1];
            if (b->group_stageable[b->group[c]] && !encode_case_maps(b, c)) {
                b->group_stageable[b->group[c]] = false;
                drop_graph(b);   // its launches chose the staged kernel for this group
            }
            dirty = true;
        }
    }
    return dirty;
}

static int blocks_for(lbm_batch* b, int g, int* blocks)
{
    int per_sm = 0;
    const int kind = KIND_TILE[g];
    cudaError_t e = dispatch(b->N, b->precision, [&](auto n, auto pr) {
        return batch_blocks_per_sm<decltype(n)::value, decltype(pr)>(kind, &per_sm);
    });
    if (e != cudaSuccess) return bcuda(b, e, "occupancy of the persistent kernel");
    if (per_sm < 1) return bfail(b, LBM_ECUDA, "the persistent kernel does not fit on an SM");
    if (b->blocks_per_sm > 0) per_sm = std::min(per_sm, b->blocks_per_sm);
    *blocks = std::min(b->group_tiles[g], per_sm * b->sms);
    return LBM_OK;
}

// The persistent launches of one call (barrier reset + one cooperative launch per group).
static int enqueue_persistent(lbm_batch* b, int nsteps, cudaStream_t st)
{
    for (int g = 0; g < NKIND; ++g) {
        if (b->group_tiles[g] == 0) continue;
        int blocks = 0;
        int rc = blocks_for(b, g, &blocks);
        if (rc != LBM_OK) return rc;
        BATCH_TRY(b, cudaMemsetAsync(b->d_bar + 2 * g, 0, 2 * sizeof(unsigned int), st));
        const BatchTable T = group_table(b, g);
        const int kind = KIND_TILE[g];
        cudaError_t e = dispatch(b->N, b->precision, [&](auto n, auto pr) {
            return launch_batch_persistent<decltype(n)::value, decltype(pr)>(T, kind, nsteps, blocks, st);
        });
        if (e != cudaSuccess) return bcuda(b, e, "persistent batch launch");
    }
    return LBM_OK;
}

// Flip every group's parity byte on the device (the per-step form after an odd number of
// steps), so that a captured call replays correctly whatever the parity it starts from.
__global__ void flip_parity_kernel(unsigned char* parity, int n)
{
    if (threadIdx.x < n) parity[threadIdx.x] ^= 1;
}

// The per-step launches of one call: one launch per group and step (in the staged mode,
// the staged kernel for the groups that allow it).
static int enqueue_per_step(lbm_batch* b, int nsteps, cudaStream_t st)
{
    for (int s = 0; s < nsteps; ++s)
        for (int g = 0; g < NKIND; ++g) {
            if (b->group_tiles[g] == 0) continue;
            const BatchTable T = group_table(b, g);
            const int kind = KIND_TILE[g];
            const bool staged = b->mode == LBM_BATCH_STAGED && b->group_stageable[g];
            const StageMaps* maps = b->d_maps;
            cudaError_t e = dispatch(b->N, b->precision, [&](auto n, auto pr) {
                if (staged) return launch_batch_staged<decltype(n)::value, decltype(pr)>(T, maps, s, st);
                return launch_batch_step<decltype(n)::value, decltype(pr)>(T, kind, s, st);
            });
            if (e != cudaSuccess) return bcuda(b, e, "batch step launch");
        }
    if (nsteps & 1) {
        flip_parity_kernel<<<1, 32, 0, st>>>(b->d_parity, NKIND);
        BATCH_TRY(b, cudaGetLastError());
    }
    return LBM_OK;
}

// One call in the current mode, as a CUDA graph of that call length (captured on first
// use, replayed afterwards), or launched directly where capture is refused.
static int run_call(lbm_batch* b, int nsteps)
{
    const bool per_step = b->mode != LBM_BATCH_PERSISTENT;
    bool& ok = per_step ? b->graph_ok_step : b->graph_ok;
    auto enqueue = [&](cudaStream_t st) {
        return per_step ? enqueue_per_step(b, nsteps, st) : enqueue_persistent(b, nsteps, st);
    };
    if (ok && (b->exec == nullptr || b->graph_steps != nsteps || b->graph_mode != b->mode)) {
        drop_graph(b);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
        int rc = LBM_OK;
        if (e == cudaSuccess) {
            rc = enqueue(b->capture);
            e = cudaStreamEndCapture(b->capture, &graph);
        }
        if (rc != LBM_OK && e == cudaSuccess) {
            cudaGraphDestroy(graph);
            return rc;
        }
        if (e == cudaSuccess && rc == LBM_OK) e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess || rc != LBM_OK) {
            // capture refused (e.g. of a cooperative launch): run the launches directly
            cudaGetLastError();
            b->exec = nullptr;
            ok = false;
        } else {
            b->graph_steps = nsteps;
            b->graph_mode = b->mode;
        }
    }
    if (ok) {
        BATCH_TRY(b, cudaGraphLaunch(b->exec, b->stream));
        return LBM_OK;
    }
    return enqueue(b->stream);
}

// One call of nsteps steps (nsteps <= INT_MAX) with the current plan.
static int batch_advance(lbm_batch* b, int nsteps)
{
    if (nsteps == 0) return LBM_OK;
    if (resync_cases(b)) {
        BATCH_TRY(b, cudaMemcpyAsync(b->d_cases, b->cases.data(), b->ncases * sizeof(BatchCase),
                                     cudaMemcpyHostToDevice, b->stream));
        BATCH_TRY(b, cudaMemcpyAsync(b->d_maps, b->maps.data(), b->maps.size() * sizeof(StageMaps),
                                     cudaMemcpyHostToDevice, b->stream));
    }
    const int rc = run_call(b, nsteps);
    if (rc != LBM_OK) return rc;
    for (int g = 0; g < NKIND; ++g) b->parity[g] ^= (unsigned char)(nsteps & 1);
    for (int c = 0; c < b->ncases; ++c) {
        lbm_handle* h = b->h[c];
        const void* now = b->cases[c].pop[b->parity[b->group[c]]];
        h->cur = now == h->pop[0] ? 0 : 1;
        h->steps += nsteps;
    }
    return LBM_OK;
}

static lbm_batch_plan current_plan(const lbm_batch* b)
{
    lbm_batch_plan p{};
    p.mode = b->mode;
    p.blocks_per_sm = b->blocks_per_sm;
    for (int k = 0; k < LBM_BATCH_CLASSES; ++k) {
        p.tile[k][0] = KIND_TX[b->class_kind[k]];
        p.tile[k][1] = KIND_TY[b->class_kind[k]];
    }
    p.graph = (b->mode == LBM_BATCH_PERSISTENT ? b->graph_ok : b->graph_ok_step) ? 1 : 0;
    return p;
}

static int apply_plan(lbm_batch* b, const lbm_batch_plan* p)
{
    if (p->mode != LBM_BATCH_PERSISTENT && p->mode != LBM_BATCH_PER_STEP && p->mode != LBM_BATCH_STAGED)
        return bfail(b, LBM_EINVAL, "plan mode must be LBM_BATCH_PERSISTENT, LBM_BATCH_PER_STEP or LBM_BATCH_STAGED");
    if (p->blocks_per_sm < 0) return bfail(b, LBM_EINVAL, "blocks_per_sm must be >= 0");
    int kinds[LBM_BATCH_CLASSES];
    for (int k = 0; k < LBM_BATCH_CLASSES; ++k) {
        kinds[k] = kind_of_shape(p->tile[k][0], p->tile[k][1]);
        if (kinds[k] < 0) return bfail(b, LBM_EINVAL, "batch tile shapes are 32x8, 64x4 or 16x16");
        if (b->precision == LBM_DF64 && KIND_TILE[kinds[k]] != TILE_32x8)
            return bfail(b, LBM_EINVAL, "the LBM_DF64 policy is compiled for the 32x8 tile only");
    }
    bool retable = false;
    for (int k = 0; k < LBM_BATCH_CLASSES; ++k) retable = retable || kinds[k] != b->class_kind[k];
    if (p->blocks_per_sm != b->blocks_per_sm) drop_graph(b);
    b->mode = p->mode;
    b->blocks_per_sm = p->blocks_per_sm;
    for (int k = 0; k < LBM_BATCH_CLASSES; ++k) b->class_kind[k] = kinds[k];
    if (retable) {
        // the groups change: bring every group to parity 0 with the handles' sets
        BATCH_TRY(b, cudaStreamSynchronize(b->stream));
        for (int g = 0; g < NKIND; ++g) b->parity[g] = 0;
        BATCH_TRY(b, cudaMemset(b->d_parity, 0, NKIND));
        return build_tables(b);
    }
    return LBM_OK;
}

static void destroy_batch(lbm_batch* b)
{
    drop_graph(b);
    free_tables(b);
    cudaFree(b->d_parity);
    cudaFree(b->d_bar);
    cudaFree(b->d_status);
    if (b->capture) cudaStreamDestroy(b->capture);
    delete b;
}

extern "C" {

int lbm_batch_create(int ncases, lbm_handle* const* cases, lbm_batch** out)
{
    if (!out) return bfail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (ncases < 1 || !cases) return bfail(nullptr, LBM_EINVAL, "a batch needs ncases >= 1 handles");
    for (int c = 0; c < ncases; ++c) {
        if (!cases[c]) return bfail(nullptr, LBM_EINVAL, "NULL handle in the batch");
        for (int d = 0; d < c; ++d)
            if (cases[d] == cases[c]) return bfail(nullptr, LBM_EINVAL, "a handle appears twice in the batch");
        if (cases[c]->N != cases[0]->N) return bfail(nullptr, LBM_EINVAL, "batch cases must share N");
        if (cases[c]->precision != cases[0]->precision)
            return bfail(nullptr, LBM_EINVAL, "batch cases must share the precision policy");
        if (cases[c]->device != cases[0]->device) return bfail(nullptr, LBM_EINVAL, "batch cases must share a device");
        if (!cases[c]->ready) return bfail(nullptr, LBM_ESTATE, "a batch case has no fields (lbm_set_fields)");
    }
    lbm_batch* b = new (std::nothrow) lbm_batch;
    if (!b) return bfail(nullptr, LBM_ENOMEM, "host allocation failed");
    b->device = cases[0]->device;
    b->N = cases[0]->N;
    b->precision = cases[0]->precision;
    b->ncases = ncases;
    b->h.assign(cases, cases + ncases);
    cudaError_t e = cudaSetDevice(b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    int coop = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_parity, NKIND);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_bar, 2 * NKIND * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_parity, 0, NKIND);
    if (e == cudaSuccess) e = cudaMemset(b->d_bar, 0, 2 * NKIND * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        destroy_batch(b);
        return bfail(nullptr, LBM_ECUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
    }
    if (!coop) {
        destroy_batch(b);
        return bfail(nullptr, LBM_ECUDA, "the device does not support cooperative launches");
    }
    // the handles' pending work must be done before the tables read their state
    for (int c = 0; c < ncases; ++c) cudaStreamSynchronize(cases[c]->stream);
    const int rc = build_tables(b);
    if (rc != LBM_OK) {
        g_batch_create_error = b->err;
        destroy_batch(b);
        return rc;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_set_stream(lbm_batch* b, void* stream)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch");
    b->stream = (cudaStream_t)stream;
    return LBM_OK;
}

int lbm_batch_set_wait_limit(lbm_batch* b, long long polls)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch");
    if (polls < 0) return bfail(b, LBM_EINVAL, "polls must be >= 0");
    BATCH_TRY(b, cudaSetDevice(b->device));
    BATCH_TRY(b, cudaStreamSynchronize(b->stream));
    b->wait_limit = polls;
    drop_graph(b);  // the limit is a kernel argument captured in the graph
    return LBM_OK;
}

int lbm_batch_set_plan(lbm_batch* b, const lbm_batch_plan* plan)
{
    if (!b || !plan) return bfail(b, LBM_EINVAL, "NULL argument");
    BATCH_TRY(b, cudaSetDevice(b->device));
    return apply_plan(b, plan);
}

int lbm_batch_get_plan(const lbm_batch* b, lbm_batch_plan* plan)
{
    if (!b || !plan) return LBM_EINVAL;
    *plan = current_plan(b);
    return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, long nsteps)
{
    const lbm::TraceRange trace_range("lbm_batch_step");
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch");
    if (nsteps < 0) return bfail(b, LBM_EINVAL, "nsteps must be >= 0");
    for (int c = 0; c < b->ncases; ++c)
        if (!b->h[c]->ready) return bfail(b, LBM_ESTATE, "a batch case has no fields (lbm_set_fields)");
    BATCH_TRY(b, cudaSetDevice(b->device));
    const long chunk = 1L << 30;
    for (long done = 0; done < nsteps;) {
        const int n = (int)std::min(chunk, nsteps - done);
        const int rc = batch_advance(b, n);
        if (rc != LBM_OK) return rc;
        done += n;
    }
    return LBM_OK;
}

int lbm_batch_sync(lbm_batch* b)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch");
    BATCH_TRY(b, cudaSetDevice(b->device));
    BATCH_TRY(b, cudaStreamSynchronize(b->stream));
    int status = 0;
    BATCH_TRY(b, cudaMemcpy(&status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status != 0) {
        BATCH_TRY(b, cudaMemset(b->d_status, 0, sizeof(int)));
        BATCH_TRY(b, cudaMemset(b->d_bar, 0, 2 * NKIND * sizeof(unsigned int)));
        return bfail(b, LBM_ETIMEOUT,
                     "a bounded wait of a batch launch gave up (a grid barrier of the persistent form, or the "
                     "tensor copies of the staged form); the state is undefined");
    }
    return LBM_OK;
}

int lbm_batch_autotune(lbm_batch* b, int trial_steps, lbm_batch_plan* best)
{
    const lbm::TraceRange trace_range("lbm_batch_autotune");
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch");
    if (trial_steps < 1) return bfail(b, LBM_EINVAL, "trial_steps must be >= 1");
    BATCH_TRY(b, cudaSetDevice(b->device));
    int rc = lbm_batch_sync(b);
    if (rc != LBM_OK) return rc;
    for (int c = 0; c < b->ncases; ++c) BATCH_TRY(b, cudaStreamSynchronize(b->h[c]->stream));
    // snapshot of every case's current sets and step count
    size_t total = 0;
    for (lbm_handle* h : b->h) total += h->pop_bytes + h->aux_bytes;
    char* snap = nullptr;
    BATCH_TRY(b, cudaMalloc(&snap, total));
    std::vector<long long> steps(b->ncases);
    size_t off = 0;
    for (int c = 0; c < b->ncases; ++c) {
        lbm_handle* h = b->h[c];
        steps[c] = h->steps;
        cudaMemcpyAsync(snap + off, h->pop[h->cur], h->pop_bytes, cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(snap + off + h->pop_bytes, h->aux[h->cur], h->aux_bytes, cudaMemcpyDeviceToDevice, b->stream);
        off += h->pop_bytes + h->aux_bytes;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_plan = [&](const lbm_batch_plan& p, float* ms) -> int {
        int r = apply_plan(b, &p);
        if (r != LBM_OK) return r;
        r = lbm_batch_step(b, trial_steps);
        if (r != LBM_OK) return r;
        BATCH_TRY(b, cudaEventRecord(e0, b->stream));
        r = lbm_batch_step(b, trial_steps);
        if (r != LBM_OK) return r;
        BATCH_TRY(b, cudaEventRecord(e1, b->stream));
        r = lbm_batch_sync(b);
        if (r != LBM_OK) return r;
        BATCH_TRY(b, cudaEventElapsedTime(ms, e0, e1));
        return LBM_OK;
    };
    lbm_batch_plan cur = current_plan(b);
    float best_ms = 0.0f;
    rc = time_plan(cur, &best_ms);
    bool present[LBM_BATCH_CLASSES] = {false, false, false, false};
    for (lbm_handle* h : b->h) present[size_class((long long)h->nx * h->ny)] = true;
    // coordinate descent: launch mode, tile shape per size class, resident blocks per SM
    auto consider = [&](lbm_batch_plan p) -> int {
        float ms = 0.0f;
        const int r = time_plan(p, &ms);
        if (r != LBM_OK) return r;
        if (ms < best_ms) {
            best_ms = ms;
            cur = p;
        }
        return LBM_OK;
    };
    bool stageable = false;
    for (int g = 0; g < NKIND; ++g) stageable = stageable || b->group_stageable[g];
    for (int mode = LBM_BATCH_PERSISTENT; mode <= LBM_BATCH_STAGED && rc == LBM_OK; ++mode) {
        if (mode == cur.mode || (mode == LBM_BATCH_STAGED && !stageable)) continue;
        lbm_batch_plan p = cur;
        p.mode = mode;
        rc = consider(p);
    }
    for (int k = 0; k < LBM_BATCH_CLASSES && rc == LBM_OK; ++k) {
        if (!present[k] || b->precision == LBM_DF64) continue;   // double words: 32x8 only
        for (int kind = 0; kind < NKIND && rc == LBM_OK; ++kind) {
            if (KIND_TX[kind] == cur.tile[k][0] && KIND_TY[kind] == cur.tile[k][1]) continue;
            lbm_batch_plan p = cur;
            p.tile[k][0] = KIND_TX[kind];
            p.tile[k][1] = KIND_TY[kind];
            rc = consider(p);
        }
    }
    if (rc == LBM_OK && cur.mode == LBM_BATCH_PERSISTENT) {
        int per_sm = 0;  // resident limit of the 32x8 kernel (the shapes are alike)
        const cudaError_t eo = dispatch(b->N, b->precision, [&](auto n, auto pr) {
            return batch_blocks_per_sm<decltype(n)::value, decltype(pr)>(TILE_32x8, &per_sm);
        });
        if (eo != cudaSuccess) rc = bcuda(b, eo, "occupancy of the persistent kernel");
        for (int bps = per_sm - 1; bps >= 1 && rc == LBM_OK; --bps) {
            lbm_batch_plan p = cur;
            p.blocks_per_sm = bps;
            rc = consider(p);
        }
    }
    // the best plan, and the state as it was
    const int rc_plan = apply_plan(b, &cur);
    cudaStreamSynchronize(b->stream);
    off = 0;
    for (int c = 0; c < b->ncases; ++c) {
        lbm_handle* h = b->h[c];
        h->steps = steps[c];
        cudaMemcpyAsync(h->pop[h->cur], snap + off, h->pop_bytes, cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(h->aux[h->cur], snap + off + h->pop_bytes, h->aux_bytes, cudaMemcpyDeviceToDevice, b->stream);
        off += h->pop_bytes + h->aux_bytes;
    }
    cudaError_t e = cudaStreamSynchronize(b->stream);
    cudaFree(snap);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LBM_OK) return rc;
    if (rc_plan != LBM_OK) return rc_plan;
    if (e != cudaSuccess) return bcuda(b, e, "restoring the batch state");
    if (best) *best = current_plan(b);
    return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b)
{
    if (!b) return g_batch_create_error.c_str();
    return b->err.c_str();
}

void lbm_batch_destroy(lbm_batch* b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    destroy_batch(b);
}

}  // extern "C"
