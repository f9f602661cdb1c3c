// lbm_slab.cu -- one lattice split into bands of rows (y slabs), one handle per band,
// with the halo exchange that makes the bands step together exactly like the whole
// lattice (the fused step of Section 3 is a one-cell stencil in every field, so a cut
// between two bands is crossed by three populations per species and by the stencil
// inputs of one row).
//
// A slab handle holds rows [y0, y1) of the global lattice plus one ghost row beyond each
// side where another band continues the lattice.  Its own lattice runs the ordinary
// fused step over all its rows, ghost rows included; a cut side is declared an adiabatic,
// neutrally wetting wall, which touches only the ghost row beyond it.  After each step:
//   phase 1: the populations that crossed the cut -- the three directions with c_y
//            pointing across it, of every species, which the step pushed into the ghost
//            row -- go to the neighbour's boundary row, replacing what its own ghost row
//            pushed there (that ghost row's collision used a wall rule beyond it);
//   phase 2: the boundary row, now complete, goes to the neighbour's ghost row: its phase
//            field and enthalpy populations (all nine directions) and its lagged mdot' and
//            Q', which are what the next step's stencil ring recomputes phi_p, rho and psi
//            from.
// Messages are packed into contiguous buffers (pack / unpack kernels), so that the same
// calls serve a device-to-device copy between two handles of one GPU and a NCCL
// send / receive between GPUs.  Nothing here changes the step kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "../../include/lbm.h"
#include "lbm_handle.hpp"
#include "lbm_trace.hpp"
#include "lbm_launch.cuh"

using namespace lbm;

namespace lbm {
void set_handle_free_error(const char* msg);
}

namespace {

constexpr int SLAB_MAX_ROWS = 64;   // rows of one message: 9 (N + 1) + 2 <= 47 for N <= 4
constexpr int SLAB_NT = 256;

struct SlabRows {
    int n;                              // rows in the message
    int nx;
    long long src[SLAB_MAX_ROWS];       // byte offset of the row in its set
    long long msg[SLAB_MAX_ROWS];       // byte offset of the row in the message
    unsigned char aux[SLAB_MAX_ROWS];   // 0: population set, 1: lagged set
    unsigned char esz[SLAB_MAX_ROWS];   // element size: 2, 4 or 8 bytes
};

template <class T>
__device__ __forceinline__ void copy_row(const char* src, char* dst, int nx)
{
    const T* s = reinterpret_cast<const T*>(src);
    T* d = reinterpret_cast<T*>(dst);
    for (int x = threadIdx.x; x < nx; x += blockDim.x) d[x] = s[x];
}

// One block per row of the message.  pack: state -> message; unpack: message -> state.
template <bool PACK>
__global__ void __launch_bounds__(SLAB_NT) slab_copy_kernel(const SlabRows L, char* pop, char* aux, char* msg)
{
    const int r = blockIdx.x;
    char* state = (L.aux[r] ? aux : pop) + L.src[r];
    char* m = msg + L.msg[r];
    const char* from = PACK ? state : m;
    char* to = PACK ? m : state;
    switch (L.esz[r]) {
        case 2: copy_row<unsigned short>(from, to, L.nx); break;
        case 4: copy_row<unsigned int>(from, to, L.nx); break;
        default: copy_row<unsigned long long>(from, to, L.nx); break;
    }
}

int sfail(lbm_handle* h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    else set_handle_free_error(msg.c_str());
    return code;
}

// Element sizes (rest, moving, lagged) of the handle's precision policy.
void elem_sizes(const lbm_handle* h, int& er, int& em, int& ea)
{
    dispatch(h->N, h->precision, [&](auto, auto pr) {
        using Pr = decltype(pr);
        er = (int)sizeof(typename Pr::TR);
        em = (int)sizeof(typename Pr::TM);
        ea = (int)sizeof(typename Pr::TA);
        return 0;
    });
}

// Rows of one message.  side 2 = y-min, 3 = y-max of the handle; `pack` selects the rows
// the handle sends on that side, else the rows it receives there.
bool message_rows(const lbm_handle* h, int side, int phase, bool pack, SlabRows& L, long long* bytes)
{
    const int N = h->N, nx = h->nx, ny = h->ny;
    const long long S = h->P.S;
    int er, em, ea;
    elem_sizes(h, er, em, ea);
    const long long rest0 = 0, move0 = (long long)(N + 2) * S * er;
    // row of the state the message touches
    int row;
    if (phase == 1) row = pack ? (side == 2 ? 0 : ny - 1) : (side == 2 ? 1 : ny - 2);
    else row = pack ? (side == 2 ? 1 : ny - 2) : (side == 2 ? 0 : ny - 1);
    L = SlabRows{};
    L.nx = nx;
    long long off = 0;
    auto add = [&](bool aux, long long plane_byte0, int esz) {
        if (L.n >= SLAB_MAX_ROWS) {  // refused below; never written past the table
            L.n = SLAB_MAX_ROWS + 1;
            return;
        }
        const int r = L.n++;
        L.aux[r] = aux ? 1 : 0;
        L.esz[r] = (unsigned char)esz;
        L.src[r] = plane_byte0 + (long long)row * nx * esz;
        L.msg[r] = off;
        off += ((long long)nx * esz + 15) / 16 * 16;  // rows start on 16-byte boundaries
    };
    if (phase == 1) {
        // directions that cross the cut: upward (2, 5, 6) through the y-max side of the
        // sender, downward (4, 7, 8) through its y-min side; the receiver gets them on its
        // opposite side
        const bool up = pack ? side == 3 : side == 2;
        const int dirs[3] = {up ? 2 : 4, up ? 5 : 7, up ? 6 : 8};
        for (int s = 0; s < N + 2; ++s)
            for (int d = 0; d < 3; ++d) add(false, move0 + (long long)(s * 8 + dirs[d] - 1) * S * em, em);
    } else {
        // phase-field and enthalpy populations (species 1 .. N + 1), all nine directions,
        // and the lagged mdot' and Q' (planes 0 and 1 of the lagged set)
        for (int s = 1; s < N + 2; ++s) {
            add(false, rest0 + (long long)s * S * er, er);
            for (int i = 1; i < 9; ++i) add(false, move0 + (long long)(s * 8 + i - 1) * S * em, em);
        }
        add(true, 0, ea);
        add(true, S * ea, ea);
    }
    if (L.n > SLAB_MAX_ROWS) return false;
    *bytes = off;
    return true;
}

// The inner tile rows of a slab handle: those whose rows and one-cell ring stay clear of
// the band's first two and last two rows (the ghost and boundary rows its halo exchange
// writes); the edge part is the other tile rows.
TileRows slab_rows(const lbm_handle* h, int part)
{
    int tx = 32, ty = 8;
    tile_dims(h->tile, tx, ty);
    const int tiles_y = (h->ny + ty - 1) / ty;
    const int lo = 1;                                              // rows >= ty, ring >= ty - 1 >= 2
    int hi = h->ny - 3 - ty >= 0 ? (h->ny - 3 - ty) / ty + 1 : 0;  // last row + 1 (ring) <= ny - 3
    hi = std::min(std::max(hi, lo), tiles_y);
    return TileRows{part == LBM_SLAB_INNER ? ROWS_INNER : ROWS_EDGE, lo, hi};
}

bool slab_side_ok(const lbm_handle* h, int side)
{
    return h->slab && (side == 2 ? h->slab_ghost[0] : side == 3 ? h->slab_ghost[1] : 0);
}

}  // namespace

extern "C" {

int lbm_slab_create(const lbm_grid* grid, int y0, int y1, int N, const lbm_phase* phases, const lbm_thermal* thermal,
                    const lbm_bc* bc, const lbm_numerics* numerics, lbm_handle** out)
{
    if (!out) return sfail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid || !bc) return sfail(nullptr, LBM_EINVAL, "NULL argument");
    if (!(0 <= y0 && y0 < y1 && y1 <= grid->ny)) return sfail(nullptr, LBM_EINVAL, "need 0 <= y0 < y1 <= ny");
    const bool yper = bc->kind[2] == LBM_BC_PERIODIC;
    const int gb = (y0 > 0 || yper) ? 1 : 0;          // ghost row below
    const int ga = (y1 < grid->ny || yper) ? 1 : 0;   // ghost row above
    if (!gb && !ga) return sfail(nullptr, LBM_EINVAL, "the band covers the whole lattice: use lbm_create");
    const int owned = y1 - y0;
    if (owned + gb + ga < 3) return sfail(nullptr, LBM_EINVAL, "a slab needs >= 3 rows with its ghost rows");
    lbm_grid g{grid->nx, owned + gb + ga};
    lbm_bc b = *bc;
    for (int side = 2; side < 4; ++side) {
        const bool cut = side == 2 ? gb : ga;
        if (!cut) continue;
        b.kind[side] = LBM_BC_WALL;
        b.tkind[side] = LBM_T_ADIABATIC;
        b.T_wall[side] = 0.0;
        for (int k = 0; k < LBM_MAXN * LBM_MAXN; ++k) b.wet_cos[side][k] = 0.0;
    }
    lbm_handle* h = nullptr;
    const int rc = lbm_create(&g, N, phases, thermal, &b, numerics, &h);
    if (rc != LBM_OK) return rc;
    h->slab = true;
    h->slab_ghost[0] = gb;
    h->slab_ghost[1] = ga;
    h->slab_y0 = y0;
    *out = h;
    return LBM_OK;
}

int lbm_slab_geometry(const lbm_handle* h, int* out4)
{
    if (!h || !out4) return LBM_EINVAL;
    if (!h->slab) return sfail(const_cast<lbm_handle*>(h), LBM_EINVAL, "not a slab handle");
    out4[0] = h->ny;
    out4[1] = h->slab_ghost[0];
    out4[2] = h->slab_ghost[1];
    out4[3] = h->slab_y0;
    return LBM_OK;
}

long long lbm_slab_message_bytes(const lbm_handle* h, int phase)
{
    if (!h || !h->slab || (phase != 1 && phase != 2)) return -1;
    SlabRows L;
    long long bytes = 0;
    if (!message_rows(h, 3, phase, true, L, &bytes)) return -1;
    return bytes;
}

static int slab_copy(lbm_handle* h, int side, int phase, bool pack, void* msg)
{
    const lbm::TraceRange trace_range(pack ? "lbm_slab_pack" : "lbm_slab_unpack");
    if (!h) return sfail(nullptr, LBM_EINVAL, "NULL handle");
    if (!msg) return sfail(h, LBM_EINVAL, "NULL message buffer");
    if (!h->ready) return sfail(h, LBM_ESTATE, "lbm_set_fields has not been called");
    if (phase != 1 && phase != 2) return sfail(h, LBM_EINVAL, "phase must be 1 or 2");
    if (!slab_side_ok(h, side)) return sfail(h, LBM_EINVAL, "side must be a cut side (2 = y-min, 3 = y-max) of a slab");
    SlabRows L;
    long long bytes = 0;
    if (!message_rows(h, side, phase, pack, L, &bytes)) return sfail(h, LBM_EINVAL, "message has too many rows");
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) {
        char* pop = (char*)h->pop[h->cur];
        char* aux = (char*)h->aux[h->cur];
        if (pack) slab_copy_kernel<true><<<L.n, SLAB_NT, 0, h->stream>>>(L, pop, aux, (char*)msg);
        else slab_copy_kernel<false><<<L.n, SLAB_NT, 0, h->stream>>>(L, pop, aux, (char*)msg);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return sfail(h, LBM_ECUDA, std::string("slab copy kernel: ") + cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_slab_pack(lbm_handle* h, int side, int phase, void* msg) { return slab_copy(h, side, phase, true, msg); }

int lbm_slab_unpack(lbm_handle* h, int side, int phase, const void* msg)
{
    return slab_copy(h, side, phase, false, const_cast<void*>(msg));
}

int lbm_slab_step_part(lbm_handle* h, int part)
{
    const lbm::TraceRange trace_range(part == LBM_SLAB_INNER ? "lbm_slab_step_part inner" : "lbm_slab_step_part edge");
    if (!h) return sfail(nullptr, LBM_EINVAL, "NULL handle");
    if (!h->slab) return sfail(h, LBM_EINVAL, "not a slab handle");
    if (!h->ready) return sfail(h, LBM_ESTATE, "lbm_set_fields has not been called");
    if (part != LBM_SLAB_INNER && part != LBM_SLAB_EDGE)
        return sfail(h, LBM_EINVAL, "part must be LBM_SLAB_INNER or LBM_SLAB_EDGE");
    if (part == LBM_SLAB_INNER && h->slab_inner_pending)
        return sfail(h, LBM_ESTATE, "the inner rows of this step were stepped already: step the edge rows");
    if (part == LBM_SLAB_EDGE && !h->slab_inner_pending)
        return sfail(h, LBM_ESTATE, "step the inner rows of this step first");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return sfail(h, LBM_ECUDA, cudaGetErrorString(e));
    const int a = h->cur, b = a ^ 1;
    const TileRows rows = slab_rows(h, part);
    e = dispatch(h->N, h->precision, [&](auto n, auto pr) {
        if (h->staged)
            return launch_staged<decltype(n)::value, decltype(pr)>(h->P, h->stage_maps[a], h->pop[a], h->pop[b],
                                                                   h->aux[a], h->aux[b], h->stage_status, h->stream,
                                                                   rows);
        return launch_step<decltype(n)::value, decltype(pr)>(h->P, h->pop[a], h->pop[b], h->aux[a], h->aux[b],
                                                             h->tile, h->stream, rows);
    });
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sfail(h, LBM_ECUDA, std::string("step kernel: ") + cudaGetErrorString(e));
    }
    if (part == LBM_SLAB_INNER) {
        h->slab_inner_pending = true;
        return LBM_OK;
    }
    h->slab_inner_pending = false;
    h->cur = b;
    h->steps++;
    return LBM_OK;
}

int lbm_slab_sums(lbm_handle* h, double* out)
{
    const lbm::TraceRange trace_range("lbm_slab_sums");
    if (!h || !out) return sfail(h, LBM_EINVAL, "NULL argument");
    if (!h->slab) return sfail(h, LBM_EINVAL, "not a slab handle");
    if (!h->ready) return sfail(h, LBM_ESTATE, "lbm_set_fields has not been called");
    const int N = h->N;
    // the diagnostics of lbm_get_diagnostics over the band's own rows
    const long long c0 = (long long)h->slab_ghost[0] * h->nx;
    const long long cells = (long long)(h->ny - h->slab_ghost[0] - h->slab_ghost[1]) * h->nx;
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess)
        e = dispatch(N, h->precision, [&](auto n, auto pr) {
            return launch_diag<decltype(n)::value, decltype(pr)>(h->P, h->pop[h->cur], h->aux[h->cur], h->diag_partial,
                                                                 h->diag_out, h->stream, c0, cells);
        });
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, h->diag_out, (2 * N + 2) * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return sfail(h, LBM_ECUDA, std::string("slab sums: ") + cudaGetErrorString(e));
    return LBM_OK;
}

}  // extern "C"
