// lbm_staged.cuh -- the fused step with its inputs staged in shared memory by the
// tensor-memory accelerator (TMA), for the 16-bit storage policies.
//
// In the one-cell step (lbm_step.cuh) every thread loads its cell's populations and
// lagged values, and the ring cells' phase-field and enthalpy populations, with ~40
// scalar global loads and their address arithmetic, waits, computes, then loads the flow
// populations and waits again.  Here thread 0 of a block copies everything the tile needs
// with six tensor copies that complete on one mbarrier:
//   A  the eight moving planes of f, own cells          [8][8][32]
//   B  the moving planes of g_p and h, tile and ring     [8(N+1)][10][32 + 2 pad]
//   C  the rest plane of f, own cells                    [1][8][32]
//   D  the rest planes of g_p and h, tile and ring        [N+1][10][32 + 2 pad]
//   E  the lagged mdot' and Q', tile and ring             [2][10][32 + 2 pad]
//   F  the other lagged planes, own cells                 [1 + 2N][8][32]
// and the tile is computed from shared memory: one memory latency per block instead of
// two, and shared-memory reads instead of global loads.  A box that includes the ring
// starts pad = 16 / element-size cells left of the tile, so its first x coordinate is on a
// 16-byte boundary (the tile's x0 is a multiple of 32), and is a multiple of 16 bytes
// wide.  Every tile is staged this way: positions of a box beyond the lattice (left of
// x = 0, below y = 0, past the right or top side) are filled with zeros by the copy and
// are either never read (beyond a wall or an outflow side: the ghost rule replaces them)
// or, across a periodic side, read again from the cells they wrap to (wrap_item).  The
// arithmetic is step_tile_l of the one-cell step with a loader that reads the stage, so
// every cell is computed exactly as the one-cell step computes it (the two forms agree
// bit for bit), and that code exists once in the kernel (a second copy for the tiles at
// the sides, reading global memory, overflowed the instruction cache).  The tiles at the
// sides run first (ring_first_tile).  Every wait on the mbarrier is bounded: a wait that
// gives up sets a status word (reported as LBM_ETIMEOUT), waits (bounded) for the copies
// in flight and leaves.
#pragma once

#include "lbm_launch.cuh"
#include "lbm_step.cuh"

namespace lbm {

constexpr int STAGE_TX = 32, STAGE_TY = 8, STAGE_NT = STAGE_TX * STAGE_TY;
// Blocks per SM the staged kernels are compiled for: the stage of N = 2 (47 KB) leaves
// room for four, that of N = 3 (60 KB) for three.
template <int N>
__host__ __device__ constexpr int stage_blocks_per_sm() { return N == 2 ? 4 : 3; }
constexpr long long STAGE_WAIT_LIMIT = 1LL << 22;   // try_wait polls of one mbarrier wait

__host__ __device__ constexpr int stage_round(int b) { return (b + 127) / 128 * 128; }

// Layout of one staged tile in shared memory (bytes; every box on a 128-byte boundary).
template <int N, class Pr>
struct StageLayout {
    static constexpr int EM = sizeof(typename Pr::TM), ER = sizeof(typename Pr::TR), EA = sizeof(typename Pr::TA);
    static constexpr int PM = 16 / EM, PR = 16 / ER, PA = 16 / EA;          // pads (cells)
    static constexpr int WM = STAGE_TX + 2 * PM, WR = STAGE_TX + 2 * PR, WA = STAGE_TX + 2 * PA;
    static constexpr int H = STAGE_TY + 2;
    static constexpr int A = 8 * STAGE_TY * STAGE_TX * EM;
    static constexpr int B = 8 * (N + 1) * H * WM * EM;
    static constexpr int C = STAGE_TY * STAGE_TX * ER;
    static constexpr int D = (N + 1) * H * WR * ER;
    static constexpr int E = 2 * H * WA * EA;
    static constexpr int F = (1 + 2 * N) * STAGE_TY * STAGE_TX * EA;
    static constexpr int OA = 0, OB = OA + stage_round(A), OC = OB + stage_round(B), OD = OC + stage_round(C),
                         OE = OD + stage_round(D), OF = OE + stage_round(E), BYTES = OF + stage_round(F);
    static constexpr int TX_BYTES = A + B + C + D + E + F;   // what the six copies deliver
    // dynamic shared memory of a block: the stage, the mbarrier, the one-cell step's tile
    // (TOTAL has 128 bytes of slack: the kernel aligns its base to 128 bytes)
    static constexpr int SMEM_ONE = tile_smem_elems<N, STAGE_TX, STAGE_TY, Pr>() * (int)sizeof(typename Pr::R);
    static constexpr int OBAR = BYTES, OONE = OBAR + 128, TOTAL = OONE + stage_round(SMEM_ONE) + 128;
};

// Reads of one staged tile; a cell is (lx, ly) of the tile with its ring.
template <int N, class Pr>
struct StagedLoader {
    using R = typename Pr::R;
    using TR = typename Pr::TR;
    using TM = typename Pr::TM;
    using TA = typename Pr::TA;
    using Lay = StageLayout<N, Pr>;
    using Cell = int;   // ly * 64 + lx
    static constexpr bool GLOBAL = false;
    const KParams& P;
    const unsigned char* st;   // the stage
    int x0, y0;                // the tile's first cell
    bool edge;                 // the ring reaches a side of the lattice
    // A position beyond a side that is not periodic is no cell (the ghost rule fills it);
    // every other position, across a periodic side too, was staged as a cell.
    __device__ __forceinline__ bool locate(int lx, int ly, Cell& cell) const
    {
        cell = ly * 64 + lx;
        if (!edge) return true;
        const int gx = x0 + lx - 1, gy = y0 + ly - 1;
        const bool bx = P.bc[0] != PERIODIC && (gx < 0 || gx >= P.nx);
        const bool by = P.bc[2] != PERIODIC && (gy < 0 || gy >= P.ny);
        return !(bx || by);
    }
    __device__ __forceinline__ Cell own(int, int, int tx, int ty) const { return (ty + 1) * 64 + tx + 1; }
    template <int KIND>
    __device__ __forceinline__ R pop(int s, int i, Cell c, int) const
    {
        const int lx = c & 63, ly = c >> 6;
        if (s == 0) {  // the flow populations: own cells only
            const int o = (ly - 1) * STAGE_TX + (lx - 1);
            if (i == 0) return (R) reinterpret_cast<const TR*>(st + Lay::OC)[o];
            return dequant<Pr, KIND>(P, reinterpret_cast<const TM*>(st + Lay::OA)[(i - 1) * STAGE_TY * STAGE_TX + o], i);
        }
        if (i == 0) return (R) reinterpret_cast<const TR*>(st + Lay::OD)[((s - 1) * Lay::H + ly) * Lay::WR + lx - 1 + Lay::PR];
        const int plane = (s - 1) * 8 + i - 1;
        return dequant<Pr, KIND>(P, reinterpret_cast<const TM*>(st + Lay::OB)[(plane * Lay::H + ly) * Lay::WM + lx - 1 + Lay::PM],
                                 i);
    }
    template <int KIND>
    __device__ __forceinline__ R pop_late(int s, int i, Cell c, int site) const
    {
        return pop<KIND>(s, i, c, site);
    }
    __device__ __forceinline__ R aux(int a, Cell c, int) const
    {
        const int lx = c & 63, ly = c >> 6;
        if (a < 2) return (R) reinterpret_cast<const TA*>(st + Lay::OE)[(a * Lay::H + ly) * Lay::WA + lx - 1 + Lay::PA];
        return (R) reinterpret_cast<const TA*>(st + Lay::OF)[((a - 2) * STAGE_TY + ly - 1) * STAGE_TX + lx - 1];
    }
};

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// Bounded wait for the phase `parity` of an mbarrier to complete.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity)
{
    for (long long k = 0; k < STAGE_WAIT_LIMIT; ++k)
        if (mbar_try(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, int x, int y, int z, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// The tile's one-cell ring lies inside the lattice: no position of the tile with its
// ring is beyond a side or across a periodic one.
__device__ __forceinline__ bool ring_inside(const KParams& P, int x0, int y0)
{
    return x0 >= 1 && x0 + STAGE_TX <= P.nx - 1 && y0 >= 1 && y0 + STAGE_TY <= P.ny - 1;
}

// Thread 0: the six copies of tile (bx, by) into `stage`, completing on `bar`.
template <int N, class Pr>
__device__ __forceinline__ void stage_issue(const StageMaps& M, unsigned char* stage, unsigned bar, int bx, int by)
{
    using Lay = StageLayout<N, Pr>;
    const int x0 = bx * STAGE_TX, y0 = by * STAGE_TY;
    mbar_expect(bar, (unsigned)Lay::TX_BYTES);
    const unsigned s = smem_addr(stage);
    tma_load_3d(s + Lay::OA, &M.m[0], x0, y0, 0, bar);
    tma_load_3d(s + Lay::OB, &M.m[1], x0 - Lay::PM, y0 - 1, 8, bar);
    tma_load_3d(s + Lay::OC, &M.m[2], x0, y0, 0, bar);
    tma_load_3d(s + Lay::OD, &M.m[3], x0 - Lay::PR, y0 - 1, 1, bar);
    tma_load_3d(s + Lay::OE, &M.m[4], x0 - Lay::PA, y0 - 1, 0, bar);
    tma_load_3d(s + Lay::OF, &M.m[5], x0, y0, 2, bar);
}

// Positions of the ring boxes (B, D, E) that lie across a periodic side: the tensor
// copies fill them with zeros (the box starts left of or below the lattice, or runs past
// its right or top side), so they are read again, with plain loads, from the cells they
// wrap to.  Positions beyond a side that is not periodic keep the zeros (the ghost rule
// replaces them); the own-cell boxes (A, C, F) are read only at cells of the lattice.
// The work is one load per (position, plane) item: the wrapped columns (10 positions
// each) and rows (34 each) of the tile with its ring, times the 8 (N + 1) + (N + 1) + 2
// planes; a corner in both lists is read twice, to the same value.  The first items of
// each thread are loaded before the wait for the tensor copies, so that their latency
// overlaps the copies', and stored once the copies have landed.
struct WrapGeom {
    int nL, cR, nB, rT, ncol, items;
};

template <int N, class Pr>
__device__ __forceinline__ WrapGeom wrap_geom(const KParams& P, int x0, int y0)
{
    using Lay = StageLayout<N, Pr>;
    constexpr int RW = STAGE_TX + 2, PLANES = 9 * (N + 1) + 2;
    const bool xper = P.bc[0] == PERIODIC, yper = P.bc[2] == PERIODIC;
    WrapGeom G;
    // wrapped columns: lx = 0 (x0 = 0) and lx = cR .. RW - 1 (past the right side);
    // wrapped rows: ly = 0 (y0 = 0) and ly = rT .. H - 1 (past the top side)
    G.nL = xper && x0 == 0 ? 1 : 0;
    G.cR = P.nx - x0 + 1;
    const int nR = xper && G.cR < RW ? RW - G.cR : 0;
    G.nB = yper && y0 == 0 ? 1 : 0;
    G.rT = P.ny - y0 + 1;
    const int nT = yper && G.rT < Lay::H ? Lay::H - G.rT : 0;
    G.ncol = (G.nL + nR) * Lay::H;
    G.items = (G.ncol + (G.nB + nT) * RW) * PLANES;
    return G;
}

template <class T>
__device__ __forceinline__ unsigned raw_bits(T v)
{
    static_assert(sizeof(T) == 2 || sizeof(T) == 4, "staged elements are 2 or 4 bytes");
    if constexpr (sizeof(T) == 2) {
        unsigned short u;
        memcpy(&u, &v, 2);
        return u;
    } else {
        unsigned u;
        memcpy(&u, &v, 4);
        return u;
    }
}

// Item e: its byte offset in the stage and the bits of its value; false for a position
// beyond a side that is not periodic (nothing to write).
template <int N, class Pr>
__device__ __forceinline__ bool wrap_item(const KParams& P, const PopView<Pr>& v, const typename Pr::TA* __restrict__ ain,
                                          int x0, int y0, const WrapGeom& G, int e, unsigned& off, unsigned& bits)
{
    using Lay = StageLayout<N, Pr>;
    using TR = typename Pr::TR;
    using TM = typename Pr::TM;
    using TA = typename Pr::TA;
    constexpr int RW = STAGE_TX + 2, PLANES = 9 * (N + 1) + 2;
    const int nx = P.nx, ny = P.ny;
    const long long S = P.S;
    const int pl = e % PLANES, pos = e / PLANES;
    int lx, ly;
    if (pos < G.ncol) {
        const int k = pos / Lay::H;
        ly = pos % Lay::H;
        lx = k < G.nL ? 0 : G.cR + (k - G.nL);
    } else {
        const int k = (pos - G.ncol) / RW;
        lx = (pos - G.ncol) % RW;
        ly = k < G.nB ? 0 : G.rT + (k - G.nB);
    }
    int gx = x0 + lx - 1, gy = y0 + ly - 1;
    const bool xout = gx < 0 || gx >= nx, yout = gy < 0 || gy >= ny;
    if ((xout && P.bc[0] != PERIODIC) || (yout && P.bc[2] != PERIODIC)) return false;
    if (xout) gx = wrap_index(gx, nx);
    if (yout) gy = wrap_index(gy, ny);
    const long long c = (long long)gy * nx + gx;
    if (pl < 8 * (N + 1)) {
        off = Lay::OB + ((pl * Lay::H + ly) * Lay::WM + lx - 1 + Lay::PM) * (unsigned)sizeof(TM);
        bits = raw_bits(LBM_LD(P, v.move, (8 + pl) * S + c, P.move_elems, 43));
    } else if (pl < 9 * (N + 1)) {
        const int s = pl - 8 * (N + 1);
        off = Lay::OD + ((s * Lay::H + ly) * Lay::WR + lx - 1 + Lay::PR) * (unsigned)sizeof(TR);
        bits = raw_bits(LBM_LD(P, v.rest, (1 + s) * S + c, P.rest_elems, 44));
    } else {
        const int a = pl - 9 * (N + 1);
        off = Lay::OE + ((a * Lay::H + ly) * Lay::WA + lx - 1 + Lay::PA) * (unsigned)sizeof(TA);
        bits = raw_bits(LBM_LD(P, ain, a * S + c, P.aux_elems, 45));
    }
    return true;
}

template <int N, class Pr>
__device__ __forceinline__ void wrap_store(unsigned char* st, unsigned off, unsigned bits)
{
    using Lay = StageLayout<N, Pr>;
    static_assert(sizeof(typename Pr::TR) == 4 && sizeof(typename Pr::TA) == 4, "the ring boxes D, E hold 4-byte values");
    if (off < (unsigned)Lay::OC) {
        if constexpr (sizeof(typename Pr::TM) == 2) *reinterpret_cast<unsigned short*>(st + off) = (unsigned short)bits;
        else *reinterpret_cast<unsigned*>(st + off) = bits;
    } else {
        *reinterpret_cast<unsigned*>(st + off) = bits;
    }
}

// The staged step of tile (bx, by), run by a block of STAGE_NT threads whose dynamic
// shared memory `dyn_raw` holds StageLayout<N, Pr>::TOTAL bytes, in two parts:
//   staged_tile_issue: thread 0 initialises the mbarrier and issues the tile's six tensor
//     copies (the caller may do other work, such as loading the parameter block, while
//     they are in flight);
//   staged_tile_finish (P must be complete and visible to every thread on entry: it is
//     read before the first block barrier): every thread waits for the copies (a block
//     barrier first, so the mbarrier is initialised before anyone waits on it), a tile at
//     a periodic side then writes its wrapped positions over the copies' zeros
//     (wrap_item), and the tile is computed from the stage.  Every tile is computed this
//     way, so the step's arithmetic is compiled once.
__device__ __forceinline__ unsigned char* stage_base(unsigned char* dyn_raw)
{
    return dyn_raw + ((128u - (smem_addr(dyn_raw) & 127u)) & 127u);
}

template <int N, class Pr>
__device__ __forceinline__ void staged_tile_issue(const StageMaps& M, int bx, int by, unsigned char* dyn_raw)
{
    using Lay = StageLayout<N, Pr>;
    unsigned char* dyn = stage_base(dyn_raw);
    if (threadIdx.x == 0) {
        const unsigned bar = smem_addr(dyn + Lay::OBAR);
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        stage_issue<N, Pr>(M, dyn, bar, bx, by);
    }
}

template <int N, class Pr>
__device__ __forceinline__ void staged_tile_finish(const KParams& P, const void* __restrict__ pin_base,
                                                   void* __restrict__ pout_base,
                                                   const typename Pr::TA* __restrict__ ain,
                                                   typename Pr::TA* __restrict__ aout, int* __restrict__ status,
                                                   int bx, int by, unsigned char* dyn_raw)
{
    using Lay = StageLayout<N, Pr>;
    using R = typename Pr::R;
    unsigned char* dyn = stage_base(dyn_raw);
    R* one = reinterpret_cast<R*>(dyn + Lay::OONE);
    const int x0 = bx * STAGE_TX, y0 = by * STAGE_TY;
    const unsigned bar = smem_addr(dyn + Lay::OBAR);
    const bool wraps = (P.bc[0] == PERIODIC && (x0 == 0 || x0 + STAGE_TX >= P.nx)) ||
                       (P.bc[2] == PERIODIC && (y0 == 0 || y0 + STAGE_TY >= P.ny));
    WrapGeom G{};
    unsigned off0 = 0, bits0 = 0, off1 = 0, bits1 = 0;
    bool has0 = false, has1 = false;
    if (wraps) {   // the first two items of this thread, loaded while the copies are in flight
        const PopView<Pr> v = pop_view<Pr>(P, pin_base);
        G = wrap_geom<N, Pr>(P, x0, y0);
        const int e0 = threadIdx.x, e1 = threadIdx.x + STAGE_NT;
        if (e0 < G.items) has0 = wrap_item<N, Pr>(P, v, ain, x0, y0, G, e0, off0, bits0);
        if (e1 < G.items) has1 = wrap_item<N, Pr>(P, v, ain, x0, y0, G, e1, off1, bits1);
    }
    __syncthreads();   // the mbarrier is initialised before anyone waits on it
    const bool ok = mbar_wait(bar, 0);
    if (!__syncthreads_and(ok)) {
        // give up: report, let the copy still in flight land, leave
        if (threadIdx.x == 0) {
            atomicExch(status, 1);
            mbar_wait(bar, 0);
        }
        __syncthreads();
        return;
    }
    const bool inside = ring_inside(P, x0, y0);
    if (wraps) {   // the wrapped positions over the copies' zeros
        if (has0) wrap_store<N, Pr>(dyn, off0, bits0);
        if (has1) wrap_store<N, Pr>(dyn, off1, bits1);
        const PopView<Pr> v = pop_view<Pr>(P, pin_base);
        for (int e = threadIdx.x + 2 * STAGE_NT; e < G.items; e += STAGE_NT) {
            unsigned off, bits;
            if (wrap_item<N, Pr>(P, v, ain, x0, y0, G, e, off, bits)) wrap_store<N, Pr>(dyn, off, bits);
        }
        __syncthreads();
    }
    const StagedLoader<N, Pr> ld{P, dyn, x0, y0, !inside};
    step_tile_l<N, STAGE_TX, STAGE_TY, true, Pr>(P, ld, pout_base, aout, ExportPtrs{}, bx, by, one);
}

// One step of one lattice: one block per tile (a one-dimensional grid of all tiles, four
// blocks per SM for N = 2 and three for N = 3, the tiles at the sides first).
template <int N, class Pr>
__global__ void __launch_bounds__(STAGE_NT, stage_blocks_per_sm<N>())
staged_tile_kernel(const KParams P, const __grid_constant__ StageMaps M, const void* __restrict__ pin_base,
                   void* __restrict__ pout_base, const typename Pr::TA* __restrict__ ain,
                   typename Pr::TA* __restrict__ aout, int* __restrict__ status, TileRows rows)
{
    extern __shared__ __align__(128) unsigned char dyn_raw[];
    int bx, by;
    tile_of_block(blockIdx.x, (P.nx + STAGE_TX - 1) / STAGE_TX, (P.ny + STAGE_TY - 1) / STAGE_TY, rows, bx, by);
    staged_tile_issue<N, Pr>(M, bx, by, dyn_raw);
    staged_tile_finish<N, Pr>(P, pin_base, pout_base, ain, aout, status, bx, by, dyn_raw);
}

}  // namespace lbm
