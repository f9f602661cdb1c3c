// lbm_prec.cuh -- storage / arithmetic precision policies of the populations.
//
// A population set holds, per species s (0 = f, 1..N = g_{s-1}, N+1 = h):
//   * the rest population (direction 0) in the "rest" block, type TR, (N + 2) planes;
//   * the eight moving populations in the "moving" block, type TM, 8 (N + 2) planes.
// Rest populations never stream and carry most of each moment (4/9 of phi_p, the
// latent part of rho H), so they stay at least FP32.  In the 16-bit policies the
// moving populations are stored as scaled / shifted values so that the stored number
// stays O(1) and in the normal range of the format:
//   f_i  -> f_i / (w_i F_SCALE)          (pressure-based f_i are small: |f_i / w_i| << 1)
//   g_ip -> g_ip / w_i                   (= phi_p (1 + 3 c_i.u) + ... in [0, 1]; no shift, so the
//                                         tail of a dense phase inside a light one keeps the
//                                         format's relative precision: a shift to [-1/2, 1/2]
//                                         left an absolute error of ~1e-4 in phi there, which a
//                                         density ratio of 100 turned into 1 % of rho and of T)
//   h_i  -> h_i / (w_i rho_ref c_p,ref)  (= T + O(u) away from walls)
// Lagged planes are stored as TA.  Arithmetic of the collision runs in R; the
// liquid fraction always comes from the FP64 enthalpy map (eq. H); policies that compute
// in FP32 or double words screen the cell first and run the FP64 map only where the
// screen cannot decide f_l (map_cell in lbm_step.cuh).
//
// NGUARD: the pairwise normal n_pq = grad phi_pq / |grad phi_pq| is set to zero where
// |grad phi_pq| is below NGUARD times its own scale (phi_q |grad phi_p| + phi_p |grad phi_q|),
// i.e. where phi_p / phi_q is uniform to within the rounding noise of the format: there
// the direction is noise while 4 phi_p phi_q / eps is not small.  FP64 keeps only the
// absolute guard of the oracle (NGUARD = 0).  NABS2 is the square of that absolute guard:
// the oracle's |grad phi_pq| > 1e-12 for FP64; for FP32 arithmetic the threshold must sit
// above the noise floor of a stencil of FP32 values (~1e-8), so 1e-5 (a pairwise fraction
// changes by O(1) over the interface width, |grad phi_pq| ~ 1/eps, even in the tails);
// 1e-3 for 16-bit storage, whose rounding noise in phi is ~1e-4 (the normal is then zero
// only in far tails, where 4 phi_p phi_q / eps < 1e-3 as well).
//
// COMPACT: compile the step for a small code footprint rather than for the most
// instruction-level parallelism (the phase-field collision loop is not unrolled).  The
// double-word policy needs it: its arithmetic is ~10 instructions per operation, and
// the fully unrolled step does not fit the instruction cache.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_df64.cuh"

namespace lbm {

constexpr float F_SCALE = 1.0f / 4096.0f;

struct PrecFP64 {
    using R = double;
    using TR = double;
    using TM = double;
    using TA = double;
    static constexpr bool QUANT = false;
    static constexpr double NABS2 = 1e-24;
    static constexpr float NGUARD = 0.0f;
    static constexpr int OCC_THREADS = 512;
    static constexpr bool COH = false;
    static constexpr bool COMPACT = false;
};
struct PrecFP32 {
    using R = float;
    using TR = float;
    using TM = float;
    using TA = float;
    static constexpr bool QUANT = false;
    static constexpr double NABS2 = 1e-10;
    static constexpr float NGUARD = 1e-3f;
    static constexpr int OCC_THREADS = 1024;
    static constexpr bool COH = false;
    static constexpr bool COMPACT = false;
};
struct PrecFP16S {
    using R = float;
    using TR = float;
    using TM = __half;
    using TA = float;
    static constexpr bool QUANT = true;
    static constexpr double NABS2 = 1e-6;
    static constexpr float NGUARD = 3e-2f;
    static constexpr int OCC_THREADS = 1024;
    static constexpr bool COH = false;
    static constexpr bool COMPACT = false;
};
struct PrecBF16S {
    using R = float;
    using TR = float;
    using TM = __nv_bfloat16;
    using TA = float;
    static constexpr bool QUANT = true;
    static constexpr double NABS2 = 1e-6;
    static constexpr float NGUARD = 3e-2f;
    static constexpr int OCC_THREADS = 1024;
    static constexpr bool COH = false;
    static constexpr bool COMPACT = false;
};

// FP64-class accuracy on the FP32 pipes: every population, lagged value and
// coefficient is a double word (lbm_df64.cuh), 8 bytes like FP64, and the collision
// arithmetic runs in double-word arithmetic; f_l comes from the FP64 eq. H map where
// the screen cannot decide it, T of a decided cell from double words.  The guard of
// the pairwise normal is the oracle's.
struct PrecDF64 {
    using R = df64;
    using TR = df64;
    using TM = df64;
    using TA = df64;
    static constexpr bool QUANT = false;
    static constexpr double NABS2 = 1e-24;
    static constexpr float NGUARD = 0.0f;
    static constexpr int OCC_THREADS = 768;
    static constexpr bool COH = false;
    static constexpr bool COMPACT = true;
};

// The same policy for a launch that runs several steps (its loads must see what
// other blocks of the launch wrote: no read-only path).
template <class Base>
struct Coherent : Base {
    static constexpr bool COH = true;
};

__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ double to_f(double v) { return v; }
template <class T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }

// Byte sizes of one population set and one lagged set.
template <class Pr>
__host__ __device__ constexpr long long pop_set_bytes(int N, long long S)
{
    return (long long)(N + 2) * S * (long long)sizeof(typename Pr::TR) +
           8LL * (N + 2) * S * (long long)sizeof(typename Pr::TM);
}
template <class Pr>
__host__ __device__ constexpr long long aux_set_bytes(int N, long long S)
{
    return (long long)(3 + 2 * N) * S * (long long)sizeof(typename Pr::TA);
}

}  // namespace lbm
