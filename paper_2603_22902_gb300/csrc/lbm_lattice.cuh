// lbm_lattice.cuh -- the D2Q9 lattice of every LB equation of the scheme (arXiv 2603.22902,
// Section 3: f, g_p and h share it, c_s^2 = 1/3): velocities, opposite directions and
// weights, usable in host and device code.
#pragma once

#include <type_traits>

#include "lbm_df64.cuh"

namespace lbm {

// D2Q9: c_0 = 0; c_1..4 = (1,0), (0,1), (-1,0), (0,-1); c_5..8 the diagonals.
__host__ __device__ constexpr int cx(int i) { return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0); }
__host__ __device__ constexpr int cy(int i) { return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0); }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i < 5 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5); }
__host__ __device__ constexpr double wgt(int i) { return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }

// D2Q9 weights as constants of the arithmetic type R.  For double words the weights are
// w_d = m / 2^54 with m = round(2^54 / 36), w_a = 4 w_d and w_0 = 1 - 20 w_d: each is
// exactly a double word (and a double, within 5e-16 of 1/36, 1/9, 4/9) and they sum to
// exactly 1.  Rounded one by one to 48 bits, the weights would sum to 1 +- 2^-49, and
// every collision would then add that fraction of the equilibrium to the conserved
// moments: a steady drift of rho H and phi_p, relative to an FP64 run, of ~1e-15 per
// step.
template <class R>
__host__ __device__ constexpr R wgt_r(int i)
{
    if constexpr (std::is_same<R, df64>::value) {
        constexpr double two54 = 18014398509481984.0;
        return R(i == 0 ? 8006399337547544.0 / two54 : (i < 5 ? 2001599834386888.0 / two54 : 500399958596722.0 / two54));
    } else {
        return R(wgt(i));
    }
}

}  // namespace lbm
