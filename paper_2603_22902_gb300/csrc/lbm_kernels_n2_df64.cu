// Kernel instantiations for N = 2 phases, precision policy PrecDF64.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(2, PrecDF64)
}  // namespace lbm
