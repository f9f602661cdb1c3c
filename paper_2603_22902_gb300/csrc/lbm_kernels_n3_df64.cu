// Kernel instantiations for N = 3 phases, precision policy PrecDF64.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(3, PrecDF64)
}  // namespace lbm
