// Kernel instantiations for N = 4 phases, precision policy PrecDF64.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(4, PrecDF64)
}  // namespace lbm
