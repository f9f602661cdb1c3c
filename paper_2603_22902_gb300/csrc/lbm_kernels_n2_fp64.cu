// Kernel instantiations for N = 2 phases, precision policy PrecFP64.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(2, PrecFP64)
}  // namespace lbm
