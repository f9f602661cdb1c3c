// Kernel instantiations for N = 4 phases, precision policy PrecFP64.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(4, PrecFP64)
}  // namespace lbm
