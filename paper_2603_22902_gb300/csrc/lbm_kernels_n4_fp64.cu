// Kernel instantiations for N = 4 phases, precision policy PrecFP64, and the adjoint of the FP64 step.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(4, PrecFP64)
LBM_INSTANTIATE_ADJ(4)
}  // namespace lbm
