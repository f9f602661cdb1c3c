// Kernel instantiations for N = 2 phases, precision policy PrecFP64, and the adjoint of the FP64 step.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(2, PrecFP64)
LBM_INSTANTIATE_ADJ(2)
}  // namespace lbm
