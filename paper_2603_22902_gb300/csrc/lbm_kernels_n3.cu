// Kernel instantiations for N = 3 phases.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(3)
}  // namespace lbm
