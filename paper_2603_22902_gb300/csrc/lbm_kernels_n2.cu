// Kernel instantiations for N = 2 phases.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(2)
}  // namespace lbm
