// Kernel instantiations for N = 4 phases.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(4)
}  // namespace lbm
