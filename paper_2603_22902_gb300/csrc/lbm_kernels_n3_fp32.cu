// Kernel instantiations for N = 3 phases, precision policy PrecFP32.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(3, PrecFP32)
}  // namespace lbm
