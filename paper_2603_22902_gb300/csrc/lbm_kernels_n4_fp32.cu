// Kernel instantiations for N = 4 phases, precision policy PrecFP32.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(4, PrecFP32)
}  // namespace lbm
