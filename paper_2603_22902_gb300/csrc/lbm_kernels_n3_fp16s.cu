// Kernel instantiations for N = 3 phases, precision policy PrecFP16S.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(3, PrecFP16S)
}  // namespace lbm
