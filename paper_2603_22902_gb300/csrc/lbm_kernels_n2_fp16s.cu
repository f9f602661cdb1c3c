// Kernel instantiations for N = 2 phases, precision policy PrecFP16S.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(2, PrecFP16S)
}  // namespace lbm
