// Kernel instantiations for N = 4 phases, precision policy PrecFP16S.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(4, PrecFP16S)
}  // namespace lbm
