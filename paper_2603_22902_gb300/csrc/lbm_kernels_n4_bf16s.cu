// Kernel instantiations for N = 4 phases, precision policy PrecBF16S.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(4, PrecBF16S)
}  // namespace lbm
