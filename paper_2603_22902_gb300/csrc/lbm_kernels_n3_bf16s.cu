// Kernel instantiations for N = 3 phases, precision policy PrecBF16S.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(3, PrecBF16S)
}  // namespace lbm
