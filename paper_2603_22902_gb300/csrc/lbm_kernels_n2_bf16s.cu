// Kernel instantiations for N = 2 phases, precision policy PrecBF16S.
#include "lbm_kernels_impl.cuh"

namespace lbm {
LBM_INSTANTIATE(2, PrecBF16S)
}  // namespace lbm
