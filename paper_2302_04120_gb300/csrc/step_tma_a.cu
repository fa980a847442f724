// Explicit instantiation of the TMA-staged step kernels, FP64 combinations
// (see sp_ops.cuh).
#include "tma_kernels.cuh"

namespace lbmk {
LBM_SP_COMBOS_A(LBM_TMA_INSTANTIATE)
LBM_SP_COMBOS_B(LBM_TMA_INSTANTIATE)
}  // namespace lbmk
