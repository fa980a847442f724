// Explicit instantiation of the TMA-staged step kernels, FP32 combinations
// (see sp_ops.cuh).
#include "tma_kernels.cuh"

namespace lbmk {
LBM_SP_COMBOS_C(LBM_TMA_INSTANTIATE)
LBM_SP_COMBOS_D(LBM_TMA_INSTANTIATE)
}  // namespace lbmk
