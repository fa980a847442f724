// Explicit instantiation of the single-phase kernels, combination group A
// (see sp_ops.cuh): split across units so that nvcc compiles them in parallel.
#include "sp_kernels.cuh"

namespace lbmk {
LBM_SP_COMBOS_A(LBM_SP_INSTANTIATE)
}  // namespace lbmk
