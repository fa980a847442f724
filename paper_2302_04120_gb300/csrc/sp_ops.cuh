// Launch entry points of the single-phase kernels for one (precision, momentum
// operator, thermal operator) combination.  The definitions are in sp_kernels.cuh;
// each combination is instantiated explicitly in one of the step_sp_*.cu units, so
// the kernels compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "lbm_internal.cuh"

namespace lbmk {

// TMA-staged step: columns per staged box (a 32-node tile plus 4, so that every box
// starts on a 16-byte boundary) and the largest ring of slots.
constexpr int kTmaBoxW = 36;
constexpr int kTmaMaxStages = 4;

template <int PREC, int FLOW, int TH>
struct SpOps {
  static cudaError_t step(const SpParams &P, dim3 block, cudaStream_t s);
  // the same step built for more resident blocks per SM (see split_blocks_per_sm)
  static cudaError_t step_occ(const SpParams &P, dim3 block, cudaStream_t s);
  static cudaError_t batch(const SpParams *table, const int4 *tiles, int ntiles, dim3 block, int grid,
                           cudaStream_t s);
  static int occupancy(int threads);
  static cudaError_t init(const SpParams &P, const double *a, const double *ux, const double *uy, const double *b,
                          dim3 block, cudaStream_t s);
  static cudaError_t moments(const SpParams &P, unsigned mask, double *out, cudaStream_t s);
  static cudaError_t integrals(const SpParams &P, double *partials, double *out4, unsigned *counter,
                               cudaStream_t s);
};

// Every supported combination, X(PREC, FLOW, TH), in four groups (one unit each).
#define LBM_SP_COMBOS_A(X) X(0, FLOW_BGK, TH_NONE) X(0, FLOW_BGK, TH_BGK) X(0, FLOW_BGK, TH_MRT) \
  X(0, FLOW_MRT, TH_NONE) X(0, FLOW_MRT, TH_BGK) X(0, FLOW_MRT, TH_MRT)
#define LBM_SP_COMBOS_B(X) X(0, FLOW_NONE, TH_BGK) X(0, FLOW_NONE, TH_MRT) X(0, FLOW_BGK, TH_BGK9) \
  X(0, FLOW_BGK, TH_MRT9) X(0, FLOW_MRT, TH_BGK9) X(0, FLOW_MRT, TH_MRT9)
#define LBM_SP_COMBOS_C(X) X(1, FLOW_BGK, TH_NONE) X(1, FLOW_BGK, TH_BGK) X(1, FLOW_BGK, TH_MRT) \
  X(1, FLOW_MRT, TH_NONE) X(1, FLOW_MRT, TH_BGK) X(1, FLOW_MRT, TH_MRT)
#define LBM_SP_COMBOS_D(X) X(1, FLOW_NONE, TH_BGK) X(1, FLOW_NONE, TH_MRT) X(1, FLOW_BGK, TH_BGK9) \
  X(1, FLOW_BGK, TH_MRT9) X(1, FLOW_MRT, TH_BGK9) X(1, FLOW_MRT, TH_MRT9)
#define LBM_SP_COMBOS(X) LBM_SP_COMBOS_A(X) LBM_SP_COMBOS_B(X) LBM_SP_COMBOS_C(X) LBM_SP_COMBOS_D(X)

}  // namespace lbmk
