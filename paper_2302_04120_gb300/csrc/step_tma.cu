// Host side of the TMA-staged single-phase step: tensor-map encoding and dispatch
// to the instantiated kernels (tma_kernels.cuh, step_tma_a.cu / step_tma_b.cu).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "lbm_internal.cuh"
#include "sp_device.cuh"
#include "sp_ops.cuh"

namespace lbmk {

template <int PREC, int FLOW, int TH>
struct TmaOps {
  static cudaError_t step(const SpParams &P, const CUtensorMap &map, int ty, int stages, int grid, int *flag,
                          unsigned long long wait_ns, int expire_probe, cudaStream_t s);
  static cudaError_t prepare();
  static int occupancy(int ty, int stages);
};

namespace {
constexpr int kBoxW = kTmaBoxW;
constexpr int kMaxStages = kTmaMaxStages;
size_t plane_bytes(int ty, int elem) { return ((size_t)kBoxW * ty * elem + 127) / 128 * 128; }
}  // namespace

int sp_tma_encode(void *base, int pitch, int ny, int nq, int elem, int ty, CUtensorMap *out) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }();
  if (!encode) return -1;
  if (ty != 4 && ty != 8) return -2;
  cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)ny, (cuuint64_t)nq};
  cuuint64_t strides[2] = {(cuuint64_t)pitch * elem, (cuuint64_t)pitch * ny * elem};
  cuuint32_t box[3] = {(cuuint32_t)kBoxW, (cuuint32_t)ty, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(out, elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims,
                      strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)r;
}

cudaError_t sp_step_tma(const SpParams &P, const CUtensorMap &map, int prec, int flow, int th, int ty, int stages,
                        int grid, int *flag, unsigned long long wait_ns, int expire_probe, cudaStream_t s) {
  if (stages < 1 || stages > kMaxStages || grid < 1 || P.local) return cudaErrorInvalidValue;
#define CALL(A, B, C) return TmaOps<A, B, C>::step(P, map, ty, stages, grid, flag, wait_ns, expire_probe, s)
  LBM_SP_DISPATCH(prec, flow, th, CALL);
#undef CALL
  return cudaErrorInvalidValue;
}

cudaError_t sp_tma_prepare(int prec, int flow, int th) {
#define CALL(A, B, C) return TmaOps<A, B, C>::prepare()
  LBM_SP_DISPATCH(prec, flow, th, CALL);
#undef CALL
  return cudaErrorInvalidValue;
}

int sp_tma_occupancy(int prec, int flow, int th, int ty, int stages) {
#define CALL(A, B, C) \
  if (prec == A && flow == B && th == C) return TmaOps<A, B, C>::occupancy(ty, stages);
  LBM_SP_COMBOS(CALL)
#undef CALL
  return 0;
}

size_t sp_tma_smem(int prec, int flow, int th, int ty, int stages) {
  const int nq = (flow != FLOW_NONE ? 9 : 0) + (th == TH_BGK9 || th == TH_MRT9 ? 9 : th != TH_NONE ? 5 : 0);
  return 128 + (size_t)stages * nq * plane_bytes(ty, prec == 0 ? 8 : 4);
}

}  // namespace lbmk
