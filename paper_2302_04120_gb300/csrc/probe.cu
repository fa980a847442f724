// FMA-rate probe: the arithmetic roofline of the FP64 (and FP32) forms of the step
// on the device at hand.  Every thread runs eight independent dependent chains of
// fused multiply-adds, so the pipe, not latency, bounds the rate.
#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "lbm_internal.cuh"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T *sink, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int c = 0; c < 8; c++) x[c] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)c;
  for (int k = 0; k < iters; k++) {
#pragma unroll
    for (int c = 0; c < 8; c++) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; c++) s += x[c];
  if (s == (T)-1.25) sink[blockIdx.x] = s;  // never true for these inputs; keeps the chains
}

template <typename T>
cudaError_t time_fma(int iters, double *gflops) {
  int dev = 0, nsm = 1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = nsm * 8, threads = 256;
  T *sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&sink, sizeof(T) * blocks);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const T a = (T)0.999999, b = (T)1e-7;
  if (e == cudaSuccess) {
    k_fma_chains<T><<<blocks, threads, 0, s>>>(sink, iters / 8, a, b);  // warm-up
    e = cudaEventRecord(e0, s);
  }
  if (e == cudaSuccess) {
    k_fma_chains<T><<<blocks, threads, 0, s>>>(sink, iters, a, b);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) *gflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e9;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(sink);
  return e;
}

}  // namespace

extern "C" lbm_status lbm_probe_fma_rate(int precision, double *gflops) {
  if (!gflops || (precision != LBM_FP64 && precision != LBM_FP32DEV)) {
    lbmk::set_global_error("lbm_probe_fma_rate: precision must be LBM_FP64 or LBM_FP32DEV, gflops non-NULL");
    return LBM_ERR_ARG;
  }
  cudaError_t e = precision == LBM_FP64 ? time_fma<double>(4096, gflops) : time_fma<float>(65536, gflops);
  if (e != cudaSuccess) {
    lbmk::set_global_error(cudaGetErrorString(e));
    return LBM_ERR_CUDA;
  }
  return LBM_OK;
}
