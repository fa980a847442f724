// Compensated FP32 sums for reductions whose result is reported in FP64: on GB300 the
// FP64 pipe runs at a small fraction of the FP32 rate, so FP32 kernels keep a pair
// hi + lo per sum (each addition's rounding error carried in lo) and convert once.
#pragma once
#include <cuda_runtime.h>

namespace lbmk {

// Error-free sum of two floats (Knuth's TwoSum): s + e equals a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// A sum of node values: FP64, or for FP32 values a compensated FP32 pair hi + lo
// (each addition's rounding error carried in lo, so the pair keeps about twice FP32's
// precision), so that the FP64 pipe, slow on GB300, is not used per node.  A plain
// aggregate (it also lives in shared memory): clear() before use.
template <typename R> struct NodeSum;
template <> struct NodeSum<double> {
  double v;
  __device__ void clear() { v = 0.0; }
  __device__ void add(double x) { v += x; }
  __device__ void merge(const NodeSum &o) { v += o.v; }
  __device__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  __device__ double value() const { return v; }
};
template <> struct NodeSum<float> {
  float hi, lo;
  __device__ void clear() { hi = 0.f; lo = 0.f; }
  __device__ void add(float x) {
    float e;
    two_sum(hi, x, hi, e);
    lo += e;
  }
  __device__ void merge(const NodeSum &o) {
    float e;
    two_sum(hi, o.hi, hi, e);
    lo += o.lo + e;
  }
  __device__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      NodeSum x;
      x.hi = __shfl_down_sync(0xffffffffu, hi, o);
      x.lo = __shfl_down_sync(0xffffffffu, lo, o);
      merge(x);
    }
  }
  __device__ double value() const { return (double)hi + (double)lo; }
};

}  // namespace lbmk
