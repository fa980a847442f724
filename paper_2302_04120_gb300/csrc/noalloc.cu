// Allocation-free field integrals.
//
// lbm_integrals() reduces through a per-handle scratch buffer of per-block
// partial sums that lbm_create obtains with cudaMalloc.  Some callers cannot
// allocate device memory at all: code running inside a memory pool or arena
// that owns every byte of the device, code under a framework allocator that
// forbids foreign cudaMalloc calls, or code that must not synchronise the
// device (cudaMalloc/cudaFree can).  This file gives them one entry point that
// allocates nothing: the same deterministic two-stage reduction as the
// integrals kernel, reading macroscopic fields the caller already holds on the
// device, with its scratch in a file-scope device array of fixed size.
//
// The array is part of the library image: every GPU that loads the library
// holds it (4 * LBM_NOALLOC_MAX_BLOCKS doubles = 128 KiB) until the process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <mutex>
#include <stdio.h>

#include "../../include/lbm.h"
#include "lbm_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 8;
constexpr int kCellsPerBlock = kThreads * kCellsPerThread;  // = LBM_NOALLOC_CELLS_PER_BLOCK
constexpr int kMaxBlocks = LBM_NOALLOC_MAX_BLOCKS;
constexpr int kMaxDevices = 64;

static_assert(kCellsPerBlock == LBM_NOALLOC_CELLS_PER_BLOCK, "header and kernel disagree on the block size");

// Shared scratch: four partials (mass, phi, max |u|, bad count) per block.
static __device__ __align__(256) double g_noalloc_partials[4 * kMaxBlocks];

// Device address of g_noalloc_partials, looked up once per device.
std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

__global__ void __launch_bounds__(kThreads) k_field_partials(const double *rho, const double *ux, const double *uy,
                                                             const double *phi, long long n, double area,
                                                             double ulim, double *partials) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const long long base = (long long)blockIdx.x * kCellsPerBlock + threadIdx.x;
#pragma unroll
  for (int k = 0; k < kCellsPerThread; k++) {
    const long long i = base + (long long)k * kThreads;
    if (i < n) {
      const double r = rho[i], u = ux[i], w = uy[i];
      const double umag = sqrt(u * u + w * w);
      const double ph = phi ? phi[i] : 0.0;
      const bool bad = !isfinite(r) || !isfinite(umag) || !isfinite(ph) || umag >= ulim;
      // a bad cell is counted and adds nothing to the sums or the maximum (as in
      // lbm_integrals)
      v[0] += bad ? 0.0 : r * area;
      v[1] += bad ? 0.0 : ph;
      v[2] = fmax(v[2], bad ? 0.0 : umag);
      v[3] += bad ? 1.0 : 0.0;
    }
  }
  // fixed shuffle tree, then warps in index order: deterministic
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v[0] += __shfl_down_sync(0xffffffffu, v[0], o);
    v[1] += __shfl_down_sync(0xffffffffu, v[1], o);
    v[2] = fmax(v[2], __shfl_down_sync(0xffffffffu, v[2], o));
    v[3] += __shfl_down_sync(0xffffffffu, v[3], o);
  }
  __shared__ double sh[kThreads / 32][4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh[warp][0] = v[0]; sh[warp][1] = v[1]; sh[warp][2] = v[2]; sh[warp][3] = v[3];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, mx = 0, cnt = 0;
    for (int w = 0; w < kThreads / 32; w++) { a += sh[w][0]; b += sh[w][1]; mx = fmax(mx, sh[w][2]); cnt += sh[w][3]; }
    // every partial the final pass reads is written here by this call
    partials[4 * blockIdx.x + 0] = a;
    partials[4 * blockIdx.x + 1] = b;
    partials[4 * blockIdx.x + 2] = mx;
    partials[4 * blockIdx.x + 3] = cnt;
  }
}

__global__ void k_field_final(const double *partials, int nb, double *out4) {
  const int lane = threadIdx.x;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = lane; b < nb; b += 32) {
    v[0] += partials[4 * b + 0];
    v[1] += partials[4 * b + 1];
    v[2] = fmax(v[2], partials[4 * b + 2]);
    v[3] += partials[4 * b + 3];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v[0] += __shfl_down_sync(0xffffffffu, v[0], o);
    v[1] += __shfl_down_sync(0xffffffffu, v[1], o);
    v[2] = fmax(v[2], __shfl_down_sync(0xffffffffu, v[2], o));
    v[3] += __shfl_down_sync(0xffffffffu, v[3], o);
  }
  if (lane == 0) { out4[0] = v[0]; out4[1] = v[1]; out4[2] = v[2]; out4[3] = v[3]; }
}

// Device address of the scratch array on the current device (set-up on first use).
cudaError_t scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (double *)p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" lbm_status lbm_field_integrals_noalloc(const double *rho, const double *ux, const double *uy,
                                                  const double *phi, int nx, int ny, double dx, double c,
                                                  double *out4, void *stream) {
  char msg[256];
  if (!rho || !ux || !uy || !out4) {
    lbmk::set_global_error("lbm_field_integrals_noalloc: rho, ux, uy and out4 must be device pointers");
    return LBM_ERR_ARG;
  }
  if (nx < 1 || ny < 1 || !(dx > 0) || !(c > 0)) {
    lbmk::set_global_error("lbm_field_integrals_noalloc: need nx, ny >= 1, dx > 0, c > 0");
    return LBM_ERR_ARG;
  }
  const long long n = (long long)nx * ny;
  if (n > (long long)kMaxBlocks * kCellsPerBlock) {
    snprintf(msg, sizeof(msg),
             "lbm_field_integrals_noalloc: %lld cells exceed the static scratch limit of %lld cells "
             "(LBM_NOALLOC_MAX_CELLS); use lbm_integrals",
             n, (long long)kMaxBlocks * kCellsPerBlock);
    lbmk::set_global_error(msg);
    return LBM_ERR_ARG;
  }
  double *scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "lbm_field_integrals_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    lbmk::set_global_error(msg);
    return LBM_ERR_CUDA;
  }
  const int nb = (int)((n + kCellsPerBlock - 1) / kCellsPerBlock);
  cudaStream_t s = (cudaStream_t)stream;
  k_field_partials<<<nb, kThreads, 0, s>>>(rho, ux, uy, phi, n, dx * dx, c, scratch);
  k_field_final<<<1, 32, 0, s>>>(scratch, nb, out4);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "lbm_field_integrals_noalloc: launch: %s", cudaGetErrorString(e));
    lbmk::set_global_error(msg);
    return LBM_ERR_CUDA;
  }
  return LBM_OK;
}
