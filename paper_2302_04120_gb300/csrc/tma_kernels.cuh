// Single-phase step with the pulled populations staged in shared memory by the
// Tensor Memory Accelerator, for sm_103a: kernels and launch entry points
// (TmaOps), instantiated in step_tma_a.cu (FP64) and step_tma_b.cu (FP32).
//
// Same arithmetic as k_step (pull streaming of Eq. eq_lattice_boltzmann_geral with
// the link-wise boundary rules of Sec. 2.1/2.2, moments, BGK/MRT collision, D2Q5
// thermal LBE), different memory pipeline:
//   * persistent CTAs (a few per SM) walk the 32 x TY node tiles of the grid with
//     a stride of gridDim.x;
//   * for each tile one elected thread issues one cp.async.bulk.tensor box per
//     population plane: plane q is read at the tile shifted by -c_q, i.e. exactly
//     the values the pull needs (the y shift is a row offset of the box; the x
//     shift is absorbed by a 36-column box whose start stays 16-byte aligned);
//   * the boxes of the next tiles are in flight (a ring of `stages` slots, each
//     completed through an mbarrier transaction count) while the current tile is
//     collided, so the DRAM latency is hidden without relying on occupancy;
//   * interior nodes read their nine (five) pulled values from shared memory;
//     nodes on the domain edge take the global-memory boundary path of k_step;
//   * post-collision values are stored straight to global memory, coalesced.
// Every mbarrier wait is bounded (one second of wall time by default, settable per
// handle); a wait that runs out sets a flag the host reads, lets the block's copies
// in flight land (bounded again, one second) and returns.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lattice.cuh"
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

namespace tma {


constexpr int kTileX = 32;      // nodes per tile row (one warp)
constexpr int kBoxW = kTmaBoxW;  // staged columns: the tile plus 4 (16-byte aligned box starts)
constexpr int kMaxStages = kTmaMaxStages;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wall-time limit of the wait that lets a block's copies in flight land before it
// exits after a failed wait (always the full second).
constexpr uint64_t kDrainWaitNs = 1000000000ull;

// Wait for the phase of parity `parity` of barrier b; false after limit_ns of wall
// time (or 2^28 tries, whichever comes first).
static __device__ __noinline__ bool mbar_wait_bounded(uint64_t *b, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(b, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < (1u << 28); ++it) {
    if (mbar_try_wait(b, parity)) return true;
    if ((it & 255u) == 255u && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// Box start relative to the tile for a population with x-velocity cx (multiples
// of 4 elements keep the start 16-byte aligned), and the staged column of the
// pulled value x - cx for node column tx: tx + 3 (cx = +1), tx + 1 (cx = -1), tx.
__host__ __device__ constexpr int box_dx(int cx) { return cx > 0 ? -4 : 0; }
__host__ __device__ constexpr int stage_dx(int cx) { return cx > 0 ? 3 : (cx < 0 ? 1 : 0); }
static_assert(stage_dx(1) == 1 * -1 - box_dx(1), "cx = +1 column");
static_assert(stage_dx(-1) == 1 - box_dx(-1), "cx = -1 column");

template <int FLOW, int TH>
struct Planes {
  static constexpr int F = FLOW != FLOW_NONE ? 9 : 0;
  static constexpr int N = F + (TH != TH_NONE ? ThLat<TH>::Q : 0);
};

// One node of a staged tile: pull (shared memory inside, boundary rules on the
// edge), moments, collision, store.  st: the tile's slot, sp: elements per staged
// plane, so: the node's offset within a staged plane.
template <int PREC, int FLOW, int TH>
__device__ __forceinline__ void step_node_staged(const SpParams &P, int i, int j, const typename Prec<PREC>::S *st,
                                                 int sp, int so) {
  typedef typename Prec<PREC>::S S;
  typedef typename Prec<PREC>::R R;
  const long long n = (long long)j * P.pitch + i;
  const S *src = (const S *)P.src;
  S *dst = (S *)P.dst;
  const bool interior = (i > 0) && (i < P.nx - 1) && (j > 0) && (j < P.ny - 1);
  constexpr int QT = ThLat<TH>::Q;
  R f[9], g[9];
  if (interior) {
    if (FLOW != FLOW_NONE) {
#pragma unroll
      for (int q = 0; q < 9; q++) f[q] = (R)st[q * sp + so + stage_dx(cx9(q))];
    }
    if (TH != TH_NONE) {
      const S *gs = st + Planes<FLOW, TH>::F * sp;
#pragma unroll
      for (int q = 0; q < QT; q++) g[q] = (R)gs[q * sp + so + stage_dx(cxT(QT, q))];
    }
  } else {
    if (P.sym) {
      if (FLOW != FLOW_NONE) pull_f<S, R, true>(P, src, i, j, false, f);
      if (TH != TH_NONE) pull_g<S, R, QT, true>(P, src, i, j, false, g);
    } else {
      if (FLOW != FLOW_NONE) pull_f<S, R>(P, src, i, j, false, f);
      if (TH != TH_NONE) pull_g<S, R, QT>(P, src, i, j, false, g);
    }
  }
  Macro<R> m;
  load_sources<S, R>(P, n, m);
  moments<R, FLOW, TH>(P, f, g, m);
  collide<R, FLOW, TH>(P, m, f, g);
  if (FLOW != FLOW_NONE) {
#pragma unroll
    for (int q = 0; q < 9; q++) dst[q * P.plane + n] = (S)f[q];
  }
  if (TH != TH_NONE) {
    S *gd = dst + (long long)P.gbase * P.plane;
#pragma unroll
    for (int q = 0; q < QT; q++) gd[q * P.plane + n] = (S)g[q];
  }
}

template <int PREC, int FLOW, int TH, int TY>
// wait_ns: wall-time limit of each ring wait.  expire_probe (self-test of the timeout
// path): each block first waits, with that limit, on a barrier of its own that nothing
// completes, so the wait runs out and the block takes the failure path below.
__global__ void __launch_bounds__(kTileX *TY) k_step_tma(const SpParams P, const __grid_constant__ CUtensorMap map,
                                                         int ntx, int ntiles, int nstages, int *flag,
                                                         unsigned long long wait_ns, int expire_probe) {
  typedef typename Prec<PREC>::S S;
  constexpr int NF = Planes<FLOW, TH>::F;
  constexpr int NQ = Planes<FLOW, TH>::N;
  constexpr uint32_t kBoxBytes = kBoxW * TY * sizeof(S);                  // one box as copied
  constexpr uint32_t kPlaneBytes = (kBoxBytes + 127u) / 128u * 128u;      // slot stride: 128-byte aligned
  constexpr int SP = kPlaneBytes / sizeof(S);                            // elements per staged plane
  constexpr uint32_t kStageBytes = NQ * kPlaneBytes;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // slots start 128-byte aligned (the dynamic size carries 128 bytes of slack)
  unsigned char *smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  __shared__ __align__(8) uint64_t full[kMaxStages];
  __shared__ __align__(8) uint64_t never;  // expire_probe only: no thread or copy completes it
  const int tid = threadIdx.y * kTileX + threadIdx.x;
  const int G = gridDim.x;
  if (tid == 0) {
    for (int s = 0; s < nstages; s++) mbar_init(&full[s], 1);
    if (expire_probe) mbar_init(&never, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  // Stage tile t into slot s: one box per population plane, read at -c_q.
  auto issue = [&](int t, int s) {
    const int i0 = (t % ntx) * kTileX, j0 = (t / ntx) * TY;
    unsigned char *slot = smem + s * kStageBytes;
    mbar_arrive_expect_tx(&full[s], NQ * kBoxBytes);
#pragma unroll
    for (int q = 0; q < NF; q++) tma_load_3d(slot + q * kPlaneBytes, &map, i0 + box_dx(cx9(q)), j0 - cy9(q), q, &full[s]);
    if (TH != TH_NONE) {
      constexpr int QT = ThLat<TH>::Q;
#pragma unroll
      for (int q = 0; q < QT; q++)
        tma_load_3d(slot + (NF + q) * kPlaneBytes, &map, i0 + box_dx(cxT(QT, q)), j0 - cyT(QT, q), P.gbase + q,
                    &full[s]);
    }
  };

  if (tid == 0) {
    for (int k = 0; k < nstages; k++) {
      const int t = blockIdx.x + k * G;
      if (t < ntiles) issue(t, k);
    }
  }
  int k = 0;
  for (int t = blockIdx.x; t < ntiles; t += G, ++k) {
    const int s = k % nstages;
    bool ok = true;
    if (expire_probe && k == 0) ok = mbar_wait_bounded(&never, 0u, wait_ns);
    if (ok) ok = mbar_wait_bounded(&full[s], (uint32_t)(k / nstages) & 1u, wait_ns);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(flag, 1);
        // let the copies this block still has in flight land before it exits
        for (int kk = k; kk < k + nstages && blockIdx.x + kk * G < ntiles; ++kk)
          mbar_wait_bounded(&full[kk % nstages], (uint32_t)(kk / nstages) & 1u, kDrainWaitNs);
      }
      __syncthreads();
      return;
    }
    const int i = (t % ntx) * kTileX + threadIdx.x, j = (t / ntx) * TY + threadIdx.y;
    if (i < P.nx && j < P.ny)
      step_node_staged<PREC, FLOW, TH>(P, i, j, (const S *)(smem + s * kStageBytes), SP, threadIdx.y * kBoxW + threadIdx.x);
    __syncthreads();  // slot s fully read
    if (tid == 0) {
      const int tn = t + nstages * G;
      if (tn < ntiles) issue(tn, s);
    }
  }
}

__host__ __device__ constexpr size_t plane_bytes(int ty, int elem) { return ((size_t)kBoxW * ty * elem + 127) / 128 * 128; }

template <int PREC, int FLOW, int TH, int TY>
size_t smem_bytes(int stages) {
  return 128 + (size_t)stages * Planes<FLOW, TH>::N * plane_bytes(TY, sizeof(typename Prec<PREC>::S));
}

template <int PREC, int FLOW, int TH, int TY>
cudaError_t launch(const SpParams &P, const CUtensorMap &map, int stages, int grid, int *flag,
                   unsigned long long wait_ns, int expire_probe, cudaStream_t s) {
  const int ntx = (P.nx + kTileX - 1) / kTileX, nty = (P.ny + TY - 1) / TY;
  const int ntiles = ntx * nty;
  if (grid > ntiles) grid = ntiles;
  k_step_tma<PREC, FLOW, TH, TY><<<grid, dim3(kTileX, TY), smem_bytes<PREC, FLOW, TH, TY>(stages), s>>>(
      P, map, ntx, ntiles, stages, flag, wait_ns, expire_probe);
  return cudaGetLastError();
}

template <int PREC, int FLOW, int TH, int TY>
cudaError_t prepare() {
  return cudaFuncSetAttribute(k_step_tma<PREC, FLOW, TH, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes<PREC, FLOW, TH, TY>(kMaxStages));
}

template <int PREC, int FLOW, int TH, int TY>
int occupancy(int stages) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_tma<PREC, FLOW, TH, TY>, kTileX * TY,
                                                    smem_bytes<PREC, FLOW, TH, TY>(stages)) != cudaSuccess)
    return 0;
  return nb;
}

}  // namespace tma

template <int PREC, int FLOW, int TH>
cudaError_t TmaOps<PREC, FLOW, TH>::step(const SpParams &P, const CUtensorMap &map, int ty, int stages, int grid,
                                         int *flag, unsigned long long wait_ns, int expire_probe, cudaStream_t s) {
  if (ty == 4) return tma::launch<PREC, FLOW, TH, 4>(P, map, stages, grid, flag, wait_ns, expire_probe, s);
  if (ty == 8) return tma::launch<PREC, FLOW, TH, 8>(P, map, stages, grid, flag, wait_ns, expire_probe, s);
  return cudaErrorInvalidValue;
}

template <int PREC, int FLOW, int TH>
cudaError_t TmaOps<PREC, FLOW, TH>::prepare() {
  cudaError_t e4 = tma::prepare<PREC, FLOW, TH, 4>(), e8 = tma::prepare<PREC, FLOW, TH, 8>();
  return e4 != cudaSuccess ? e4 : e8;
}

template <int PREC, int FLOW, int TH>
int TmaOps<PREC, FLOW, TH>::occupancy(int ty, int stages) {
  return ty == 4 ? tma::occupancy<PREC, FLOW, TH, 4>(stages) : tma::occupancy<PREC, FLOW, TH, 8>(stages);
}

#define LBM_TMA_INSTANTIATE(A, B, C) template struct TmaOps<A, B, C>;

}  // namespace lbmk
