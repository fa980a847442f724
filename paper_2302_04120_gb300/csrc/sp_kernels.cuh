// Single-phase kernels of the dimensional lattice Boltzmann method and the
// definitions of their launch entry points (SpOps); included by the step_sp_*.cu
// units, which instantiate them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lattice.cuh"
#include "lbm_internal.cuh"
#include "sp_device.cuh"
#include "sp_ops.cuh"
#include "compensated.cuh"

namespace lbmk {

// ----------------------------------------------------------------------------
// Kernels
// ----------------------------------------------------------------------------
// One node: pull with boundary links, moments, collision, store.  INNER: the
// caller guarantees an interior node of a non-local step (no boundary code).
template <int PREC, int FLOW, int TH, bool INNER = false, bool SYM = false>
__device__ __forceinline__ void step_node(const SpParams &P, int i, int j) {
  typedef typename Prec<PREC>::S S;
  typedef typename Prec<PREC>::R R;
  const long long n = (long long)j * P.pitch + i;
  const S *src = (const S *)P.src;
  S *dst = (S *)P.dst;
  const bool interior = INNER || (!P.local && (i > 0) && (i < P.nx - 1) && (j > 0) && (j < P.ny - 1));
  R f[9], g[9];
  if (FLOW != FLOW_NONE) pull_f<S, R, SYM>(P, src, i, j, interior, f);
  if (TH != TH_NONE) pull_g<S, R, ThLat<TH>::Q, SYM>(P, src, i, j, interior, g);
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
    for (int q = 0; q < ThLat<TH>::Q; q++) gd[q * P.plane + n] = (S)g[q];
  }
}

// Boundary frame of the grid: rows j = 0 and j = ny - 1, then the columns i = 0
// and i = nx - 1 between them (each node once, also for nx or ny < 3).  Gives the
// node of frame index f, or false past the last one.
__device__ __forceinline__ bool frame_node(int nx, int ny, int f, int &i, int &j) {
  const int rows = ny >= 2 ? 2 : 1, cols = nx >= 2 ? 2 : 1;
  if (f < rows * nx) {
    i = f % nx;
    j = (f / nx) ? ny - 1 : 0;
    return true;
  }
  f -= rows * nx;
  const int inner = ny - 2;
  if (inner <= 0 || f >= cols * inner) return false;
  i = (f / inner) ? nx - 1 : 0;
  j = 1 + f % inner;
  return true;
}


// A step after the first, on a grid of gridDim.x tiles per row: the first fy rows of
// blocks take the boundary frame (the boundary rules, whose gathers and velocity
// reconstructions make these nodes the longest-running; they start first), the
// other rows the interior tiles, with the boundary code compiled out.  Keeping the
// frame in warps of its own spares the interior warps that touch the inlet or
// outlet column from running both paths one after the other.
// FP32 momentum-only solves move 9 values per node: at 64 registers (4 blocks of 256
// per SM) too few bytes are in flight to cover HBM latency, so they run 6 blocks per
// SM (40 registers, with some spilling) -- measured 0.78 -> 0.88 (BGK) and 0.83 -> 0.96
// (MRT) of the copy bandwidth on an 8192 x 4096 grid.  FP32 solves with a thermal
// lattice have two builds: 4 blocks per SM (64 registers, OCC = false), the faster on
// short launches such as the 2048 x 256 channel (16.3 against 20.4 us per step), and 6
// (40 registers, OCC = true), the faster on large grids (8192 x 4096: 549 against
// 578 us, 1.01 against 0.96 of the measured copy bandwidth); the launch kind picks one.
template <int PREC, bool OCC, int TH>
constexpr int split_blocks_per_sm() {
  return PREC == 1 ? ((TH == TH_NONE || OCC) ? 6 : 4) : 3;
}

template <int PREC, int FLOW, int TH, bool SYM, bool OCC = false>
__global__ void __launch_bounds__(256, split_blocks_per_sm<PREC, OCC, TH>()) k_step_split(const SpParams P, int fy) {
  if ((int)blockIdx.y < fy) {
    const int nt = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    int i, j;
    if (frame_node(P.nx, P.ny, (blockIdx.y * gridDim.x + blockIdx.x) * nt + tid, i, j))
      step_node<PREC, FLOW, TH, false, SYM>(P, i, j);
    return;
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = (blockIdx.y - fy) * blockDim.y + threadIdx.y;
  if (i <= 0 || j <= 0 || i >= P.nx - 1 || j >= P.ny - 1) return;
  step_node<PREC, FLOW, TH, true>(P, i, j);
}

// Every node in one pass (the first step after initialisation, whose pull is local).
template <int PREC, int FLOW, int TH, bool SYM>
__global__ void __launch_bounds__(256) k_step(const SpParams P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= P.nx || j >= P.ny) return;
  step_node<PREC, FLOW, TH, false, SYM>(P, i, j);
}

// Many independent solves in one launch: blocks walk a flattened list of entries
// with a grid stride; the channel's parameters (sizes, boundaries, rates, buffers of
// this parity) sit in a device table.  An entry (channel, x0, y0, 0) is one
// blockDim.x x blockDim.y tile of the channel's interior; an entry (channel, f0, 0, 1)
// is blockDim.x * blockDim.y consecutive nodes of its boundary frame from frame
// index f0 (the list puts these first), as in k_step_split.
#ifndef LBM_BATCH_FP32_BLOCKS_PER_SM
#define LBM_BATCH_FP32_BLOCKS_PER_SM 4
#endif
template <int PREC, int FLOW, int TH>
__global__ void __launch_bounds__(256, PREC == 1 ? LBM_BATCH_FP32_BLOCKS_PER_SM : 3) k_batch_step(const SpParams *__restrict__ table, const int4 *__restrict__ tiles,
                                                     int ntiles) {
  int4 next = blockIdx.x < ntiles ? tiles[blockIdx.x] : make_int4(0, 0, 0, 0);
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int4 tl = next;
    if (t + gridDim.x < ntiles) next = tiles[t + gridDim.x];  // the next entry's load overlaps this tile
    const SpParams &P = table[tl.x];
    if (tl.w == 1) {
      int i, j;
      const int f = tl.y + threadIdx.y * blockDim.x + threadIdx.x;
      if (!frame_node(P.nx, P.ny, f, i, j)) continue;
      if (P.sym) step_node<PREC, FLOW, TH, false, true>(P, i, j);
      else step_node<PREC, FLOW, TH>(P, i, j);
      continue;
    }
    const int i = tl.y + threadIdx.x, j = tl.z + threadIdx.y;
    if (i <= 0 || j <= 0 || i >= P.nx - 1 || j >= P.ny - 1) continue;  // frame entries
    if (P.local) step_node<PREC, FLOW, TH>(P, i, j);  // local pull: no boundary links
    else step_node<PREC, FLOW, TH, true>(P, i, j);
  }
}

// Equilibrium from fields (Eqs. feq_geral, geq_geral): the pre-collision state of
// time 0, stored in deviation form; the first step collides it in place.
template <int PREC, int FLOW, int TH>
__global__ void __launch_bounds__(256) k_init(const SpParams P, const double *A, const double *UX,
                                               const double *UY, const double *B) {
  typedef typename Prec<PREC>::S S;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= P.nx || j >= P.ny) return;
  const long long n = (long long)j * P.pitch + i;
  const int k = j * P.nx + i;
  S *dst = (S *)P.dst;
  const double rho = A ? A[k] : P.rho0;
  const double u0 = (FLOW != FLOW_NONE) ? (UX ? UX[k] : 0.0) : P.ux_pres;
  const double v0 = (FLOW != FLOW_NONE) ? (UY ? UY[k] : 0.0) : P.uy_pres;
  const double T = B ? B[k] : P.T0;
  const double c = P.c, inv_cs2 = 3.0 / (c * c);
  if (FLOW != FLOW_NONE) {
    const double usq = u0 * u0 + v0 * v0;
#pragma unroll
    for (int q = 0; q < 9; q++) {
      double cu = c * (cx9(q) * u0 + cy9(q) * v0);
      dst[q * P.plane + n] = (S)(w9<double>(q) * ((rho - P.rho0) + rho * (cu * inv_cs2 + 0.5 * cu * cu * inv_cs2 * inv_cs2 - 0.5 * usq * inv_cs2)));
    }
  }
  if (TH != TH_NONE) {
    constexpr int QT = ThLat<TH>::Q;
    S *gd = dst + (long long)P.gbase * P.plane;
#pragma unroll
    for (int q = 0; q < QT; q++) {
      double cu = c * (cxT(QT, q) * u0 + cyT(QT, q) * v0);
      gd[q * P.plane + n] = (S)(wT<double>(QT, q) * ((T - P.T0) + T * cu * inv_cs2));
    }
  }
}

// Macroscopic fields of the current time: pull (with boundary rules) + moments.
template <int PREC, int FLOW, int TH, bool SYM>
__global__ void __launch_bounds__(256) k_moments(const SpParams P, unsigned mask, double *out) {
  typedef typename Prec<PREC>::S S;
  typedef typename Prec<PREC>::R R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= P.nx || j >= P.ny) return;
  const long long n = (long long)j * P.pitch + i;
  const S *src = (const S *)P.src;
  const bool interior = !P.local && (i > 0) && (i < P.nx - 1) && (j > 0) && (j < P.ny - 1);
  R f[9], g[9];
  if (FLOW != FLOW_NONE) pull_f<S, R, SYM>(P, src, i, j, interior, f);
  if (TH != TH_NONE) pull_g<S, R, ThLat<TH>::Q, SYM>(P, src, i, j, interior, g);
  Macro<R> m;
  load_sources<S, R>(P, n, m);
  moments<R, FLOW, TH>(P, f, g, m);
  const long long N = (long long)P.nx * P.ny;
  const long long k = (long long)j * P.nx + i;
  int slot = 0;
  // rho, ux, uy, T, p (= c_s^2 (rho - rho0)), phi (0)
  if (mask & 1u) out[(slot++) * N + k] = (double)P.rho0 + (double)m.drho;
  if (mask & 2u) out[(slot++) * N + k] = (double)m.ux;
  if (mask & 4u) out[(slot++) * N + k] = (double)m.uy;
  if (mask & 8u) out[(slot++) * N + k] = (TH != TH_NONE) ? (double)P.T0 + (double)m.sumg + 0.5 * P.dt * (double)m.qd : 0.0;
  if (mask & 16u) out[(slot++) * N + k] = P.cs2 * (double)m.drho;
  if (mask & 32u) out[(slot++) * N + k] = 0.0;
}

// Deterministic integrals.  Per node: the density deviation rho - rho0 and |u|^2 in
// FP64 from the working-precision moments (no square root per node), and a health
// flag; warp sums in a fixed shuffle tree; per-block FP64 partials (sum of
// rho - rho0, 0, max |u|^2, bad-node count); a one-block final pass in a fixed order
// adds (N - bad) rho0 and takes the one square root.  Bad nodes (a non-finite value or
// |u| >= c) add nothing to the mass or to max |u|: they are only counted.
// One block's partials in the working precision: sum of drho, max |u|^2, bad count.
template <typename R> struct Part {
  NodeSum<R> s;
  R u2;
  int bad;
  __device__ void clear() { s.clear(); u2 = (R)0; bad = 0; }
  __device__ void merge(const Part &o) {
    s.merge(o.s);
    u2 = u2 > o.u2 ? u2 : o.u2;
    bad += o.bad;
  }
};
// Partials written by other blocks of the launch: read through L2 (__ldcg).
__device__ __forceinline__ Part<float> load_part(const Part<float> *p) {
  const float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
  Part<float> r;
  r.s.hi = v.x; r.s.lo = v.y; r.u2 = v.z; r.bad = __float_as_int(v.w);
  return r;
}
__device__ __forceinline__ Part<double> load_part(const Part<double> *p) {
  Part<double> r;
  r.s.v = __ldcg(&p->s.v); r.u2 = __ldcg(&p->u2); r.bad = __ldcg(&p->bad);
  return r;
}

// Per-block partials in a fixed order: lane tree, then the warps in order.
template <typename R>
__device__ __forceinline__ void block_partials(Part<R> a, Part<R> *out) {
  a.s.warp_reduce();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const R u = __shfl_down_sync(0xffffffffu, a.u2, o);
    a.u2 = a.u2 > u ? a.u2 : u;
    a.bad += __shfl_down_sync(0xffffffffu, a.bad, o);
  }
  __shared__ Part<R> sh[8];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
  if (lane == 0) sh[warp] = a;
  __syncthreads();
  if (tid == 0) {
    Part<R> b = sh[0];
    for (int w = 1; w < nw; w++) b.merge(sh[w]);
    *out = b;
  }
}

// Fixed-order sum of the nb per-block partials by one 256-thread block: thread t
// merges partials t, t + 256, ... in order, then a fixed tree, in the working
// precision; one thread forms the FP64 results.  mass = ((N - bad) rho0 + sum over
// healthy nodes of (rho - rho0)) dx^2, max |u| = sqrt(max |u|^2).
template <typename R>
__device__ __forceinline__ void final_reduce(const Part<R> *parts, int nb, double n_rho0, double rho0, double area,
                                             double *out4) {
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  Part<R> a;
  a.clear();
  for (int k = t; k < nb; k += 256) a.merge(load_part(parts + k));
  __shared__ Part<R> sh[256];
  sh[t] = a;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (t < w) sh[t].merge(sh[t + w]);
    __syncthreads();
  }
  if (t == 0) {
    const double bad = (double)sh[0].bad;
    out4[0] = (n_rho0 - bad * rho0 + sh[0].s.value()) * area;
    out4[1] = 0.0;
    out4[2] = sqrt((double)sh[0].u2);
    out4[3] = bad;
  }
}

// Integrals in one launch: every block writes its partials; the block that counts
// last (a device counter, 0 on entry and reset by that block) makes the final pass.
// The first fy rows of blocks take the boundary frame, one node per thread (its pull
// rules are the long path); in the others each thread takes the interior nodes of its
// column in `steps` groups of rows, with the pull compiled without boundary code.
// drho is summed exactly enough for FP64 (NodeSum); |u|^2, its maximum and the health
// test are taken in the working precision.  On GB300 the FP64 pipe bounded the form
// with every quantity in FP64 (49 us on 2048 x 256, 57 % FP64 pipe).
template <typename S, typename R, int FLOW, int TH, bool SYM, bool INNER>
__device__ __forceinline__ void integrate_node(const SpParams &P, int i, int j, R c2, Part<R> &acc) {
  const S *src = (const S *)P.src;
  const bool interior = INNER || (!P.local && (i > 0) && (i < P.nx - 1) && (j > 0) && (j < P.ny - 1));
  R f[9], g[9];
  if (FLOW != FLOW_NONE) pull_f<S, R, SYM && !INNER>(P, src, i, j, interior, f);
  if (TH != TH_NONE) pull_g<S, R, ThLat<TH>::Q, SYM && !INNER>(P, src, i, j, interior, g);
  Macro<R> m;
  load_sources<S, R>(P, (long long)j * P.pitch + i, m);
  moments<R, FLOW, TH>(P, f, g, m);
  const R uu = m.ux * m.ux + m.uy * m.uy;
  const R Tchk = (TH != TH_NONE) ? m.T : (R)0;
  if (!isfinite(m.drho) || !isfinite(uu) || !isfinite(Tchk) || uu >= c2) {
    acc.bad++;
  } else {
    acc.s.add(m.drho);
    acc.u2 = acc.u2 > uu ? acc.u2 : uu;
  }
}

template <int PREC, int FLOW, int TH, bool SYM>
__global__ void __launch_bounds__(256, 3) k_integrals(const SpParams P, int steps, int fy, double *partials,
                                                      double n_rho0, double area, double *out4, unsigned *counter) {
  // n_rho0 = N rho0 of the whole grid; final_reduce removes rho0 per bad node
  typedef typename Prec<PREC>::S S;
  typedef typename Prec<PREC>::R R;
  const R c2 = K<R>(P).c * K<R>(P).c;
  Part<R> acc;
  acc.clear();
  if ((int)blockIdx.y < fy) {
    const int nt = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    int i, j;
    if (frame_node(P.nx, P.ny, (blockIdx.y * gridDim.x + blockIdx.x) * nt + tid, i, j))
      integrate_node<S, R, FLOW, TH, SYM, false>(P, i, j, c2, acc);
  } else {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > 0 && i < P.nx - 1) {
#pragma unroll 1
      for (int r = 0; r < steps; r++) {
        const int j = ((blockIdx.y - fy) * steps + r) * blockDim.y + threadIdx.y;
        if (j >= P.ny - 1) break;
        if (j < 1) continue;
        if (P.local) integrate_node<S, R, FLOW, TH, SYM, false>(P, i, j, c2, acc);
        else integrate_node<S, R, FLOW, TH, SYM, true>(P, i, j, c2, acc);
      }
    }
  }
  Part<R> *parts = reinterpret_cast<Part<R> *>(partials);  // sizeof(Part<R>) <= 4 doubles
  block_partials<R>(acc, parts + blockIdx.y * gridDim.x + blockIdx.x);
  const unsigned nb = gridDim.x * gridDim.y;
  __shared__ bool last;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();  // this block's partials before its count
    last = atomicAdd(counter, 1u) == nb - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    final_reduce<R>(parts, (int)nb, n_rho0, P.rho0, area, out4);
    if (threadIdx.x == 0 && threadIdx.y == 0) *counter = 0u;
  }
}

// ----------------------------------------------------------------------------
// Launch entry points
// ----------------------------------------------------------------------------
inline dim3 grid_for(int nx, int ny, dim3 b) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y); }

template <int PREC, int FLOW, int TH>
cudaError_t SpOps<PREC, FLOW, TH>::step(const SpParams &P, dim3 block, cudaStream_t s) {
  dim3 grid = grid_for(P.nx, P.ny, block);
  const int nt = block.x * block.y;
  const int nfb = (frame_nodes(P.nx, P.ny) + nt - 1) / nt;  // frame blocks
  const int fy = (nfb + (int)grid.x - 1) / (int)grid.x;      // rows of them
  if (!P.local && grid.y + fy <= 65535u) {                   // else the one-pass kernel
    if (P.sym) k_step_split<PREC, FLOW, TH, true><<<dim3(grid.x, grid.y + fy), block, 0, s>>>(P, fy);
    else k_step_split<PREC, FLOW, TH, false><<<dim3(grid.x, grid.y + fy), block, 0, s>>>(P, fy);
  } else {
    if (P.sym) k_step<PREC, FLOW, TH, true><<<grid, block, 0, s>>>(P);
    else k_step<PREC, FLOW, TH, false><<<grid, block, 0, s>>>(P);
  }
  return cudaGetLastError();
}

template <int PREC, int FLOW, int TH>
cudaError_t SpOps<PREC, FLOW, TH>::step_occ(const SpParams &P, dim3 block, cudaStream_t s) {
  dim3 grid = grid_for(P.nx, P.ny, block);
  const int nt = block.x * block.y;
  const int nfb = (frame_nodes(P.nx, P.ny) + nt - 1) / nt;  // frame blocks
  const int fy = (nfb + (int)grid.x - 1) / (int)grid.x;      // rows of them
  if (P.local || grid.y + fy > 65535u) return step(P, block, s);
  if (P.sym) k_step_split<PREC, FLOW, TH, true, true><<<dim3(grid.x, grid.y + fy), block, 0, s>>>(P, fy);
  else k_step_split<PREC, FLOW, TH, false, true><<<dim3(grid.x, grid.y + fy), block, 0, s>>>(P, fy);
  return cudaGetLastError();
}

template <int PREC, int FLOW, int TH>
cudaError_t SpOps<PREC, FLOW, TH>::batch(const SpParams *table, const int4 *tiles, int ntiles, dim3 block, int grid,
                                         cudaStream_t s) {
  k_batch_step<PREC, FLOW, TH><<<grid, block, 0, s>>>(table, tiles, ntiles);
  return cudaGetLastError();
}

template <int PREC, int FLOW, int TH>
int SpOps<PREC, FLOW, TH>::occupancy(int threads) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_step<PREC, FLOW, TH>, threads, 0) != cudaSuccess)
    return 0;
  return nb;
}

template <int PREC, int FLOW, int TH>
cudaError_t SpOps<PREC, FLOW, TH>::init(const SpParams &P, const double *a, const double *ux, const double *uy,
                                        const double *b, dim3 block, cudaStream_t s) {
  k_init<PREC, FLOW, TH><<<grid_for(P.nx, P.ny, block), block, 0, s>>>(P, a, ux, uy, b);
  return cudaGetLastError();
}

template <int PREC, int FLOW, int TH>
cudaError_t SpOps<PREC, FLOW, TH>::moments(const SpParams &P, unsigned mask, double *out, cudaStream_t s) {
  const dim3 block(64, 4);
  if (P.sym) k_moments<PREC, FLOW, TH, true><<<grid_for(P.nx, P.ny, block), block, 0, s>>>(P, mask, out);
  else k_moments<PREC, FLOW, TH, false><<<grid_for(P.nx, P.ny, block), block, 0, s>>>(P, mask, out);
  return cudaGetLastError();
}

template <int PREC, int FLOW, int TH>
cudaError_t SpOps<PREC, FLOW, TH>::integrals(const SpParams &P, double *partials, double *out4, unsigned *counter,
                                             cudaStream_t s) {
  const dim3 block(kRedBX, kRedBY);
  const double n_rho0 = (double)P.nx * P.ny * P.rho0, area = P.dx * P.dx;
  int steps, fy;
  const dim3 grid = integral_grid(P.nx, P.ny, &steps, &fy);
  if (P.sym)
    k_integrals<PREC, FLOW, TH, true><<<grid, block, 0, s>>>(P, steps, fy, partials, n_rho0, area, out4, counter);
  else
    k_integrals<PREC, FLOW, TH, false><<<grid, block, 0, s>>>(P, steps, fy, partials, n_rho0, area, out4, counter);
  return cudaGetLastError();
}

#define LBM_SP_INSTANTIATE(A, B, C) template struct SpOps<A, B, C>;

}  // namespace lbmk
