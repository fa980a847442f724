// Single-phase kernels of the dimensional lattice Boltzmann method
// (Martins, Alvarino & Cabezas-Gomez, arXiv:2302.04120) for sm_103a.
//
// One thread = one lattice node.  Each step is ONE kernel launch that
//   1. pulls f_i(x, t) = f_i*(x - c_i dt, t - dt) from the post-collision buffer
//      of the previous step (Eq. eq_lattice_boltzmann_geral, streaming part),
//      replacing links that leave the domain by the link-wise boundary rules
//      (Eqs. BB_vel, anti_BB_vel, anti_BB_T, BB_T, periodic and outlet
//      extrapolation of Sec. 2.1/2.2);
//   2. takes the moments (Eqs. zero_moment_f, first_moment_f, zero_moment_g);
//   3. collides: BGK (Eq. eq_lattice_boltzmann_BGK with Guo forcing, Eq.
//      forcing_term) or MRT (Eq. colisao_MRT with [M]_dim, Eq. M_matrix_dim,
//      and the dimensional rates of Sec. 3), and the D2Q5 thermal LBE (Eqs.
//      eq_lattice_boltzmann_BGK_T, forcing_term_g, geq_geral);
//   4. stores the post-collision values into the other ping-pong buffer.
//
// Storage is structure-of-arrays: plane q holds population q on an ny x pitch
// grid, so the 32 lanes of a warp touch 32 consecutive nodes of one plane.
// Populations are stored as deviations from the rest equilibrium
// (f_i - w_i rho0, g_i - w_i T0): in FP32 this keeps the non-equilibrium
// digits of f_i ~ 1e3 kg m^-3; in FP64 it costs nothing because the deviation
// form of every formula has the same operation count.
//
// MRT without matrices: [M]_dim = D [M] with D = diag(c^n), so the relaxation
// is done on the lattice-scaled moments M f (integer combinations) with the
// equilibrium and forcing moments divided by c^n, and [M]_dim^-1 is applied as
// M^T diag(1/|row|^2) D^-1 -- the same arithmetic as the matrices of Sec. 3 /
// App. A up to rounding order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lattice.cuh"
#include "lbm_internal.cuh"
#include "sp_device.cuh"

namespace lbmk {

// ----------------------------------------------------------------------------
// Kernels
// ----------------------------------------------------------------------------
// One node: pull with boundary links, moments, collision, store.  INNER: the
// caller guarantees an interior node of a non-local step (no boundary code).
template <int PREC, int FLOW, int TH, bool INNER = false>
__device__ __forceinline__ void step_node(const SpParams &P, int i, int j) {
  typedef typename Prec<PREC>::S S;
  typedef typename Prec<PREC>::R R;
  const long long n = (long long)j * P.pitch + i;
  const S *src = (const S *)P.src;
  S *dst = (S *)P.dst;
  const bool interior = INNER || (!P.local && (i > 0) && (i < P.nx - 1) && (j > 0) && (j < P.ny - 1));
  R f[9], g[5];
  if (FLOW != FLOW_NONE) pull_f<S, R>(P, src, i, j, interior, f);
  if (TH != TH_NONE) pull_g<S, R>(P, src, i, j, interior, g);
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
    for (int q = 0; q < 5; q++) gd[q * P.plane + n] = (S)g[q];
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
template <int PREC, int FLOW, int TH>
__global__ void __launch_bounds__(256, PREC == 1 ? 4 : 3) k_step_split(const SpParams P, int fy) {
  if ((int)blockIdx.y < fy) {
    const int nt = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    int i, j;
    if (frame_node(P.nx, P.ny, (blockIdx.y * gridDim.x + blockIdx.x) * nt + tid, i, j))
      step_node<PREC, FLOW, TH>(P, i, j);
    return;
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = (blockIdx.y - fy) * blockDim.y + threadIdx.y;
  if (i <= 0 || j <= 0 || i >= P.nx - 1 || j >= P.ny - 1) return;
  step_node<PREC, FLOW, TH, true>(P, i, j);
}

// Every node in one pass (the first step after initialisation, whose pull is local).
template <int PREC, int FLOW, int TH>
__global__ void __launch_bounds__(256) k_step(const SpParams P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= P.nx || j >= P.ny) return;
  step_node<PREC, FLOW, TH>(P, i, j);
}

// Many independent solves in one launch: blocks walk a flattened list of entries
// with a grid stride; the channel's parameters (sizes, boundaries, rates, buffers of
// this parity) sit in a device table.  An entry (channel, x0, y0, 0) is one
// blockDim.x x blockDim.y tile of the channel's interior; an entry (channel, f0, 0, 1)
// is blockDim.x * blockDim.y consecutive nodes of its boundary frame from frame
// index f0 (the list puts these first), as in k_step_split.
template <int PREC, int FLOW, int TH>
__global__ void __launch_bounds__(256, PREC == 1 ? 4 : 3) k_batch_step(const SpParams *__restrict__ table, const int4 *__restrict__ tiles,
                                                     int ntiles) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int4 tl = tiles[t];
    const SpParams &P = table[tl.x];
    if (tl.w == 1) {
      int i, j;
      const int f = tl.y + threadIdx.y * blockDim.x + threadIdx.x;
      if (frame_node(P.nx, P.ny, f, i, j)) step_node<PREC, FLOW, TH>(P, i, j);
      continue;
    }
    const int i = tl.y + threadIdx.x, j = tl.z + threadIdx.y;
    if (i <= 0 || j <= 0 || i >= P.nx - 1 || j >= P.ny - 1) continue;  // frame entries
    if (P.local) step_node<PREC, FLOW, TH>(P, i, j);
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
    S *gd = dst + (long long)P.gbase * P.plane;
#pragma unroll
    for (int q = 0; q < 5; q++) {
      double cu = c * (cx5(q) * u0 + cy5(q) * v0);
      gd[q * P.plane + n] = (S)(w5<double>(q) * ((T - P.T0) + T * cu * inv_cs2));
    }
  }
}

// Macroscopic fields of the current time: pull (with boundary rules) + moments.
template <int PREC, int FLOW, int TH>
__global__ void __launch_bounds__(256) k_moments(const SpParams P, unsigned mask, double *out) {
  typedef typename Prec<PREC>::S S;
  typedef typename Prec<PREC>::R R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= P.nx || j >= P.ny) return;
  const long long n = (long long)j * P.pitch + i;
  const S *src = (const S *)P.src;
  const bool interior = !P.local && (i > 0) && (i < P.nx - 1) && (j > 0) && (j < P.ny - 1);
  R f[9], g[5];
  if (FLOW != FLOW_NONE) pull_f<S, R>(P, src, i, j, interior, f);
  if (TH != TH_NONE) pull_g<S, R>(P, src, i, j, interior, g);
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
// adds N rho0 and takes the one square root.
__device__ __forceinline__ void block_partials(double drho, double u2, int bad, double *out) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    drho += __shfl_down_sync(0xffffffffu, drho, o);
    u2 = fmax(u2, __shfl_down_sync(0xffffffffu, u2, o));
  }
  const int nbad = __popc(__ballot_sync(0xffffffffu, bad));
  __shared__ double sh[8][3];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
  if (lane == 0) { sh[warp][0] = drho; sh[warp][1] = u2; sh[warp][2] = (double)nbad; }
  __syncthreads();
  if (tid == 0) {
    double a = 0, mx = 0, cnt = 0;
    for (int w = 0; w < nw; w++) { a += sh[w][0]; mx = fmax(mx, sh[w][1]); cnt += sh[w][2]; }
    out[0] = a; out[1] = 0.0; out[2] = mx; out[3] = cnt;
  }
}

// Fixed-order sum of the nb per-block partials by one 256-thread block: thread t sums
// partials t, t + 256, ... in order, then a fixed tree.  mass = (N rho0 + sum (rho -
// rho0)) dx^2, max |u| = sqrt(max |u|^2).
__device__ __forceinline__ void final_reduce(const double *partials, int nb, double n_rho0, double area,
                                             double *out4) {
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  double a = 0, b = 0, mx = 0, cnt = 0;
  for (int k = t; k < nb; k += 256) {
    a += __ldcg(partials + 4 * k + 0);
    b += __ldcg(partials + 4 * k + 1);
    mx = fmax(mx, __ldcg(partials + 4 * k + 2));
    cnt += __ldcg(partials + 4 * k + 3);
  }
  __shared__ double sh[4][256];
  sh[0][t] = a; sh[1][t] = b; sh[2][t] = mx; sh[3][t] = cnt;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (t < w) {
      sh[0][t] += sh[0][t + w];
      sh[1][t] += sh[1][t + w];
      sh[2][t] = fmax(sh[2][t], sh[2][t + w]);
      sh[3][t] += sh[3][t + w];
    }
    __syncthreads();
  }
  if (t == 0) {
    out4[0] = (n_rho0 + sh[0][0]) * area;
    out4[1] = sh[1][0];
    out4[2] = sqrt(sh[2][0]);
    out4[3] = sh[3][0];
  }
}

// Integrals in one launch: every block writes its partials; the block that counts
// last (a device counter, 0 on entry and reset by that block) makes the final pass.
template <int PREC, int FLOW, int TH>
__global__ void __launch_bounds__(256) k_integrals(const SpParams P, double *partials, double n_rho0, double area,
                                                   double *out4, unsigned *counter) {
  typedef typename Prec<PREC>::S S;
  typedef typename Prec<PREC>::R R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  double drho = 0.0, u2 = 0.0;
  int bad = 0;
  if (i < P.nx && j < P.ny) {
    const long long n = (long long)j * P.pitch + i;
    const S *src = (const S *)P.src;
    const bool interior = !P.local && (i > 0) && (i < P.nx - 1) && (j > 0) && (j < P.ny - 1);
    R f[9], g[5];
    if (FLOW != FLOW_NONE) pull_f<S, R>(P, src, i, j, interior, f);
    if (TH != TH_NONE) pull_g<S, R>(P, src, i, j, interior, g);
    Macro<R> m;
    load_sources<S, R>(P, n, m);
    moments<R, FLOW, TH>(P, f, g, m);
    const double ux = (double)m.ux, uy = (double)m.uy;
    drho = (double)m.drho;
    u2 = ux * ux + uy * uy;
    const R Tchk = (TH != TH_NONE) ? m.T : (R)0;
    bad = !isfinite(drho) || !isfinite(u2) || !isfinite(Tchk) || u2 >= P.c * P.c;
    if (bad) { drho = 0.0; u2 = 0.0; }
  }
  block_partials(drho, u2, bad, partials + 4ll * (blockIdx.y * gridDim.x + blockIdx.x));
  const unsigned nb = gridDim.x * gridDim.y;
  __shared__ bool last;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();  // this block's partials before its count
    last = atomicAdd(counter, 1u) == nb - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    final_reduce(partials, (int)nb, n_rho0, area, out4);
    if (threadIdx.x == 0 && threadIdx.y == 0) *counter = 0u;
  }
}

// ----------------------------------------------------------------------------
// Dispatch
// ----------------------------------------------------------------------------
static dim3 grid_for(int nx, int ny, dim3 b) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y); }


cudaError_t sp_step(const SpParams &P, int prec, int flow, int th, dim3 block, cudaStream_t s) {
  dim3 grid = grid_for(P.nx, P.ny, block);
  const int nt = block.x * block.y;
  const int nfb = (frame_nodes(P.nx, P.ny) + nt - 1) / nt;  // frame blocks
  const int fy = (nfb + (int)grid.x - 1) / (int)grid.x;      // rows of them
  if (!P.local && grid.y + fy <= 65535u) {                   // else the one-pass kernel
    const dim3 g2(grid.x, grid.y + fy);
#define CALL_SPLIT(A, B, C) k_step_split<A, B, C><<<g2, block, 0, s>>>(P, fy)
    LBM_SP_DISPATCH(prec, flow, th, CALL_SPLIT);
#undef CALL_SPLIT
    return cudaGetLastError();
  }
#define CALL_STEP(A, B, C) k_step<A, B, C><<<grid, block, 0, s>>>(P)
  LBM_SP_DISPATCH(prec, flow, th, CALL_STEP);
#undef CALL_STEP
  return cudaGetLastError();
}

cudaError_t sp_batch_step(const SpParams *table, const int4 *tiles, int ntiles, int prec, int flow, int th, dim3 block,
                          int grid, cudaStream_t s) {
#define CALL_BATCH(A, B, C) k_batch_step<A, B, C><<<grid, block, 0, s>>>(table, tiles, ntiles)
  LBM_SP_DISPATCH(prec, flow, th, CALL_BATCH);
#undef CALL_BATCH
  return cudaGetLastError();
}

int sp_batch_occupancy(int prec, int flow, int th, int threads) {
  int nb = 0;
#define CALL_OCC(A, B, C) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_step<A, B, C>, threads, 0)
  do {
    if (prec == 0) {
      if (flow == FLOW_BGK && th == TH_NONE) CALL_OCC(0, FLOW_BGK, TH_NONE);
      else if (flow == FLOW_BGK && th == TH_BGK) CALL_OCC(0, FLOW_BGK, TH_BGK);
      else if (flow == FLOW_BGK && th == TH_MRT) CALL_OCC(0, FLOW_BGK, TH_MRT);
      else if (flow == FLOW_MRT && th == TH_NONE) CALL_OCC(0, FLOW_MRT, TH_NONE);
      else if (flow == FLOW_MRT && th == TH_BGK) CALL_OCC(0, FLOW_MRT, TH_BGK);
      else if (flow == FLOW_MRT && th == TH_MRT) CALL_OCC(0, FLOW_MRT, TH_MRT);
      else if (flow == FLOW_NONE && th == TH_BGK) CALL_OCC(0, FLOW_NONE, TH_BGK);
      else if (flow == FLOW_NONE && th == TH_MRT) CALL_OCC(0, FLOW_NONE, TH_MRT);
    } else {
      if (flow == FLOW_BGK && th == TH_NONE) CALL_OCC(1, FLOW_BGK, TH_NONE);
      else if (flow == FLOW_BGK && th == TH_BGK) CALL_OCC(1, FLOW_BGK, TH_BGK);
      else if (flow == FLOW_BGK && th == TH_MRT) CALL_OCC(1, FLOW_BGK, TH_MRT);
      else if (flow == FLOW_MRT && th == TH_NONE) CALL_OCC(1, FLOW_MRT, TH_NONE);
      else if (flow == FLOW_MRT && th == TH_BGK) CALL_OCC(1, FLOW_MRT, TH_BGK);
      else if (flow == FLOW_MRT && th == TH_MRT) CALL_OCC(1, FLOW_MRT, TH_MRT);
      else if (flow == FLOW_NONE && th == TH_BGK) CALL_OCC(1, FLOW_NONE, TH_BGK);
      else if (flow == FLOW_NONE && th == TH_MRT) CALL_OCC(1, FLOW_NONE, TH_MRT);
    }
  } while (0);
#undef CALL_OCC
  return nb;
}

cudaError_t sp_init(const SpParams &P, int prec, int flow, int th, const double *a, const double *ux,
                    const double *uy, const double *b, dim3 block, cudaStream_t s) {
  dim3 grid = grid_for(P.nx, P.ny, block);
#define CALL_INIT(A, B, C) k_init<A, B, C><<<grid, block, 0, s>>>(P, a, ux, uy, b)
  LBM_SP_DISPATCH(prec, flow, th, CALL_INIT);
#undef CALL_INIT
  return cudaGetLastError();
}

cudaError_t sp_moments(const SpParams &P, int prec, int flow, int th, unsigned mask, double *out,
                       cudaStream_t s) {
  dim3 block(64, 4);
  dim3 grid = grid_for(P.nx, P.ny, block);
#define CALL_MOM(A, B, C) k_moments<A, B, C><<<grid, block, 0, s>>>(P, mask, out)
  LBM_SP_DISPATCH(prec, flow, th, CALL_MOM);
#undef CALL_MOM
  return cudaGetLastError();
}

static const dim3 kRedBlock(64, 4);

int sp_integral_blocks(int nx, int ny) {
  dim3 g = grid_for(nx, ny, kRedBlock);
  return (int)(g.x * g.y);
}

cudaError_t sp_integrals(const SpParams &P, int prec, int flow, int th, double *partials, int max_blocks,
                         double *out4, unsigned *counter, cudaStream_t s) {
  dim3 grid = grid_for(P.nx, P.ny, kRedBlock);
  if ((int)(grid.x * grid.y) > max_blocks) return cudaErrorInvalidValue;
  const double n_rho0 = (double)P.nx * P.ny * P.rho0, area = P.dx * P.dx;
#define CALL_INT(A, B, C) k_integrals<A, B, C><<<grid, kRedBlock, 0, s>>>(P, partials, n_rho0, area, out4, counter)
  LBM_SP_DISPATCH(prec, flow, th, CALL_INT);
#undef CALL_INT
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Layout helpers
// ----------------------------------------------------------------------------
template <typename S>
__global__ void k_to_storage(const double *in, S *out, int nx, int ny, int pitch, int nplanes,
                             long long plane, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  for (int p = 0; p < nplanes; p++)
    out[p * plane + (long long)j * pitch + i] = (S)(scale * in[(long long)p * nx * ny + (long long)j * nx + i]);
}

cudaError_t to_storage(const double *in, void *out, int nx, int ny, int pitch, int nplanes, long long plane,
                       int prec, double scale, cudaStream_t s) {
  dim3 b(64, 4), g = grid_for(nx, ny, b);
  if (prec == 0) k_to_storage<double><<<g, b, 0, s>>>(in, (double *)out, nx, ny, pitch, nplanes, plane, scale);
  else k_to_storage<float><<<g, b, 0, s>>>(in, (float *)out, nx, ny, pitch, nplanes, plane, scale);
  return cudaGetLastError();
}

template <typename S>
__global__ void k_pack(const S *state, S *packed, int nx, int ny, int pitch, int nq, long long plane, int unpack) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  for (int q = 0; q < nq; q++) {
    long long a = q * plane + (long long)j * pitch + i;
    long long b = ((long long)q * ny + j) * nx + i;
    if (unpack) ((S *)state)[a] = packed[b];
    else packed[b] = state[a];
  }
}

cudaError_t pack_state(const void *state, void *packed, int nx, int ny, int pitch, int nq, long long plane,
                       int elem, int unpack, cudaStream_t s) {
  dim3 b(64, 4), g = grid_for(nx, ny, b);
  if (elem == 8) k_pack<double><<<g, b, 0, s>>>((const double *)state, (double *)packed, nx, ny, pitch, nq, plane, unpack);
  else k_pack<float><<<g, b, 0, s>>>((const float *)state, (float *)packed, nx, ny, pitch, nq, plane, unpack);
  return cudaGetLastError();
}

}  // namespace lbmk
