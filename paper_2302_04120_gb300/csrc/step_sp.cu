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
#include "sp_ops.cuh"

namespace lbmk {

// ----------------------------------------------------------------------------
// Dispatch on (precision, momentum operator, thermal operator); the kernels are
// instantiated in step_sp_a.cu ... step_sp_d.cu
// ----------------------------------------------------------------------------
static dim3 grid_for(int nx, int ny, dim3 b) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y); }

cudaError_t sp_step(const SpParams &P, int prec, int flow, int th, dim3 block, cudaStream_t s) {
#define CALL(A, B, C) return SpOps<A, B, C>::step(P, block, s)
  LBM_SP_DISPATCH(prec, flow, th, CALL);
#undef CALL
  return cudaErrorInvalidValue;
}

cudaError_t sp_step_occ(const SpParams &P, int prec, int flow, int th, dim3 block, cudaStream_t s) {
#define CALL(A, B, C) return SpOps<A, B, C>::step_occ(P, block, s)
  LBM_SP_DISPATCH(prec, flow, th, CALL);
#undef CALL
  return cudaErrorInvalidValue;
}

cudaError_t sp_batch_step(const SpParams *table, const int4 *tiles, int ntiles, int prec, int flow, int th, dim3 block,
                          int grid, cudaStream_t s) {
#define CALL(A, B, C) return SpOps<A, B, C>::batch(table, tiles, ntiles, block, grid, s)
  LBM_SP_DISPATCH(prec, flow, th, CALL);
#undef CALL
  return cudaErrorInvalidValue;
}

int sp_batch_occupancy(int prec, int flow, int th, int threads) {
#define CALL(A, B, C) \
  if (prec == A && flow == B && th == C) return SpOps<A, B, C>::occupancy(threads);
  LBM_SP_COMBOS(CALL)
#undef CALL
  return 0;
}

cudaError_t sp_init(const SpParams &P, int prec, int flow, int th, const double *a, const double *ux,
                    const double *uy, const double *b, dim3 block, cudaStream_t s) {
#define CALL(A, B, C) return SpOps<A, B, C>::init(P, a, ux, uy, b, block, s)
  LBM_SP_DISPATCH(prec, flow, th, CALL);
#undef CALL
  return cudaErrorInvalidValue;
}

cudaError_t sp_moments(const SpParams &P, int prec, int flow, int th, unsigned mask, double *out,
                       cudaStream_t s) {
#define CALL(A, B, C) return SpOps<A, B, C>::moments(P, mask, out, s)
  LBM_SP_DISPATCH(prec, flow, th, CALL);
#undef CALL
  return cudaErrorInvalidValue;
}

int sp_integral_blocks(int nx, int ny) {
  int steps, fy;
  dim3 g = integral_grid(nx, ny, &steps, &fy);
  return (int)(g.x * g.y);
}

cudaError_t sp_integrals(const SpParams &P, int prec, int flow, int th, double *partials, int max_blocks,
                         double *out4, unsigned *counter, cudaStream_t s) {
  int steps, fy;
  dim3 grid = integral_grid(P.nx, P.ny, &steps, &fy);
  if ((int)(grid.x * grid.y) > max_blocks) return cudaErrorInvalidValue;
#define CALL(A, B, C) return SpOps<A, B, C>::integrals(P, partials, out4, counter, s)
  LBM_SP_DISPATCH(prec, flow, th, CALL);
#undef CALL
  return cudaErrorInvalidValue;
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
