// Lagged linear heat sink of the fuse problem (Sec. 4.1 of Martins, Alvarino &
// Cabezas-Gomez, arXiv:2302.04120, Eq. conver_energy_fuse): the source of a step is
// qdot(t) = qbase - conv (T(t - dt) - T_inf), with T of the previous step so that the
// update stays explicit.
//
// T(t - dt) is rebuilt at each node from the node's own post-collision populations
// of that step, which the pull step has not moved yet: the thermal collision keeps
// the zeroth moment and adds dt qdot to it (BGK with the (1 - dt/2tau_T) source
// factor, and MRT with a zero rate on the zeroth moment), so
//     T(t - dt) = T0 + sum_q g*_q - dt qdot(t - dt) / 2      (deviation storage),
// and right after initialisation (the buffer holds g(0) itself) T(-dt) = T0 + sum g.
// The two qdot fields ping-pong with the state buffers: qprev is the one used by the
// step that wrote `src`, qnext the one for the step that reads it, so the kernel can
// run again on the same state with the same result.
#include <cuda_runtime.h>

#include "lbm_internal.cuh"

namespace lbmk {

namespace {

template <typename S>
__global__ void k_lagged_qdot(const S *src, const S *qprev, const S *qbase, S *qnext, int nx, int ny, int pitch,
                              long long plane, int gbase, int qg, double T0, double dt, double conv, double Tinf,
                              int pre) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const long long n = (long long)j * pitch + i;
  const S *g = src + (long long)gbase * plane + n;
  double s = 0.0;
  for (int q = 0; q < qg; q++) s += (double)g[q * plane];
  const double Tp = T0 + s - (pre ? 0.0 : 0.5 * dt * (double)qprev[n]);
  const double b = qbase ? (double)qbase[n] : 0.0;
  qnext[n] = (S)(b - conv * (Tp - Tinf));
}

}  // namespace

cudaError_t lagged_qdot(const void *src, const void *qprev, const void *qbase, void *qnext, int nx, int ny, int pitch,
                        long long plane, int gbase, int qg, double T0, double dt, double conv, double Tinf, int pre,
                        int precision, cudaStream_t s) {
  const dim3 b(64, 4), g((nx + 63) / 64, (ny + 3) / 4);
  if (precision == 0)
    k_lagged_qdot<double><<<g, b, 0, s>>>((const double *)src, (const double *)qprev, (const double *)qbase,
                                          (double *)qnext, nx, ny, pitch, plane, gbase, qg, T0, dt, conv, Tinf, pre);
  else
    k_lagged_qdot<float><<<g, b, 0, s>>>((const float *)src, (const float *)qprev, (const float *)qbase,
                                         (float *)qnext, nx, ny, pitch, plane, gbase, qg, T0, dt, conv, Tinf, pre);
  return cudaGetLastError();
}

}  // namespace lbmk
