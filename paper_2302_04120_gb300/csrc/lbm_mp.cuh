// Internal declarations of the two-phase kernels (step_mp.cu).
#pragma once
#include <cuda_runtime.h>

namespace lbmk {

// Constants of a two-phase solve in the working precision R (host-filled, so the
// FP32 kernels convert nothing per thread on GB300's slow FP64 pipe).
template <typename R>
struct MpConst {
  R c, dt, inv_cs2, g3, l6, beta, kappa, rho_g, drl, nu_g, dnu, zg, dzeta, inv_cs2dt;
  R Fx, Fy, hdt, pcoef, om_h, sfac_h, aint_coef, inv_dt, ic;
};

// Two-phase solve; each axis periodic or bounded by resting half-way walls on both
// sides.  State planes: z_0..8, h_0..4, (phi u)_x, (phi u)_y of the previous step.
struct MpParams {
  int nx, ny, pitch;
  long long plane;
  double c, cs2, dt, dx;
  double rho_l, rho_g, nu_l, nu_g;
  double kappa, beta, W, tauphi;
  // derived constants (host-side): 1/c_s^2, 3/dx, 6/dx^2, 1/(c_s^2 dt), dt/tau_phi,
  // (1 - dt/(2 tau_phi)) dt, 4 c_s^2 / W, 1/dt
  double inv_cs2, g3, l6, inv_cs2dt, om_h, sfac_h, aint_coef, inv_dt;
  int nu_rule, z_mrt, qy_literal;
  int xwall, ywall;  // 1: the axis ends at resting walls (bounce-back, mirrored phi)
  double Fx, Fy;
  MpConst<double> kd;
  MpConst<float> kf;
  const void *force;  // 2 planes or null
  int local;          // 1: src holds the pre-collision state itself (after init)
  const void *src;
  void *dst;
};

template <typename R>
__device__ __forceinline__ const MpConst<R> &KM(const MpParams &P);
template <>
__device__ __forceinline__ const MpConst<double> &KM<double>(const MpParams &P) { return P.kd; }
template <>
__device__ __forceinline__ const MpConst<float> &KM<float>(const MpParams &P) { return P.kf; }

cudaError_t mp_step(const MpParams &P, int prec, cudaStream_t s);
// Equilibria of the given fields (pre-collision state of time 0) into P.dst.
cudaError_t mp_init(const MpParams &P, int prec, const double *phi0, const double *ux0, const double *uy0,
                    const double *p0, cudaStream_t s);
cudaError_t mp_moments(const MpParams &P, int prec, unsigned mask, double *out, cudaStream_t s);
cudaError_t mp_integrals(const MpParams &P, int prec, double *partials, int max_blocks, double *out4,
                         cudaStream_t s);
int mp_integral_blocks(int nx, int ny);

}  // namespace lbmk
