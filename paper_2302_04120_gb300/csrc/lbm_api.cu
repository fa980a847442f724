// Host side of the C ABI declared in include/lbm.h: parameter validation,
// derived constants (Sec. 3 of the paper), device buffer ownership, boundary
// upload, launches and status reporting.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "../../include/lbm.h"
#include "lbm_internal.cuh"
#include "lbm_mp.cuh"

using lbmk::SpParams;

struct lbm_s {
  lbm_params p;
  cudaStream_t stream;
  // derived SI constants
  double c, cs2, tau, tauT, tauphi;
  int pitch;
  long long plane;
  int nq;          // planes in one state buffer
  size_t elem;     // bytes per stored value
  void *buf[2];    // ping-pong post-collision buffers
  int cur;         // index of the buffer holding the latest state
  int pre;         // 1: buf[cur] holds the pre-collision state f(t) itself (after init)
  int initialised;
  long steps;
  // boundaries
  int bc[4], tbc[4];
  double rho_w[4];
  double *d_uw[4], *d_tw[4];
  double *h_stage[4];        // pinned staging of the boundary arrays, one slot per side
  cudaEvent_t stage_done[4];  // the slot's last upload has been consumed
  int uw_zero[4], tw_zero[4];  // the device array holds zeros (no upload since the last fill)
  // sources (storage precision, pitched)
  void *d_qdot, *d_force;
  // lagged heat sink (lbm_set_lagged_sink): qdot = qbase - conv (T(t - dt) - T_inf); the
  // two qdot fields ping-pong with buf[]: d_qs[b] is the one the step writing buf[b] used
  double sink_conv, sink_Tinf;
  void *d_qbase, *d_qs[2];
  // reductions
  double *d_partials;
  int max_blocks;
  double *d_out4;  // 4 integrals, the step kernels' error flag (an int in slot 4) and the
                   // integrals' block counter (an unsigned in slot 5, zero between calls)
  double *h_out4;  // pinned, 5 doubles
  dim3 block;
  // single-phase step launch: LBM_LAUNCH_GRID (one node per thread, `block`) or
  // LBM_LAUNCH_TMA (persistent CTAs of 32 x tma_ty threads, boxes staged by TMA)
  int launch_kind;
  int tma_ty, tma_stages, tma_ctas;  // tma_ctas: CTAs per SM
  unsigned long long tma_wait_ns;    // wall-time limit of each staged-copy wait
  int tma_expire_next;               // self-test: the next TMA-staged step's waits run out
  // health check inside lbm_step: every `check_every` steps (0 = off); the step count
  // of the last check that found every cell healthy (-1: none since init)
  long check_every, last_good;
  int nsm;
  CUtensorMap tmap[2];  // one per state buffer, boxes 36 x tmap_ty
  int tmap_ty;          // 0 until encoded
  // Replay of kGraphSteps consecutive grid-launched steps as one CUDA graph, captured
  // on a private stream (capture only records) and launched on `stream`.  One graph
  // per parity of the buffer a run starts from; each stays valid while the launch
  // parameters it was captured with (gkey) are unchanged.
  cudaStream_t cap_stream;
  cudaGraphExec_t gexec[2];
  struct StepKey *gkey[2];
  char err[512];
};

// Everything a run of grid-launched steps depends on besides device memory contents:
// the kernel choice and the parameter blocks of both buffer parities.
struct StepKey {
  int two_phase, prec, flow, th, kind;
  dim3 block;
  double sink_conv, sink_Tinf;
  lbmk::MpParams mp[2];
  SpParams sp[2];
};
static constexpr long kGraphSteps = 64;  // even: the ping-pong buffers end where they start

static char g_create_err[512];

void lbmk::set_global_error(const char *msg) { snprintf(g_create_err, sizeof(g_create_err), "%s", msg); }

static lbm_status fail(lbm_t h, lbm_status st, const char *fmt, ...) {
  char *dst = h ? h->err : g_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return st;
}

#define CU(h, call)                                                                      \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(h, LBM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

extern "C" void lbm_params_default(lbm_params *p) {
  memset(p, 0, sizeof(*p));
  p->flow = LBM_D2Q9;
  p->flow_op = LBM_BGK;
  p->thermal = LBM_NONE;
  p->thermal_op = LBM_BGK;
  p->phase = LBM_NONE;
  p->z_op = LBM_MRT;
  p->precision = LBM_FP64;
  p->nx = p->ny = 1;
  p->dx = 1.0;
  p->dt = 1.0;
  p->rho0 = 1000.0;
  p->nu = 1e-6;
  p->cp = 4180.0;
  p->k = 0.6;
  p->T0 = 300.0;
  p->W = 1.0;
  p->omega_e_dt = 1.0;
  p->omega_eps_dt = 1.0;
}

static int two_phase(const lbm_t h) { return h->p.phase != LBM_NONE; }

// Thermal kernel kind of a parameter set: lattice (D2Q5 / D2Q9) x operator.
static int th_kind(const lbm_params &p) {
  if (!p.thermal) return lbmk::TH_NONE;
  if (p.thermal == LBM_D2Q9) return p.thermal_op == LBM_MRT ? lbmk::TH_MRT9 : lbmk::TH_BGK9;
  return p.thermal_op == LBM_MRT ? lbmk::TH_MRT : lbmk::TH_BGK;
}

static int axis_periodic(const lbm_t h, int axis, int thermal) {
  int a = axis == 0 ? 0 : 2, b = a + 1;
  if (thermal) return h->tbc[a] == LBM_TBC_NONE && h->tbc[b] == LBM_TBC_NONE;
  return h->bc[a] == LBM_BC_PERIODIC && h->bc[b] == LBM_BC_PERIODIC;
}

template <typename R>
static void fill_const(const SpParams &P, lbmk::SpConst<R> &k) {
  k.c = (R)P.c; k.cs2 = (R)P.cs2; k.dt = (R)P.dt; k.rho0 = (R)P.rho0; k.T0 = (R)P.T0;
  // the same IEEE divisions the kernels would take per thread, taken once here
  k.inv_c = (R)1 / k.c; k.inv_cs2 = (R)1 / k.cs2; k.three_inv_c2 = (R)3 / (k.c * k.c);
  k.hdt = (R)0.5 * k.dt;
  k.fk_e = ((R)1 - (R)0.5 * (R)P.s_e) * k.dt;
  k.fk_eps = ((R)1 - (R)0.5 * (R)P.s_eps) * k.dt;
  k.fk_q = ((R)1 - (R)0.5 * (R)P.s_q) * k.dt;
  k.fk_nu = ((R)1 - (R)0.5 * (R)P.s_nu) * k.dt;
  k.Fx = (R)P.Fx; k.Fy = (R)P.Fy; k.ux_pres = (R)P.ux_pres; k.uy_pres = (R)P.uy_pres;
  k.omega = (R)P.omega; k.s_e = (R)P.s_e; k.s_eps = (R)P.s_eps; k.s_q = (R)P.s_q; k.s_nu = (R)P.s_nu;
  k.omegaT = (R)P.omegaT; k.tsrc_fac = (R)P.tsrc_fac; k.flux_coef = (R)P.flux_coef;
  k.bgx = (R)P.bgx; k.bgy = (R)P.bgy; k.T_ref = (R)P.T_ref;
  for (int s = 0; s < 4; s++) k.rho_w[s] = (R)P.side[s].rho_w;
}

static SpParams sp_params(const lbm_t h, int from_buf) {
  SpParams P;
  memset(&P, 0, sizeof(P));
  const lbm_params &p = h->p;
  P.nx = p.nx; P.ny = p.ny; P.pitch = h->pitch; P.plane = h->plane;
  P.xper = axis_periodic(h, 0, 0); P.yper = axis_periodic(h, 1, 0);
  P.txper = axis_periodic(h, 0, 1); P.typer = axis_periodic(h, 1, 1);
  P.gbase = p.flow == LBM_D2Q9 ? 9 : 0;
  P.qg = p.thermal ? p.thermal : 0;
  P.fysym = (h->bc[2] == LBM_BC_SYMMETRY ? 1 : 0) | (h->bc[3] == LBM_BC_SYMMETRY ? 2 : 0);
  P.tysym = (h->tbc[2] == LBM_TBC_SYMMETRY ? 1 : 0) | (h->tbc[3] == LBM_TBC_SYMMETRY ? 2 : 0);
  P.sym = 0;
  // the boundary-rule variant of the kernels: symmetry sides and wet-node sides
  for (int s = 0; s < 4; s++)
    P.sym |= h->bc[s] == LBM_BC_SYMMETRY || h->tbc[s] == LBM_TBC_SYMMETRY || h->tbc[s] == LBM_TBC_WETNODE;
  for (int s = 0; s < 4; s++) {
    P.side[s].kind = h->bc[s];
    P.side[s].tkind = h->tbc[s];
    P.side[s].rho_w = h->rho_w[s];
    P.side[s].uw = h->d_uw[s];
    P.side[s].tw = h->d_tw[s];
  }
  P.c = h->c; P.cs2 = h->cs2; P.dt = p.dt; P.dx = p.dx;
  P.rho0 = p.rho0; P.T0 = p.T0;
  P.Fx = p.body_force[0]; P.Fy = p.body_force[1];
  P.ux_pres = p.u_prescribed[0]; P.uy_pres = p.u_prescribed[1];
  P.omega = p.dt / h->tau;
  // dimensional MRT rates (Sec. 3) times dt
  const double wnu = 1.0 / h->tau;
  const double wq = (3.0 / p.dt) * (2.0 / p.dt - wnu) / (3.0 / p.dt - wnu);
  P.s_e = p.omega_e_dt; P.s_eps = p.omega_eps_dt; P.s_q = wq * p.dt; P.s_nu = wnu * p.dt;
  if (p.thermal) {
    P.omegaT = p.dt / h->tauT;
    const double tau_sg = (p.literal & 1) ? h->tau : h->tauT;  // reading R1
    P.tsrc_fac = 1.0 - p.dt / (2.0 * tau_sg);
    P.flux_coef = p.dt / (p.dx * p.rho0 * p.cp);
    if (p.flow && p.beta_exp != 0.0) {
      P.buoy = 1;
      P.bgx = -p.rho_ref * p.beta_exp * p.gravity[0];
      P.bgy = -p.rho_ref * p.beta_exp * p.gravity[1];
      P.T_ref = p.T_ref;
    }
  }
  P.qdot = h->sink_conv != 0.0 ? h->d_qs[1 - from_buf] : h->d_qdot;
  P.force = h->d_force;
  fill_const(P, P.kd);
  fill_const(P, P.kf);
  P.local = h->pre;
  P.src = h->buf[from_buf];
  P.dst = h->buf[1 - from_buf];
  return P;
}

template <typename R>
static void fill_mp_const(const lbmk::MpParams &P, lbmk::MpConst<R> &k) {
  k.c = (R)P.c; k.dt = (R)P.dt; k.inv_cs2 = (R)P.inv_cs2; k.g3 = (R)P.g3; k.l6 = (R)P.l6;
  k.beta = (R)P.beta; k.kappa = (R)P.kappa; k.rho_g = (R)P.rho_g; k.drl = (R)(P.rho_l - P.rho_g);
  k.nu_g = (R)P.nu_g; k.dnu = (R)(P.nu_l - P.nu_g); k.zg = (R)(P.rho_g * P.nu_g);
  k.dzeta = (R)(P.rho_l * P.nu_l - P.rho_g * P.nu_g); k.inv_cs2dt = (R)P.inv_cs2dt;
  k.Fx = (R)P.Fx; k.Fy = (R)P.Fy; k.hdt = (R)(0.5 * P.dt); k.pcoef = (R)(P.cs2 * 1.8);
  k.om_h = (R)P.om_h; k.sfac_h = (R)P.sfac_h; k.aint_coef = (R)P.aint_coef; k.inv_dt = (R)P.inv_dt;
  k.ic = (R)1 / (R)P.c;
}

static lbmk::MpParams mp_params(const lbm_t h, int from_buf) {
  lbmk::MpParams P;
  memset(&P, 0, sizeof(P));
  const lbm_params &p = h->p;
  P.nx = p.nx; P.ny = p.ny; P.pitch = h->pitch; P.plane = h->plane;
  P.c = h->c; P.cs2 = h->cs2; P.dt = p.dt; P.dx = p.dx;
  P.rho_l = p.rho_l; P.rho_g = p.rho_g; P.nu_l = p.nu_l; P.nu_g = p.nu_g;
  P.kappa = 1.5 * p.sigma * p.W;   // kappa = 3 sigma W / 2
  P.beta = 12.0 * p.sigma / p.W;   // beta = 12 sigma / W
  P.W = p.W;
  P.tauphi = h->tauphi;
  P.inv_cs2 = 1.0 / h->cs2;
  P.g3 = 3.0 / p.dx;
  P.l6 = 6.0 / (p.dx * p.dx);
  P.inv_cs2dt = 1.0 / (h->cs2 * p.dt);
  P.om_h = p.dt / h->tauphi;
  P.sfac_h = (1.0 - p.dt / (2.0 * h->tauphi)) * p.dt;
  P.aint_coef = 4.0 * h->cs2 / p.W;
  P.inv_dt = 1.0 / p.dt;
  P.nu_rule = p.nu_rule;
  P.z_mrt = p.z_op == LBM_MRT;
  P.qy_literal = (p.literal & 2) ? 1 : 0;
  P.xwall = h->bc[0] != LBM_BC_PERIODIC || h->bc[1] != LBM_BC_PERIODIC;
  P.ywall = h->bc[2] != LBM_BC_PERIODIC || h->bc[3] != LBM_BC_PERIODIC;
  P.Fx = p.body_force[0]; P.Fy = p.body_force[1];
  P.force = h->d_force;
  P.local = h->pre;
  P.src = h->buf[from_buf];
  P.dst = h->buf[1 - from_buf];
  fill_mp_const(P, P.kd);  // after every field it reads is set
  fill_mp_const(P, P.kf);
  return P;
}

extern "C" const char *lbm_last_error(lbm_t h) { return h ? h->err : g_create_err; }

extern "C" lbm_status lbm_create(const lbm_params *pin, void *stream, lbm_t *out) {
  if (!out) return fail(NULL, LBM_ERR_ARG, "out is NULL");
  *out = NULL;
  if (!pin) return fail(NULL, LBM_ERR_ARG, "params is NULL");
  const lbm_params p = *pin;
  if (p.nx < 1 || p.ny < 1) return fail(NULL, LBM_ERR_ARG, "nx, ny must be >= 1 (got %d, %d)", p.nx, p.ny);
  if ((long long)p.nx * p.ny > (1ll << 31)) return fail(NULL, LBM_ERR_ARG, "grid too large");
  if (!(p.dx > 0) || !(p.dt > 0)) return fail(NULL, LBM_ERR_ARG, "dx and dt must be positive");
  if (p.precision != LBM_FP64 && p.precision != LBM_FP32DEV) return fail(NULL, LBM_ERR_ARG, "precision");
  if (p.flow != LBM_D2Q9 && p.flow != LBM_NONE) return fail(NULL, LBM_ERR_ARG, "flow lattice must be D2Q9 or NONE");
  if (p.thermal != LBM_D2Q5 && p.thermal != LBM_D2Q9 && p.thermal != LBM_NONE)
    return fail(NULL, LBM_ERR_ARG, "thermal lattice must be D2Q5, D2Q9 or NONE");
  if (p.thermal == LBM_D2Q9 && p.flow != LBM_D2Q9)
    return fail(NULL, LBM_ERR_ARG, "a D2Q9 thermal LBE needs the D2Q9 momentum LBE");
  if (p.phase != LBM_D2Q5 && p.phase != LBM_NONE) return fail(NULL, LBM_ERR_ARG, "phase lattice must be D2Q5 or NONE");
  if (p.flow_op != LBM_BGK && p.flow_op != LBM_MRT) return fail(NULL, LBM_ERR_ARG, "flow_op");
  if (p.thermal_op != LBM_BGK && p.thermal_op != LBM_MRT) return fail(NULL, LBM_ERR_ARG, "thermal_op");
  if (p.flow == LBM_NONE && p.thermal == LBM_NONE) return fail(NULL, LBM_ERR_ARG, "nothing to solve");
  if (p.phase != LBM_NONE) {
    if (p.flow != LBM_D2Q9 || p.thermal != LBM_NONE)
      return fail(NULL, LBM_ERR_ARG, "two-phase solves need flow = D2Q9 (z_i) and no thermal LBE");
    if (!(p.rho_l > 0) || !(p.rho_g > 0) || !(p.nu_l > 0) || !(p.nu_g > 0) || !(p.W > 0) || !(p.mobility > 0) ||
        !(p.sigma >= 0))
      return fail(NULL, LBM_ERR_ARG, "two-phase properties rho_l, rho_g, nu_l, nu_g, W, mobility must be positive");
  } else if (!(p.rho0 > 0)) {
    return fail(NULL, LBM_ERR_ARG, "rho0 must be positive");
  }
  if (p.beta_exp != 0.0 && (p.flow != LBM_D2Q9 || p.thermal == LBM_NONE || p.phase != LBM_NONE))
    return fail(NULL, LBM_ERR_ARG, "buoyancy needs a single-phase D2Q9 flow with a thermal LBE");
  if (!(p.omega_e_dt > 0 && p.omega_e_dt < 2) || !(p.omega_eps_dt > 0 && p.omega_eps_dt < 2))
    return fail(NULL, LBM_ERR_ARG, "free MRT rates times dt must lie in (0, 2)");

  lbm_t h = (lbm_t)calloc(1, sizeof(struct lbm_s));
  if (!h) return fail(NULL, LBM_ERR_NOMEM, "host allocation failed");
  h->p = p;
  h->stream = (cudaStream_t)stream;
  h->c = p.dx / p.dt;                   // c = dx/dt (Sec. 2.1)
  h->cs2 = h->c * h->c / 3.0;           // c_s = c/sqrt(3)
  const double eps = 1e-12 * p.dt;
  if (p.flow == LBM_D2Q9 && p.phase == LBM_NONE) {
    if (!(p.nu > 0)) { free(h); return fail(NULL, LBM_ERR_UNSTABLE_TAU, "nu must be positive (tau > dt/2)"); }
    h->tau = p.nu / h->cs2 + 0.5 * p.dt;  // Eq. eq_kinematic_viscosity
    if (!(h->tau > 0.5 * p.dt + eps)) { free(h); return fail(NULL, LBM_ERR_UNSTABLE_TAU, "tau <= dt/2"); }
  } else {
    h->tau = 1.0;
  }
  if (p.thermal) {
    if (!(p.k > 0) || !(p.cp > 0)) { free(h); return fail(NULL, LBM_ERR_UNSTABLE_TAU, "k and cp must be positive (tau_T > dt/2)"); }
    h->tauT = (p.k / (p.rho0 * p.cp)) / h->cs2 + 0.5 * p.dt;
  }
  if (p.phase) {
    h->tauphi = p.mobility / h->cs2 + 0.5 * p.dt;  // M = (tau_phi - dt/2) c_s^2
    h->tau = p.nu_l / h->cs2 + 0.5 * p.dt;         // liquid tau, reported only
  }
  // storage layout: pitch rounded to 32 elements (128 B FP32 / 256 B FP64 rows)
  h->elem = p.precision == LBM_FP64 ? 8 : 4;
  h->pitch = (p.nx + 31) / 32 * 32;
  h->plane = (long long)h->pitch * p.ny;
  if (p.phase) h->nq = 9 + 5 + 2;   // z, h, (phi u)_prev
  else h->nq = (p.flow ? 9 : 0) + (p.thermal ? p.thermal : 0);
  h->block = dim3(64, 4);
  for (int s = 0; s < 4; s++) {
    h->bc[s] = LBM_BC_PERIODIC;
    h->tbc[s] = LBM_TBC_NONE;
    h->rho_w[s] = p.phase ? p.rho_l : p.rho0;
  }
  size_t bytes = (size_t)h->nq * h->plane * h->elem;
  cudaError_t e;
  for (int b = 0; b < 2; b++) {
    e = cudaMalloc(&h->buf[b], bytes);
    if (e != cudaSuccess) { lbm_destroy(h); return fail(NULL, LBM_ERR_NOMEM, "cudaMalloc state (%zu B): %s", bytes, cudaGetErrorString(e)); }
    cudaMemsetAsync(h->buf[b], 0, bytes, h->stream);
  }
  for (int s = 0; s < 4; s++) {
    int len = s < 2 ? p.ny : p.nx;
    e = cudaMalloc(&h->d_uw[s], sizeof(double) * 2 * len);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_tw[s], sizeof(double) * len);
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_stage[s], sizeof(double) * 3 * len);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->stage_done[s], cudaEventDisableTiming);
    if (e != cudaSuccess) { lbm_destroy(h); return fail(NULL, LBM_ERR_NOMEM, "cudaMalloc boundary arrays"); }
    cudaMemsetAsync(h->d_uw[s], 0, sizeof(double) * 2 * len, h->stream);
    cudaMemsetAsync(h->d_tw[s], 0, sizeof(double) * len, h->stream);
    h->uw_zero[s] = h->tw_zero[s] = 1;
  }
  h->max_blocks = lbmk::sp_integral_blocks(p.nx, p.ny);
  int mpb = lbmk::mp_integral_blocks(p.nx, p.ny);
  if (mpb > h->max_blocks) h->max_blocks = mpb;
  e = cudaMalloc(&h->d_partials, sizeof(double) * 4 * h->max_blocks);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_out4, sizeof(double) * 6);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_out4, 0, sizeof(double) * 6, h->stream);
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_out4, sizeof(double) * 6);
  if (e != cudaSuccess) { lbm_destroy(h); return fail(NULL, LBM_ERR_NOMEM, "cudaMalloc reduction scratch"); }
  {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) h->nsm = 1;
  }
  h->launch_kind = LBM_LAUNCH_GRID;
  h->tma_ty = 8;
  h->tma_stages = 3;
  h->tma_ctas = 2;
  h->tma_wait_ns = 1000000000ull;
  h->tmap_ty = 0;
  h->last_good = -1;
  if (!p.phase && (p.flow || p.thermal)) {
    int fk = p.flow ? (p.flow_op == LBM_MRT ? lbmk::FLOW_MRT : lbmk::FLOW_BGK) : lbmk::FLOW_NONE;
    int tk = th_kind(p);
    lbmk::sp_tma_prepare(p.precision, fk, tk);  // failure leaves only the grid launch usable
    cudaGetLastError();
  }
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) { lbm_destroy(h); return fail(NULL, LBM_ERR_CUDA, "create: %s", cudaGetErrorString(e)); }
  *out = h;
  h->err[0] = 0;
  // advisory: lattice Mach number of the prescribed velocity (not an error)
  return LBM_OK;
}

extern "C" void lbm_destroy(lbm_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  for (int b = 0; b < 2; b++) cudaFree(h->buf[b]);
  for (int s = 0; s < 4; s++) {
    cudaFree(h->d_uw[s]);
    cudaFree(h->d_tw[s]);
    if (h->h_stage[s]) cudaFreeHost(h->h_stage[s]);
    if (h->stage_done[s]) cudaEventDestroy(h->stage_done[s]);
  }
  cudaFree(h->d_qdot);
  cudaFree(h->d_qbase);
  cudaFree(h->d_qs[0]);
  cudaFree(h->d_qs[1]);
  cudaFree(h->d_force);
  cudaFree(h->d_partials);
  cudaFree(h->d_out4);
  if (h->h_out4) cudaFreeHost(h->h_out4);
  for (int k = 0; k < 2; k++) {
    if (h->gexec[k]) cudaGraphExecDestroy(h->gexec[k]);
    free(h->gkey[k]);
  }
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  free(h);
}

extern "C" lbm_status lbm_constants(lbm_t h, double out[5]) {
  if (!h || !out) return fail(h, LBM_ERR_ARG, "NULL argument");
  out[0] = h->c; out[1] = h->cs2; out[2] = h->tau; out[3] = h->tauT; out[4] = h->tauphi;
  return LBM_OK;
}

extern "C" lbm_status lbm_set_bc(lbm_t h, int side, int kind, const double *uw, double rho_w, int tkind,
                                 const double *tw) {
  if (!h) return fail(h, LBM_ERR_ARG, "NULL handle");
  if (side < 0 || side > 3) return fail(h, LBM_ERR_ARG, "side must be 0..3");
  if (kind < LBM_BC_PERIODIC || kind > LBM_BC_SYMMETRY) return fail(h, LBM_ERR_ARG, "kind");
  if (tkind < LBM_TBC_NONE || tkind > LBM_TBC_WETNODE) return fail(h, LBM_ERR_ARG, "tkind");
  if (tkind == LBM_TBC_WETNODE && (side > 1 || h->p.thermal != LBM_D2Q5))
    return fail(h, LBM_ERR_ARG, "wet-node sides are x-sides of a D2Q5 thermal lattice");
  const int len = side < 2 ? h->p.ny : h->p.nx;
  if (two_phase(h)) {
    if ((kind != LBM_BC_PERIODIC && kind != LBM_BC_WALL) || tkind != LBM_TBC_NONE)
      return fail(h, LBM_ERR_ARG, "two-phase solves support periodic sides and resting walls only");
    for (int k = 0; uw && k < 2 * len; k++)
      if (uw[k] != 0.0) return fail(h, LBM_ERR_ARG, "two-phase walls are at rest (uw must be NULL or zero)");
  }
  const int normal_len = side < 2 ? h->p.nx : h->p.ny;
  if ((kind == LBM_BC_PRESSURE || tkind == LBM_TBC_OUTFLOW) && normal_len < 2)
    return fail(h, LBM_ERR_ARG, "pressure/outflow sides need at least 2 nodes along the normal");
  if (!(rho_w > 0) && kind != LBM_BC_PERIODIC) return fail(h, LBM_ERR_ARG, "rho_w must be positive");
  h->bc[side] = kind;
  h->tbc[side] = tkind;
  h->rho_w[side] = rho_w > 0 ? rho_w : h->p.rho0;
  // Copy through this side's pinned staging slot so the call returns without a stream
  // synchronisation (the caller may reuse its arrays at once); wait only until the
  // slot's previous upload has been consumed.  A missing array zero-fills the device
  // copy, unless it already holds zeros.
  double *st = h->h_stage[side];
  if (uw || tw) CU(h, cudaEventSynchronize(h->stage_done[side]));
  if (uw) {
    memcpy(st, uw, sizeof(double) * 2 * len);
    CU(h, cudaMemcpyAsync(h->d_uw[side], st, sizeof(double) * 2 * len, cudaMemcpyHostToDevice, h->stream));
    h->uw_zero[side] = 0;
  } else if (!h->uw_zero[side]) {
    CU(h, cudaMemsetAsync(h->d_uw[side], 0, sizeof(double) * 2 * len, h->stream));
    h->uw_zero[side] = 1;
  }
  if (tw) {
    memcpy(st + 2 * len, tw, sizeof(double) * len);
    CU(h, cudaMemcpyAsync(h->d_tw[side], st + 2 * len, sizeof(double) * len, cudaMemcpyHostToDevice, h->stream));
    h->tw_zero[side] = 0;
  } else if (!h->tw_zero[side]) {
    CU(h, cudaMemsetAsync(h->d_tw[side], 0, sizeof(double) * len, h->stream));
    h->tw_zero[side] = 1;
  }
  if (uw || tw) CU(h, cudaEventRecord(h->stage_done[side], h->stream));
  return LBM_OK;
}

// Copy an nx*ny*nplanes double field (host or device) into a pitched storage array.
static lbm_status upload_field(lbm_t h, const double *src, int nplanes, int on_device, void **dst, double scale) {
  const size_t n = (size_t)h->p.nx * h->p.ny * nplanes;
  if (!*dst) {
    cudaError_t e = cudaMalloc(dst, (size_t)nplanes * h->plane * h->elem);
    if (e != cudaSuccess) return fail(h, LBM_ERR_NOMEM, "cudaMalloc source field");
    CU(h, cudaMemsetAsync(*dst, 0, (size_t)nplanes * h->plane * h->elem, h->stream));
  }
  const double *dsrc = src;
  double *tmp = NULL;
  if (!on_device) {
    CU(h, cudaMalloc(&tmp, n * sizeof(double)));
    CU(h, cudaMemcpyAsync(tmp, src, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    dsrc = tmp;
  }
  cudaError_t e = lbmk::to_storage(dsrc, *dst, h->p.nx, h->p.ny, h->pitch, nplanes, h->plane, h->p.precision, scale, h->stream);
  if (tmp) {
    cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
  }
  if (e != cudaSuccess) return fail(h, LBM_ERR_CUDA, "to_storage: %s", cudaGetErrorString(e));
  return LBM_OK;
}

extern "C" lbm_status lbm_set_source(lbm_t h, const double *q3, const double *force, int on_device) {
  if (!h) return fail(h, LBM_ERR_ARG, "NULL handle");
  lbm_status st;
  if (q3) {
    if (!h->p.thermal) return fail(h, LBM_ERR_ARG, "heat source needs a thermal LBE");
    // qdot = q'''/(rho c_p) in K/s (Sec. 2.2); with a lagged sink it is the sink's base
    st = upload_field(h, q3, 1, on_device, h->sink_conv != 0.0 ? &h->d_qbase : &h->d_qdot,
                      1.0 / (h->p.rho0 * h->p.cp));
    if (st != LBM_OK) return st;
  } else if (h->sink_conv != 0.0) {
    CU(h, cudaMemsetAsync(h->d_qbase, 0, (size_t)h->plane * h->elem, h->stream));
  } else if (h->d_qdot) {
    CU(h, cudaStreamSynchronize(h->stream));
    cudaFree(h->d_qdot);
    h->d_qdot = NULL;
  }
  if (force) {
    if (!h->p.flow) return fail(h, LBM_ERR_ARG, "force field needs a momentum LBE");
    st = upload_field(h, force, 2, on_device, &h->d_force, 1.0);
    if (st != LBM_OK) return st;
  } else if (h->d_force) {
    CU(h, cudaStreamSynchronize(h->stream));
    cudaFree(h->d_force);
    h->d_force = NULL;
  }
  CU(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

extern "C" lbm_status lbm_set_lagged_sink(lbm_t h, double conv_coef, double T_inf) {
  if (!h) return fail(h, LBM_ERR_ARG, "NULL handle");
  const lbm_params &p = h->p;
  if (!p.thermal) return fail(h, LBM_ERR_ARG, "the lagged sink needs a thermal LBE");
  if (!isfinite(conv_coef) || !isfinite(T_inf)) return fail(h, LBM_ERR_ARG, "non-finite sink coefficients");
  const size_t bytes = (size_t)h->plane * h->elem;
  if (conv_coef == 0.0) {
    if (h->sink_conv != 0.0) {  // back to the plain source field, which is the base
      CU(h, cudaStreamSynchronize(h->stream));
      cudaFree(h->d_qdot);
      h->d_qdot = h->d_qbase;
      h->d_qbase = NULL;
      cudaFree(h->d_qs[0]);
      cudaFree(h->d_qs[1]);
      h->d_qs[0] = h->d_qs[1] = NULL;
    }
    h->sink_conv = 0.0;
    return LBM_OK;
  }
  if (p.literal & 1) return fail(h, LBM_ERR_ARG, "the lagged sink needs the tau_T source factor (literal bit 0 off)");
  if (p.beta_exp != 0.0) return fail(h, LBM_ERR_ARG, "the lagged sink is not combined with buoyancy");
  if (h->sink_conv == 0.0) {
    void **f[3] = {&h->d_qbase, &h->d_qs[0], &h->d_qs[1]};
    for (int k = 0; k < 3; k++) {
      if (cudaMalloc(f[k], bytes) != cudaSuccess) {
        *f[k] = NULL;
        return fail(h, LBM_ERR_NOMEM, "cudaMalloc lagged-sink field");
      }
      CU(h, cudaMemsetAsync(*f[k], 0, bytes, h->stream));
    }
    if (h->d_qdot) {  // the source so far is the base and the field the last step used
      CU(h, cudaMemcpyAsync(h->d_qbase, h->d_qdot, bytes, cudaMemcpyDeviceToDevice, h->stream));
      CU(h, cudaMemcpyAsync(h->d_qs[h->cur], h->d_qdot, bytes, cudaMemcpyDeviceToDevice, h->stream));
    }
  }
  h->sink_conv = conv_coef;
  h->sink_Tinf = T_inf;
  CU(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

extern "C" lbm_status lbm_init_fields(lbm_t h, const double *a, const double *ux, const double *uy,
                                      const double *b, int on_device) {
  if (!h) return fail(h, LBM_ERR_ARG, "NULL handle");
  const size_t n = (size_t)h->p.nx * h->p.ny;
  const double *in[4] = {a, ux, uy, b};
  const double *d_in[4] = {NULL, NULL, NULL, NULL};
  double *tmp = NULL;
  if (!on_device) {
    int cnt = 0;
    for (int k = 0; k < 4; k++) cnt += in[k] != NULL;
    if (cnt) {
      CU(h, cudaMalloc(&tmp, n * sizeof(double) * cnt));
      int slot = 0;
      for (int k = 0; k < 4; k++) {
        if (!in[k]) continue;
        CU(h, cudaMemcpyAsync(tmp + slot * n, in[k], n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        d_in[k] = tmp + slot * n;
        slot++;
      }
    }
  } else {
    for (int k = 0; k < 4; k++) d_in[k] = in[k];
  }
  cudaError_t e;
  h->cur = 1;  // init writes buffer 0 (dst of a launch reading buffer 1)
  h->pre = 0;
  if (two_phase(h)) {
    lbmk::MpParams P = mp_params(h, 1);
    e = lbmk::mp_init(P, h->p.precision, d_in[0], d_in[1], d_in[2], d_in[3], h->stream);
  } else {
    SpParams P = sp_params(h, 1);
    int flow = h->p.flow ? (h->p.flow_op == LBM_MRT ? lbmk::FLOW_MRT : lbmk::FLOW_BGK) : lbmk::FLOW_NONE;
    int th = th_kind(h->p);
    e = lbmk::sp_init(P, h->p.precision, flow, th, d_in[0], d_in[1], d_in[2], d_in[3], h->block, h->stream);
  }
  if (tmp) {
    cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
  }
  if (e != cudaSuccess) return fail(h, LBM_ERR_CUDA, "init launch: %s", cudaGetErrorString(e));
  h->cur = 0;
  h->pre = 1;  // buffer 0 holds f(0) itself; the first step collides it in place
  h->steps = 0;
  h->last_good = -1;
  h->initialised = 1;
  if (!on_device) CU(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

static void sp_kinds(const lbm_t h, int *flow, int *th) {
  *flow = h->p.flow ? (h->p.flow_op == LBM_MRT ? lbmk::FLOW_MRT : lbmk::FLOW_BGK) : lbmk::FLOW_NONE;
  *th = th_kind(h->p);
}

static int *step_flag(lbm_t h) { return (int *)(h->d_out4 + 4); }

// qdot of the lagged sink for the step (or moments) that reads buffer `from`
// (pre: the buffer holds the initial state itself); nothing without a sink.
static cudaError_t sink_refresh(const lbm_t h, int from, int pre, cudaStream_t st) {
  if (h->sink_conv == 0.0) return cudaSuccess;
  const lbm_params &p = h->p;
  return lbmk::lagged_qdot(h->buf[from], h->d_qs[from], h->d_qbase, h->d_qs[1 - from], p.nx, p.ny, h->pitch, h->plane,
                           p.flow == LBM_D2Q9 ? 9 : 0, p.thermal, p.T0, p.dt, h->sink_conv, h->sink_Tinf, pre,
                           p.precision, st);
}

// One grid-launched step reading buffer `from` (two-phase or single phase).
static cudaError_t launch_grid_step(const lbm_t h, int from, int flow, int th, cudaStream_t st) {
  if (two_phase(h)) return lbmk::mp_step(mp_params(h, from), h->p.precision, st);
  const cudaError_t e = sink_refresh(h, from, 0, st);
  if (e != cudaSuccess) return e;
  if (h->launch_kind == LBM_LAUNCH_GRID_OCC)
    return lbmk::sp_step_occ(sp_params(h, from), h->p.precision, flow, th, h->block, st);
  return lbmk::sp_step(sp_params(h, from), h->p.precision, flow, th, h->block, st);
}

static void step_key(const lbm_t h, int flow, int th, StepKey *k) {
  memset(k, 0, sizeof(*k));
  k->two_phase = two_phase(h);
  k->prec = h->p.precision;
  k->flow = flow;
  k->th = th;
  k->kind = h->launch_kind;
  k->block = h->block;
  k->sink_conv = h->sink_conv;
  k->sink_Tinf = h->sink_Tinf;
  for (int b = 0; b < 2; b++) {
    const int from = (h->cur + b) & 1;
    if (k->two_phase) k->mp[b] = mp_params(h, from);
    else k->sp[b] = sp_params(h, from);
  }
}

// The graph of kGraphSteps steps starting from buffer h->cur, captured now if absent
// or stale; NULL if capture is not possible (the caller then launches step by step).
static cudaGraphExec_t step_graph(lbm_t h, int flow, int th) {
  StepKey key;
  step_key(h, flow, th, &key);
  const int slot = h->cur;
  if (h->gexec[slot] && memcmp(h->gkey[slot], &key, sizeof(key)) == 0) return h->gexec[slot];
  if (h->gexec[slot]) {
    cudaGraphExecDestroy(h->gexec[slot]);
    h->gexec[slot] = NULL;
  }
  if (!h->gkey[slot] && !(h->gkey[slot] = (StepKey *)malloc(sizeof(StepKey)))) return NULL;
  if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    h->cap_stream = NULL;
    return NULL;
  }
  if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return NULL;
  cudaError_t e = cudaSuccess;
  for (long s = 0; s < kGraphSteps && e == cudaSuccess; s++) e = launch_grid_step(h, (h->cur + s) & 1, flow, th, h->cap_stream);
  cudaGraph_t g = NULL;
  const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &g);
  cudaGraphExec_t x = NULL;
  if (e == cudaSuccess && ec == cudaSuccess && g && cudaGraphInstantiate(&x, g, 0) != cudaSuccess) x = NULL;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();  // a failed capture leaves no sticky error; clear the last one
  if (!x) return NULL;
  h->gexec[slot] = x;
  memcpy(h->gkey[slot], &key, sizeof(key));
  return x;
}

static lbm_status advance(lbm_t h, long n) {
  int flow, th;
  sp_kinds(h, &flow, &th);
  for (long s = 0; s < n;) {
    cudaError_t e;
    // long runs of grid-launched steps replay a captured graph (no per-step host work)
    if (!h->pre && n - s >= kGraphSteps && (two_phase(h) || h->launch_kind != LBM_LAUNCH_TMA)) {
      cudaGraphExec_t x = step_graph(h, flow, th);
      if (x) {
        e = cudaGraphLaunch(x, h->stream);
        if (e != cudaSuccess) return fail(h, LBM_ERR_CUDA, "step graph launch: %s", cudaGetErrorString(e));
        s += kGraphSteps;
        h->steps += kGraphSteps;
        continue;
      }
    }
    if (!two_phase(h)) {
      e = sink_refresh(h, h->cur, h->pre, h->stream);
      if (e != cudaSuccess) return fail(h, LBM_ERR_CUDA, "sink launch: %s", cudaGetErrorString(e));
    }
    if (two_phase(h)) {
      lbmk::MpParams P = mp_params(h, h->cur);
      e = lbmk::mp_step(P, h->p.precision, h->stream);
    } else if (h->launch_kind == LBM_LAUNCH_TMA && !h->pre) {
      SpParams P = sp_params(h, h->cur);
      e = lbmk::sp_step_tma(P, h->tmap[h->cur], h->p.precision, flow, th, h->tma_ty, h->tma_stages,
                            h->nsm * h->tma_ctas, step_flag(h), h->tma_wait_ns, h->tma_expire_next, h->stream);
      h->tma_expire_next = 0;
    } else {
      SpParams P = sp_params(h, h->cur);
      e = h->launch_kind == LBM_LAUNCH_GRID_OCC ? lbmk::sp_step_occ(P, h->p.precision, flow, th, h->block, h->stream)
                                             : lbmk::sp_step(P, h->p.precision, flow, th, h->block, h->stream);
    }
    if (e != cudaSuccess) return fail(h, LBM_ERR_CUDA, "step launch: %s", cudaGetErrorString(e));
    h->cur = 1 - h->cur;
    h->pre = 0;
    h->steps++;
    s++;
  }
  return LBM_OK;
}

extern "C" lbm_status lbm_step(lbm_t h, long n) {
  if (!h) return fail(h, LBM_ERR_ARG, "NULL handle");
  if (n < 0) return fail(h, LBM_ERR_ARG, "n must be >= 0");
  if (!h->initialised) return fail(h, LBM_ERR_STATE, "lbm_init_fields has not been called");
  if (h->check_every <= 0) return advance(h, n);
  // health check at every multiple of check_every of the step count
  while (n > 0) {
    const long k = std::min(n, h->check_every - h->steps % h->check_every);
    lbm_status st = advance(h, k);
    if (st != LBM_OK) return st;
    n -= k;
    if (h->steps % h->check_every == 0) {
      double v[4];
      st = lbm_integrals(h, v);
      if (st != LBM_OK) return st;
      if (v[3] > 0)
        return fail(h, LBM_ERR_DIVERGED, "%.0f cells non-finite or |u| >= c at step %ld; last healthy check at step %ld",
                    v[3], h->steps, h->last_good);
      h->last_good = h->steps;
    }
  }
  return LBM_OK;
}

extern "C" lbm_status lbm_set_check_interval(lbm_t h, long every) {
  if (!h) return fail(h, LBM_ERR_ARG, "NULL handle");
  if (every < 0) return fail(h, LBM_ERR_ARG, "the check interval must be >= 0 (0 = off)");
  h->check_every = every;
  return LBM_OK;
}

extern "C" long lbm_last_good_step(lbm_t h) { return h ? h->last_good : -1; }

extern "C" lbm_status lbm_set_wait_limit(lbm_t h, double seconds, int expire_next) {
  if (!h) return fail(h, LBM_ERR_ARG, "NULL handle");
  if (!(seconds > 0) || seconds > 10.0) return fail(h, LBM_ERR_ARG, "wait limit must lie in (0, 10] s");
  h->tma_wait_ns = (unsigned long long)(seconds * 1e9);
  h->tma_expire_next = expire_next ? 1 : 0;
  return LBM_OK;
}

extern "C" long lbm_steps_done(lbm_t h) { return h ? h->steps : -1; }

extern "C" lbm_status lbm_moments(lbm_t h, unsigned mask, double *out, int on_device) {
  if (!h || !out) return fail(h, LBM_ERR_ARG, "NULL argument");
  if (!h->initialised) return fail(h, LBM_ERR_STATE, "not initialised");
  if (mask == 0 || mask > 63u) return fail(h, LBM_ERR_ARG, "mask must select 1..6 of RHO|UX|UY|T|P|PHI");
  int nsel = 0;
  for (int b = 0; b < 6; b++) nsel += (mask >> b) & 1u;
  const size_t n = (size_t)h->p.nx * h->p.ny;
  double *dout = out;
  if (!on_device) CU(h, cudaMalloc(&dout, n * nsel * sizeof(double)));
  cudaError_t e;
  if (two_phase(h)) {
    lbmk::MpParams P = mp_params(h, h->cur);
    e = lbmk::mp_moments(P, h->p.precision, mask, dout, h->stream);
  } else {
    int flow, th;
    sp_kinds(h, &flow, &th);
    SpParams P = sp_params(h, h->cur);
    e = sink_refresh(h, h->cur, h->pre, h->stream);
    if (e == cudaSuccess) e = lbmk::sp_moments(P, h->p.precision, flow, th, mask, dout, h->stream);
  }
  if (e != cudaSuccess) {
    if (!on_device) cudaFree(dout);
    return fail(h, LBM_ERR_CUDA, "moments launch: %s", cudaGetErrorString(e));
  }
  if (!on_device) {
    cudaError_t e2 = cudaMemcpyAsync(out, dout, n * nsel * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    cudaError_t e3 = cudaStreamSynchronize(h->stream);
    cudaFree(dout);
    if (e2 != cudaSuccess || e3 != cudaSuccess)
      return fail(h, LBM_ERR_CUDA, "moments copy: %s", cudaGetErrorString(e2 != cudaSuccess ? e2 : e3));
  }
  return LBM_OK;
}

extern "C" lbm_status lbm_integrals(lbm_t h, double out[4]) {
  if (!h || !out) return fail(h, LBM_ERR_ARG, "NULL argument");
  if (!h->initialised) return fail(h, LBM_ERR_STATE, "not initialised");
  cudaError_t e;
  if (two_phase(h)) {
    lbmk::MpParams P = mp_params(h, h->cur);
    e = lbmk::mp_integrals(P, h->p.precision, h->d_partials, h->max_blocks, h->d_out4, h->stream);
  } else {
    int flow, th;
    sp_kinds(h, &flow, &th);
    SpParams P = sp_params(h, h->cur);
    e = lbmk::sp_integrals(P, h->p.precision, flow, th, h->d_partials, h->max_blocks, h->d_out4,
                           (unsigned *)(h->d_out4 + 5), h->stream);
  }
  if (e != cudaSuccess) return fail(h, LBM_ERR_CUDA, "integrals launch: %s", cudaGetErrorString(e));
  CU(h, cudaMemcpyAsync(h->h_out4, h->d_out4, 5 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  memcpy(out, h->h_out4, 4 * sizeof(double));
  int flag;
  memcpy(&flag, h->h_out4 + 4, sizeof(int));
  if (flag) {  // reported once: clear it for the steps that follow
    CU(h, cudaMemsetAsync(step_flag(h), 0, sizeof(int), h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    return fail(h, LBM_ERR_TIMEOUT, "a step kernel gave up waiting for its staged copies (flag %d)", flag);
  }
  return LBM_OK;
}

extern "C" lbm_status lbm_check(lbm_t h) {
  double v[4];
  lbm_status st = lbm_integrals(h, v);
  if (st != LBM_OK) return st;
  if (v[3] > 0) return fail(h, LBM_ERR_DIVERGED, "%.0f cells non-finite or |u| >= c after %ld steps", v[3], h->steps);
  return LBM_OK;
}

extern "C" size_t lbm_state_bytes(lbm_t h) {
  if (!h) return 0;
  return (size_t)h->nq * h->p.nx * h->p.ny * h->elem;
}

static lbm_status state_copy(lbm_t h, void *host, size_t bytes, int unpack) {
  if (!h || !host) return fail(h, LBM_ERR_ARG, "NULL argument");
  if (bytes != lbm_state_bytes(h)) return fail(h, LBM_ERR_ARG, "state size is %zu bytes", lbm_state_bytes(h));
  if (!unpack && !h->initialised) return fail(h, LBM_ERR_STATE, "not initialised");
  if (!unpack && h->pre) return fail(h, LBM_ERR_STATE, "no step taken since lbm_init_fields: no post-collision state yet");
  void *tmp = NULL;
  CU(h, cudaMalloc(&tmp, bytes));
  cudaError_t e = cudaSuccess;
  if (unpack) {
    e = cudaMemcpyAsync(tmp, host, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
      e = lbmk::pack_state(h->buf[h->cur], tmp, h->p.nx, h->p.ny, h->pitch, h->nq, h->plane, (int)h->elem, 1, h->stream);
  } else {
    e = lbmk::pack_state(h->buf[h->cur], tmp, h->p.nx, h->p.ny, h->pitch, h->nq, h->plane, (int)h->elem, 0, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, tmp, bytes, cudaMemcpyDeviceToHost, h->stream);
  }
  cudaError_t e2 = cudaStreamSynchronize(h->stream);
  cudaFree(tmp);
  if (e != cudaSuccess || e2 != cudaSuccess)
    return fail(h, LBM_ERR_CUDA, "state copy: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  if (unpack) { h->initialised = 1; h->pre = 0; }
  if (unpack && h->sink_conv != 0.0)  // the lag restarts from the base qdot
    CU(h, cudaMemcpyAsync(h->d_qs[h->cur], h->d_qbase, (size_t)h->plane * h->elem, cudaMemcpyDeviceToDevice, h->stream));
  return LBM_OK;
}

extern "C" lbm_status lbm_get_state(lbm_t h, void *dst, size_t bytes) { return state_copy(h, dst, bytes, 0); }
extern "C" lbm_status lbm_set_state(lbm_t h, const void *src, size_t bytes) { return state_copy(h, (void *)src, bytes, 1); }

extern "C" lbm_status lbm_synchronize(lbm_t h) {
  if (!h) return fail(h, LBM_ERR_ARG, "NULL handle");
  CU(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// Batched solves: many independent single-phase channels, one launch per step
// ---------------------------------------------------------------------------
struct lbm_batch_s {
  int n;
  lbm_t *ch;              // channel handles (own their buffers and boundaries)
  cudaStream_t stream;
  int own_stream;
  int prec, flow, th;
  // device tables: parity p, channel k at [p * n + k]; local variant at [2n + k]
  SpParams *h_tab, *d_tab;
  int tab_valid;
  // tile list for the chosen tile shape
  int4 *d_tiles;
  int ntiles, tiles_bx, tiles_by;
  int bx, by, grid;       // launch configuration (autotuned or set)
  cudaGraph_t graph;
  cudaGraphExec_t exec;   // two steps: parity 0 then parity 1
  char err[512];
};

static lbm_status bfail(lbm_batch_t b, lbm_status st, const char *fmt, ...) {
  char *dst = b ? b->err : g_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return st;
}

#define BCU(b, call)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

extern "C" const char *lbm_batch_last_error(lbm_batch_t b) { return b ? b->err : g_create_err; }

static void batch_drop_graph(lbm_batch_t b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = NULL;
  b->graph = NULL;
}

extern "C" void lbm_batch_destroy(lbm_batch_t b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  for (int k = 0; k < b->n; k++) lbm_destroy(b->ch[k]);
  free(b->ch);
  free(b->h_tab);
  cudaFree(b->d_tab);
  cudaFree(b->d_tiles);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  free(b);
}

extern "C" lbm_status lbm_batch_create(const lbm_params *params, int n, void *stream, lbm_batch_t *out) {
  if (!out) return bfail(NULL, LBM_ERR_ARG, "out is NULL");
  *out = NULL;
  if (!params || n < 1) return bfail(NULL, LBM_ERR_ARG, "need n >= 1 channel parameter blocks");
  for (int k = 0; k < n; k++) {
    const lbm_params &p = params[k];
    if (p.phase != LBM_NONE) return bfail(NULL, LBM_ERR_ARG, "batched solves are single phase (channel %d)", k);
    if (p.precision != params[0].precision || p.flow != params[0].flow || p.flow_op != params[0].flow_op ||
        p.thermal != params[0].thermal || p.thermal_op != params[0].thermal_op)
      return bfail(NULL, LBM_ERR_ARG, "all channels need the same precision, lattices and operators (channel %d)", k);
  }
  lbm_batch_t b = (lbm_batch_t)calloc(1, sizeof(struct lbm_batch_s));
  if (!b) return bfail(NULL, LBM_ERR_NOMEM, "host allocation failed");
  b->n = n;
  b->ch = (lbm_t *)calloc(n, sizeof(lbm_t));
  b->h_tab = (SpParams *)calloc(3 * (size_t)n, sizeof(SpParams));
  if (!b->ch || !b->h_tab) { lbm_batch_destroy(b); return bfail(NULL, LBM_ERR_NOMEM, "host allocation failed"); }
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {  // graph capture needs a stream other than the legacy default one
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      lbm_batch_destroy(b);
      return bfail(NULL, LBM_ERR_CUDA, "cudaStreamCreate failed");
    }
    b->own_stream = 1;
  }
  for (int k = 0; k < n; k++) {
    lbm_status st = lbm_create(&params[k], b->stream, &b->ch[k]);
    if (st != LBM_OK) {
      char msg[512];
      snprintf(msg, sizeof(msg), "channel %d: %s", k, g_create_err);
      lbm_batch_destroy(b);
      return bfail(NULL, st, "%s", msg);
    }
  }
  b->prec = params[0].precision;
  sp_kinds(b->ch[0], &b->flow, &b->th);
  if (cudaMalloc(&b->d_tab, 3 * (size_t)n * sizeof(SpParams)) != cudaSuccess) {
    lbm_batch_destroy(b);
    return bfail(NULL, LBM_ERR_NOMEM, "cudaMalloc parameter table");
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->bx = 64;
  b->by = 4;
  int occ = lbmk::sp_batch_occupancy(b->prec, b->flow, b->th, 256);
  b->grid = sms * (occ > 0 ? occ : 4);
  *out = b;
  return LBM_OK;
}

extern "C" lbm_t lbm_batch_channel(lbm_batch_t b, int k) {
  if (!b || k < 0 || k >= b->n) return NULL;
  return b->ch[k];
}

extern "C" int lbm_batch_size(lbm_batch_t b) { return b ? b->n : 0; }

// (Re)build the entry list for a tile shape: every channel's boundary frame in
// chunks of bx*by nodes first (the longest-running nodes start first), then the
// interior tiles.
static lbm_status batch_tiles(lbm_batch_t b, int bx, int by) {
  if (b->d_tiles && b->tiles_bx == bx && b->tiles_by == by) return LBM_OK;
  const int chunk = bx * by;
  long long total = 0;
  for (int k = 0; k < b->n; k++) {
    const int nx = b->ch[k]->p.nx, ny = b->ch[k]->p.ny;
    total += (lbmk::frame_nodes(nx, ny) + chunk - 1) / chunk;
    total += (long long)((nx + bx - 1) / bx) * ((ny + by - 1) / by);
  }
  if (total > (1ll << 31) - 1) return bfail(b, LBM_ERR_ARG, "too many tiles");
  int4 *h = (int4 *)malloc(sizeof(int4) * (size_t)total);
  if (!h) return bfail(b, LBM_ERR_NOMEM, "host allocation failed");
  long long t = 0;
  for (int k = 0; k < b->n; k++) {
    const int nf = lbmk::frame_nodes(b->ch[k]->p.nx, b->ch[k]->p.ny);
    for (int f0 = 0; f0 < nf; f0 += chunk) h[t++] = make_int4(k, f0, 0, 1);
  }
  for (int k = 0; k < b->n; k++) {
    const int nx = b->ch[k]->p.nx, ny = b->ch[k]->p.ny;
    for (int y0 = 0; y0 < ny; y0 += by)
      for (int x0 = 0; x0 < nx; x0 += bx) h[t++] = make_int4(k, x0, y0, 0);
  }
  cudaStreamSynchronize(b->stream);
  cudaFree(b->d_tiles);
  b->d_tiles = NULL;
  cudaError_t e = cudaMalloc(&b->d_tiles, sizeof(int4) * (size_t)total);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_tiles, h, sizeof(int4) * (size_t)total, cudaMemcpyHostToDevice);
  free(h);
  if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "tile list: %s", cudaGetErrorString(e));
  b->ntiles = (int)total;
  b->tiles_bx = bx;
  b->tiles_by = by;
  batch_drop_graph(b);
  return LBM_OK;
}

// Parameter tables for the current state of every channel; upload when changed.
static lbm_status batch_tables(lbm_batch_t b, int *cur, int *pre) {
  const int c0 = b->ch[0]->cur, p0 = b->ch[0]->pre;
  for (int k = 0; k < b->n; k++) {
    lbm_t h = b->ch[k];
    if (!h->initialised) return bfail(b, LBM_ERR_STATE, "channel %d is not initialised", k);
    if (h->cur != c0 || h->pre != p0)
      return bfail(b, LBM_ERR_STATE, "channel %d is not in step with channel 0 (step it through the batch only)", k);
  }
  SpParams *tmp = (SpParams *)malloc(3 * (size_t)b->n * sizeof(SpParams));
  if (!tmp) return bfail(b, LBM_ERR_NOMEM, "host allocation failed");
  for (int k = 0; k < b->n; k++) {
    lbm_t h = b->ch[k];
    const int save = h->pre;
    h->pre = 0;
    tmp[k] = sp_params(h, 0);
    tmp[b->n + k] = sp_params(h, 1);
    h->pre = 1;
    tmp[2 * b->n + k] = sp_params(h, c0);
    h->pre = save;
  }
  if (!b->tab_valid || memcmp(tmp, b->h_tab, 3 * (size_t)b->n * sizeof(SpParams)) != 0) {
    memcpy(b->h_tab, tmp, 3 * (size_t)b->n * sizeof(SpParams));
    cudaError_t e = cudaMemcpyAsync(b->d_tab, b->h_tab, 3 * (size_t)b->n * sizeof(SpParams), cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // h_tab may change before the copy runs
    if (e != cudaSuccess) { free(tmp); return bfail(b, LBM_ERR_CUDA, "table upload: %s", cudaGetErrorString(e)); }
    b->tab_valid = 1;
  }
  free(tmp);
  *cur = c0;
  *pre = p0;
  return LBM_OK;
}

static cudaError_t batch_launch(lbm_batch_t b, const SpParams *table) {
  return lbmk::sp_batch_step(table, b->d_tiles, b->ntiles, b->prec, b->flow, b->th, dim3(b->bx, b->by), b->grid,
                             b->stream);
}

static void batch_advance(lbm_batch_t b, long n) {
  for (int k = 0; k < b->n; k++) {
    lbm_t h = b->ch[k];
    h->cur = (int)((h->cur + n) & 1);
    h->pre = 0;
    h->steps += n;
  }
}

extern "C" lbm_status lbm_batch_config(lbm_batch_t b, int bx, int by, int grid) {
  if (!b) return bfail(b, LBM_ERR_ARG, "NULL batch");
  if (bx < 1 || by < 1 || bx * by > 256 || (bx * by) % 32 || grid < 1)
    return bfail(b, LBM_ERR_ARG, "tile must be a multiple of 32 threads, at most 256; grid >= 1");
  lbm_status st = batch_tiles(b, bx, by);
  if (st != LBM_OK) return st;
  if (b->bx != bx || b->by != by || b->grid != grid) batch_drop_graph(b);
  b->bx = bx;
  b->by = by;
  b->grid = grid;
  return LBM_OK;
}

extern "C" lbm_status lbm_batch_step(lbm_batch_t b, long n) {
  if (!b) return bfail(b, LBM_ERR_ARG, "NULL batch");
  if (n < 0) return bfail(b, LBM_ERR_ARG, "n must be >= 0");
  if (n == 0) return LBM_OK;
  for (int k = 0; k < b->n; k++)  // the batched launch does not refresh a lagged qdot
    if (b->ch[k]->sink_conv != 0.0) return bfail(b, LBM_ERR_ARG, "channel %d has a lagged sink", k);
  lbm_status st = batch_tiles(b, b->bx, b->by);
  if (st != LBM_OK) return st;
  int cur, pre;
  st = batch_tables(b, &cur, &pre);
  if (st != LBM_OK) return st;
  if (pre) {  // first step after initialisation: collide the stored f(0) in place
    BCU(b, batch_launch(b, b->d_tab + 2 * b->n));
    batch_advance(b, 1);
    n--;
    cur = 1 - cur;
  }
  if (n > 0 && cur == 1) {  // align to parity 0 for the two-step graph
    BCU(b, batch_launch(b, b->d_tab + b->n));
    batch_advance(b, 1);
    n--;
  }
  if (n >= 2) {
    if (!b->exec) {  // capture: step with parity 0 (buf0 -> buf1), then parity 1
      BCU(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e1 = batch_launch(b, b->d_tab);
      cudaError_t e2 = batch_launch(b, b->d_tab + b->n);
      cudaError_t e3 = cudaStreamEndCapture(b->stream, &b->graph);
      if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        batch_drop_graph(b);
        return bfail(b, LBM_ERR_CUDA, "graph capture failed");
      }
      BCU(b, cudaGraphInstantiate(&b->exec, b->graph, 0));
    }
    for (long k = 0; k < n / 2; k++) BCU(b, cudaGraphLaunch(b->exec, b->stream));
    batch_advance(b, 2 * (n / 2));
    n -= 2 * (n / 2);
  }
  if (n == 1) {
    BCU(b, batch_launch(b, b->d_tab));
    batch_advance(b, 1);
  }
  return LBM_OK;
}

extern "C" lbm_status lbm_batch_autotune(lbm_batch_t b, int out_cfg[3]) {
  if (!b) return bfail(b, LBM_ERR_ARG, "NULL batch");
  int cur, pre;
  lbm_status st = batch_tables(b, &cur, &pre);
  if (st != LBM_OK) return st;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  static const int shapes[][2] = {{32, 4}, {64, 4}, {128, 2}, {32, 8}, {256, 1}, {64, 2}, {128, 1}};
  static const int mults[] = {1, 2, 4, 8, 16};
  // Timing launches re-run the step that the next lbm_batch_step would take (same
  // source buffer, same destination), so the solution does not advance.
  const SpParams *table = pre ? b->d_tab + 2 * b->n : b->d_tab + (size_t)cur * b->n;
  cudaEvent_t e0, e1;
  BCU(b, cudaEventCreate(&e0));
  BCU(b, cudaEventCreate(&e1));
  float best = 1e30f;
  int bb[3] = {b->bx, b->by, b->grid};
  for (const auto &sh : shapes) {
    st = batch_tiles(b, sh[0], sh[1]);
    if (st != LBM_OK) break;
    const int occ = lbmk::sp_batch_occupancy(b->prec, b->flow, b->th, sh[0] * sh[1]);
    // grid-stride launches of a few blocks per SM, and one block per entry (the block
    // scheduler then hands out the tiles)
    for (int mi = 0; mi <= (int)(sizeof(mults) / sizeof(mults[0])); mi++) {
      const int m = mi < (int)(sizeof(mults) / sizeof(mults[0])) ? mults[mi] : 0;
      if (m > (occ > 0 ? occ : 1) * 2) continue;
      const int grid = m ? sms * m : b->ntiles;
      b->bx = sh[0];
      b->by = sh[1];
      b->grid = grid;
      batch_launch(b, table);  // warm-up
      cudaEventRecord(e0, b->stream);
      for (int r = 0; r < 3; r++) batch_launch(b, table);
      cudaEventRecord(e1, b->stream);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) { st = bfail(b, LBM_ERR_CUDA, "autotune: %s", cudaGetErrorString(e)); break; }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; bb[0] = sh[0]; bb[1] = sh[1]; bb[2] = grid; }
    }
    if (st != LBM_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LBM_OK) return st;
  st = lbm_batch_config(b, bb[0], bb[1], bb[2]);
  batch_drop_graph(b);
  if (out_cfg) { out_cfg[0] = b->bx; out_cfg[1] = b->by; out_cfg[2] = b->grid; }
  return st;
}

// ---------------------------------------------------------------------------
// Reverse-time adjoint of the fused step (D2Q9 MRT + D2Q5 MRT, FP64)
// ---------------------------------------------------------------------------
extern "C" lbm_status lbm_adjoint(lbm_t h, long steps, int ckpt_every, const double *T_target, double *loss,
                                  double *g_q3, double *g_qwall, double *g_nu) {
  if (!h || !T_target || !loss) return fail(h, LBM_ERR_ARG, "NULL argument");
  const lbm_params &p = h->p;
  if (p.phase || p.flow != LBM_D2Q9 || p.flow_op != LBM_MRT || p.thermal != LBM_D2Q5 || p.thermal_op != LBM_MRT)
    return fail(h, LBM_ERR_ARG, "the adjoint covers single-phase D2Q9 MRT + D2Q5 MRT solves");
  for (int s = 0; s < 4; s++)
    if (h->bc[s] == LBM_BC_SYMMETRY || h->tbc[s] == LBM_TBC_SYMMETRY || h->tbc[s] == LBM_TBC_WETNODE)
      return fail(h, LBM_ERR_ARG, "the adjoint does not cover symmetry or wet-node sides");
  if (h->sink_conv != 0.0) return fail(h, LBM_ERR_ARG, "the adjoint does not cover the lagged sink");
  if (p.beta_exp != 0.0) return fail(h, LBM_ERR_ARG, "the adjoint does not cover the buoyancy coupling");
  if (p.nx < 2) return fail(h, LBM_ERR_ARG, "nx must be >= 2 (loss on the x+ column)");
  if (steps < 1 || ckpt_every < 1) return fail(h, LBM_ERR_ARG, "steps and ckpt_every must be >= 1");
  if (!h->initialised || !h->pre)
    return fail(h, LBM_ERR_STATE, "call lbm_adjoint right after lbm_init_fields (it runs the forward itself)");
  const int K = ckpt_every;
  const long M = (steps + K - 1) / K;          // segments
  // states and adjoint variables in the storage precision (FP64, or FP32 for the
  // deviation form); parameter gradients in FP64
  const size_t sbytes = (size_t)h->nq * h->plane * h->elem;
  const size_t pbytes = (size_t)h->plane * sizeof(double);
  const int nx = p.nx, ny = p.ny;
  dim3 ag = lbmk::adj_grid(nx, ny);
  const int nblk = (int)(ag.x * ag.y);
  double *ck = NULL, *seg = NULL, *lp = NULL, *gq = NULL, *gf = NULL, *nup = NULL, *tt = NULL, *lr = NULL, *o2 = NULL;
  lbm_status st = LBM_OK;
  cudaError_t e = cudaSuccess;
#define ACU(call)                                                                       \
  do {                                                                                  \
    e = (call);                                                                         \
    if (e != cudaSuccess) { st = fail(h, LBM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e)); goto done; } \
  } while (0)
#define AAL(ptr, bytes)                                                                 \
  do {                                                                                  \
    if (cudaMalloc(&(ptr), (bytes)) != cudaSuccess) { st = fail(h, LBM_ERR_NOMEM, "adjoint: cudaMalloc %zu B", (size_t)(bytes)); goto done; } \
  } while (0)
  {
    AAL(ck, sbytes * (size_t)M);
    AAL(seg, sbytes * (size_t)(K + 1));
    AAL(lp, sbytes * 2);
    AAL(gq, pbytes);
    AAL(gf, sizeof(double) * 2 * nx);
    AAL(nup, sizeof(double) * 2 * nblk);
    AAL(tt, sizeof(double) * ny);
    AAL(lr, sizeof(double) * ny);
    AAL(o2, sizeof(double) * 2);
    ACU(cudaMemsetAsync(gq, 0, pbytes, h->stream));
    ACU(cudaMemsetAsync(gf, 0, sizeof(double) * 2 * nx, h->stream));
    ACU(cudaMemsetAsync(nup, 0, sizeof(double) * 2 * nblk, h->stream));
    ACU(cudaMemcpyAsync(tt, T_target, sizeof(double) * ny, cudaMemcpyHostToDevice, h->stream));
    // forward with checkpoints: ck[m] = X_{mK-1} (ck[0] = pre-collision initial state)
    ACU(cudaMemcpyAsync(ck, h->buf[h->cur], sbytes, cudaMemcpyDeviceToDevice, h->stream));
    // (whole segments through lbm_step, so that long ones replay the captured step graph)
    for (long t = 0; t < steps;) {
      const long k = std::min((long)K - t % K, steps - t);
      st = lbm_step(h, k);
      if (st != LBM_OK) goto done;
      t += k;
      if (t % K == 0 && t / K < M)
        ACU(cudaMemcpyAsync((char *)ck + sbytes * (size_t)(t / K), h->buf[h->cur], sbytes, cudaMemcpyDeviceToDevice,
                            h->stream));
    }
    // loss at time N and the seed Lam_pre(N)
    int cur = 0;
    ACU(cudaMemsetAsync(lp, 0, sbytes * 2, h->stream));
    SpParams P = sp_params(h, h->cur);
    ACU(lbmk::adj_loss(P, p.precision, tt, lp, gq, lr, h->stream));
    for (long m = M - 1; m >= 0; m--) {
      const long s0 = m * K, s1 = (m + 1) * K < steps ? (m + 1) * K - 1 : steps - 1;
      // recompute X_{s0-1} .. X_{s1} into seg[0 .. s1-s0+1]
      ACU(cudaMemcpyAsync(seg, (char *)ck + sbytes * (size_t)m, sbytes, cudaMemcpyDeviceToDevice, h->stream));
      for (long k = 1; k <= s1 - s0 + 1; k++) {
        SpParams Q = sp_params(h, 0);
        Q.local = (m == 0 && k == 1) ? 1 : 0;
        Q.src = (char *)seg + sbytes * (size_t)(k - 1);
        Q.dst = (char *)seg + sbytes * (size_t)k;
        ACU(lbmk::sp_step(Q, p.precision, lbmk::FLOW_MRT, lbmk::TH_MRT, h->block, h->stream));
      }
      for (long t = s1; t >= s0; t--) {
        const long k = t - s0 + 1;
        SpParams Q = sp_params(h, 0);
        Q.local = (t == 0) ? 1 : 0;
        Q.src = (char *)seg + sbytes * (size_t)(k - 1);
        Q.dst = NULL;
        const void *Xt = (const char *)seg + sbytes * (size_t)k;
        void *LPn = (char *)lp + sbytes * (size_t)cur;
        void *LPo = (char *)lp + sbytes * (size_t)(1 - cur);
        ACU(lbmk::adj_step(Q, p.precision, Xt, LPn, LPo, gq, gf, gf + nx, nup, h->stream));
        cur = 1 - cur;
      }
    }
    ACU(lbmk::adj_final(nup, nblk, o2, h->stream));
    // results to the host
    double *hl = (double *)malloc(sizeof(double) * ny);
    double ho2[2];
    if (!hl) { st = fail(h, LBM_ERR_NOMEM, "host allocation"); goto done; }
    ACU(cudaMemcpyAsync(hl, lr, sizeof(double) * ny, cudaMemcpyDeviceToHost, h->stream));
    ACU(cudaMemcpyAsync(ho2, o2, sizeof(double) * 2, cudaMemcpyDeviceToHost, h->stream));
    if (g_qwall) ACU(cudaMemcpyAsync(g_qwall, gf, sizeof(double) * 2 * nx, cudaMemcpyDeviceToHost, h->stream));
    if (g_q3) {
      // dL/dq''' = dL/dqdot / (rho0 c_p); unpitch on the host
      double *tmp = (double *)malloc(pbytes);
      if (!tmp) { free(hl); st = fail(h, LBM_ERR_NOMEM, "host allocation"); goto done; }
      e = cudaMemcpyAsync(tmp, gq, pbytes, cudaMemcpyDeviceToHost, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      // per node an FP64 sum, or in the FP32 form a compensated FP32 pair (hi, lo)
      const float *pair = (const float *)tmp;
      if (e == cudaSuccess)
        for (int j = 0; j < ny; j++)
          for (int i = 0; i < nx; i++) {
            const size_t k = (size_t)j * h->pitch + i;
            const double g = h->elem == 4 ? (double)pair[2 * k] + (double)pair[2 * k + 1] : tmp[k];
            g_q3[(size_t)j * nx + i] = g / (p.rho0 * p.cp);
          }
      free(tmp);
      if (e != cudaSuccess) { free(hl); st = fail(h, LBM_ERR_CUDA, "gradient copy: %s", cudaGetErrorString(e)); goto done; }
    }
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) { free(hl); st = fail(h, LBM_ERR_CUDA, "adjoint: %s", cudaGetErrorString(e)); goto done; }
    double L = 0;
    for (int j = 0; j < ny; j++) L += hl[j];
    free(hl);
    *loss = L;
    if (g_nu) {
      // s_nu = dt/tau, s_q = dt omega_q(1/tau), tau = nu/c_s^2 + dt/2
      const double dt = p.dt, tau = h->tau, w = 1.0 / tau;
      const double dw_dnu = -1.0 / (tau * tau * h->cs2);
      const double dsnu = dt * dw_dnu;
      const double a = 3.0 / dt - w;
      const double dwq_dw = -3.0 / (dt * dt * a * a);
      const double dsq = dt * dwq_dw * dw_dnu;
      *g_nu = ho2[0] * dsnu + ho2[1] * dsq;
    }
  }
done:
  cudaStreamSynchronize(h->stream);
  cudaFree(ck); cudaFree(seg); cudaFree(lp); cudaFree(gq); cudaFree(gf); cudaFree(nup); cudaFree(tt); cudaFree(lr);
  cudaFree(o2);
#undef ACU
#undef AAL
  return st;
}

// ---------------------------------------------------------------------------
// Launch-shape autotuning of the single-solve step kernel
// ---------------------------------------------------------------------------
// Encode the tensor maps of both state buffers for boxes of height ty.
static lbm_status ensure_tmaps(lbm_t h, int ty) {
  if (h->tmap_ty == ty) return LBM_OK;
  for (int b = 0; b < 2; b++) {
    int r = lbmk::sp_tma_encode(h->buf[b], h->pitch, h->p.ny, h->nq, (int)h->elem, ty, &h->tmap[b]);
    if (r != 0) {
      h->tmap_ty = 0;
      return fail(h, LBM_ERR_CUDA, "tensor map encoding failed (%d)", r);
    }
  }
  h->tmap_ty = ty;
  return LBM_OK;
}

static lbm_status check_launch(lbm_t h, const int cfg[4]) {
  if (two_phase(h)) return fail(h, LBM_ERR_ARG, "two-phase solves use a fixed 32 x 8 tile");
  if (cfg[0] == LBM_LAUNCH_GRID || cfg[0] == LBM_LAUNCH_GRID_OCC) {
    if (cfg[1] < 32 || cfg[1] % 32 != 0 || cfg[2] < 1 || cfg[1] * cfg[2] > 256)
      return fail(h, LBM_ERR_ARG, "grid launch: block_x a multiple of 32, block_x * block_y <= 256");
    return LBM_OK;
  }
  if (cfg[0] == LBM_LAUNCH_TMA) {
    int flow, th;
    sp_kinds(h, &flow, &th);
    if (cfg[1] != 4 && cfg[1] != 8) return fail(h, LBM_ERR_ARG, "TMA launch: tile height 4 or 8");
    if (cfg[2] < 1 || cfg[2] > 4) return fail(h, LBM_ERR_ARG, "TMA launch: 1..4 stages");
    int occ = lbmk::sp_tma_occupancy(h->p.precision, flow, th, cfg[1], cfg[2]);
    if (cfg[3] < 1 || cfg[3] > occ)
      return fail(h, LBM_ERR_ARG, "TMA launch: 1..%d CTAs per SM fit for this tile and stage count", occ);
    return ensure_tmaps(h, cfg[1]);
  }
  return fail(h, LBM_ERR_ARG, "launch kind must be LBM_LAUNCH_GRID, LBM_LAUNCH_GRID_OCC or LBM_LAUNCH_TMA");
}

static void apply_launch(lbm_t h, const int cfg[4]) {
  h->launch_kind = cfg[0];
  if (cfg[0] != LBM_LAUNCH_TMA) {
    h->block = dim3(cfg[1], cfg[2]);
  } else {
    h->tma_ty = cfg[1];
    h->tma_stages = cfg[2];
    h->tma_ctas = cfg[3];
  }
}

extern "C" lbm_status lbm_set_launch(lbm_t h, const int cfg[4]) {
  if (!h || !cfg) return fail(h, LBM_ERR_ARG, "NULL argument");
  lbm_status st = check_launch(h, cfg);
  if (st != LBM_OK) return st;
  apply_launch(h, cfg);
  return LBM_OK;
}

extern "C" lbm_status lbm_launch_config(lbm_t h, int cfg[4]) {
  if (!h || !cfg) return fail(h, LBM_ERR_ARG, "NULL argument");
  cfg[0] = h->launch_kind;
  if (h->launch_kind != LBM_LAUNCH_TMA) {
    cfg[1] = (int)h->block.x;
    cfg[2] = (int)h->block.y;
    cfg[3] = 0;
  } else {
    cfg[1] = h->tma_ty;
    cfg[2] = h->tma_stages;
    cfg[3] = h->tma_ctas;
  }
  return LBM_OK;
}

extern "C" lbm_status lbm_autotune(lbm_t h, int out_block[2]) {
  if (!h) return fail(h, LBM_ERR_ARG, "NULL handle");
  if (!h->initialised) return fail(h, LBM_ERR_STATE, "not initialised");
  if (two_phase(h)) return fail(h, LBM_ERR_ARG, "two-phase solves use a fixed 32 x 8 tile");
  int flow, th;
  sp_kinds(h, &flow, &th);
  // candidates: grid launches of 32..256 threads, then TMA launches
  int cands[64][4];
  int nc = 0;
  static const int shapes[][2] = {{32, 2}, {32, 4}, {32, 8}, {64, 1}, {64, 2}, {64, 4}, {128, 1}, {128, 2}, {256, 1}};
  for (int kind = LBM_LAUNCH_GRID; kind <= LBM_LAUNCH_GRID_OCC; kind += LBM_LAUNCH_GRID_OCC - LBM_LAUNCH_GRID)
    for (const auto &sh : shapes) {
      cands[nc][0] = kind; cands[nc][1] = sh[0]; cands[nc][2] = sh[1]; cands[nc][3] = 0;
      nc++;
    }
  for (int ty = 4; ty <= 8; ty += 4)
    for (int stages = 2; stages <= 4; stages++) {
      int occ = lbmk::sp_tma_occupancy(h->p.precision, flow, th, ty, stages);
      for (int ctas = 1; ctas <= occ && ctas <= 4; ctas++) {
        cands[nc][0] = LBM_LAUNCH_TMA; cands[nc][1] = ty; cands[nc][2] = stages; cands[nc][3] = ctas;
        nc++;
      }
    }
  // The timed launches repeat the next step (same source, same destination) with
  // the non-local pull; the destination is rewritten in full by the next real
  // step, so the stored state does not change.
  SpParams P = sp_params(h, h->cur);
  P.local = 0;
  cudaEvent_t e0, e1;
  CU(h, cudaEventCreate(&e0));
  CU(h, cudaEventCreate(&e1));
  float best = 1e30f;
  int bestc = -1;
  lbm_status st = LBM_OK;
  for (int c = 0; c < nc; c++) {
    const int *cf = cands[c];
    if (cf[0] == LBM_LAUNCH_TMA && ensure_tmaps(h, cf[1]) != LBM_OK) continue;  // TMA unavailable: grid only
    auto launch = [&]() -> cudaError_t {
      if (cf[0] == LBM_LAUNCH_GRID) return lbmk::sp_step(P, h->p.precision, flow, th, dim3(cf[1], cf[2]), h->stream);
      if (cf[0] == LBM_LAUNCH_GRID_OCC)
        return lbmk::sp_step_occ(P, h->p.precision, flow, th, dim3(cf[1], cf[2]), h->stream);
      return lbmk::sp_step_tma(P, h->tmap[h->cur], h->p.precision, flow, th, cf[1], cf[2], h->nsm * cf[3],
                               step_flag(h), h->tma_wait_ns, 0, h->stream);
    };
    cudaError_t e = launch();  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
    for (int r = 0; r < 5 && e == cudaSuccess; r++) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) { st = fail(h, LBM_ERR_CUDA, "autotune: %s", cudaGetErrorString(e)); break; }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; bestc = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LBM_OK) return st;
  h->err[0] = 0;
  if (bestc >= 0) {
    if (cands[bestc][0] == LBM_LAUNCH_TMA) ensure_tmaps(h, cands[bestc][1]);
    apply_launch(h, cands[bestc]);
  }
  if (out_block) {
    out_block[0] = h->launch_kind != LBM_LAUNCH_TMA ? (int)h->block.x : 32;
    out_block[1] = h->launch_kind != LBM_LAUNCH_TMA ? (int)h->block.y : h->tma_ty;
  }
  return LBM_OK;
}
