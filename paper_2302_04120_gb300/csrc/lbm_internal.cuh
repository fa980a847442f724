// Internal declarations shared by the host C-ABI (lbm_api.cu) and the kernels.
// Not part of the public interface (include/lbm.h is).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmk {

// Boundary description of one side, device pointers.
struct DevSide {
  int kind;          // LBM_BC_*
  int tkind;         // LBM_TBC_*
  double rho_w;      // boundary density of Eqs. BB_vel / anti_BB_vel
  const double *uw;  // 2*len: u_x then u_y at each boundary node
  const double *tw;  // len: q'' (FLUX) or T_w (TEMP)
};

// Constants of a single-phase solve in the working precision R, filled on the host:
// the FP32 kernels must not convert double parameters per thread (on GB300 each
// conversion is an instruction of the slow FP64 pipe).
template <typename R>
struct SpConst {
  R c, cs2, dt, rho0, T0, Fx, Fy, ux_pres, uy_pres;
  R inv_c, inv_cs2, three_inv_c2;  // 1/c, 1/cs2, 3/(c c), each rounded once in R
  R hdt;                            // dt / 2
  R fk_e, fk_eps, fk_q, fk_nu;      // MRT forcing factors (1 - s_k / 2) dt, s_k = dt Lambda_k
  R omega, s_e, s_eps, s_q, s_nu, omegaT, tsrc_fac, flux_coef, bgx, bgy, T_ref;
  R rho_w[4];
};

// Everything a single-phase kernel needs; passed by value.
struct SpParams {
  int nx, ny, pitch;
  long long plane;        // elements per population plane (ny * pitch)
  int xper, yper;         // momentum lattice periodic along x / y
  int txper, typer;       // thermal lattice periodic along x / y
  int gbase;              // plane index of g_0 (9 with a momentum LBE, else 0)
  int qg;                 // thermal populations (5 or 9; 0 without a thermal LBE)
  int fysym, tysym;       // y-sides that are symmetry planes (bit 0: y = 0, bit 1: y = ny - 1),
                          // momentum and thermal lattice
  int sym;                // any side of either lattice is a symmetry plane (selects the
                          // kernels compiled with the symmetry rules)
  DevSide side[4];
  // SI constants
  double c, cs2, dt, dx;
  double rho0, T0;        // storage offsets (deviation form)
  double Fx, Fy;          // uniform body force
  double ux_pres, uy_pres;
  // momentum collision
  double omega;           // BGK: dt/tau
  double s_e, s_eps, s_q, s_nu;  // MRT: dt * Lambda_k for e, eps, q, nu moments
  // thermal collision
  double omegaT;          // dt/tau_T
  double tsrc_fac;        // BGK thermal source prefactor (1 - dt/(2 tau_sg))
  double flux_coef;       // dt / (dx rho0 cp): q'' -> K per step (Eq. BB_T, lambda = 1)
  // Boussinesq buoyancy (App. D): F += (bgx, bgy) (T - T_ref), (bgx, bgy) = -rho_ref beta_exp g
  int buoy;
  double bgx, bgy, T_ref;
  // optional per-cell fields (storage precision, pitched planes)
  const void *qdot;       // thermal source qdot [K/s], or null
  const void *force;      // 2 planes F_x, F_y [N m^-3], or null
  SpConst<double> kd;     // the constants above, in FP64 ...
  SpConst<float> kf;      // ... and in FP32
  // state
  int local;              // 1: src holds pre-collision f(t) itself (right after init)
  const void *src;        // post-collision populations of the previous step
  void *dst;              // post-collision populations written by this step
};

template <typename R>
__device__ __forceinline__ const SpConst<R> &K(const SpParams &P);
template <>
__device__ __forceinline__ const SpConst<double> &K<double>(const SpParams &P) { return P.kd; }
template <>
__device__ __forceinline__ const SpConst<float> &K<float>(const SpParams &P) { return P.kf; }

enum { FLOW_NONE = 0, FLOW_BGK = 1, FLOW_MRT = 2 };

// Nodes of the boundary frame of an nx x ny grid: rows j = 0 and ny - 1, then the
// columns i = 0 and nx - 1 between them (each node once, also for nx or ny < 3).
__host__ __device__ inline int frame_nodes(int nx, int ny) {
  return (ny >= 2 ? 2 : 1) * nx + (nx >= 2 ? 2 : 1) * (ny > 2 ? ny - 2 : 0);
}
// Grid of the single-phase integrals: 64 x 4 blocks.  The first *fy rows of blocks
// take the boundary frame, one node per thread; in the others each thread takes the
// interior nodes of its column in *steps consecutive groups of 4 rows: at most
// kRedParts blocks write partials, and grids of 1024 or more row groups take at least
// two nodes per thread (measured on GB300: 2048 x 256 in 28 us at two nodes per thread
// against 38 us at one, 8192 x 4096 in 348 us at 32).  Fixed for a grid size, so the
// reduction order is too.
constexpr int kRedBX = 64, kRedBY = 4, kRedParts = 4096;
__host__ __device__ inline dim3 integral_grid(int nx, int ny, int *steps, int *fy) {
  const int gx = (nx + kRedBX - 1) / kRedBX, groups = (ny + kRedBY - 1) / kRedBY;
  const int nfb = (frame_nodes(nx, ny) + kRedBX * kRedBY - 1) / (kRedBX * kRedBY);
  *fy = (nfb + gx - 1) / gx;
  const long long blocks1 = (long long)gx * groups;  // blocks at one node per thread
  int st = (int)((blocks1 + kRedParts - 1) / kRedParts);
  if (blocks1 >= 1024 && st < 2) st = 2;
  if (st > groups) st = groups;
  *steps = st;
  return dim3(gx, (groups + st - 1) / st + *fy);
}
enum { TH_NONE = 0, TH_BGK = 1, TH_MRT = 2, TH_BGK9 = 3, TH_MRT9 = 4 };
// populations of the thermal lattice of a TH kind: D2Q5, or the paper's D2Q9
template <int TH>
struct ThLat {
  static constexpr int Q = (TH == TH_BGK9 || TH == TH_MRT9) ? 9 : 5;
};

// Launchers (step_sp.cu).  prec: 0 FP64, 1 FP32 deviation.  Return cudaGetLastError().
cudaError_t sp_step(const SpParams &P, int prec, int flow, int th, dim3 block, cudaStream_t s);
// The same step built for more resident blocks per SM (FP32 with a thermal lattice: 6
// blocks of 256 at 40 registers instead of 4 at 64; other kinds: the same kernel).
cudaError_t sp_step_occ(const SpParams &P, int prec, int flow, int th, dim3 block, cudaStream_t s);
// qdot of the lagged heat sink for the step reading `src` (csrc/sink.cu): qnext =
// qbase - conv (T(t - dt) - T_inf), T(t - dt) rebuilt from src and qprev (pre: src
// holds the initial state itself).  Storage precision fields, one plane each.
cudaError_t lagged_qdot(const void *src, const void *qprev, const void *qbase, void *qnext, int nx, int ny, int pitch,
                        long long plane, int gbase, int qg, double T0, double dt, double conv, double Tinf, int pre,
                        int precision, cudaStream_t s);
// One step of many solves: table[k] holds the parameters (with this step's src/dst)
// of channel k; tiles lists the frame chunks (channel, f0, 0, 1) and the interior
// tiles (channel, x0, y0, 0) of every channel.
cudaError_t sp_batch_step(const SpParams *table, const int4 *tiles, int ntiles, int prec, int flow, int th,
                          dim3 block, int grid, cudaStream_t s);
int sp_batch_occupancy(int prec, int flow, int th, int threads);
// TMA-staged persistent step (step_tma.cu).  sp_tma_encode fills the tensor map of
// one state buffer (3-D: pitch x ny x nq planes, 36 x ty boxes; ty 4 or 8) and
// returns 0, or nonzero when the driver refuses it.  sp_tma_prepare raises the
// dynamic shared-memory limit of the kernels of one (prec, flow, th).  The step
// runs `grid` CTAs of 32 x ty threads with `stages` (1..4) slots of boxes in
// flight; flag (device int) receives 1 if a copy wait ran out (each ring wait is
// limited to wait_ns of wall time; expire_probe makes every block's first wait run
// out, a self-test of that path).  P.local must be 0.
int sp_tma_encode(void *base, int pitch, int ny, int nq, int elem, int ty, CUtensorMap *out);
cudaError_t sp_tma_prepare(int prec, int flow, int th);
int sp_tma_occupancy(int prec, int flow, int th, int ty, int stages);
size_t sp_tma_smem(int prec, int flow, int th, int ty, int stages);
cudaError_t sp_step_tma(const SpParams &P, const CUtensorMap &map, int prec, int flow, int th, int ty, int stages,
                        int grid, int *flag, unsigned long long wait_ns, int expire_probe, cudaStream_t s);
// Equilibrium initialisation (pre-collision state of time 0) from double fields (device).
cudaError_t sp_init(const SpParams &P, int prec, int flow, int th, const double *a,
                    const double *ux, const double *uy, const double *b, dim3 block,
                    cudaStream_t s);
// Macroscopic fields of the current state into nx*ny double planes (mask bit order).
cudaError_t sp_moments(const SpParams &P, int prec, int flow, int th, unsigned mask,
                       double *out, cudaStream_t s);
// Per-block partial integrals (4 doubles per block) then a fixed-order final reduction.
// counter: a device unsigned that is 0 on entry; the kernel's last block resets it.
cudaError_t sp_integrals(const SpParams &P, int prec, int flow, int th, double *partials,
                         int max_blocks, double *out4, unsigned *counter, cudaStream_t s);
int sp_integral_blocks(int nx, int ny);

// Convert nx*ny double planes into pitched storage planes (sources, forces).
cudaError_t to_storage(const double *in, void *out, int nx, int ny, int pitch, int nplanes,
                       long long plane, int prec, double scale, cudaStream_t s);
// Adjoint (adjoint.cu): loss at the outlet column + seed, one reverse step, final sum.
// prec 0: FP64 states and adjoint variables; 1: FP32 deviation states, FP32 adjoint
// variables (LP, LPn float); the parameter gradients are FP64 in both.
cudaError_t adj_loss(const SpParams &P, int prec, const double *Ttarget, void *LP, double *grad_qdot,
                     double *loss_rows, cudaStream_t s);
cudaError_t adj_step(const SpParams &P, int prec, const void *Xt, const void *LPn, void *LP, double *grad_qdot,
                     double *grad_flux2, double *grad_flux3, double *nu_partials, cudaStream_t s);
cudaError_t adj_final(const double *nu_partials, int nb, double *out2, cudaStream_t s);
dim3 adj_grid(int nx, int ny);

// Text for lbm_last_error(NULL) from entry points that take no handle.
void set_global_error(const char *msg);

// State <-> packed (unpitched) copies for checkpointing.
cudaError_t pack_state(const void *state, void *packed, int nx, int ny, int pitch, int nq,
                       long long plane, int elem, int unpack, cudaStream_t s);

}  // namespace lbmk
