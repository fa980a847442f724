/*
 * lbm.h -- C ABI of the GB300 dimensional lattice Boltzmann library.
 *
 * Method: Martins, Alvarino & Cabezas-Gomez, "Dimensional lattice Boltzmann
 * method for transport phenomena simulation without conversion to lattice
 * units" (arXiv:2302.04120).  The lattice Boltzmann equation is integrated
 * directly in SI units: dx [m], dt [s], c = dx/dt [m/s], f_i [kg m^-3],
 * T [K], forces [N m^-3], heat sources [W m^-3], heat fluxes [W m^-2]
 * (Sec. 3).  Every call below takes and returns SI quantities.
 *
 * Conventions
 *  - Grids are nx columns (x index i) by ny rows (y index j).  Host and device
 *    field arrays are row-major doubles, element (j, i) at j*nx + i, node
 *    (i, j) located at ((i+1/2) dx, (j+1/2) dx).  Half-way walls lie on cell
 *    faces (link-wise boundaries, Sec. 2.1).
 *  - The caller owns every array it passes; set/init calls copy before they
 *    return.  The handle owns its device state and frees it in lbm_destroy.
 *  - All work runs asynchronously on the CUDA stream bound at lbm_create
 *    (NULL = the legacy default stream).  Calls that write to host memory
 *    synchronise that stream before returning.
 *  - Every call returns an lbm_status; lbm_last_error() gives the text of the
 *    last failure on that handle.  No call aborts the process.
 *  - Pointer arguments flagged "on_device" are device pointers when the flag is
 *    non-zero, host pointers otherwise.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_s *lbm_t;

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,           /* bad argument, size or combination           */
  LBM_ERR_UNSTABLE_TAU = -2,  /* a relaxation time tau <= dt/2 (Sec. 4 intro)  */
  LBM_ERR_NOMEM = -3,         /* device or host allocation failed            */
  LBM_ERR_CUDA = -4,          /* a CUDA runtime call failed                  */
  LBM_ERR_DIVERGED = -5,      /* NaN/Inf or |u| >= c found by lbm_check       */
  LBM_ERR_TIMEOUT = -6,       /* a bounded device wait gave up                */
  LBM_ERR_STATE = -7          /* call not valid in the handle's current state */
} lbm_status;

/* lattices */
enum { LBM_NONE = 0, LBM_D2Q5 = 5, LBM_D2Q9 = 9 };
/* collision operators */
enum { LBM_BGK = 0, LBM_MRT = 1 };
/* storage/arithmetic precision */
enum {
  LBM_FP64 = 0,   /* FP64 storage and arithmetic                                      */
  LBM_FP32DEV = 1 /* FP32 storage of deviations f_i - w_i rho0, g_i - w_i T0; FP32 math */
};
/* momentum boundary kinds, per side */
enum {
  LBM_BC_PERIODIC = 0, /* Sec. 2.1: f_i(x_b) = f_i*(x_b + L - c_i dt); both sides of an axis */
  LBM_BC_WALL = 1,     /* half-way bounce-back with wall velocity, Eq. BB_vel               */
  LBM_BC_VELOCITY = 2, /* velocity inlet, Eq. BB_vel with u_w = inlet velocity              */
  LBM_BC_PRESSURE = 3, /* outlet, Eq. anti_BB_vel; u_w = u(x_b) + (u(x_b) - u(x_b-1))/2      */
  LBM_BC_SYMMETRY = 4  /* symmetry plane, Eq. simetria: mirrored populations of the
                          tangential neighbour; at a corner with another side the link
                          that crosses both takes that side's rule                       */
};
/* thermal boundary kinds, per side (LBM_TBC_NONE = periodic for the thermal lattice) */
enum {
  LBM_TBC_NONE = 0,
  LBM_TBC_FLUX = 1,    /* prescribed heat flux into the fluid, Eq. BB_T                     */
  LBM_TBC_TEMP = 2,    /* prescribed temperature, Eq. anti_BB_T                             */
  LBM_TBC_OUTFLOW = 3, /* first-order extrapolation of the unknown populations (Sec. 2.2)   */
  LBM_TBC_SYMMETRY = 4, /* symmetry plane for the thermal lattice, Eq. simetria             */
  LBM_TBC_WETNODE = 5   /* wet-node Dirichlet T_w (App. B): the boundary node lies on the
                           boundary (x = 0 or x = L) and its single unknown population is
                           T_w - dt qdot/2 - (sum of the others), so its T is T_w; D2Q5,
                           x-sides only                                                  */
};
/* sides */
enum { LBM_SIDE_XMIN = 0, LBM_SIDE_XMAX = 1, LBM_SIDE_YMIN = 2, LBM_SIDE_YMAX = 3 };
/* moment selection bits for lbm_moments */
enum { LBM_RHO = 1, LBM_UX = 2, LBM_UY = 4, LBM_T = 8, LBM_P = 16, LBM_PHI = 32 };

/*
 * Solver parameters, all SI.
 *  flow       LBM_D2Q9 (momentum LBE, Sec. 2.1) or LBM_NONE (velocity prescribed
 *             by u_prescribed; thermal-only problems).
 *  flow_op    LBM_BGK (Eq. eq_lattice_boltzmann_BGK) or LBM_MRT (Eq. colisao_MRT with
 *             [M]_dim of Eq. M_matrix_dim and the dimensional rates of Sec. 3:
 *             omega_nu = 1/tau, omega_q = (3/dt)(2/dt - omega_nu)/(3/dt - omega_nu),
 *             omega_e = omega_e_dt/dt, omega_eps = omega_eps_dt/dt).
 *  thermal    LBM_NONE, LBM_D2Q5 or LBM_D2Q9 (double-distribution thermal LBE, Sec. 2.2,
 *             linear g_eq of Eq. geq_geral; D2Q5: w = 1/3, 1/6 x4, c_s^2 = c^2/3; D2Q9, the
 *             paper's lattice, needs flow = D2Q9).
 *  thermal_op LBM_BGK (Eq. eq_lattice_boltzmann_BGK_T) or LBM_MRT: on D2Q9 the thermal MRT
 *             of Sec. 2.2, [Lambda_T] = diag(0, 1, 1, 1/tau_T, 1, 1/tau_T, 1, 1, 1) with
 *             the unit rates taken as 1/dt, on the momentum matrices; on D2Q5 its analogue,
 *             moments (1, c_x, c_y, 5|c|^2-4c^2, c_x^2-c_y^2) relaxed at (0, 1/tau_T, 1/tau_T,
 *             1/dt, 1/dt).  Both with the source dt (I - dt Lambda/2) M (w qdot).
 *  phase      LBM_NONE (single phase) or LBM_D2Q5 (two-phase model of Sec. 2.3: Allen-Cahn
 *             h_i on D2Q5, pressure-evolution z_i on D2Q9 with operator z_op).
 *  nu_rule    two-phase viscosity: 0 linear in phi, 1 nu = zeta/rho with zeta linear in phi.
 *  literal    bit 0: thermal source prefactor with the momentum tau as printed in
 *             Eq. forcing_term_g (default uses tau_T); bit 1: multiphase q_y moment
 *             relaxed at 1/dt as printed in Sec. 3 (default uses omega_q2 for q_x and q_y).
 *  precision  LBM_FP64 or LBM_FP32DEV.
 *  nx, ny     grid size, each >= 1 (>= 2 along an axis with a pressure/outflow side).
 *  dx, dt     lattice spacing [m] and time step [s]; c = dx/dt.
 *  rho0       reference density [kg m^-3] (single phase; storage offset for FP32DEV).
 *  nu         kinematic viscosity [m^2 s^-1]; tau = nu/c_s^2 + dt/2 (Eq. eq_kinematic_viscosity).
 *  cp, k      specific heat [J kg^-1 K^-1] and conductivity [W m^-1 K^-1];
 *             alpha = k/(rho0 cp) = (tau_T - dt/2) c_s^2.
 *  T0         reference temperature [K] (default initial T; storage offset for FP32DEV).
 *  rho_l, rho_g, nu_l, nu_g, sigma, W, mobility: two-phase properties (Sec. 2.3);
 *             kappa = 3 sigma W/2, beta = 12 sigma/W, M = (tau_phi - dt/2) c_s^2.
 *  omega_e_dt, omega_eps_dt: free MRT rates times dt (paper: between 1 and 2; default 1).
 *  body_force uniform body force F_b [N m^-3].
 *  u_prescribed velocity used when flow == LBM_NONE [m s^-1].
 *  gravity, beta_exp, T_ref, rho_ref: Boussinesq two-way coupling of App. D, Eq. buoyancy_force:
 *             F_b = -rho_ref beta_exp (T - T_ref) g added to the momentum force with the
 *             node's temperature of the same step (beta_exp = 0 disables it).  Needs
 *             flow = D2Q9 and a thermal LBE.
 */
typedef struct {
  int flow, flow_op, thermal, thermal_op, phase, z_op, nu_rule, literal, precision;
  int nx, ny;
  double dx, dt;
  double rho0, nu, cp, k, T0;
  double rho_l, rho_g, nu_l, nu_g, sigma, W, mobility;
  double omega_e_dt, omega_eps_dt;
  double body_force[2];
  double u_prescribed[2];
  double gravity[2];
  double beta_exp, T_ref, rho_ref;
} lbm_params;

/* Fill *p with defaults: D2Q9 BGK, no thermal, single phase, FP64, water-like
   rho0 = 1000, nu = 1e-6, cp = 4180, k = 0.6, T0 = 300, free MRT rates 1/dt. */
void lbm_params_default(lbm_params *p);

/*
 * Create a solver.  Validates the parameters (tau, tau_T, tau_phi > dt/2 as required
 * by Eq. eq_kinematic_viscosity and the stability remark of Sec. 4; sizes; lattice
 * combinations), derives c, c_s^2 and the relaxation times, allocates the device
 * state (two ping-pong structure-of-arrays buffers) and leaves it uninitialised until
 * lbm_init_fields.  All sides start periodic.  stream: a cudaStream_t or NULL.
 * Errors: LBM_ERR_ARG, LBM_ERR_UNSTABLE_TAU, LBM_ERR_NOMEM, LBM_ERR_CUDA; *out = NULL then.
 */
lbm_status lbm_create(const lbm_params *p, void *stream, lbm_t *out);

/*
 * Boundary of one side (0 x-, 1 x+, 2 y-, 3 y+), both lattices at once.
 *  kind  momentum rule (LBM_BC_*); rho_w the boundary density of Eqs. BB_vel/anti_BB_vel.
 *  uw    host array of 2*len doubles (u_x[len] then u_y[len]), len = ny for x-sides and
 *        nx for y-sides: wall/inlet velocity at each boundary node, also used by the
 *        thermal anti-bounce-back; NULL = zero.
 *  tkind thermal rule (LBM_TBC_*); tw host array of len doubles: q'' [W m^-2, positive
 *        into the fluid] for FLUX, T_w [K] for TEMP, ignored otherwise; NULL = zero.
 *        FLUX on D2Q9 weights the unknowns with lambda_i = 6 w_i (4/6 axial, 1/6
 *        diagonal), on D2Q5 the single unknown with 1.
 * Both sides of an axis must be periodic together, for each lattice.  A link that
 * leaves through a corner takes the y-side rule, unless the y-side is a symmetry
 * side: then the other side's rule.
 * Two-phase solves (Sec. 4.4, layered flow between plates) take LBM_BC_PERIODIC or
 * LBM_BC_WALL at rest (uw NULL or zero) and LBM_TBC_NONE: half-way bounce-back of z
 * and h, and phi beyond the wall mirrored from the boundary node in the gradient
 * and Laplacian stencils; an axis with a wall on either side is walled.
 * The arrays are copied before the call returns (through pinned staging, without
 * synchronising the stream).  The kernels keep post-collision populations and rebuild
 * the incoming ones, boundary links included, by the pull: after n steps the state of
 * time n is formed when it is next read (lbm_moments, lbm_integrals) or advanced
 * (lbm_step).  New boundary values therefore apply from the boundary links of the
 * current time n on; a collide-then-push formulation would apply them from time n + 1,
 * one step later.
 * Errors: LBM_ERR_ARG (side, kind, pairing, a moving or non-wall two-phase side),
 * LBM_ERR_CUDA.
 */
lbm_status lbm_set_bc(lbm_t h, int side, int kind, const double *uw, double rho_w, int tkind,
                      const double *tw);

/*
 * Per-cell sources.  q3: nx*ny volumetric heat generation q''' [W m^-3]; the thermal
 * source is qdot = q'''/(rho0 cp) [K s^-1] (Eqs. forcing_term_g, zero_moment_g).
 * force: 2*nx*ny doubles (F_x plane then F_y plane) [N m^-3], added to body_force
 * (Eqs. forcing_term, first_moment_f).  NULL removes the field.  on_device: pointers
 * are device pointers.  Errors: LBM_ERR_ARG, LBM_ERR_NOMEM, LBM_ERR_CUDA.
 */
lbm_status lbm_set_source(lbm_t h, const double *q3, const double *force, int on_device);

/*
 * Lagged linear heat sink of the fuse problem (Sec. 4.1, Eq. conver_energy_fuse):
 * qdot(t) = q'''/(rho0 cp) - conv_coef (T(t - dt) - T_inf), the temperature of the
 * previous step, so that the update stays explicit.  Before every step (and before
 * lbm_moments) a kernel rebuilds T(t - dt) at each node from its own post-collision
 * populations, T = T0 + sum g* - dt qdot/2 (the collision adds dt qdot to sum g), and
 * writes this step's qdot; after lbm_init_fields T(-dt) is the initial T.
 *  conv_coef [s^-1] (4 hbar / (rho cp d) for the fuse); 0 removes the sink.
 *  T_inf     [K].
 * q''' of lbm_set_source stays the base of qdot.  Needs a thermal LBE; not with
 * buoyancy, the literal thermal-source flag (literal bit 0) or the adjoint.
 * After lbm_set_state the lag restarts from the base qdot.
 * Errors: LBM_ERR_ARG, LBM_ERR_NOMEM, LBM_ERR_CUDA.
 */
lbm_status lbm_set_lagged_sink(lbm_t h, double conv_coef, double T_inf);

/*
 * Initialise every distribution at its equilibrium (Eqs. feq_geral, geq_geral,
 * heq_liang, zeq_liang) from nx*ny fields; NULL takes the default.
 *  single phase: a = rho (default rho0), ux, uy (default 0), b = T (default T0);
 *  two-phase:    a = phi (default 1), ux, uy, b = p (default 0); (phi u)_prev = phi u.
 * The first step then collides this state (the pull kernel stores post-collision
 * values, so the initial collision is folded into this call).
 * Errors: LBM_ERR_ARG, LBM_ERR_CUDA.
 */
lbm_status lbm_init_fields(lbm_t h, const double *a, const double *ux, const double *uy,
                           const double *b, int on_device);

/*
 * Advance n >= 0 time steps: fused pull-stream + boundary links + moments + collision
 * (Eqs. eq_lattice_boltzmann_geral, colisao_MRT, ...), one kernel launch per step,
 * asynchronous on the stream.  With a health-check interval K > 0
 * (lbm_set_check_interval) the call also runs the integrals of lbm_integrals each time
 * the step count reaches a multiple of K (one stream synchronisation per check) and
 * stops there if a cell is bad (non-finite, or |u| >= c).
 * Errors: LBM_ERR_STATE (not initialised), LBM_ERR_CUDA, LBM_ERR_DIVERGED (a check
 * found bad cells: the state is that of the failing step, lbm_last_good_step gives
 * the step count of the last check that passed), LBM_ERR_TIMEOUT (see lbm_set_launch).
 */
lbm_status lbm_step(lbm_t h, long n);

/*
 * Health check inside lbm_step (no counterpart in the paper: a run-time guard for
 * long runs).  every = K > 0 checks at each multiple of K steps; 0 (the default)
 * turns the checks off, keeping lbm_step fully asynchronous.  lbm_last_good_step
 * returns the step count of the last passed check since lbm_init_fields (-1: none).
 * Errors: LBM_ERR_ARG (every < 0).
 */
lbm_status lbm_set_check_interval(lbm_t h, long every);
long lbm_last_good_step(lbm_t h);

/*
 * Wall-time limit of each wait of the TMA-staged step for its staged copies (no
 * counterpart in the paper; default 1 s, allowed (0, 10] s).  A wait that runs out
 * marks the handle, lets the block's copies in flight land and ends the block; the
 * next lbm_integrals / lbm_check reports LBM_ERR_TIMEOUT once and clears the mark.
 * The results of a step whose waits ran out are not valid: restore a state saved with
 * lbm_get_state.  expire_next = 1 is a self-test of that failure path: in the next
 * TMA-staged step every block first waits, with this limit, on a barrier that nothing
 * completes, so its wait runs out.  Errors: LBM_ERR_ARG.
 */
lbm_status lbm_set_wait_limit(lbm_t h, double seconds, int expire_next);

/*
 * Pick the launch of the single-solve step kernel by timing candidates (grid launches
 * of 32..256 threads and TMA-staged persistent launches, see lbm_set_launch) on the
 * next step, without advancing the solution (the timed launches repeat that step into
 * the same destination).  out_block (may be NULL) receives the chosen thread-block
 * shape {block_x, block_y}.  Single-phase solves only; the default is a 64 x 4 grid
 * launch.
 * Errors: LBM_ERR_STATE (not initialised), LBM_ERR_ARG, LBM_ERR_CUDA.
 */
lbm_status lbm_autotune(lbm_t h, int out_block[2]);

/*
 * DIAGNOSTIC, not part of the solver: FMA-rate probe used by the benchmark to state
 * the arithmetic roofline of the FP64 and FP32 forms on the current device (no
 * counterpart in the paper).  Runs eight independent chains of fused
 * multiply-adds per thread on every SM and returns the rate in GFLOP/s (2 flops per
 * FMA) in *gflops.  Synchronous; allocates and frees its own scratch.
 * precision: LBM_FP64 or LBM_FP32DEV.  Errors: LBM_ERR_ARG, LBM_ERR_CUDA (text in
 * lbm_last_error(NULL)).
 */
lbm_status lbm_probe_fma_rate(int precision, double *gflops);

/*
 * Launch configuration of the single-phase step (no counterpart in the paper: a
 * choice of memory pipeline for the same arithmetic).  cfg[4]:
 *  {LBM_LAUNCH_GRID, block_x, block_y, 0}: one thread per node, block_x a multiple
 *     of 32, block_x * block_y <= 256 (the default, 64 x 4);
 *  {LBM_LAUNCH_GRID_OCC, block_x, block_y, 0}: the same kernel built for more
 *     resident blocks per SM (FP32 with a thermal lattice: 6 blocks of 256 threads at
 *     40 registers instead of 4 at 64; faster on large grids, slower on short
 *     launches; the same kernel for the other kinds);
 *  {LBM_LAUNCH_TMA, tile_height (4 or 8), stages (1..4), CTAs per SM}: persistent
 *     CTAs of 32 x tile_height threads; per tile, the pulled values of every
 *     population plane arrive as tensor-memory-accelerator boxes in shared memory,
 *     `stages` tiles ahead (the first step after lbm_init_fields always uses the
 *     grid launch).  A wait for a box that runs out (about 1 s) marks the handle;
 *     the next lbm_integrals / lbm_check then fails with LBM_ERR_TIMEOUT.
 * lbm_autotune chooses among all three kinds; lbm_launch_config reads the current one.
 * Errors: LBM_ERR_ARG (two-phase handle, out-of-range value, more CTAs per SM than
 * fit), LBM_ERR_CUDA (the driver refused the tensor maps).
 */
#define LBM_LAUNCH_GRID 0
#define LBM_LAUNCH_TMA 1
#define LBM_LAUNCH_GRID_OCC 2
lbm_status lbm_set_launch(lbm_t h, const int cfg[4]);
lbm_status lbm_launch_config(lbm_t h, int cfg[4]);

/* Steps taken since lbm_init_fields (time = steps * dt). */
long lbm_steps_done(lbm_t h);

/*
 * Macroscopic fields at the current time (pulled from the stored post-collision
 * populations, so they include the boundary rules):
 *  LBM_RHO rho (Eq. zero_moment_f, or rho(phi)), LBM_UX / LBM_UY velocity
 *  (Eq. first_moment_f or Eq. u_Liang), LBM_T temperature (Eq. zero_moment_g),
 *  LBM_P pressure (two-phase: Eq. p_Liang; single phase: c_s^2 (rho - rho0)),
 *  LBM_PHI order parameter (Eq. zero_moment_h).
 * out receives one nx*ny row-major plane per selected bit, in bit order.
 * Host output synchronises the stream.  Errors: LBM_ERR_ARG, LBM_ERR_STATE, LBM_ERR_CUDA.
 */
lbm_status lbm_moments(lbm_t h, unsigned mask, double *out, int on_device);

/*
 * Integrals with deterministic FP64 reductions (fixed tree order).  A bad cell is one
 * with a non-finite rho, u, T (thermal) or p (two-phase), or with |u| >= c; it is
 * counted in out[3] and adds nothing to out[0..2].  Single-phase FP32 solves form
 * |u|^2, its maximum and the |u| >= c test in FP32 (the precision of their u); the
 * mass is summed in FP64 in every precision:
 *  out[0] = sum of rho dx^2 over the healthy cells (mass per unit depth, kg/m),
 *  out[1] = sum of phi over the healthy cells (two-phase, else 0),
 *  out[2] = max |u| over the healthy cells [m/s], out[3] = number of bad cells.
 * out is host memory of 4 doubles; the call synchronises the stream.
 * Errors: LBM_ERR_STATE, LBM_ERR_CUDA, LBM_ERR_TIMEOUT (a TMA-staged step gave up
 * waiting for a staged copy since the last call; out is still written).
 */
lbm_status lbm_integrals(lbm_t h, double out[4]);

/* lbm_integrals + status: LBM_ERR_DIVERGED when out[3] > 0 (or LBM_ERR_TIMEOUT). */
lbm_status lbm_check(lbm_t h);

/*
 * Raw state for checkpoint/restart: the current post-collision buffer, the step
 * counter excluded.  lbm_state_bytes gives the size; get copies device -> host,
 * set copies host -> device.  Layout: planes of ny*nx values (no padding) in the
 * order f_0..8, g_0..4 (single phase) or z_0..8, h_0..4, (phi u)_x, (phi u)_y
 * (two-phase); FP32DEV stores deviations f_i - w_i rho0 and g_i - w_i T0 as float.
 * Errors: LBM_ERR_ARG (size), LBM_ERR_STATE, LBM_ERR_CUDA.
 */
size_t lbm_state_bytes(lbm_t h);
lbm_status lbm_get_state(lbm_t h, void *dst, size_t bytes);
lbm_status lbm_set_state(lbm_t h, const void *src, size_t bytes);

/* Derived constants: out[0] c, [1] c_s^2, [2] tau, [3] tau_T, [4] tau_phi (seconds). */
lbm_status lbm_constants(lbm_t h, double out[5]);

/* Wait for all work on the handle's stream. */
lbm_status lbm_synchronize(lbm_t h);

/* Text of the last error on h (or of the last failed lbm_create when h is NULL). */
const char *lbm_last_error(lbm_t h);

/* Free the device state.  NULL is ignored. */
void lbm_destroy(lbm_t h);

/*
 * Batched solves: many independent single-phase channels of uneven size advanced
 * together, one kernel launch per time step over a flattened (channel, tile) list,
 * replayed from a CUDA graph.  Each channel is an ordinary lbm_t owned by the batch:
 * set its boundaries, sources and initial fields and read its moments with the calls
 * above (lbm_batch_channel), but advance it only with lbm_batch_step.
 *  lbm_batch_create  n parameter blocks (same precision, lattices and operators; single
 *                    phase); stream NULL = a private non-blocking stream (graph capture
 *                    cannot use the legacy default stream).  Errors as lbm_create.
 *  lbm_batch_step    advance every channel n steps; all channels must be initialised and
 *                    in step.  Asynchronous on the batch stream.  Errors: LBM_ERR_STATE,
 *                    LBM_ERR_ARG (a channel with a lagged sink), LBM_ERR_CUDA.
 *  lbm_batch_autotune time candidate tile shapes (32..256 threads) and grid sizes (1..16
 *                    blocks per SM) on the next step without advancing the solution; keeps
 *                    the fastest; out_cfg (may be NULL) receives {tile_x, tile_y, grid}.
 *  lbm_batch_config  set tile shape and grid explicitly (tile_x * tile_y a multiple of 32,
 *                    at most 256).
 * Every channel's result equals stepping it alone with lbm_step (same arithmetic).
 */
typedef struct lbm_batch_s *lbm_batch_t;
lbm_status lbm_batch_create(const lbm_params *params, int n, void *stream, lbm_batch_t *out);
lbm_t lbm_batch_channel(lbm_batch_t b, int k);
int lbm_batch_size(lbm_batch_t b);
lbm_status lbm_batch_step(lbm_batch_t b, long n);
lbm_status lbm_batch_autotune(lbm_batch_t b, int out_cfg[3]);
lbm_status lbm_batch_config(lbm_batch_t b, int tile_x, int tile_y, int grid);
const char *lbm_batch_last_error(lbm_batch_t b);
void lbm_batch_destroy(lbm_batch_t b);

/*
 * Reverse-time discrete adjoint of the fused step for single-phase D2Q9 MRT + D2Q5 MRT
 * solves, in the handle's precision: FP64, or FP32 (the forward in FP32 deviation
 * storage, the adjoint variables and their arithmetic in FP32, the parameter gradients
 * accumulated to FP64 precision (the per-cell q''' gradient and the nu sums in
 * compensated FP32 pairs, converted once); its gradient is that of the FP32 forward
 * map, to FP32 rounding).  Call right after lbm_init_fields (and lbm_set_bc, lbm_set_source):
 * it runs the forward `steps` steps itself, keeping a checkpoint every ckpt_every
 * steps, then walks the steps backwards, recomputing each segment's states from its
 * checkpoint.  Device memory: (steps/ckpt_every + ckpt_every + 3) state buffers.  On
 * return the handle holds the forward state of time steps * dt.
 *  loss     L = (1/ny) sum_j (T(nx-1, j; steps) - T_target[j])^2: mean squared error of
 *           the temperature of the x+ column against T_target (ny host doubles) [K^2]
 *  g_q3     nx*ny host array (or NULL): dL/dq for the per-cell volumetric heat source
 *           set by lbm_set_source [K^2 per W m^-3]
 *  g_qwall  2*nx host array (or NULL): dL/dq_wall per node of the y- wall, then of the
 *           y+ wall, for sides with LBM_TBC_FLUX [K^2 per W m^-2]
 *  g_nu     host scalar (or NULL): dL/dnu [K^2 per m^2 s^-1]
 * The gradient is that of the discrete forward map (exact up to rounding).
 * Errors: LBM_ERR_ARG (configuration), LBM_ERR_STATE (not freshly initialised),
 * LBM_ERR_NOMEM, LBM_ERR_CUDA.
 */
lbm_status lbm_adjoint(lbm_t h, long steps, int ckpt_every, const double *T_target, double *loss, double *g_q3,
                       double *g_qwall, double *g_nu);

/*
 * Allocation-free integrals over macroscopic fields the caller already holds on
 * the device.  The paper has no counterpart: this is a service for callers that
 * cannot call cudaMalloc (code that runs inside a memory pool or arena owning the
 * whole device, under a framework allocator that forbids foreign allocations, or
 * where an allocation's implicit device synchronisation is not allowed).
 *
 * Computes the four quantities of lbm_integrals from the given fields, with a
 * deterministic two-stage FP64 reduction (fixed order, so repeated calls agree bit
 * for bit; the summation order differs from lbm_integrals', so the two agree to
 * rounding).  A bad cell has a non-finite rho, u or phi, or |u| >= c (there is no
 * temperature field here, so a non-finite T is not seen); it is counted and adds
 * nothing to the sums or the maximum:
 *   out4[0] = sum of rho dx^2 over the healthy cells, out4[1] = sum of phi over the
 *   healthy cells (0 when phi is NULL), out4[2] = max |u| over the healthy cells,
 *   out4[3] = number of bad cells.
 * rho, ux, uy (and phi, or NULL): device arrays of nx*ny doubles, row-major;
 * out4: device array of 4 doubles written by the call; dx [m]; c = dx/dt [m/s];
 * stream: a cudaStream_t or NULL.  Asynchronous on that stream; it allocates
 * nothing and calls no allocating routine.
 *
 * Scratch: a file-scope device array of LBM_NOALLOC_MAX_BLOCKS x 4 doubles (128 KiB)
 * that every GPU loading the library holds until the process exits.  Grids larger
 * than LBM_NOALLOC_MAX_CELLS cells are rejected with LBM_ERR_ARG (message in
 * lbm_last_error(NULL)); use lbm_integrals for them.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share the
 * array and each call rewrites every entry it reads, so calls that overlap on the
 * GPU (different streams, or different host threads on one device) race: order
 * them on one stream.  The looked-up address is kept for the life of the process:
 * do not call this after a cudaDeviceReset of a device it has already run on.
 * Errors: LBM_ERR_ARG (NULL pointer, sizes), LBM_ERR_CUDA.
 */
#define LBM_NOALLOC_MAX_BLOCKS 4096
#define LBM_NOALLOC_CELLS_PER_BLOCK 2048
#define LBM_NOALLOC_MAX_CELLS (LBM_NOALLOC_MAX_BLOCKS * LBM_NOALLOC_CELLS_PER_BLOCK)
lbm_status lbm_field_integrals_noalloc(const double *rho, const double *ux, const double *uy,
                                       const double *phi, int nx, int ny, double dx, double c,
                                       double *out4, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
