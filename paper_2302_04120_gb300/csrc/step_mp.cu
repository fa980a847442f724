// Two-phase kernels: conservative Allen-Cahn h_i (D2Q5, BGK) coupled to the
// pressure-evolution z_i (D2Q9, MRT or BGK) of the model described in Sec. 2.3
// of Martins, Alvarino & Cabezas-Gomez (arXiv:2302.04120), all in SI units.
//
// A step is ONE launch (k_mp_collide) over 32 x 8 tiles:
//   * pull h_i for the tile and for a one-node halo ring (periodic, or beyond a
//     resting wall the mirror image of the boundary node) and stage
//     phi = sum h_i (Eq. zero_moment_h) in shared memory (the node's own h stay
//     in registers; halo h re-reads hit L2, so DRAM sees each h once);
//   * isotropic gradient and Laplacian (Eqs. gradient, laplacian, D2Q9 weights),
//     chemical potential (Eq. chemical_potential), guarded normal, F_s = mu grad
//     phi, grad rho; pull z_i; recover u (Eq. u_Liang) and p (Eq. p_Liang);
//   * collide h (Eqs. eq_lattice_boltzmann_interface, heq_liang,
//     source_term_interface) and z (Eq. colisao_MRT with the multiphase
//     [Lambda]_dim of Sec. 3, Eqs. zeq_liang, s_i_Liang,
//     forcing_term_pressure_evolution); store h*, z* and phi u for the next
//     explicit d_t(phi u).
// In the FP32 form the populations and (phi u) are stored in FP32 and the
// collision runs in FP32, while rho(phi), u and p are recovered in FP64 across the
// interface and in the gas (phi < 0.999): at the ~43000 density ratio of saturated
// water u = j / rho divides by rho_g = 0.023.  In the liquid bulk FP32 resolves them.
#include <cuda_runtime.h>

#include "lattice.cuh"
#include "lbm_mp.cuh"

namespace lbmk {

namespace {

// Tiles are 32 nodes wide and BY = 8 rows high, or 2 rows on grids too small to give
// every SM several 32 x 8 tiles (the FP64 collision is then spread over more SMs).
constexpr int BX = 32;
constexpr int kSmallGridBlocks = 608;  // 4 x 152 SMs: fewer 32 x 8 tiles take BY = 2

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }
__device__ __forceinline__ int modi(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

// Source of the pull of population q (velocity (cx, cy), opposite o) at node (i, j):
// the upstream node, wrapped on a periodic axis; on a walled axis a link whose
// upstream node lies beyond the wall is the node's own opposite population
// (half-way bounce-back at a resting wall).  Returns the element offset.
__device__ __forceinline__ long long pull_src(const MpParams &P, int q, int o, int cx, int cy, int i, int j) {
  if (P.local) return q * P.plane + (long long)j * P.pitch + i;
  const int si = i - cx, sj = j - cy;
  const bool out = (P.xwall && (si < 0 || si >= P.nx)) || (P.ywall && (sj < 0 || sj >= P.ny));
  if (out) return o * P.plane + (long long)j * P.pitch + i;
  return q * P.plane + (long long)wrapi(sj, P.ny) * P.pitch + wrapi(si, P.nx);
}

// Node whose phi stands at stencil position a along an axis of n nodes: wrapped on a
// periodic axis; on a walled axis the mirror image of the boundary node for the one
// layer beyond the wall (further positions are never read by a live node).
__device__ __forceinline__ int stencil_node(int a, int n, int wall) {
  if (wall) return a < 0 ? 0 : (a >= n ? n - 1 : a);
  return a < 0 || a >= n ? modi(a, n) : a;
}

template <typename S, typename R>
__device__ __forceinline__ void pull_h(const MpParams &P, const S *src, int i, int j, R h[5]) {
  const S *hs = src + 9ll * P.plane;
#pragma unroll
  for (int q = 0; q < 5; q++) h[q] = (R)hs[pull_src(P, q, opp5(q), cx5(q), cy5(q), i, j)];
}

// The same pulls for a node whose sources cannot wrap (blocks away from the grid's
// periodic seams): sn points at the node in plane 0; every plane offset is uniform.
template <typename S, typename R>
__device__ __forceinline__ void pull_h_at(const MpParams &P, const S *sn, R h[5]) {
  const S *hs = sn + 9ll * P.plane;
#pragma unroll
  for (int q = 0; q < 5; q++) h[q] = (R)hs[q * P.plane - (long long)cy5(q) * P.pitch - cx5(q)];
}

template <typename S, typename R>
__device__ __forceinline__ void pull_z_at(const MpParams &P, const S *sn, R z[9]) {
#pragma unroll
  for (int q = 0; q < 9; q++) z[q] = (R)sn[q * P.plane - (long long)cy9(q) * P.pitch - cx9(q)];
}

// Quotient in the working precision: exact in FP64; in FP32 the approximate
// reciprocal-based divide (about 2 ulp), which spares the IEEE divide sequence.
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
// 1 / |g| for g2 = |g|^2 > 0, else 0 (same precision split).
__device__ __forceinline__ double inv_norm(double g2) { return g2 != 0.0 ? 1.0 / sqrt(g2) : 0.0; }
__device__ __forceinline__ float inv_norm(float g2) { return g2 != 0.0f ? rsqrtf(g2) : 0.0f; }

template <typename S, typename R>
__device__ __forceinline__ void pull_z(const MpParams &P, const S *src, int i, int j, R z[9]) {
#pragma unroll
  for (int q = 0; q < 9; q++) z[q] = (R)src[pull_src(P, q, opp9(q), cx9(q), cy9(q), i, j)];
}

// Macroscopic state of a node.  The order parameter, its stencils, the chemical
// potential, the forces and the relaxation rates are in the working precision R;
// rho, u and p -- the recovery that divides by rho_g ~ 0.023 at the interface --
// are in FP64 in both forms.
template <typename R>
struct MpMacro {
  R phi, mu, gx, gy, nxv, nyv, Fx, Fy, drx, dry, wb;  // wb = dt / tau
  R rho, ux, uy, p;
};

// Gradient/Laplacian from the shared tile, then rho, nu, tau, F, u, p.
// Liquid nodes with phi above this use the working-precision recovery of rho, u, p;
// all others (the interface, its tanh tails and the gas) recover in FP64.
constexpr float kPhiFp64Below = 0.999f;

template <typename R>
__device__ __forceinline__ void mp_macro(const MpParams &P, const R (*tile)[BX + 2], int tx, int ty,
                                         const R z[9], R fext_x, R fext_y, MpMacro<R> &m) {
  // D2Q9 neighbours phi(x + c_i dt)
  const R pc = tile[ty][tx];
  const R pE = tile[ty][tx + 1], pW = tile[ty][tx - 1];
  const R pN = tile[ty + 1][tx], pS = tile[ty - 1][tx];
  const R pNE = tile[ty + 1][tx + 1], pNW = tile[ty + 1][tx - 1];
  const R pSW = tile[ty - 1][tx - 1], pSE = tile[ty - 1][tx + 1];
  // Eq. gradient: sum_i w_i c_i phi_i / (c_s^2 dt) = (3/dx) sum_i w_i e_i phi_i
  const MpConst<R> &K = KM<R>(P);
  const R g3 = K.g3;
  m.gx = g3 * ((pE - pW) * ((R)1 / (R)9) + ((pNE - pNW) + (pSE - pSW)) * ((R)1 / (R)36));
  m.gy = g3 * ((pN - pS) * ((R)1 / (R)9) + ((pNE - pSE) + (pNW - pSW)) * ((R)1 / (R)36));
  // Eq. laplacian: sum_i 2 w_i (phi_i - phi) / (c_s^2 dt^2) = (6/dx^2) sum_i w_i (phi_i - phi)
  const R lap = K.l6 * (((pE + pW) + (pN + pS) - (R)4 * pc) * ((R)1 / (R)9) +
                           ((pNE + pNW) + (pSE + pSW) - (R)4 * pc) * ((R)1 / (R)36));
  m.phi = pc;
  // Eq. chemical_potential
  m.mu = (R)4 * K.beta * pc * (pc - (R)1) * (pc - (R)0.5) - K.kappa * lap;
  // normal only where |grad phi| != 0
  const R rg = inv_norm(m.gx * m.gx + m.gy * m.gy);
  m.nxv = m.gx * rg;
  m.nyv = m.gy * rg;
  const R drl = K.drl;
  R nu;
  if (P.nu_rule == 0) nu = K.nu_g + pc * K.dnu;
  else nu = qdiv(K.zg + pc * K.dzeta, K.rho_g + pc * drl);
  // tau / dt = nu / (c_s^2 dt) + 1/2 (Eq. eq_kinematic_viscosity)
  m.wb = qdiv((R)1, nu * K.inv_cs2dt + (R)0.5);
  m.drx = drl * m.gx;
  m.dry = drl * m.gy;
  m.Fx = m.mu * m.gx + K.Fx + fext_x;
  m.Fy = m.mu * m.gy + K.Fy + fext_y;
  // recovery of rho(phi), Eq. u_Liang, then Eq. p_Liang (u first)
  if (sizeof(R) == 8 || pc < (R)kPhiFp64Below) {
    // FP64 across the interface and in the gas, where u = j / rho divides by rho_g
    double zd[9];
#pragma unroll
    for (int q = 0; q < 9; q++) zd[q] = (double)z[q];
    const double c = P.c;
    const double jx = c * ((zd[1] - zd[3]) + (zd[5] - zd[6]) + (zd[8] - zd[7]));
    const double jy = c * ((zd[2] - zd[4]) + (zd[5] - zd[8]) + (zd[6] - zd[7]));
    const double znz = ((zd[1] + zd[2]) + (zd[3] + zd[4])) + ((zd[5] + zd[6]) + (zd[7] + zd[8]));
    const double rho = P.rho_g + (double)pc * (P.rho_l - P.rho_g);
    const double inv = 1.0 / rho;
    const double ux = (jx + 0.5 * P.dt * (double)m.Fx) * inv;
    const double uy = (jy + 0.5 * P.dt * (double)m.Fy) * inv;
    const double usq = ux * ux + uy * uy;
    const double s0 = (4.0 / 9.0) * (-0.5 * usq * P.inv_cs2);  // s_0(u), Eq. s_i_Liang
    m.rho = (R)rho;
    m.ux = (R)ux;
    m.uy = (R)uy;
    m.p = (R)(P.cs2 * 1.8 * (znz + 0.5 * P.dt * (ux * (double)m.drx + uy * (double)m.dry) + rho * s0));
  } else {
    // liquid (rho within 0.1 % of rho_l): the working precision resolves u and p
    const R c = K.c;
    const R jx = c * ((z[1] - z[3]) + (z[5] - z[6]) + (z[8] - z[7]));
    const R jy = c * ((z[2] - z[4]) + (z[5] - z[8]) + (z[6] - z[7]));
    const R znz = ((z[1] + z[2]) + (z[3] + z[4])) + ((z[5] + z[6]) + (z[7] + z[8]));
    const R rho = K.rho_g + pc * K.drl;
    const R inv = qdiv((R)1, rho);
    const R hdt = K.hdt;
    const R ux = (jx + hdt * m.Fx) * inv, uy = (jy + hdt * m.Fy) * inv;
    const R s0 = (R)(4.0 / 9.0) * ((R)-0.5 * (ux * ux + uy * uy) * K.inv_cs2);
    m.rho = rho;
    m.ux = ux;
    m.uy = uy;
    m.p = K.pcoef * (znz + hdt * (ux * m.drx + uy * m.dry) + rho * s0);
  }
}

template <typename R>
__device__ __forceinline__ void collide_h(const MpParams &P, const MpMacro<R> &m, R dpux, R dpuy, R h[5]) {
  const MpConst<R> &K = KM<R>(P);
  const R c = K.c, inv_cs2 = K.inv_cs2;
  const R om = K.om_h;
  const R sfac = K.sfac_h;
  const R a_int = K.aint_coef * m.phi * ((R)1 - m.phi);  // c_s^2 4 phi (1 - phi) / W
  const R ax = dpux + a_int * m.nxv, ay = dpuy + a_int * m.nyv;
  const R phi = m.phi, ux = m.ux, uy = m.uy;
  R heq_sum = 0;
#pragma unroll
  for (int q = 1; q < 5; q++) {
    const R cxq = c * (R)cx5(q), cyq = c * (R)cy5(q);
    const R heq = phi * w5<R>(q) * ((R)1 + (cxq * ux + cyq * uy) * inv_cs2);  // Eq. heq_liang
    const R Sh = w5<R>(q) * (cxq * ax + cyq * ay) * inv_cs2;                    // Eq. source_term_interface
    heq_sum += heq;
    h[q] = h[q] - om * (h[q] - heq) + sfac * Sh;
  }
  // h_0^eq = phi w_0 = phi - sum_{q>=1} h_q^eq: sum h_eq = phi exactly in the working
  // precision (in FP32 the rounded weights sum to 1 + 3e-8, a systematic phase gain)
  h[0] = h[0] - om * (h[0] - (phi - heq_sum));
}

template <typename R>
__device__ __forceinline__ void collide_z(const MpParams &P, const MpMacro<R> &m, R z[9]) {
  const MpConst<R> &K = KM<R>(P);
  const R c = K.c;
  const R rho = m.rho, ux = m.ux, uy = m.uy;
  const R Fx = m.Fx, Fy = m.Fy, gx = m.drx, gy = m.dry;
  if (!P.z_mrt) {
    // BGK, Eq. eq_lattice_boltzmann_pressure
    const R inv_cs2 = K.inv_cs2;
    const R om = m.wb, sfac = ((R)1 - (R)0.5 * m.wb) * K.dt;
    const R Pp = m.p * K.inv_cs2;
    const R hu = (R)0.5 * (ux * ux + uy * uy) * inv_cs2;
#pragma unroll
    for (int q = 0; q < 9; q++) {
      const R cxq = c * (R)cx9(q), cyq = c * (R)cy9(q);
      const R cu = cxq * ux + cyq * uy;
      const R si = w9<R>(q) * (cu * inv_cs2 * ((R)1 + (R)0.5 * cu * inv_cs2) - hu);
      const R zeq = Pp * (w9<R>(q) - (q == 0 ? (R)1 : (R)0)) + rho * si;  // Eq. zeq_liang
      const R Fz = w9<R>(q) * ((cxq * Fx + cyq * Fy) + cu * (cxq * gx + cyq * gy)) * inv_cs2;
      z[q] = z[q] - om * (z[q] - zeq) + sfac * Fz;
    }
    return;
  }
  // MRT on lattice-scaled moments (see step_sp.cu): equilibrium moments of z_eq
  // are M f_eq(rho, u) - rho M w + (p/c_s^2)(M w - M e_0); forcing moments of
  // F_hat^z = w_i [c_i.F + (c_i.u)(c_i.grad rho)] / c_s^2.
  const R ic = K.ic;
  const R hx = ux * ic, hy = uy * ic, usq = hx * hx + hy * hy;
  const R Pp = m.p * K.inv_cs2;
  const R s14 = (z[1] + z[2]) + (z[3] + z[4]);
  const R s58 = (z[5] + z[6]) + (z[7] + z[8]);
  const R m0 = z[0] + s14 + s58;
  const R m_e = -(R)4 * z[0] - s14 + (R)2 * s58;
  const R m_ep = (R)4 * z[0] - (R)2 * s14 + s58;
  const R d58 = z[5] - z[7], d68 = z[6] - z[8];
  const R m_jx = (z[1] - z[3]) + d58 - d68;
  const R m_jy = (z[2] - z[4]) + d58 + d68;
  const R m_qx = (R)2 * (z[3] - z[1]) + d58 - d68;
  const R m_qy = (R)2 * (z[4] - z[2]) + d58 + d68;
  const R m_xx = (z[1] + z[3]) - (z[2] + z[4]);
  const R m_xy = (z[5] + z[7]) - (z[6] + z[8]);
  const R eq_e = (R)3 * rho * usq + (R)2 * Pp;
  const R eq_ep = -(R)3 * rho * usq - (R)3 * Pp;
  const R eq_jx = rho * hx, eq_jy = rho * hy;
  const R eq_xx = rho * (hx * hx - hy * hy), eq_xy = rho * hx * hy;
  const R ug = ux * gx + uy * gy;
  const R F0 = ug, Fep = -ug;
  const R Fjx = Fx * ic, Fjy = Fy * ic;
  const R Fxx = (R)(2.0 / 3.0) * (ux * gx - uy * gy), Fxy = (R)(1.0 / 3.0) * (ux * gy + uy * gx);
  // multiphase [Lambda]_dim (Sec. 3): 1/dt everywhere except omega_q2 (q_x, and
  // q_y by the isotropic reading) and 1/tau for the stress moments
  // omega_q2 dt = 3 (2 - omega_nu dt) / (3 - omega_nu dt), omega_nu dt = dt / tau (Sec. 3)
  const R snu = m.wb;
  const R sq = qdiv((R)3 * ((R)2 - snu), (R)3 - snu);
  const R sqy = P.qy_literal ? (R)1 : sq;
  const R rdt = K.dt, one = (R)1, half = (R)0.5;
  const R d0 = m0 - half * rdt * F0;                 // s = 1: (m - 0) - (1 - 1/2) dt F
  const R d_e = (m_e - eq_e);                        // F_e = 0
  const R d_ep = (m_ep - eq_ep) - half * rdt * Fep;
  const R d_jx = (m_jx - eq_jx) - half * rdt * Fjx;
  const R d_jy = (m_jy - eq_jy) - half * rdt * Fjy;
  const R d_qx = sq * (m_qx + eq_jx) + (one - half * sq) * rdt * Fjx;   // eq_qx = -rho u_x/c, F_qx = -F_x/c
  const R d_qy = sqy * (m_qy + eq_jy) + (one - half * sqy) * rdt * Fjy;
  const R d_xx = snu * (m_xx - eq_xx) - (one - half * snu) * rdt * Fxx;
  const R d_xy = snu * (m_xy - eq_xy) - (one - half * snu) * rdt * Fxy;
  const R a0 = d0 * ((R)1 / (R)9);
  const R a1 = d_e * ((R)1 / (R)36), a2 = d_ep * ((R)1 / (R)36);
  const R a3 = d_jx * ((R)1 / (R)6), a4 = d_qx * ((R)1 / (R)12);
  const R a5 = d_jy * ((R)1 / (R)6), a6 = d_qy * ((R)1 / (R)12);
  const R a7 = d_xx * (R)0.25, a8 = d_xy * (R)0.25;
  const R ax = a0 - a1 - (R)2 * a2;
  const R dg = a0 + (R)2 * a1 + a2;
  z[0] -= a0 + (R)4 * (a2 - a1);
  z[1] -= ax + a3 - (R)2 * a4 + a7;
  z[2] -= ax + a5 - (R)2 * a6 - a7;
  z[3] -= ax - a3 + (R)2 * a4 + a7;
  z[4] -= ax - a5 + (R)2 * a6 - a7;
  const R p34 = a3 + a4, p56 = a5 + a6;
  z[5] -= dg + p34 + p56 + a8;
  z[6] -= dg - p34 + p56 - a8;
  z[7] -= dg - p34 - p56 + a8;
  z[8] -= dg + p34 - p56 - a8;
}

enum { MODE_STEP = 0, MODE_MOMENTS = 2, MODE_INTEGRALS = 3 };

template <int BY>
__device__ __forceinline__ void reduce4_block(double v[4], double *out) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v[0] += __shfl_down_sync(0xffffffffu, v[0], o);
    v[1] += __shfl_down_sync(0xffffffffu, v[1], o);
    v[2] = fmax(v[2], __shfl_down_sync(0xffffffffu, v[2], o));
    v[3] += __shfl_down_sync(0xffffffffu, v[3], o);
  }
  __shared__ double sh[8][4];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if ((tid & 31) == 0) { sh[tid >> 5][0] = v[0]; sh[tid >> 5][1] = v[1]; sh[tid >> 5][2] = v[2]; sh[tid >> 5][3] = v[3]; }
  __syncthreads();
  if (tid == 0) {
    double a = 0, b = 0, mx = 0, cnt = 0;
    for (int w = 0; w < (BX * BY) / 32; w++) { a += sh[w][0]; b += sh[w][1]; mx = fmax(mx, sh[w][2]); cnt += sh[w][3]; }
    out[0] = a; out[1] = b; out[2] = mx; out[3] = cnt;
  }
}

// Resident 32 x 8 blocks per SM asked of the compiler for the FP32 form: 5 caps it
// at 48 registers (the unbounded build takes 56, i.e. 4 blocks), more warps to cover
// the HBM latency of the pulls.
#ifndef LBM_MP_FP32_BLOCKS_PER_SM
#define LBM_MP_FP32_BLOCKS_PER_SM 5
#endif

// pass 2 (and its init / moments / integrals variants)
template <int PREC, int MODE, int BY>
__global__ void __launch_bounds__(BX * BY, (PREC == 1 && BY == 8) ? LBM_MP_FP32_BLOCKS_PER_SM : 0) k_mp_collide(const MpParams P, const double *A, const double *UX,
                                                         const double *UY, const double *B, unsigned mask,
                                                         double *out) {
  typedef typename Prec<PREC>::S S;
  typedef typename Prec<PREC>::R R;
  __shared__ R tile[BY + 2][BX + 2];
  const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
  const int tid = threadIdx.y * BX + threadIdx.x;
  const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
  const bool live = (i < P.nx) && (j < P.ny);
  const S *src = (const S *)P.src;
  // phi = sum_i h_i (Eq. zero_moment_h) of the tile and of a one-node periodic halo,
  // from pulled h: this node's h stays in registers for its collision
  // a block whose tile, halo and their pull sources stay off the periodic seams
  // (the bulk of the grid) pulls with plain offsets: no wrap, no modulo
  const bool inner = !P.local && i0 >= 2 && j0 >= 2 && i0 + BX + 2 <= P.nx && j0 + BY + 2 <= P.ny;
  R h[5];
  if (inner) {
    pull_h_at<S, R>(P, src + ((long long)j * P.pitch + i), h);
  } else {
    pull_h<S, R>(P, src, stencil_node(i, P.nx, P.xwall), stencil_node(j, P.ny, P.ywall), h);
  }
  // the node's z, (phi u)_prev and force do not depend on the tile: their loads are
  // issued here, so that they are in flight during the halo pulls and the barrier
  const long long n = (long long)j * P.pitch + i;
  R z[9];
  R prevx = 0, prevy = 0, fex = 0, fey = 0;
  if (live) {
    if (P.force) {
      fex = (R)((const S *)P.force)[n];
      fey = (R)((const S *)P.force)[P.plane + n];
    }
    if (inner) pull_z_at<S, R>(P, src + n, z);
    else pull_z<S, R>(P, src, i, j, z);
    if (MODE == MODE_STEP) {
      prevx = (R)src[14ll * P.plane + n];
      prevy = (R)src[15ll * P.plane + n];
    }
  }
  tile[threadIdx.y + 1][threadIdx.x + 1] = (h[0] + h[1]) + (h[2] + h[3]) + h[4];
  constexpr int kHalo = 2 * (BX + 2) + 2 * BY;
  for (int t = tid; t < kHalo; t += BX * BY) {
    int tx, ty;
    if (t < BX + 2) { tx = t; ty = 0; }                            // row below the tile
    else if (t < 2 * (BX + 2)) { tx = t - (BX + 2); ty = BY + 1; }  // row above
    else if (t < 2 * (BX + 2) + BY) { tx = 0; ty = t - 2 * (BX + 2) + 1; }  // left column
    else { tx = BX + 1; ty = t - 2 * (BX + 2) - BY + 1; }           // right column
    R hh[5];
    if (inner) {
      pull_h_at<S, R>(P, src + ((long long)(j0 + ty - 1) * P.pitch + (i0 + tx - 1)), hh);
    } else {
      pull_h<S, R>(P, src, stencil_node(i0 + tx - 1, P.nx, P.xwall), stencil_node(j0 + ty - 1, P.ny, P.ywall), hh);
    }
    tile[ty][tx] = (hh[0] + hh[1]) + (hh[2] + hh[3]) + hh[4];
  }
  __syncthreads();
  double red[4] = {0.0, 0.0, 0.0, 0.0};
  if (live) {
    MpMacro<R> m;
    mp_macro<R>(P, tile, threadIdx.x + 1, threadIdx.y + 1, z, fex, fey, m);
    if (MODE == MODE_STEP) {
      const R pux = m.phi * m.ux, puy = m.phi * m.uy;
      const R dpux = (pux - prevx) * KM<R>(P).inv_dt, dpuy = (puy - prevy) * KM<R>(P).inv_dt;  // explicit Euler d_t(phi u)
      collide_h<R>(P, m, dpux, dpuy, h);
      collide_z<R>(P, m, z);
      S *dst = (S *)P.dst;
#pragma unroll
      for (int q = 0; q < 9; q++) dst[q * P.plane + n] = (S)z[q];
#pragma unroll
      for (int q = 0; q < 5; q++) dst[(9 + q) * P.plane + n] = (S)h[q];
      dst[14ll * P.plane + n] = (S)pux;
      dst[15ll * P.plane + n] = (S)puy;
    } else if (MODE == MODE_MOMENTS) {
      const long long N = (long long)P.nx * P.ny, k = (long long)j * P.nx + i;
      int slot = 0;
      if (mask & 1u) out[(slot++) * N + k] = (double)m.rho;
      if (mask & 2u) out[(slot++) * N + k] = (double)m.ux;
      if (mask & 4u) out[(slot++) * N + k] = (double)m.uy;
      if (mask & 8u) out[(slot++) * N + k] = 0.0;
      if (mask & 16u) out[(slot++) * N + k] = (double)m.p;
      if (mask & 32u) out[(slot++) * N + k] = (double)m.phi;
    } else {
      const double ux = (double)m.ux, uy = (double)m.uy, rho = (double)m.rho, p = (double)m.p;
      const double umag = sqrt(ux * ux + uy * uy);
      const bool bad = !isfinite(rho) || !isfinite(umag) || !isfinite(p) || umag >= P.c;
      // a bad node (non-finite, or |u| >= c) is counted and adds nothing else
      red[0] = bad ? 0.0 : rho * P.dx * P.dx;
      red[1] = bad ? 0.0 : (double)m.phi;
      red[2] = bad ? 0.0 : umag;
      red[3] = bad ? 1.0 : 0.0;
    }
  }
  if (MODE == MODE_INTEGRALS) reduce4_block<BY>(red, out + 4ll * (blockIdx.y * gridDim.x + blockIdx.x));
}

__global__ void k_mp_final(const double *partials, int nb, double *out4) {
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

// Equilibria of the given fields (Eqs. heq_liang, zeq_liang, s_i_Liang) as the
// pre-collision state of time 0; (phi u)_prev = phi0 u0.  Defaults: phi 1, u 0, p 0.
template <typename S>
__global__ void k_mp_init(const MpParams P, const double *A, const double *UX, const double *UY, const double *B) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= P.nx || j >= P.ny) return;
  const long long n = (long long)j * P.pitch + i;
  const int k = j * P.nx + i;
  S *dst = (S *)P.dst;
  const double c = P.c;
  const double ph = A ? A[k] : 1.0, u0 = UX ? UX[k] : 0.0, v0 = UY ? UY[k] : 0.0, p0 = B ? B[k] : 0.0;
  const double rho = P.rho_g + ph * (P.rho_l - P.rho_g);
  const double usq = u0 * u0 + v0 * v0;
#pragma unroll
  for (int q = 0; q < 9; q++) {
    const double cu = c * (cx9(q) * u0 + cy9(q) * v0);
    const double si = w9<double>(q) * (cu / P.cs2 + 0.5 * cu * cu / (P.cs2 * P.cs2) - 0.5 * usq / P.cs2);
    dst[q * P.plane + n] = (S)(p0 / P.cs2 * (w9<double>(q) - (q == 0 ? 1.0 : 0.0)) + rho * si);
  }
#pragma unroll
  for (int q = 0; q < 5; q++)
    dst[(9 + q) * P.plane + n] = (S)(ph * w5<double>(q) * (1.0 + c * (cx5(q) * u0 + cy5(q) * v0) / P.cs2));
  dst[14ll * P.plane + n] = (S)(ph * u0);
  dst[15ll * P.plane + n] = (S)(ph * v0);
}

dim3 mp_grid(int nx, int ny, int by) { return dim3((nx + BX - 1) / BX, (ny + by - 1) / by); }
int mp_rows(int nx, int ny) { return (int)(mp_grid(nx, ny, 8).x * mp_grid(nx, ny, 8).y) >= kSmallGridBlocks ? 8 : 2; }

template <int PREC, int MODE>
void launch_collide(const MpParams &P, unsigned mask, double *out, cudaStream_t s) {
  const int by = mp_rows(P.nx, P.ny);
  const dim3 g = mp_grid(P.nx, P.ny, by);
  if (by == 8) k_mp_collide<PREC, MODE, 8><<<g, dim3(BX, 8), 0, s>>>(P, nullptr, nullptr, nullptr, nullptr, mask, out);
  else k_mp_collide<PREC, MODE, 2><<<g, dim3(BX, 2), 0, s>>>(P, nullptr, nullptr, nullptr, nullptr, mask, out);
}

}  // namespace

int mp_integral_blocks(int nx, int ny) {
  dim3 g = mp_grid(nx, ny, mp_rows(nx, ny));
  return (int)(g.x * g.y);
}

cudaError_t mp_step(const MpParams &P, int prec, cudaStream_t s) {
  if (prec == 0) launch_collide<0, MODE_STEP>(P, 0u, nullptr, s);
  else launch_collide<1, MODE_STEP>(P, 0u, nullptr, s);
  return cudaGetLastError();
}

cudaError_t mp_init(const MpParams &P, int prec, const double *phi0, const double *ux0, const double *uy0,
                    const double *p0, cudaStream_t s) {
  dim3 b(BX, 8), g = mp_grid(P.nx, P.ny, 8);
  if (prec == 0) k_mp_init<double><<<g, b, 0, s>>>(P, phi0, ux0, uy0, p0);
  else k_mp_init<float><<<g, b, 0, s>>>(P, phi0, ux0, uy0, p0);
  return cudaGetLastError();
}

cudaError_t mp_moments(const MpParams &P, int prec, unsigned mask, double *out, cudaStream_t s) {
  if (prec == 0) launch_collide<0, MODE_MOMENTS>(P, mask, out, s);
  else launch_collide<1, MODE_MOMENTS>(P, mask, out, s);
  return cudaGetLastError();
}

cudaError_t mp_integrals(const MpParams &P, int prec, double *partials, int max_blocks, double *out4, cudaStream_t s) {
  const int nb = mp_integral_blocks(P.nx, P.ny);
  if (nb > max_blocks) return cudaErrorInvalidValue;
  if (prec == 0) launch_collide<0, MODE_INTEGRALS>(P, 0u, partials, s);
  else launch_collide<1, MODE_INTEGRALS>(P, 0u, partials, s);
  k_mp_final<<<1, 32, 0, s>>>(partials, nb, out4);
  return cudaGetLastError();
}

}  // namespace lbmk
