// Single-phase device helpers shared by the step kernels (step_sp.cu) and the
// adjoint kernels (adjoint.cu): pull-streaming with the link-wise boundary rules,
// moments and the BGK / MRT collisions, all in deviation form.
#pragma once
#include <cuda_runtime.h>

#include "lattice.cuh"
#include "lbm_internal.cuh"

namespace lbmk {

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_VELOCITY = 2, BC_PRESSURE = 3, BC_SYMMETRY = 4 };
enum { TBC_NONE = 0, TBC_FLUX = 1, TBC_TEMP = 2, TBC_OUTFLOW = 3, TBC_SYMMETRY = 4, TBC_WETNODE = 5 };

__device__ __forceinline__ int wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// Position of node (i, j) along a side, and the side's length.
__device__ __forceinline__ int along(int side, int i, int j) { return side < 2 ? j : i; }
__device__ __forceinline__ int side_len(const SpParams &P, int side) { return side < 2 ? P.ny : P.nx; }

// Node (i, j) lies on side s (0: x = 0, 1: x = nx - 1, 2: y = 0, 3: y = ny - 1).
__device__ __forceinline__ bool on_side(const SpParams &P, int s, int i, int j) {
  return (s == 0 && i == 0) || (s == 1 && i == P.nx - 1) || (s == 2 && j == 0) || (s == 3 && j == P.ny - 1);
}

// Which side the link arriving at (i, j) along c = (cx, cy) comes through (source
// node (i - cx, j - cy) outside the domain), or -1.  A link through a corner takes
// the y-side, unless that y-side is a symmetry side (ysym: bit 0 for y = 0, bit 1
// for y = ny - 1): the mirror image of the link also comes through the x-side, whose
// rule then applies.
__device__ __forceinline__ int entry_side(int i, int j, int cx, int cy, int nx, int ny, int xper, int yper,
                                          int ysym = 0) {
  const int si = i - cx, sj = j - cy;
  const int xs = xper ? -1 : (si < 0 ? 0 : (si >= nx ? 1 : -1));
  if (!yper) {
    if (sj < 0) return (ysym & 1) && xs >= 0 ? xs : 2;
    if (sj >= ny) return (ysym & 2) && xs >= 0 ? xs : 3;
  }
  return xs;
}

// Source of a link entering node (i, j) through symmetry side `side` (Eq. simetria):
// population mirror(q) of the tangential neighbour (i, j) - c_{q,tan} dt, wrapped
// where the tangential axis is periodic, else the node itself where the neighbour
// falls outside.  Returns the element offset of that value.
template <int Q>
__device__ __forceinline__ long long symmetry_source(const SpParams &P, int side, int q, int i, int j, int tper) {
  const int cx = Q == 9 ? cx9(q) : cx5(q), cy = Q == 9 ? cy9(q) : cy5(q);
  int si = i, sj = j, qm;
  if (side >= 2) {
    qm = Q == 9 ? my9(q) : my5(q);
    si = i - cx;
    if (si < 0 || si >= P.nx) si = tper ? wrap(si, P.nx) : i;
  } else {
    qm = Q == 9 ? mx9(q) : mx5(q);
    sj = j - cy;
    if (sj < 0 || sj >= P.ny) sj = tper ? wrap(sj, P.ny) : j;
  }
  return qm * P.plane + (long long)sj * P.pitch + si;
}

// Pre-collision velocity of time t at node n rebuilt from its post-collision
// populations: rho = sum f*, rho u = sum c f* - dt F / 2 (the collision adds dt F
// to the momentum, Eqs. first_moment_f and forcing_term).
template <typename S, typename R>
__device__ __forceinline__ void post_velocity(const SpParams &P, const S *src, int i, int j, R &ux, R &uy) {
  long long n = (long long)j * P.pitch + i;
  R f[9];
#pragma unroll
  for (int q = 0; q < 9; q++) f[q] = (R)src[q * P.plane + n];
  R drho = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
  R rho = K<R>(P).rho0 + drho;
  R c = K<R>(P).c;
  R jx = c * ((f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]));
  R jy = c * ((f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]));
  R Fx = K<R>(P).Fx, Fy = K<R>(P).Fy;
  if (P.force) {
    const S *fo = (const S *)P.force;
    Fx += (R)fo[n];
    Fy += (R)fo[P.plane + n];
  }
  if (P.buoy) {
    // buoyancy of T(t) = T0 + sum g* - dt qdot / 2 at this node
    const S *gs = src + (long long)P.gbase * P.plane;
    R sg = (R)0;
#pragma unroll
    for (int q = 0; q < 9; q++)
      if (q < P.qg) sg += (R)gs[q * P.plane + n];
    const R qd = P.qdot ? (R)((const S *)P.qdot)[n] : (R)0;
    const R dT = (K<R>(P).T0 - K<R>(P).T_ref) + sg - (R)0.5 * K<R>(P).dt * qd;
    Fx += K<R>(P).bgx * dT;
    Fy += K<R>(P).bgy * dT;
  }
  ux = (jx - (R)0.5 * K<R>(P).dt * Fx) / rho;
  uy = (jy - (R)0.5 * K<R>(P).dt * Fy) / rho;
}

// Pull of all momentum populations at node (i, j), with boundary links.  SYM: the
// solve has symmetry sides (compiled separately, so that solves without them run the
// shorter boundary code).
template <typename S, typename R, bool SYM = false>
__device__ __forceinline__ void pull_f(const SpParams &P, const S *src, int i, int j, bool interior, R f[9]) {
  const long long n = (long long)j * P.pitch + i;
  if (interior) {
#pragma unroll
    for (int q = 0; q < 9; q++) f[q] = (R)src[q * P.plane + n - (long long)cy9(q) * P.pitch - cx9(q)];
    return;
  }
  if (P.local) {  // src holds f(t) itself (first step after initialisation)
#pragma unroll
    for (int q = 0; q < 9; q++) f[q] = (R)src[q * P.plane + n];
    return;
  }
  const R c = K<R>(P).c, inv_cs2 = K<R>(P).inv_cs2;
  // 1. gather, branch-free so that all nine loads are in flight together: the
  //    streaming source (periodic wrap included), or for a link entering through a
  //    side the outgoing population o = opp(q) of this node
  //    (a symmetry side gives the mirrored population of the tangential neighbour)
  int side[9];
  bool sym[9];
  R raw[9];
#pragma unroll
  for (int q = 0; q < 9; q++) {
    side[q] = entry_side(i, j, cx9(q), cy9(q), P.nx, P.ny, P.xper, P.yper, SYM ? P.fysym : 0);
    sym[q] = false;
    if (SYM) {
#pragma unroll
      for (int s = 0; s < 4; s++)
        if (side[q] == s) sym[q] = P.side[s].kind == BC_SYMMETRY;
    }
    long long at = side[q] < 0 ? q * P.plane + (long long)wrap(j - cy9(q), P.ny) * P.pitch + wrap(i - cx9(q), P.nx)
                               : opp9(q) * P.plane + n;
    if (sym[q]) at = symmetry_source<9>(P, side[q], q, i, j, side[q] >= 2 ? P.xper : P.yper);
    raw[q] = (R)src[at];
  }
  // 2. wall / inlet velocities of the sides this node lies on, loaded up front
  R uws[4][2];
#pragma unroll
  for (int s = 0; s < 4; s++) {
    const double *uw = P.side[s].uw;
    const bool ld = on_side(P, s, i, j) && uw != nullptr;
    const int a = along(s, i, j), len = side_len(P, s);
    uws[s][0] = ld ? (R)uw[a] : (R)0;
    uws[s][1] = ld ? (R)uw[len + a] : (R)0;
  }
  // 3. outlet velocity extrapolation, Eq. anti_BB_vel and the rule below it (reading:
  //    pre-collision velocities of time t at the boundary node and its inner neighbour)
  R uwp[4][2];
#pragma unroll
  for (int s = 0; s < 4; s++) { uwp[s][0] = 0; uwp[s][1] = 0; }
#pragma unroll
  for (int s = 0; s < 4; s++) {
    if (on_side(P, s, i, j) && P.side[s].kind == BC_PRESSURE) {
      int ii = i + (s == 0) - (s == 1), jj = j + (s == 2) - (s == 3);
      R ub, vb, ui, vi;
      post_velocity<S, R>(P, src, i, j, ub, vb);
      post_velocity<S, R>(P, src, ii, jj, ui, vi);
      uwp[s][0] = ub + (R)0.5 * (ub - ui);
      uwp[s][1] = vb + (R)0.5 * (vb - vi);
    }
  }
  // 4. boundary links (side values picked with compile-time side indices)
#pragma unroll
  for (int q = 0; q < 9; q++) {
    if (side[q] < 0 || sym[q]) {
      f[q] = raw[q];
      continue;
    }
    const int o = opp9(q);
    const R fo = raw[q];
    int kind = BC_WALL;
    R rw = 0, ux = 0, uy = 0;
#pragma unroll
    for (int s = 0; s < 4; s++) {
      if (side[q] == s) {
        kind = P.side[s].kind;
        rw = K<R>(P).rho_w[s];
        ux = kind == BC_PRESSURE ? uwp[s][0] : uws[s][0];
        uy = kind == BC_PRESSURE ? uwp[s][1] : uws[s][1];
      }
    }
    const R cox = c * (R)cx9(o), coy = c * (R)cy9(o);
    if (kind == BC_PRESSURE) {
      // Eq. anti_BB_vel in deviation form: f_q - w rho0 = -(f_o* - w rho0) + 2 w [rho_w(...) - rho0]
      R cu = cox * ux + coy * uy;
      R uu = ux * ux + uy * uy;
      f[q] = -fo + (R)2 * w9<R>(o) * (rw * ((R)1 + (R)0.5 * cu * cu * inv_cs2 * inv_cs2 - (R)0.5 * uu * inv_cs2) - K<R>(P).rho0);
    } else {
      // Eq. BB_vel (walls and velocity inlet): f_q = f_o* - 2 w_o rho_w c_o.u_w / c_s^2
      f[q] = fo - (R)2 * w9<R>(o) * rw * (cox * ux + coy * uy) * inv_cs2;
    }
  }
}

// Pull of the thermal populations (QT = 5: D2Q5, 9: D2Q9) at node (i, j) with
// boundary links.
template <typename S, typename R, int QT = 5, bool SYM = false>
__device__ __forceinline__ void pull_g(const SpParams &P, const S *src, int i, int j, bool interior, R g[QT]) {
  const long long n = (long long)j * P.pitch + i;
  const S *gsrc = src + (long long)P.gbase * P.plane;
  if (interior) {
#pragma unroll
    for (int q = 0; q < QT; q++) g[q] = (R)gsrc[q * P.plane + n - (long long)cyT(QT, q) * P.pitch - cxT(QT, q)];
    return;
  }
  if (P.local) {
#pragma unroll
    for (int q = 0; q < QT; q++) g[q] = (R)gsrc[q * P.plane + n];
    return;
  }
  const R c = K<R>(P).c, inv_cs2 = K<R>(P).inv_cs2;
  // 1. gather (branch-free, all loads in flight together)
  int side[QT], tk[QT];
  R raw[QT];
#pragma unroll
  for (int q = 0; q < QT; q++) {
    side[q] = entry_side(i, j, cxT(QT, q), cyT(QT, q), P.nx, P.ny, P.txper, P.typer, SYM ? P.tysym : 0);
    tk[q] = TBC_NONE;
#pragma unroll
    for (int s = 0; s < 4; s++)
      if (side[q] == s) tk[q] = P.side[s].tkind;
    long long at;
    if (side[q] < 0) {
      at = q * P.plane + (long long)wrap(j - cyT(QT, q), P.ny) * P.pitch + wrap(i - cxT(QT, q), P.nx);
    } else if (SYM && tk[q] == TBC_SYMMETRY) {
      at = symmetry_source<QT>(P, side[q], q, i, j, side[q] >= 2 ? P.txper : P.typer);
    } else if (tk[q] == TBC_OUTFLOW) {
      // g_q(x_b, t+dt) = g_q(x_b-1, t+dt): the inner node's pull of q (Sec. 2.2, outlet);
      // where that pull itself crosses a symmetry side (the outlet's corner with a
      // symmetry plane) it is that side's mirrored value
      const int ii = i + (side[q] == 0) - (side[q] == 1), jj = j + (side[q] == 2) - (side[q] == 3);
      const int si = ii - cxT(QT, q), sj = jj - cyT(QT, q);
      at = q * P.plane + (long long)min(max(sj, 0), P.ny - 1) * P.pitch + min(max(si, 0), P.nx - 1);
      if (SYM) {
        const int cs = entry_side(ii, jj, cxT(QT, q), cyT(QT, q), P.nx, P.ny, P.txper, P.typer, P.tysym);
        bool csym = false;
#pragma unroll
        for (int s = 0; s < 4; s++)
          if (cs == s) csym = P.side[s].tkind == TBC_SYMMETRY;
        if (csym) at = symmetry_source<QT>(P, cs, q, ii, jj, cs >= 2 ? P.txper : P.typer);
      }
    } else {
      at = oppT(QT, q) * P.plane + n;
    }
    raw[q] = (R)gsrc[at];
  }
  // 2. wall temperatures / fluxes and velocities of the sides this node lies on
  R tws[4], uws[4][2];
#pragma unroll
  for (int s = 0; s < 4; s++) {
    const bool on = on_side(P, s, i, j);
    const double *tw = P.side[s].tw, *uw = P.side[s].uw;
    const int a = along(s, i, j), len = side_len(P, s);
    tws[s] = (on && tw) ? (R)tw[a] : (R)0;
    uws[s][0] = (on && uw) ? (R)uw[a] : (R)0;
    uws[s][1] = (on && uw) ? (R)uw[len + a] : (R)0;
  }
  // 3. boundary links
#pragma unroll
  for (int q = 0; q < QT; q++) {
    if (side[q] < 0 || tk[q] == TBC_OUTFLOW || (SYM && (tk[q] == TBC_SYMMETRY || tk[q] == TBC_WETNODE))) {
      g[q] = raw[q];
      continue;
    }
    const int o = oppT(QT, q);
    const R go = raw[q];
    R Tw = 0, ux = 0, uy = 0;
#pragma unroll
    for (int s = 0; s < 4; s++) {
      if (side[q] == s) {
        Tw = tws[s];
        ux = uws[s][0];
        uy = uws[s][1];
      }
    }
    if (tk[q] == TBC_TEMP) {
      // Eq. anti_BB_T in deviation form
      R cu = c * ((R)cxT(QT, o) * ux + (R)cyT(QT, o) * uy);
      R uu = ux * ux + uy * uy;
      g[q] = -go + (R)2 * wT<R>(QT, o) * (Tw * ((R)1 + (R)0.5 * cu * cu * inv_cs2 * inv_cs2 - (R)0.5 * uu * inv_cs2) - K<R>(P).T0);
    } else if (QT == 9) {
      // Eq. BB_T with lambda_o = 6 w_o on D2Q9 (4/6 axial, 1/6 diagonal; FLUX, zero flux = adiabatic)
      g[q] = go + (R)6 * w9<R>(o) * K<R>(P).flux_coef * Tw;
    } else {
      // Eq. BB_T with lambda = 1 for the single D2Q5 unknown (FLUX; zero flux = adiabatic)
      g[q] = go + K<R>(P).flux_coef * Tw;
    }
  }
  // 4. wet-node x-sides (App. B, Eq. BCs_1D_advection_diffusion): the boundary node lies
  //    on the boundary; its single D2Q5 unknown closes T of Eq. zero_moment_g at T_w,
  //    g_unknown = T_w - dt qdot/2 - (sum of the others), in deviation form
  if (SYM && QT == 5) {
#pragma unroll
    for (int s = 0; s < 2; s++) {
      if (P.side[s].tkind != TBC_WETNODE || i != (s == 0 ? 0 : P.nx - 1)) continue;
      const int qu = s == 0 ? 1 : 3;
      R others = (R)0;
#pragma unroll
      for (int k = 0; k < QT; k++)
        if (k != qu) others += g[k];
      const R qd = P.qdot ? (R)((const S *)P.qdot)[n] : (R)0;
      g[qu] = (tws[s] - K<R>(P).T0) - (R)0.5 * K<R>(P).dt * qd - others;
    }
  }
}

// ----------------------------------------------------------------------------
// Moments and collisions (deviation form)
// ----------------------------------------------------------------------------
template <typename R>
struct Macro {
  R drho, rho, ux, uy, Fx, Fy;  // momentum
  R sumg, qd, T;                // thermal
};

template <typename S, typename R>
__device__ __forceinline__ void load_sources(const SpParams &P, long long n, Macro<R> &m) {
  m.Fx = K<R>(P).Fx;
  m.Fy = K<R>(P).Fy;
  if (P.force) {
    const S *fo = (const S *)P.force;
    m.Fx += (R)fo[n];
    m.Fy += (R)fo[P.plane + n];
  }
  m.qd = P.qdot ? (R)((const S *)P.qdot)[n] : (R)0;
}

template <typename R, int FLOW, int TH>
__device__ __forceinline__ void moments(const SpParams &P, const R f[9], const R *g, Macro<R> &m) {
  if (TH != TH_NONE) {
    // Eq. zero_moment_g
    if (ThLat<TH>::Q == 9) m.sumg = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    else m.sumg = (g[0] + g[1]) + (g[2] + g[3]) + g[4];
    m.T = K<R>(P).T0 + m.sumg + K<R>(P).hdt * m.qd;
    if (FLOW != FLOW_NONE && P.buoy) {
      // Boussinesq buoyancy with this step's temperature (Eq. buoyancy_force)
      const R dT = (K<R>(P).T0 - K<R>(P).T_ref) + m.sumg + K<R>(P).hdt * m.qd;
      m.Fx += K<R>(P).bgx * dT;
      m.Fy += K<R>(P).bgy * dT;
    }
  }
  if (FLOW != FLOW_NONE) {
    // Eqs. zero_moment_f and first_moment_f
    m.drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    m.rho = K<R>(P).rho0 + m.drho;
    const R c = K<R>(P).c, hdt = K<R>(P).hdt;
    const R jx = c * ((f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]));
    const R jy = c * ((f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]));
    const R inv = (R)1 / m.rho;
    m.ux = (jx + hdt * m.Fx) * inv;
    m.uy = (jy + hdt * m.Fy) * inv;
  } else {
    m.drho = 0;
    m.rho = K<R>(P).rho0;
    m.ux = K<R>(P).ux_pres;
    m.uy = K<R>(P).uy_pres;
  }
}

template <typename R>
__device__ __forceinline__ void collide_bgk9(const SpParams &P, const Macro<R> &m, R f[9]) {
  const R c = K<R>(P).c, inv_cs2 = K<R>(P).three_inv_c2, inv_cs4 = inv_cs2 * inv_cs2;
  const R om = K<R>(P).omega;
  const R fac = ((R)1 - (R)0.5 * om) * K<R>(P).dt;  // (1 - dt/(2 tau)) dt
  const R hu = (R)0.5 * (m.ux * m.ux + m.uy * m.uy) * inv_cs2;  // u^2 / (2 c_s^2)
  const R uF = m.ux * m.Fx + m.uy * m.Fy;
  // q >= 1 first; the rest population takes the remainders so that sum f_eq = rho
  // and sum F_hat = 0 hold exactly in the working precision (the rounded weights
  // do not sum to one in FP32)
  R feq_sum = 0, fh_sum = 0;
#pragma unroll
  for (int q = 1; q < 9; q++) {
    const R cxq = c * (R)cx9(q), cyq = c * (R)cy9(q);
    const R cu = cxq * m.ux + cyq * m.uy;
    // f_eq - w rho0 (Eq. feq_geral, deviation form: no O(rho0) cancellation)
    const R feq = w9<R>(q) * (m.drho + m.rho * (cu * inv_cs2 * ((R)1 + (R)0.5 * cu * inv_cs2) - hu));
    // Guo forcing F_hat (Eq. forcing_term)
    const R cF = cxq * m.Fx + cyq * m.Fy;
    const R Fh = w9<R>(q) * ((cF - uF) * inv_cs2 + cu * cF * inv_cs4);
    feq_sum += feq;
    fh_sum += Fh;
    f[q] = f[q] - om * (f[q] - feq) + fac * Fh;
  }
  f[0] = f[0] - om * (f[0] - (m.drho - feq_sum)) + fac * (-fh_sum);
}

template <typename R>
__device__ __forceinline__ void collide_mrt9(const SpParams &P, const Macro<R> &m, R f[9]) {
  const R c = K<R>(P).c, ic = K<R>(P).inv_c;
  const R dt = K<R>(P).dt;
  // lattice-scaled moments of the deviations (rows of Eq. M_matrix)
  const R s14 = (f[1] + f[2]) + (f[3] + f[4]);
  const R s58 = (f[5] + f[6]) + (f[7] + f[8]);
  const R m_e = -(R)4 * f[0] - s14 + (R)2 * s58;
  const R m_ep = (R)4 * f[0] - (R)2 * s14 + s58;
  const R d58 = (f[5] - f[7]), d68 = (f[6] - f[8]);
  const R m_qx = (R)2 * (f[3] - f[1]) + d58 - d68;
  const R m_qy = (R)2 * (f[4] - f[2]) + d58 + d68;
  const R m_xx = (f[1] + f[3]) - (f[2] + f[4]);
  const R m_xy = (f[5] + f[7]) - (f[6] + f[8]);
  // equilibrium and forcing moments divided by c^n (Eq. M_matrix_dim row orders)
  const R ux = m.ux * ic, uy = m.uy * ic, usq = ux * ux + uy * uy;
  const R Fx = m.Fx * ic, Fy = m.Fy * ic, uF = ux * Fx + uy * Fy;
  const R eq_e = -(R)2 * m.drho + (R)3 * m.rho * usq;
  const R eq_ep = m.drho - (R)3 * m.rho * usq;
  const R eq_qx = -m.rho * ux, eq_qy = -m.rho * uy;
  const R eq_xx = m.rho * (ux * ux - uy * uy), eq_xy = m.rho * ux * uy;
  const R s_e = K<R>(P).s_e, s_ep = K<R>(P).s_eps, s_q = K<R>(P).s_q, s_nu = K<R>(P).s_nu;
  // Delta m_k = dt Lambda_k (m_k - m_k^eq) - dt (1 - dt Lambda_k / 2) F_k  (Eq. colisao_MRT)
  // (the factors (1 - dt Lambda_k / 2) dt come from the host-filled constants)
  const R d_e = s_e * (m_e - eq_e) - K<R>(P).fk_e * ((R)6 * uF);
  const R d_ep = s_ep * (m_ep - eq_ep) + K<R>(P).fk_eps * ((R)6 * uF);
  const R d_jx = -dt * Fx, d_jy = -dt * Fy;
  const R d_qx = s_q * (m_qx - eq_qx) + K<R>(P).fk_q * Fx;
  const R d_qy = s_q * (m_qy - eq_qy) + K<R>(P).fk_q * Fy;
  const R d_xx = s_nu * (m_xx - eq_xx) - K<R>(P).fk_nu * ((R)2 * (ux * Fx - uy * Fy));
  const R d_xy = s_nu * (m_xy - eq_xy) - K<R>(P).fk_nu * (ux * Fy + uy * Fx);
  // back to populations: M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
  const R a1 = d_e * ((R)1 / (R)36), a2 = d_ep * ((R)1 / (R)36);
  const R a3 = d_jx * ((R)1 / (R)6), a4 = d_qx * ((R)1 / (R)12);
  const R a5 = d_jy * ((R)1 / (R)6), a6 = d_qy * ((R)1 / (R)12);
  const R a7 = d_xx * (R)0.25, a8 = d_xy * (R)0.25;
  const R ax = -a1 - (R)2 * a2;   // common to i = 1..4
  const R dg = (R)2 * a1 + a2;    // common to i = 5..8
  f[0] -= (R)4 * (a2 - a1);
  f[1] -= ax + a3 - (R)2 * a4 + a7;
  f[2] -= ax + a5 - (R)2 * a6 - a7;
  f[3] -= ax - a3 + (R)2 * a4 + a7;
  f[4] -= ax - a5 + (R)2 * a6 - a7;
  const R p34 = a3 + a4, p56 = a5 + a6;
  f[5] -= dg + p34 + p56 + a8;
  f[6] -= dg - p34 + p56 - a8;
  f[7] -= dg - p34 - p56 + a8;
  f[8] -= dg + p34 - p56 - a8;
}

// Thermal BGK with source (Eqs. eq_lattice_boltzmann_BGK_T, forcing_term_g,
// geq_geral) on the thermal lattice QT.
template <typename R, int QT = 5>
__device__ __forceinline__ void collide_bgk5(const SpParams &P, const Macro<R> &m, R *g) {
  const R c = K<R>(P).c, inv_cs2 = K<R>(P).three_inv_c2;
  const R om = K<R>(P).omegaT;
  const R src = K<R>(P).tsrc_fac * K<R>(P).dt * m.qd;
  const R dT = m.T - K<R>(P).T0;
  R geq_sum = 0, s_sum = 0;
#pragma unroll
  for (int q = 1; q < QT; q++) {
    const R cu = c * ((R)cxT(QT, q) * m.ux + (R)cyT(QT, q) * m.uy);
    const R geq = wT<R>(QT, q) * (dT + m.T * cu * inv_cs2);  // Eq. geq_geral minus w T0
    const R sq = wT<R>(QT, q) * src;                         // Eq. forcing_term_g
    geq_sum += geq;
    s_sum += sq;
    g[q] = g[q] - om * (g[q] - geq) + sq;
  }
  // rest population from the remainders: sum g_eq = T - T0, sum S = source, exactly
  g[0] = g[0] - om * (g[0] - (dT - geq_sum)) + (src - s_sum);
}

// Thermal MRT on D2Q9 (Sec. 2.2): the momentum transformation matrices and
// [Lambda_T] = diag(0, 1, 1, omega_T, 1, omega_T, 1, 1, 1), the unit rates read as
// 1/dt; source Delta t (I - dt Lambda/2) M (w qdot).  Lattice-scaled moments of the
// deviations g - w T0; equilibrium moments of g_eq - w T0 from Eq. geq_geral:
// (T - T0, -2 (T - T0), T - T0, T u_x/c, -T u_x/c, T u_y/c, -T u_y/c, 0, 0).
template <typename R>
__device__ __forceinline__ void collide_mrt9T(const SpParams &P, const Macro<R> &m, R g[9]) {
  const R ic = K<R>(P).inv_c, dt = K<R>(P).dt;
  const R dT = m.T - K<R>(P).T0;
  const R sT = K<R>(P).omegaT;  // dt / tau_T
  const R qd = m.qd;
  const R s14 = (g[1] + g[2]) + (g[3] + g[4]);
  const R s58 = (g[5] + g[6]) + (g[7] + g[8]);
  const R m_e = -(R)4 * g[0] - s14 + (R)2 * s58;
  const R m_ep = (R)4 * g[0] - (R)2 * s14 + s58;
  const R d58 = g[5] - g[7], d68 = g[6] - g[8];
  const R m_jx = (g[1] - g[3]) + d58 - d68;
  const R m_jy = (g[2] - g[4]) + d58 + d68;
  const R m_qx = (R)2 * (g[3] - g[1]) + d58 - d68;
  const R m_qy = (R)2 * (g[4] - g[2]) + d58 + d68;
  const R m_xx = (g[1] + g[3]) - (g[2] + g[4]);
  const R m_xy = (g[5] + g[7]) - (g[6] + g[8]);
  const R Tux = m.T * m.ux * ic, Tuy = m.T * m.uy * ic;
  // Delta m_k = dt Lambda_k (m_k - m_k^eq) - dt (1 - dt Lambda_k / 2) S_k, S = qdot (1, -2, 1, 0, ...)
  const R d0 = -dt * qd;                                       // Lambda_0 = 0
  const R d_e = (m_e + (R)2 * dT) + dt * qd;                   // rate 1/dt: -(dt/2)(-2 qdot)
  const R d_ep = (m_ep - dT) - (R)0.5 * dt * qd;
  const R d_jx = sT * (m_jx - Tux), d_jy = sT * (m_jy - Tuy);  // rate omega_T
  const R d_qx = m_qx + Tux, d_qy = m_qy + Tuy;                // rate 1/dt, eq -T u/c
  const R d_xx = m_xx, d_xy = m_xy;                            // rate 1/dt, eq 0
  // back to populations: M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
  const R a0 = d0 * ((R)1 / (R)9);
  const R a1 = d_e * ((R)1 / (R)36), a2 = d_ep * ((R)1 / (R)36);
  const R a3 = d_jx * ((R)1 / (R)6), a4 = d_qx * ((R)1 / (R)12);
  const R a5 = d_jy * ((R)1 / (R)6), a6 = d_qy * ((R)1 / (R)12);
  const R a7 = d_xx * (R)0.25, a8 = d_xy * (R)0.25;
  const R ax = a0 - a1 - (R)2 * a2;  // common to i = 1..4
  const R dg = a0 + (R)2 * a1 + a2;  // common to i = 5..8
  g[0] -= a0 + (R)4 * (a2 - a1);
  g[1] -= ax + a3 - (R)2 * a4 + a7;
  g[2] -= ax + a5 - (R)2 * a6 - a7;
  g[3] -= ax - a3 + (R)2 * a4 + a7;
  g[4] -= ax - a5 + (R)2 * a6 - a7;
  const R p34 = a3 + a4, p56 = a5 + a6;
  g[5] -= dg + p34 + p56 + a8;
  g[6] -= dg - p34 + p56 - a8;
  g[7] -= dg - p34 - p56 + a8;
  g[8] -= dg + p34 - p56 - a8;
}

template <typename R>
__device__ __forceinline__ void collide_mrt5(const SpParams &P, const Macro<R> &m, R g[5]) {
  // D2Q5 moments (1, c_x, c_y, 5|c|^2 - 4c^2, c_x^2 - c_y^2) scaled by c^-n; rates
  // (0, 1/tau_T, 1/tau_T, 1/dt, 1/dt); source Delta t (I - dt Lambda/2) M (w qdot).
  const R ic = K<R>(P).inv_c, dt = K<R>(P).dt;
  const R dT = m.T - K<R>(P).T0;
  const R m1 = g[1] - g[3], m2 = g[2] - g[4];
  const R m3 = -(R)4 * g[0] + ((g[1] + g[2]) + (g[3] + g[4]));
  const R m4 = (g[1] + g[3]) - (g[2] + g[4]);
  const R sT = K<R>(P).omegaT;
  const R d0 = -dt * m.qd;
  const R d1 = sT * (m1 - m.T * m.ux * ic);
  const R d2 = sT * (m2 - m.T * m.uy * ic);
  // e-moment: rate 1/dt, equilibrium -(2/3) dT, source -(2/3) qdot with factor 1/2
  const R d3 = (m3 + (R)(2.0 / 3.0) * dT) - K<R>(P).hdt * (-(R)(2.0 / 3.0) * m.qd);
  const R d4 = m4;
  const R a0 = d0 * (R)0.2, a1 = d1 * (R)0.5, a2 = d2 * (R)0.5, a3 = d3 * (R)0.05, a4 = d4 * (R)0.25;
  g[0] -= a0 - (R)4 * a3;
  g[1] -= a0 + a1 + a3 + a4;
  g[2] -= a0 + a2 + a3 - a4;
  g[3] -= a0 - a1 + a3 + a4;
  g[4] -= a0 - a2 + a3 - a4;
}

template <typename R, int FLOW, int TH>
__device__ __forceinline__ void collide(const SpParams &P, const Macro<R> &m, R f[9], R *g) {
  if (FLOW == FLOW_BGK) collide_bgk9<R>(P, m, f);
  if (FLOW == FLOW_MRT) collide_mrt9<R>(P, m, f);
  if (TH == TH_BGK) collide_bgk5<R, 5>(P, m, g);
  if (TH == TH_MRT) collide_mrt5<R>(P, m, g);
  if (TH == TH_BGK9) collide_bgk5<R, 9>(P, m, g);
  if (TH == TH_MRT9) collide_mrt9T<R>(P, m, g);
}

// Dispatch of a launcher body over the supported (precision, momentum operator,
// thermal operator) combinations; CALL(PREC, FLOW, TH) names one instantiation.
#define LBM_SP_DISPATCH(PREC_, FLOW_, TH_, CALL)                                      \
  do {                                                                                \
    if (PREC_ == 0) {                                                                 \
      if (FLOW_ == FLOW_BGK && TH_ == TH_NONE) { CALL(0, FLOW_BGK, TH_NONE); }        \
      else if (FLOW_ == FLOW_BGK && TH_ == TH_BGK) { CALL(0, FLOW_BGK, TH_BGK); }     \
      else if (FLOW_ == FLOW_BGK && TH_ == TH_MRT) { CALL(0, FLOW_BGK, TH_MRT); }     \
      else if (FLOW_ == FLOW_MRT && TH_ == TH_NONE) { CALL(0, FLOW_MRT, TH_NONE); }   \
      else if (FLOW_ == FLOW_MRT && TH_ == TH_BGK) { CALL(0, FLOW_MRT, TH_BGK); }     \
      else if (FLOW_ == FLOW_MRT && TH_ == TH_MRT) { CALL(0, FLOW_MRT, TH_MRT); }     \
      else if (FLOW_ == FLOW_NONE && TH_ == TH_BGK) { CALL(0, FLOW_NONE, TH_BGK); }   \
      else if (FLOW_ == FLOW_NONE && TH_ == TH_MRT) { CALL(0, FLOW_NONE, TH_MRT); }   \
      else if (FLOW_ == FLOW_BGK && TH_ == TH_BGK9) { CALL(0, FLOW_BGK, TH_BGK9); }   \
      else if (FLOW_ == FLOW_BGK && TH_ == TH_MRT9) { CALL(0, FLOW_BGK, TH_MRT9); }   \
      else if (FLOW_ == FLOW_MRT && TH_ == TH_BGK9) { CALL(0, FLOW_MRT, TH_BGK9); }   \
      else if (FLOW_ == FLOW_MRT && TH_ == TH_MRT9) { CALL(0, FLOW_MRT, TH_MRT9); }   \
      else return cudaErrorInvalidValue;                                              \
    } else {                                                                          \
      if (FLOW_ == FLOW_BGK && TH_ == TH_NONE) { CALL(1, FLOW_BGK, TH_NONE); }        \
      else if (FLOW_ == FLOW_BGK && TH_ == TH_BGK) { CALL(1, FLOW_BGK, TH_BGK); }     \
      else if (FLOW_ == FLOW_BGK && TH_ == TH_MRT) { CALL(1, FLOW_BGK, TH_MRT); }     \
      else if (FLOW_ == FLOW_MRT && TH_ == TH_NONE) { CALL(1, FLOW_MRT, TH_NONE); }   \
      else if (FLOW_ == FLOW_MRT && TH_ == TH_BGK) { CALL(1, FLOW_MRT, TH_BGK); }     \
      else if (FLOW_ == FLOW_MRT && TH_ == TH_MRT) { CALL(1, FLOW_MRT, TH_MRT); }     \
      else if (FLOW_ == FLOW_NONE && TH_ == TH_BGK) { CALL(1, FLOW_NONE, TH_BGK); }   \
      else if (FLOW_ == FLOW_NONE && TH_ == TH_MRT) { CALL(1, FLOW_NONE, TH_MRT); }   \
      else if (FLOW_ == FLOW_BGK && TH_ == TH_BGK9) { CALL(1, FLOW_BGK, TH_BGK9); }   \
      else if (FLOW_ == FLOW_BGK && TH_ == TH_MRT9) { CALL(1, FLOW_BGK, TH_MRT9); }   \
      else if (FLOW_ == FLOW_MRT && TH_ == TH_BGK9) { CALL(1, FLOW_MRT, TH_BGK9); }   \
      else if (FLOW_ == FLOW_MRT && TH_ == TH_MRT9) { CALL(1, FLOW_MRT, TH_MRT9); }   \
      else return cudaErrorInvalidValue;                                              \
    }                                                                                 \
  } while (0)

}  // namespace lbmk
