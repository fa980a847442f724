// Reverse-time (discrete) adjoint of the single-phase fused step: D2Q9 MRT
// momentum + D2Q5 MRT thermal, FP64 or FP32 (the adjoint of the FP32 deviation
// form: states stored as FP32 deviations, adjoint variables and arithmetic in FP32,
// parameter gradients accumulated to FP64 precision: FP64 sums, or in the FP32 form
// compensated FP32 pairs), with the channel boundary rules
// (BB-velocity inlet and walls, anti-BB pressure outlet with extrapolated
// velocity, anti-BB temperature inlet, heat-flux walls, thermal outflow).
//
// Forward (step_sp.cu): X_t = C(P(X_{t-1})), where P is the pull with boundary
// links and C the local collision; X_{-1} is the pre-collision initial state.
// Loss: L = (1/ny) sum_j (T(nx-1, j; N) - T_target(j))^2 with T of P(X_{N-1}).
// Reverse step t (N-1 >= t >= 0), one launch per node grid:
//   Lam_X(t)   = P^T Lam_pre(t+1)       gather from the consumers of X_t: the
//                                        streaming neighbour, the node's own
//                                        reflected links, the thermal outflow,
//                                        and the outlet velocity extrapolation;
//   Lam_pre(t) = C'(pre(t))^T Lam_X(t)   local transposed Jacobian of the MRT
//                                        collisions (moments, equilibria,
//                                        forcing, u = j/rho, T = sum g + dt qdot/2),
// with pre(t) recomputed by pulling X_{t-1}.  Parameter gradients accumulate per
// node (qdot, wall flux) or per block (the two nu-dependent MRT rates), so the
// result does not depend on scheduling.
#include <cuda_runtime.h>

#include "lattice.cuh"
#include "lbm_internal.cuh"
#include "sp_device.cuh"
#include "compensated.cuh"

namespace lbmk {

namespace {

__device__ __forceinline__ long long nidx(const SpParams &P, int i, int j) { return (long long)j * P.pitch + i; }

// The link arriving at node (i, j) along q is an ordinary streaming link (its
// source is inside the domain or wraps periodically).
__device__ __forceinline__ bool streams_in(const SpParams &P, int i, int j, int cx, int cy, int xper, int yper) {
  return entry_side(i, j, cx, cy, P.nx, P.ny, xper, yper) < 0;
}

// d(pre_p)/d(u_w) of the anti-BB outlet rule for outgoing direction o.
template <typename R>
__device__ __forceinline__ void dpre_duw(const SpParams &P, int o, R rw, R uwx, R uwy, R &gx, R &gy) {
  const R c = K<R>(P).c, ics2 = K<R>(P).inv_cs2;
  const R cx = c * (R)cx9(o), cy = c * (R)cy9(o);
  const R cu = cx * uwx + cy * uwy;
  const R k = (R)2 * w9<R>(o) * rw;
  gx = k * (cu * cx * ics2 * ics2 - uwx * ics2);
  gy = k * (cu * cy * ics2 * ics2 - uwy * ics2);
}

// G = sum over the outlet's unknown populations p of Lam_pre_p * d(pre_p)/d(u_w) at
// boundary node (bi, bj) of pressure side s; also returns u_w inputs.
template <typename S, typename R>
__device__ void outlet_G(const SpParams &P, const S *Xt, const R *LPn, int s, int bi, int bj, R &Gx, R &Gy) {
  const int ii = bi + (s == 0) - (s == 1), jj = bj + (s == 2) - (s == 3);
  R ub, vb, ui, vi;
  post_velocity<S, R>(P, Xt, bi, bj, ub, vb);
  post_velocity<S, R>(P, Xt, ii, jj, ui, vi);
  const R uwx = ub + (R)0.5 * (ub - ui), uwy = vb + (R)0.5 * (vb - vi);
  Gx = 0;
  Gy = 0;
  const long long nb = nidx(P, bi, bj);
#pragma unroll
  for (int p = 0; p < 9; p++) {
    if (entry_side(bi, bj, cx9(p), cy9(p), P.nx, P.ny, P.xper, P.yper) != s) continue;
    R gx, gy;
    dpre_duw<R>(P, opp9(p), K<R>(P).rho_w[s], uwx, uwy, gx, gy);
    const R lam = LPn[p * P.plane + nb];
    Gx += lam * gx;
    Gy += lam * gy;
  }
}

// Post-collision density and velocity of X at a node (for d u / d X).
template <typename S, typename R>
__device__ __forceinline__ void post_rho_u(const SpParams &P, const S *X, int i, int j, R &rho, R &ux, R &uy) {
  const long long n = nidx(P, i, j);
  R s = 0;
#pragma unroll
  for (int q = 0; q < 9; q++) s += (R)X[q * P.plane + n];
  rho = K<R>(P).rho0 + s;
  post_velocity<S, R>(P, X, i, j, ux, uy);
}

}  // namespace

// Per-node parameter-gradient accumulators (8 bytes per node): an FP64 sum, or in the
// FP32 form a compensated FP32 pair (hi, lo) in the same 8 bytes, so that the reverse
// step runs no FP64 instruction per node.  grad_value() gives the FP64 value.
__device__ __forceinline__ void grad_add(double *g, long long n, double v) { g[n] += v; }
__device__ __forceinline__ void grad_add(double *g, long long n, float v) {
  float2 *g2 = reinterpret_cast<float2 *>(g);
  float2 a = g2[n];
  float e;
  two_sum(a.x, v, a.x, e);
  a.y += e;
  g2[n] = a;
}
// An FP64 value into the accumulator of a form with working precision R.
template <typename R> __device__ __forceinline__ void grad_add_fp64(double *g, long long n, double v);
template <> __device__ __forceinline__ void grad_add_fp64<double>(double *g, long long n, double v) { g[n] += v; }
template <> __device__ __forceinline__ void grad_add_fp64<float>(double *g, long long n, double v) {
  const float hi = (float)v, lo = (float)(v - (double)hi);  // v = hi + lo to ~2^-48
  float2 *g2 = reinterpret_cast<float2 *>(g);
  float2 a = g2[n];
  float e;
  two_sum(a.x, hi, a.x, e);
  a.y += e + lo;
  g2[n] = a;
}

// Loss at the outlet column and the seed Lam_pre(N).  One thread per row j.  T - T_target
// is formed in FP64 in both forms (FP32 would resolve T ~ 300 K only to ~3e-5 K).
template <typename S, typename R>
__global__ void k_adj_loss(const SpParams P, const double *Ttarget, R *LP, double *grad_qdot, double *loss_rows) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P.ny) return;
  const int i = P.nx - 1;
  const S *src = (const S *)P.src;
  const bool interior = false;
  R g[5];
  pull_g<S, R>(P, src, i, j, interior, g);
  const long long n = nidx(P, i, j);
  const double qd = P.qdot ? (double)((const S *)P.qdot)[n] : 0.0;
  const double T = P.T0 + (double)((g[0] + g[1]) + (g[2] + g[3]) + g[4]) + 0.5 * P.dt * qd;
  const double e = T - Ttarget[j];
  loss_rows[j] = e * e / P.ny;
  const double dLdT = 2.0 * e / P.ny;
  R *LPg = LP + (long long)P.gbase * P.plane;
#pragma unroll
  for (int q = 0; q < 5; q++) LPg[q * P.plane + n] = (R)dLdT;
  grad_add_fp64<R>(grad_qdot, n, 0.5 * P.dt * dLdT);
}

// One reverse step.  P.src = X_{t-1} (P.local = 1 when t = 0), Xt = X_t,
// LPn = Lam_pre(t+1), LP = Lam_pre(t) (output).
// The FP32 reverse step is latency-bound (long-scoreboard stalls, 22 % warps active at
// 100 registers and 2 blocks per SM): built for 4 resident blocks (64 registers, a few
// spills) the gradient run of the 1024 x 128 workload takes 99.7 ms instead of 113.6 ms
// (3 blocks: no gain).  The FP64 step is bound by the FP64 pipe: 2 blocks.
#ifndef LBM_ADJ_FP32_BLOCKS_PER_SM
#define LBM_ADJ_FP32_BLOCKS_PER_SM 4
#endif
template <typename S, typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? LBM_ADJ_FP32_BLOCKS_PER_SM : 2) k_adj_step(const SpParams P, const S *__restrict__ Xt,
                                                  const R *__restrict__ LPn, R *__restrict__ LP,
                                                  double *grad_qdot, double *grad_flux2, double *grad_flux3,
                                                  double *nu_partials) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  R dsnu = 0, dsq = 0;
  if (i < P.nx && j < P.ny) {
    const long long n = nidx(P, i, j);
    const R c = K<R>(P).c, ic = K<R>(P).inv_c;
    // ---- (1) Lam_X(t) = P^T Lam_pre(t+1) at this node --------------------------
    R lx[9], lg[5];
    const R *LPng = LPn + (long long)P.gbase * P.plane;
    if (i >= 2 && i <= P.nx - 3 && j >= 2 && j <= P.ny - 3) {
      // two or more cells from every side: every consumer of this node's populations is
      // an ordinary streaming link (no reflection, outlet extrapolation, flux or outflow
      // rule reaches it), so Lam_X is the plain gather
#pragma unroll
      for (int q = 0; q < 9; q++) lx[q] = LPn[q * P.plane + n + (long long)cy9(q) * P.pitch + cx9(q)];
#pragma unroll
      for (int q = 0; q < 5; q++) lg[q] = LPng[q * P.plane + n + (long long)cy5(q) * P.pitch + cx5(q)];
    } else {
#pragma unroll
      for (int q = 0; q < 9; q++) {
        R acc = 0;
        // streaming consumer: node y + c_q pulls population q from here
        int xi = i + cx9(q), xj = j + cy9(q);
        if (P.xper) xi = wrap(xi, P.nx);
        if (P.yper) xj = wrap(xj, P.ny);
        if (xi >= 0 && xi < P.nx && xj >= 0 && xj < P.ny && streams_in(P, xi, xj, cx9(q), cy9(q), P.xper, P.yper))
          acc += LPn[q * P.plane + nidx(P, xi, xj)];
        // reflection consumer: the incoming p = opp(q) at this node built from X_q here
        const int p = opp9(q);
        const int side = entry_side(i, j, cx9(p), cy9(p), P.nx, P.ny, P.xper, P.yper);
        if (side >= 0) acc += (P.side[side].kind == BC_PRESSURE ? (R)-1 : (R)1) * LPn[p * P.plane + n];
        lx[q] = acc;
      }
      // outlet velocity extrapolation u_w = 1.5 u(x_b) - 0.5 u(x_b - n)
#pragma unroll
      for (int s = 0; s < 4; s++) {
        if (P.side[s].kind != BC_PRESSURE) continue;
        const bool on = (s == 0 && i == 0) || (s == 1 && i == P.nx - 1) || (s == 2 && j == 0) || (s == 3 && j == P.ny - 1);
        const int bi = i - (s == 0) + (s == 1), bj = j - (s == 2) + (s == 3);  // boundary node outward of here
        const bool inner = !on && ((s == 0 && i == 1) || (s == 1 && i == P.nx - 2) || (s == 2 && j == 1) ||
                                   (s == 3 && j == P.ny - 2));
        if (!on && !inner) continue;
        R Gx, Gy;
        if (on) outlet_G<S, R>(P, Xt, LPn, s, i, j, Gx, Gy);
        else outlet_G<S, R>(P, Xt, LPn, s, bi, bj, Gx, Gy);
        R rho, ux, uy;
        post_rho_u<S, R>(P, Xt, i, j, rho, ux, uy);
        const R coef = (on ? (R)1.5 : (R)-0.5) / rho;  // one division for the nine links
#pragma unroll
        for (int q = 0; q < 9; q++) lx[q] += coef * (Gx * (c * (R)cx9(q) - ux) + Gy * (c * (R)cy9(q) - uy));
      }
#pragma unroll
      for (int q = 0; q < 5; q++) {
        R acc = 0;
        int xi = i + cx5(q), xj = j + cy5(q);
        if (P.txper) xi = wrap(xi, P.nx);
        if (P.typer) xj = wrap(xj, P.ny);
        if (xi >= 0 && xi < P.nx && xj >= 0 && xj < P.ny && streams_in(P, xi, xj, cx5(q), cy5(q), P.txper, P.typer))
          acc += LPng[q * P.plane + nidx(P, xi, xj)];
        const int p = opp5(q);
        const int side = entry_side(i, j, cx5(p), cy5(p), P.nx, P.ny, P.txper, P.typer);
        if (side >= 0) {
          const int tk = P.side[side].tkind;
          if (tk == TBC_FLUX) acc += LPng[p * P.plane + n];
          else if (tk == TBC_TEMP) acc -= LPng[p * P.plane + n];
        }
        // outflow consumer: the unknown q of an outflow side reads X_q of this node
        const int qside = entry_side(i, j, cx5(q), cy5(q), P.nx, P.ny, P.txper, P.typer);
        if (qside >= 0 && P.side[qside].tkind == TBC_OUTFLOW) acc += LPng[q * P.plane + n];
        lg[q] = acc;
      }
      // wall heat flux gradient: pre_p = X_o + flux_coef q''(a) on flux sides
#pragma unroll
      for (int p = 1; p < 5; p++) {
        const int side = entry_side(i, j, cx5(p), cy5(p), P.nx, P.ny, P.txper, P.typer);
        if (side >= 2 && P.side[side].tkind == TBC_FLUX) {
          double *gf = side == 2 ? grad_flux2 : grad_flux3;
          gf[i] += P.flux_coef * (double)LPng[p * P.plane + n];
        }
      }
    }

    // ---- (2) pre(t) and the forward intermediates -----------------------------
    const S *src = (const S *)P.src;
    const bool interior = !P.local && (i > 0) && (i < P.nx - 1) && (j > 0) && (j < P.ny - 1);
    R f[9], g[5];
    pull_f<S, R>(P, src, i, j, interior, f);
    pull_g<S, R>(P, src, i, j, interior, g);
    Macro<R> m;
    load_sources<S, R>(P, n, m);
    moments<R, FLOW_MRT, TH_MRT>(P, f, g, m);
    const R rho = m.rho, irho = (R)1 / rho;
    const R hx = m.ux * ic, hy = m.uy * ic, usq = hx * hx + hy * hy;
    const R Fx = m.Fx * ic, Fy = m.Fy * ic;
    const R dt = K<R>(P).dt;
    const R two = 2, three = 3, four = 4, six = 6, half = 0.5;

    // ---- (3) momentum MRT: transpose ------------------------------------------
    // moments of Lam_X (same integer rows as the moments of f)
    const R s14 = (lx[1] + lx[2]) + (lx[3] + lx[4]), s58 = (lx[5] + lx[6]) + (lx[7] + lx[8]);
    const R d58 = lx[5] - lx[7], d68 = lx[6] - lx[8];
    const R M_e = -four * lx[0] - s14 + two * s58;
    const R M_ep = four * lx[0] - two * s14 + s58;
    const R M_qx = two * (lx[3] - lx[1]) + d58 - d68;
    const R M_qy = two * (lx[4] - lx[2]) + d58 + d68;
    const R M_xx = (lx[1] + lx[3]) - (lx[2] + lx[4]);
    const R M_xy = (lx[5] + lx[7]) - (lx[6] + lx[8]);
    // dL/dd_k = -(M Lam)_k / |row_k|^2
    // (products with the rounded reciprocals: a divide is a long sequence on the FP64 pipe)
    const R de = -M_e * ((R)1 / (R)36), dep = -M_ep * ((R)1 / (R)36);
    const R dqx = -M_qx * ((R)1 / (R)12), dqy = -M_qy * ((R)1 / (R)12);
    const R dxx = -M_xx * (R)0.25, dxy = -M_xy * (R)0.25;
    const R se = K<R>(P).s_e, sep = K<R>(P).s_eps, sq = K<R>(P).s_q, snu = K<R>(P).s_nu;
    // dL/dm_k = s_k dL/dd_k; dL/deq_k = -s_k dL/dd_k
    const R lme = se * de, lmep = sep * dep, lmqx = sq * dqx, lmqy = sq * dqy, lmxx = snu * dxx, lmxy = snu * dxy;
    // equilibria of the moments
    const R mf58 = f[5] - f[7], mf68 = f[6] - f[8];
    const R m_qx = two * (f[3] - f[1]) + mf58 - mf68, m_qy = two * (f[4] - f[2]) + mf58 + mf68;
    const R m_xx = (f[1] + f[3]) - (f[2] + f[4]), m_xy = (f[5] + f[7]) - (f[6] + f[8]);
    const R eq_qx = -rho * hx, eq_qy = -rho * hy, eq_xx = rho * (hx * hx - hy * hy), eq_xy = rho * hx * hy;
    // nu enters through s_nu (stress moments) and s_q (third-order moments)
    const R hdt = K<R>(P).hdt;
    dsnu = dxx * ((m_xx - eq_xx) + hdt * two * (hx * Fx - hy * Fy)) + dxy * ((m_xy - eq_xy) + hdt * (hx * Fy + hy * Fx));
    dsq = dqx * ((m_qx - eq_qx) - hdt * Fx) + dqy * ((m_qy - eq_qy) - hdt * Fy);
    const R le = -se * de, lep = -sep * dep, lqx = -sq * dqx, lqy = -sq * dqy, lxx = -snu * dxx, lxy = -snu * dxy;
    R l_drho = le * (-two + three * usq) + lep * ((R)1 - three * usq) + lqx * (-hx) + lqy * (-hy) +
               lxx * (hx * hx - hy * hy) + lxy * (hx * hy);
    R l_hx = le * (six * rho * hx) + lep * (-six * rho * hx) + lqx * (-rho) + lxx * (two * rho * hx) + lxy * (rho * hy);
    R l_hy = le * (six * rho * hy) + lep * (-six * rho * hy) + lqy * (-rho) + lxx * (-two * rho * hy) + lxy * (rho * hx);
    // forcing moments that depend on u
    // (1 - dt Lambda_k / 2) dt from the host-filled constants
    const R l_uF = -six * K<R>(P).fk_e * de + six * K<R>(P).fk_eps * dep;
    const R l_Fxx = -K<R>(P).fk_nu * dxx * two, l_Fxy = -K<R>(P).fk_nu * dxy;
    l_hx += l_uF * Fx + l_Fxx * Fx + l_Fxy * Fy;
    l_hy += l_uF * Fy - l_Fxx * Fy + l_Fxy * Fx;

    // ---- (4) thermal D2Q5 MRT: transpose --------------------------------------
    const R B0 = -((lg[0] + lg[1]) + (lg[2] + lg[3]) + lg[4]);
    const R B1 = -(lg[1] - lg[3]), B2 = -(lg[2] - lg[4]);
    const R B3 = -(-four * lg[0] + ((lg[1] + lg[2]) + (lg[3] + lg[4])));
    const R B4 = -((lg[1] + lg[3]) - (lg[2] + lg[4]));
    const R t0 = B0 * (R)0.2, t1 = B1 * half, t2 = B2 * half, t3 = B3 * (R)0.05, t4 = B4 * (R)0.25;
    const R sT = K<R>(P).omegaT;
    const R lm1 = sT * t1, lm2 = sT * t2, lm3 = t3, lm4 = t4;
    const R lT = -sT * hx * t1 - sT * hy * t2 + (two / three) * t3;
    l_hx += -sT * m.T * t1;
    l_hy += -sT * m.T * t2;
    grad_add(grad_qdot, n, (R)(hdt * lT - dt * t0 + (dt * ((R)1 / three)) * t3));

    // ---- (5) back to the pre-collision populations ----------------------------
    R out[14];
#pragma unroll
    for (int q = 0; q < 9; q++) {
      const int cxq = cx9(q), cyq = cy9(q);
      // transpose of the moment rows: sum_k M[k][q] lm_k
      const R e_row = q == 0 ? -four : (q <= 4 ? (R)-1 : two);
      const R ep_row = q == 0 ? four : (q <= 4 ? -two : (R)1);
      const R qx_row = q == 0 ? (R)0 : (q <= 4 ? -two * (R)cxq : (R)cxq);
      const R qy_row = q == 0 ? (R)0 : (q <= 4 ? -two * (R)cyq : (R)cyq);
      const R xx_row = (q >= 1 && q <= 4) ? (R)(cxq * cxq - cyq * cyq) : (R)0;
      const R xy_row = q >= 5 ? (R)(cxq * cyq) : (R)0;
      R v = lx[q] + e_row * lme + ep_row * lmep + qx_row * lmqx + qy_row * lmqy + xx_row * lmxx + xy_row * lmxy;
      v += l_drho + (l_hx * ((R)cxq - hx) + l_hy * ((R)cyq - hy)) * irho;
      out[q] = v;
    }
#pragma unroll
    for (int q = 0; q < 5; q++) {
      const R r1 = (R)cx5(q), r2 = (R)cy5(q);
      const R r3 = q == 0 ? -four : (R)1;
      const R r4 = (q == 1 || q == 3) ? (R)1 : (q == 0 ? (R)0 : (R)-1);
      out[9 + q] = lg[q] + r1 * lm1 + r2 * lm2 + r3 * lm3 + r4 * lm4 + lT;
    }
#pragma unroll
    for (int q = 0; q < 14; q++) LP[q * P.plane + n] = out[q];
  }
  // per-block, fixed-order sums of the nu-rate sensitivities (working precision,
  // compensated in FP32), added to the block's FP64 partials by one thread
  NodeSum<R> dn, dq;
  dn.clear();
  dq.clear();
  dn.add(dsnu);
  dq.add(dsq);
  dn.warp_reduce();
  dq.warp_reduce();
  __shared__ NodeSum<R> sh[8][2];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if ((tid & 31) == 0) { sh[tid >> 5][0] = dn; sh[tid >> 5][1] = dq; }
  __syncthreads();
  if (tid == 0) {
    NodeSum<R> a = sh[0][0], b = sh[0][1];
    for (int w = 1; w < (int)(blockDim.x * blockDim.y) / 32; w++) { a.merge(sh[w][0]); b.merge(sh[w][1]); }
    double *acc = nu_partials + 2ll * (blockIdx.y * gridDim.x + blockIdx.x);
    acc[0] += a.value();
    acc[1] += b.value();
  }
}

__global__ void k_adj_final(const double *nu_partials, int nb, double *out2) {
  const int lane = threadIdx.x;
  double a = 0, b = 0;
  for (int k = lane; k < nb; k += 32) { a += nu_partials[2 * k]; b += nu_partials[2 * k + 1]; }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if (lane == 0) { out2[0] = a; out2[1] = b; }
}

cudaError_t adj_loss(const SpParams &P, int prec, const double *Ttarget, void *LP, double *grad_qdot,
                     double *loss_rows, cudaStream_t s) {
  const dim3 g((P.ny + 127) / 128), b(128);
  if (prec == 0) k_adj_loss<double, double><<<g, b, 0, s>>>(P, Ttarget, (double *)LP, grad_qdot, loss_rows);
  else k_adj_loss<float, float><<<g, b, 0, s>>>(P, Ttarget, (float *)LP, grad_qdot, loss_rows);
  return cudaGetLastError();
}

dim3 adj_grid(int nx, int ny) { return dim3((nx + 63) / 64, (ny + 3) / 4); }

cudaError_t adj_step(const SpParams &P, int prec, const void *Xt, const void *LPn, void *LP, double *grad_qdot,
                     double *grad_flux2, double *grad_flux3, double *nu_partials, cudaStream_t s) {
  const dim3 g = adj_grid(P.nx, P.ny), b(64, 4);
  if (prec == 0)
    k_adj_step<double, double><<<g, b, 0, s>>>(P, (const double *)Xt, (const double *)LPn, (double *)LP, grad_qdot,
                                               grad_flux2, grad_flux3, nu_partials);
  else
    k_adj_step<float, float><<<g, b, 0, s>>>(P, (const float *)Xt, (const float *)LPn, (float *)LP, grad_qdot,
                                             grad_flux2, grad_flux3, nu_partials);
  return cudaGetLastError();
}

cudaError_t adj_final(const double *nu_partials, int nb, double *out2, cudaStream_t s) {
  k_adj_final<<<1, 32, 0, s>>>(nu_partials, nb, out2);
  return cudaGetLastError();
}

}  // namespace lbmk
