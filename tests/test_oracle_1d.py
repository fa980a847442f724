"""Pins of the oracle's one-dimensional cases (Sec. 4.1 and App. B): D2Q5 on one
periodic row is the D1Q3 lattice the paper uses (aggregated weights 4/6, 1/6, 1/6).

* wet-node Dirichlet sides (Eq. BCs_1D_advection_diffusion, with the node's T of
  Eq. zero_moment_g set to T_w, reading R37): pure diffusion gives the straight
  line and a uniform source the parabola T_w + q''' x (L - x)/(2k), both exactly,
  with the boundary nodes on x = 0 and x = L;
* App. B advection-diffusion with wet nodes against the closed form (reading R19):
  E2 = 0.036 % measured, the paper prints 0.030 %; link-wise ends give 0.061 % and
  wet-node values placed at half-way positions 0.70 %;
* the fuse of Sec. 4.1 (Joule heating, lagged convective loss, anti-bounce-back ends)
  against a forward-time central-space solution of Eq. conver_energy_fuse on the same
  nodes, as the paper compares its transient (plain numpy, written here).
"""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")


def _paper():
    with open(GOLDEN) as fh:
        return json.load(fh)


def _wet_rod(nx, dx, dt, k, rho, cp, T0, TL, u=0.0, q3=None, op=0):
    o = oracle.Oracle(dict(nx=nx, ny=1, flow=0, thermal=5, thermal_op=op, dx=dx, dt=dt, rho0=rho, cp=cp, k=k,
                           T0=T0, u_prescribed=(u, 0.0)))
    for side, T in ((0, T0), (1, TL)):
        o.set_bc(side, oracle.BC_PERIODIC, uw=np.array([u, 0.0]), tkind=oracle.TBC_WETNODE, tw=np.array([T]))
    if q3 is not None:
        o.set_source(q3=np.full(nx, q3))
    o.init()
    return o


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("nx,tau_bar", [(9, 0.8), (12, 1.3)])
def test_wet_node_linear_and_source_exact(op, nx, tau_bar):
    dx, k, rho, cp = 0.01, 1.0, 1.0, 1.0
    dt = (tau_bar - 0.5) * dx * dx / (3 * k / (rho * cp))
    x = np.arange(nx) * dx
    L = (nx - 1) * dx
    o = _wet_rod(nx, dx, dt, k, rho, cp, 300.0, 350.0, op=op)
    o.step(20000)
    T = o.moments()["T"][0]
    assert np.abs(T - (300.0 + 50.0 * x / L)).max() < 1e-9
    o = _wet_rod(nx, dx, dt, k, rho, cp, 300.0, 300.0, q3=1e4, op=op)
    o.step(20000)
    T = o.moments()["T"][0]
    ex = 300.0 + 1e4 * x * (L - x) / (2 * k)
    assert np.abs(T - ex).max() / (ex.max() - 300.0) < 1e-9


def test_app_b_wet_node():
    bp = _paper()["appB_problem"]
    nx = int(round(bp["L"] / bp["dx"])) + 1
    o = _wet_rod(nx, bp["dx"], bp["dt"], bp["k"], bp["rho"], bp["cp"], bp["T0"], bp["TL"], u=bp["u"])
    o.step(200000)
    T = o.moments()["T"][0]
    x = np.arange(nx) * bp["dx"]
    Pe = bp["rho"] * bp["cp"] * bp["u"] * bp["L"] / bp["k"]
    ex = bp["T0"] + (bp["TL"] - bp["T0"]) * np.expm1(Pe * x / bp["L"]) / np.expm1(Pe)
    e2 = oracle.e2_percent(ex, T)
    assert e2 < 1.5 * _paper()["appB_E2_percent"]["value"]
    assert abs(T[0] - bp["T0"]) < 1e-9 and abs(T[-1] - bp["TL"]) < 1e-9


def fuse_setup():
    fp = _paper()["fuse_problem"]
    Tinf = 273.15 + fp["T_inf_C"]
    q3 = 16 * fp["I"] ** 2 * fp["res"] / (np.pi ** 2 * fp["d"] ** 4)
    conv = 4 * fp["hbar"] / (fp["rho"] * fp["cp"] * fp["d"])
    nx = int(round(fp["L"] / fp["dx"]))
    return fp, Tinf, q3, conv, nx


def ftcs_fuse(nx, dx, dt, alpha, qd, conv, Tinf, steps):
    """Forward time, central space on the nodes x_i = (i + 1/2) dx, ends held at T_inf on
    the faces x = 0, L through mirrored ghost nodes (T_ghost = 2 T_w - T_boundary)."""
    T = np.full(nx, Tinf)
    for _ in range(steps):
        Tg = np.concatenate([[2 * Tinf - T[0]], T, [2 * Tinf - T[-1]]])
        T = T + dt * (alpha * (Tg[2:] - 2 * T + Tg[:-2]) / dx ** 2 + qd - conv * (T - Tinf))
    return T


def test_fuse_transient_against_ftcs():
    fp, Tinf, q3, conv, nx = fuse_setup()
    o = oracle.Oracle(dict(nx=nx, ny=1, flow=0, thermal=5, thermal_op=0, dx=fp["dx"], dt=fp["dt"], rho0=fp["rho"],
                           cp=fp["cp"], k=fp["k"], T0=Tinf, conv_coef=conv, T_inf=Tinf))
    for side in (0, 1):
        o.set_bc(side, oracle.BC_PERIODIC, tkind=oracle.TBC_TEMP, tw=np.array([Tinf]))
    o.set_source(q3=np.full(nx, q3))
    o.init()
    alpha = fp["k"] / (fp["rho"] * fp["cp"])
    done = 0
    for steps in (4000, 40000):       # t = 1 s and 10 s
        o.step(steps - done)
        done = steps
        T = o.moments()["T"][0]
        Tf = ftcs_fuse(nx, fp["dx"], fp["dt"], alpha, q3 / (fp["rho"] * fp["cp"]), conv, Tinf, steps)
        assert oracle.e2_percent(Tf - Tinf, T - Tinf) < 0.05   # 0.020 % at 1 s, 0.005 % at 10 s measured


@pytest.mark.parametrize("thermal,op", [(5, 0), (5, 1), (9, 0), (9, 1)])
@pytest.mark.parametrize("conv", [0.0, 3.0])
def test_thermal_collision_adds_dt_qdot(thermal, op, conv):
    """Each thermal collision (BGK with the (1 - dt/2tau_T) source factor, Eq.
    forcing_term_g; MRT with a zero rate on the zeroth moment and the source
    dt (I - dt Lambda/2) M (w qdot)) adds exactly dt qdot to sum_i g_i at every node,
    qdot = q'''/(rho0 c_p) - conv (T(t - dt) - T_inf).  The GPU's lagged sink rebuilds
    T(t - dt) from the post-collision populations through this identity."""
    rng = np.random.default_rng(7)
    nx, ny, dx, dt = 6, 5, 1e-3, 2e-3
    rho0, cp, k = 1000.0, 4180.0, 0.6
    o = oracle.Oracle(dict(nx=nx, ny=ny, flow=9, flow_op=0, thermal=thermal, thermal_op=op, dx=dx, dt=dt,
                           rho0=rho0, cp=cp, k=k, nu=1e-6, T0=300.0, conv_coef=conv, T_inf=295.0))
    q3 = 1e6 * rng.standard_normal((ny, nx))
    o.set_source(q3=q3)
    T0 = 300.0 + rng.standard_normal((ny, nx))
    o.init(None, 1e-3 * rng.standard_normal((ny, nx)), 1e-3 * rng.standard_normal((ny, nx)), T0)
    g0 = o.dist("g")
    o.step(1)
    gs = o.dist("g", post=True)
    qdot = q3 / (rho0 * cp) - conv * (T0 - 295.0)
    np.testing.assert_allclose(gs.sum(0) - g0.sum(0), dt * qdot, rtol=1e-9, atol=1e-12)
