"""Seeded synthetic workloads shaped like the paper's test problems.

This module is the ONLY code shared by the CUDA path's tests/bench and the CPU
oracle.  It holds inputs only: SI parameters, grid sizes, boundary values and
initial fields.  None of the lattice Boltzmann arithmetic lives here.

Every workload is a dict:
    params : SI parameter dict (keys of ``lbm_params`` / the oracle's params)
    bcs    : list of (side, kind, uw[2*len] or None, rho_w, tkind, tw[len] or None)
             side 0 = x-, 1 = x+, 2 = y-, 3 = y+
    init   : dict(a=..., ux=..., uy=..., b=...) arrays of shape (ny, nx) or None
             (a = rho or phi, b = T or p)
    q3     : q''' field (W m^-3), shape (ny, nx), or None
    steps  : step count of the full workload

Node (i, j) sits at x = (i + 1/2) dx, y = (j + 1/2) dx; half-way walls lie on
cell faces (Sec. 2.1, link-wise boundaries).
"""
from __future__ import annotations

import numpy as np

# boundary kinds (same numbering as include/lbm.h and the oracle)
BC_PERIODIC, BC_WALL, BC_VELOCITY, BC_PRESSURE, BC_SYMMETRY = 0, 1, 2, 3, 4
TBC_NONE, TBC_FLUX, TBC_TEMP, TBC_OUTFLOW, TBC_SYMMETRY, TBC_WETNODE = 0, 1, 2, 3, 4, 5

# Water of the forced-convection workload (rho, c_p, k) and Pr = 7.
WATER = dict(rho0=1000.0, cp=4180.0, k=0.6)
# The four two-phase systems of the property table of Sec. 4.3 (rho_g, rho_l in
# kg m^-3, nu_g, nu_l in m^2 s^-1, sigma in N m^-1).
AIR_WATER_25C = dict(rho_g=1.184, rho_l=997.048, nu_g=155.770e-7, nu_l=8.927e-7, sigma=0.072)
SAT_WATER_100C = dict(rho_g=0.598, rho_l=958.349, nu_g=204.493e-7, nu_l=2.938e-7, sigma=0.059)
SAT_WATER_80C = dict(rho_g=0.294, rho_l=971.766, nu_g=392.919e-7, nu_l=3.643e-7, sigma=0.063)
SAT_WATER_25C = dict(rho_g=0.023, rho_l=997.003, nu_g=4204.120e-7, nu_l=8.927e-7, sigma=0.072)
TWO_PHASE_SYSTEMS = {"air_water_25C": AIR_WATER_25C, "sat_water_100C": SAT_WATER_100C,
                     "sat_water_80C": SAT_WATER_80C, "sat_water_25C": SAT_WATER_25C}


def node_y(ny, dx):
    return (np.arange(ny) + 0.5) * dx


def node_x(nx, dx):
    return (np.arange(nx) + 0.5) * dx


def parabola(ny, dx, u_mean):
    """Developed channel profile u(y) = 6 u_m (y/H - y^2/H^2), Eq. velocity_prof."""
    H = ny * dx
    y = node_y(ny, dx)
    return 6.0 * u_mean * (y / H - (y / H) ** 2)


# ---------------------------------------------------------------------------
# Workload 1: isothermal Poiseuille channel, D2Q9 BGK, FP64
# ---------------------------------------------------------------------------
def poiseuille(nx=64, ny=33, steps=20000, u_max=1e-3, tau_bar_dt=9.765625e-5, flow_op=0):
    """64 x 33 periodic channel with half-way walls; H = 1 mm resolved by dx = H/32.

    33 fluid rows between half-way walls give an effective height 33 dx; the
    body force is chosen so the centreline speed of the continuum parabola over
    that height is u_max.  dt = 9.765625e-5 s gives tau/dt = 0.8 for nu = 1e-6.
    """
    dx = 1e-3 / 32
    rho, nu = 1000.0, 1e-6
    H = ny * dx
    Fb = 8.0 * rho * nu * u_max / H ** 2
    params = dict(nx=nx, ny=ny, flow=9, flow_op=flow_op, thermal=0, phase=0, dx=dx,
                  dt=tau_bar_dt, rho0=rho, nu=nu, Fb=(Fb, 0.0))
    bcs = [(2, BC_WALL, None, rho, TBC_NONE, None), (3, BC_WALL, None, rho, TBC_NONE, None)]
    return dict(name=f"poiseuille_d2q9_{nx}x{ny}", params=params, bcs=bcs, init=None, q3=None,
                steps=steps, H=H, Fb=Fb)


# ---------------------------------------------------------------------------
# Workload 2: developing forced convection, D2Q9 MRT + D2Q5 thermal
# ---------------------------------------------------------------------------
def channel(nx=2048, ny=256, steps=50000, Re=100.0, Pr=7.0, qflux=4e4, T_in=300.0,
            dx=2.5e-6, dt=6.25e-7, flow_op=1, thermal_op=1, q3=None, literal=0):
    """Full channel with two heated walls (constant flux q''), parabolic inflow,
    uniform inlet temperature, anti-bounce-back pressure outlet.

    Water with c_p = 4180 J/kg/K, k = 0.6 W/m/K, rho = 1000; nu = Pr * alpha;
    Re = u_m D_h / nu with D_h = 2H.  dx, dt are the paper's developing-flow
    values (Sec. 4.2).  Initial state: inlet parabola everywhere, T = T_in.
    """
    rho0, cp, k = WATER["rho0"], WATER["cp"], WATER["k"]
    alpha = k / (rho0 * cp)
    nu = Pr * alpha
    H = ny * dx
    u_m = Re * nu / (2.0 * H)
    uin = parabola(ny, dx, u_m)
    params = dict(nx=nx, ny=ny, flow=9, flow_op=flow_op, thermal=5, thermal_op=thermal_op,
                  phase=0, dx=dx, dt=dt, rho0=rho0, nu=nu, cp=cp, k=k, T0=T_in, literal=literal)
    uw_in = np.concatenate([uin, np.zeros(ny)])
    bcs = [
        (0, BC_VELOCITY, uw_in, rho0, TBC_TEMP, np.full(ny, T_in)),
        (1, BC_PRESSURE, None, rho0, TBC_OUTFLOW, None),
        (2, BC_WALL, None, rho0, TBC_FLUX, np.full(nx, qflux)),
        (3, BC_WALL, None, rho0, TBC_FLUX, np.full(nx, qflux)),
    ]
    ux0 = np.tile(uin[:, None], (1, nx))
    init = dict(a=None, ux=ux0, uy=np.zeros((ny, nx)), b=np.full((ny, nx), T_in))
    return dict(name=f"channel_d2q9mrt_d2q5_{nx}x{ny}", params=params, bcs=bcs, init=init,
                q3=q3, steps=steps, u_m=u_m, H=H, nu=nu, alpha=alpha, qflux=qflux, T_in=T_in)


# ---------------------------------------------------------------------------
# The paper's heated-channel cases (Sec. 4.2): D2Q9 BGK flow + D2Q9 MRT thermal
# ---------------------------------------------------------------------------
# Water at 301 K (property table of Sec. 4.2).
WATER_301K = dict(rho0=996.279, nu=8.382e-7, k=0.611, cp=4180.333)


def heated_channel(case=2, nx=None, ny=None, steps=0, half=True, flow_op=0, thermal=9, thermal_op=1,
                   q_mean=4e4, dq=4e4, L_h=1e-3, T_in=300.0, H=5e-4, L=1e-2, u_m=None):
    """Forced convection between two plates heated with the same flux (Sec. 4.2).

    case 1: hydrodynamically and thermally developed inlet, u(y) = 6 u_m (y/H - y^2/H^2)
            with u_m = 0.2 m/s and the developed T(y) of Eq. temp_prof; oscillating flux
            q''(x) = q_mean + dq sign(sin(2 pi x / L_h)) (Eq. var_flux); dx = 5e-6, dt = 2e-6.
    case 2: developing flow, uniform inlet u_m = 0.02 m/s and T_in; constant flux q_mean;
            dx = 2.5e-6, dt = 6.25e-7.
    case 3: case 2 with the oscillating flux.
    half=True simulates the lower half (y in [0, H/2]) with a symmetry top, as the paper
    does; half=False the full channel with two heated walls.  nx, ny default to the
    paper's L/dx and (H/2)/dx (H/dx for the full channel); smaller values give a
    shorter channel with the same dx, dt and inlet data; u_m overrides the case's mean
    inlet speed.  Initial state: the inlet fields everywhere.
    """
    w = WATER_301K
    rho0, nu, k, cp = w["rho0"], w["nu"], w["k"], w["cp"]
    dx, dt, um = (5e-6, 2e-6, 0.2) if case == 1 else (2.5e-6, 6.25e-7, 0.02)
    u_m = um if u_m is None else u_m
    if nx is None:
        nx = int(round(L / dx))
    if ny is None:
        ny = int(round((H / 2 if half else H) / dx))
    y = node_y(ny, dx)                        # from the bottom plate
    s = y / H
    if case == 1:
        uin = 6.0 * u_m * (s - s * s)
        Tin = T_in + q_mean * H / k * (-s ** 4 + 2 * s ** 3 - s + 0.243)   # Eq. temp_prof
    else:
        uin = np.full(ny, u_m)
        Tin = np.full(ny, T_in)
    x = node_x(nx, dx)
    if case in (1, 3):
        qw = q_mean + dq * np.sign(np.sin(2.0 * np.pi * x / L_h))          # Eq. var_flux
    else:
        qw = np.full(nx, q_mean)
    params = dict(nx=nx, ny=ny, flow=9, flow_op=flow_op, thermal=thermal, thermal_op=thermal_op, phase=0,
                  dx=dx, dt=dt, rho0=rho0, nu=nu, cp=cp, k=k, T0=T_in)
    bcs = [
        (0, BC_VELOCITY, np.concatenate([uin, np.zeros(ny)]), rho0, TBC_TEMP, Tin.copy()),
        (1, BC_PRESSURE, None, rho0, TBC_OUTFLOW, None),
        (2, BC_WALL, None, rho0, TBC_FLUX, qw.copy()),
    ]
    if half:
        bcs.append((3, BC_SYMMETRY, None, rho0, TBC_SYMMETRY, None))
    else:
        bcs.append((3, BC_WALL, None, rho0, TBC_FLUX, qw.copy()))
    init = dict(a=None, ux=np.tile(uin[:, None], (1, nx)), uy=np.zeros((ny, nx)),
                b=np.tile(Tin[:, None], (1, nx)))
    return dict(name=f"heated_channel_case{case}_{nx}x{ny}{'_half' if half else ''}", params=params, bcs=bcs,
                init=init, q3=None, steps=steps, u_m=u_m, H=H, qwall=qw, T_in=T_in, k=k, dx=dx)


# ---------------------------------------------------------------------------
# Workload 3: static bubble, D2Q9 MRT z + D2Q5 h
# ---------------------------------------------------------------------------
def bubble(n=512, R_cells=64.0, W_cells=5.0, steps=100000, dx=5e-6, dt=1e-7, mobility=1e-5,
           fluid=SAT_WATER_25C, z_op=1, ny=None):
    """Periodic box with a centred gas bubble; phi = 0 gas, 1 liquid.

    Initial phi is the equilibrium tanh profile with gas inside radius R
    (Eq. diffuse_interface with the sign that puts gas inside), u = 0, p = 0.
    """
    nx = n
    ny = n if ny is None else ny
    W = W_cells * dx
    R = R_cells * dx
    x = node_x(nx, dx)[None, :]
    y = node_y(ny, dx)[:, None]
    xc, yc = 0.5 * nx * dx, 0.5 * ny * dx
    r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    phi0 = 0.5 + 0.5 * np.tanh(2.0 * (r - R) / W)
    params = dict(nx=nx, ny=ny, flow=9, flow_op=1, thermal=0, phase=5, z_op=z_op, dx=dx, dt=dt,
                  rho0=fluid["rho_l"], W=W, mobility=mobility, **fluid)
    init = dict(a=phi0, ux=None, uy=None, b=None)
    return dict(name=f"bubble_{nx}x{ny}_R{R_cells:g}", params=params, bcs=[], init=init, q3=None,
                steps=steps, R=R, W=W, r=r, xc=xc, yc=yc)


# ---------------------------------------------------------------------------
# Workload 3b: layered two-phase Poiseuille flow (Sec. 4.4)
# ---------------------------------------------------------------------------
def layered_poiseuille(fluid="air_water_25C", H=0.5e-3, dx=1.25e-6, dt=1.25e-8, nx=10, W=25e-6,
                       mobility=1e-5, u_c=1e-4, steps=0, z_op=1, literal=0):
    """Channel of height H between resting walls (y sides), periodic in x, liquid in
    the lower half and gas in the upper half.

    phi(y) = 1/2 - 1/2 tanh((2y - H)/W) (Eq. diffuse_interface across the plane y = H/2,
    liquid below), so zeta = phi zeta_l + (1 - phi) zeta_g is the profile of
    Eq. viscosity_prof; nu = zeta/rho (nu_rule 1); body force F_x = u_c (zeta_l +
    zeta_g)/H^2; u = 0 and p = 0 at t = 0.  The paper uses 10 columns, W = 25 um,
    M = 1e-5 m^2/s and dx = 1.25 um, D2Q5 h with BGK and MRT for the momentum (z)
    equation.  It states dt = 1.25e-7 s, and 1.25e-8 s at the same dx in its refinement
    study; at the real surface tension 1.25e-7 s diverges within ~100 steps, so the
    default is 1.25e-8 s.
    """
    fl = TWO_PHASE_SYSTEMS[fluid] if isinstance(fluid, str) else fluid
    ny = int(round(H / dx))
    y = node_y(ny, dx)
    phi_y = 0.5 - 0.5 * np.tanh((2.0 * y - H) / W)
    phi0 = np.repeat(phi_y[:, None], nx, axis=1)
    zeta_l, zeta_g = fl["rho_l"] * fl["nu_l"], fl["rho_g"] * fl["nu_g"]
    Fx = u_c * (zeta_l + zeta_g) / H ** 2
    params = dict(nx=nx, ny=ny, flow=9, flow_op=1, thermal=0, phase=5, z_op=z_op, nu_rule=1, literal=literal,
                  dx=dx, dt=dt, rho0=fl["rho_l"], W=W, mobility=mobility, Fb=(Fx, 0.0), **fl)
    bcs = [(2, BC_WALL, None, fl["rho_l"], TBC_NONE, None), (3, BC_WALL, None, fl["rho_l"], TBC_NONE, None)]
    init = dict(a=phi0, ux=None, uy=None, b=None)
    name = fluid if isinstance(fluid, str) else "custom"
    return dict(name=f"layered_poiseuille_{name}_{nx}x{ny}", params=params, bcs=bcs, init=init, q3=None,
                steps=steps, H=H, W=W, Fx=Fx, zeta_l=zeta_l, zeta_g=zeta_g, u_c=u_c, y=y)


# ---------------------------------------------------------------------------
# Workload 4: many independent channels of uneven size
# ---------------------------------------------------------------------------
def channel_batch_specs(count=256, seed=4, nx_range=(128, 4096), ny_range=(32, 512)):
    """Per-channel (nx, ny, Re, Pr, dx, dt) of the batched workload: Nx ~ U{128..4096},
    Ny ~ U{32..512}, Re ~ U(10, 200), Pr in {0.7, 7} (numpy PCG64 seed 4, draws in that
    order per channel).

    dt per channel: the largest dt with a lattice Mach number <= 0.1 based on
    1.5 u_m, clipped so that both relaxation times stay in [0.51, 2.0] dt.
    """
    rng = np.random.default_rng(seed)
    dx = 2.5e-6
    rho0, cp, k = WATER["rho0"], WATER["cp"], WATER["k"]
    alpha = k / (rho0 * cp)
    out = []
    for _ in range(count):
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1))
        Re = float(rng.uniform(10.0, 200.0))
        Pr = float(rng.choice([0.7, 7.0]))
        nu = Pr * alpha
        H = ny * dx
        u_m = Re * nu / (2.0 * H)
        dmin, dmax = min(nu, alpha), max(nu, alpha)
        dt_ma = 0.1 * dx / (np.sqrt(3.0) * 1.5 * u_m)
        dt_lo = 0.01 * dx * dx / (3.0 * dmin)
        dt_hi = 0.5 * dx * dx / dmax
        dt = max(dt_lo, min(dt_ma, dt_hi))
        out.append(dict(nx=nx, ny=ny, Re=Re, Pr=Pr, dx=dx, dt=dt))
    return out


def channel_from_spec(spec, steps=5000):
    w = channel(nx=spec["nx"], ny=spec["ny"], steps=steps, Re=spec["Re"], Pr=spec["Pr"], dx=spec["dx"],
                dt=spec["dt"])
    w["Re"], w["Pr"] = spec["Re"], spec["Pr"]
    return w


def channel_batch(count=256, seed=4, steps=5000, nx_range=(128, 4096), ny_range=(32, 512)):
    """The batched workload as full workload dicts (see channel_batch_specs)."""
    return [channel_from_spec(sp, steps) for sp in channel_batch_specs(count, seed, nx_range, ny_range)]


# ---------------------------------------------------------------------------
# Workload 5: heat-source field for the gradient workload
# ---------------------------------------------------------------------------
def smooth_source(nx=1024, ny=128, seed=5, sigma_cells=8.0, scale=1e6):
    """Gaussian-filtered N(0,1) field (periodic in x, reflected in y), renormalised
    to unit standard deviation and scaled to W m^-3."""
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal((ny, nx))
    rad = int(np.ceil(4 * sigma_cells))
    t = np.arange(-rad, rad + 1)
    ker = np.exp(-0.5 * (t / sigma_cells) ** 2)
    ker /= ker.sum()
    # x: periodic
    acc = np.zeros_like(xi)
    for s, w in zip(t, ker):
        acc += w * np.roll(xi, s, axis=1)
    # y: reflect
    pad = np.pad(acc, ((rad, rad), (0, 0)), mode="symmetric")
    out = np.zeros_like(acc)
    for s, w in zip(t, ker):
        out += w * pad[rad + s: rad + s + ny, :]
    out = (out - out.mean()) / out.std()
    return scale * out


def adjoint_channel(nx=1024, ny=128, steps=2000, Re=50.0):
    w = channel(nx=nx, ny=ny, steps=steps, Re=Re, q3=smooth_source(nx, ny))
    return w


def random_state_like(shape, seed, scale=1.0):
    """Seeded perturbation field for parity tests off the equilibrium manifold."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(shape)


# ---------------------------------------------------------------------------
# Natural convection in a square cavity (two-way coupling through buoyancy)
# ---------------------------------------------------------------------------
AIR_333K = dict(rho0=1.059, cp=1008.045, k=0.029, nu=1.90e-5, beta_exp=3.004e-3)


def natural_convection(L=0.013, T_h=373.15, T_c=293.85, T_ref=333.5, dx=2e-4, dt=2e-4, steps=40000,
                       flow_op=0, thermal_op=1, n=None):
    """Square cavity of side L (air at 333.5 K, App. D): hot left wall T_h, cold right
    wall T_c, adiabatic top and bottom, no-slip walls, gravity (0, -9.81) m/s^2.
    L = 13 mm gives Ra ~ 1e4 (App. D).  Start at rest at T_c."""
    n = int(round(L / dx)) if n is None else n
    a = AIR_333K
    params = dict(nx=n, ny=n, flow=9, flow_op=flow_op, thermal=5, thermal_op=thermal_op, phase=0, dx=dx, dt=dt,
                  rho0=a["rho0"], nu=a["nu"], cp=a["cp"], k=a["k"], T0=T_c, gravity=(0.0, -9.81),
                  beta_exp=a["beta_exp"], T_ref=T_ref, rho_ref=a["rho0"])
    bcs = [
        (0, BC_WALL, None, a["rho0"], TBC_TEMP, np.full(n, T_h)),
        (1, BC_WALL, None, a["rho0"], TBC_TEMP, np.full(n, T_c)),
        (2, BC_WALL, None, a["rho0"], TBC_FLUX, np.zeros(n)),
        (3, BC_WALL, None, a["rho0"], TBC_FLUX, np.zeros(n)),
    ]
    init = dict(a=None, ux=np.zeros((n, n)), uy=np.zeros((n, n)), b=np.full((n, n), T_c))
    alpha = a["k"] / (a["rho0"] * a["cp"])
    Ra = 9.81 * a["beta_exp"] * (n * dx) ** 3 * (T_h - T_c) / (a["nu"] * alpha)
    return dict(name=f"cavity_{n}x{n}", params=params, bcs=bcs, init=init, q3=None, steps=steps,
                alpha=alpha, dT=T_h - T_c, Ra=Ra, L=n * dx)
