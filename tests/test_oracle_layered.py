"""Pins of the oracle's two-phase solve between walls (layered Poiseuille flow, Sec. 4.4).

The paper states no wall rule for the two-phase LBEs; the oracle takes half-way
bounce-back at resting walls for z (Eq. BB_vel with u_w = 0) and for h, and the
mirror image of the boundary node for the phi stencils (readings R34, R35).  These
tests pin that against things other than the oracle:

* one fluid (phi = 1 everywhere): the z-LBE between walls driven by a body force
  must reach the exact discrete steady state of half-way bounce-back, the parabola
  plus the slip (F dx^2/(rho nu))(16 Lambda - 3)/24 with Lambda = 1/12 for the
  multiphase MRT (omega_q2 rule of Sec. 3) and (tau/dt - 1/2)^2 for BGK;
* air-water layers: the steady profile converges at second order to the
  quadrature of Eq. NSE_for_layered_poiseuille with zeta(y) of Eq. viscosity_prof
  (nu = zeta/rho, Sec. 4.4), with the interface width held fixed in metres;
* the walls let no phi through: sum phi is conserved.
"""
import numpy as np
import pytest

import oracle
from _helpers import run_oracle
from _layered import e2, reference_for
from paper_2302_04120_gb300 import workloads as wl


@pytest.mark.parametrize("z_op", [1, 0])
@pytest.mark.parametrize("ny,tau_bar", [(6, 0.8), (9, 1.3)])
def test_one_fluid_between_walls_exact(z_op, ny, tau_bar):
    H, nu, rho = 1e-3, 1e-6, 1000.0
    dx = H / ny
    dt = (tau_bar - 0.5) * dx * dx / (3.0 * nu)
    fl = dict(rho_g=rho, rho_l=rho, nu_g=nu, nu_l=nu, sigma=1e-4)
    # tau_phi = dt (mobility free here: phi stays 1)
    w = wl.layered_poiseuille(fl, H=H, dx=dx, dt=dt, nx=2, W=2 * dx, steps=20000, z_op=z_op,
                              mobility=0.5 * dx * dx / (3.0 * dt))
    w["init"] = dict(w["init"], a=np.ones_like(w["init"]["a"]))
    u = run_oracle(w).moments()["ux"]
    y = (np.arange(ny) + 0.5) * dx
    F = w["Fx"]
    lam = 1.0 / 12.0 if z_op == 1 else (tau_bar - 0.5) ** 2
    exact = F / (2 * rho * nu) * y * (H - y) + F * dx * dx / (rho * nu) * (16 * lam - 3) / 24
    assert np.abs(u - exact[:, None]).max() / exact.max() < 1e-12


def _air_water(ny, steps):
    H = 0.5e-3
    dx = H / ny
    dt = 0.1 * dx * dx / (3.0 * wl.AIR_WATER_25C["nu_l"])  # tau_l = 0.6 dt
    # sigma does not enter the planar steady state; the paper's 0.072 N/m makes the
    # interface forces at 4-8 cells per W too stiff for this dt
    fl = dict(wl.AIR_WATER_25C, sigma=1e-4)
    return wl.layered_poiseuille(fl, H=H, dx=dx, dt=dt, nx=2, W=H / 10, steps=steps)


def test_air_water_layers_converge_to_quadrature():
    """E2 against the quadrature at W = 4 and 8 cells: 21 % and 5.4 % measured, a
    ratio of 3.9 (second order).  A wrong wall rule, viscosity rule or force term
    leaves an O(1) error that does not shrink."""
    errs = []
    for ny, steps in ((40, 60000), (80, 200000)):
        w = _air_water(ny, steps)
        u = run_oracle(w).moments()["ux"].mean(axis=1)
        errs.append(e2(u, reference_for(w)))
    assert errs[0] < 0.25 and errs[1] < 0.07
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_walls_conserve_phase():
    w = _air_water(40, 3000)
    o = oracle.Oracle(w["params"])
    for bc in w["bcs"]:
        o.set_bc(*bc)
    o.init(**w["init"])
    s0 = o.moments()["phi"].sum()
    o.step(3000)
    m = o.moments()
    assert abs(m["phi"].sum() - s0) / s0 < 1e-12
    # x-invariant inputs stay x-invariant (columns agree to rounding)
    assert np.abs(m["ux"] - m["ux"][:, :1]).max() <= 1e-12 * np.abs(m["ux"]).max()


def test_property_table_consistent_with_printed_columns():
    """The four fluid systems typed into the workloads (rho_g, rho_l, nu_g, nu_l of the
    table of Sec. 4.3) reproduce the table's own derived columns: zeta = rho nu and the
    density, viscosity and zeta ratios, to the printed rounding."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")) as fh:
        table = json.load(fh)["two_phase_property_table"]
    for name, fl in wl.TWO_PHASE_SYSTEMS.items():
        row = table[name]
        zg, zl = fl["rho_g"] * fl["nu_g"] / 1e-5, fl["rho_l"] * fl["nu_l"] / 1e-5
        # 0.5 %: the printed inputs carry 2 to 5 significant digits (rho_g = 0.023 at
        # 25 C alone leaves zeta_g uncertain by 2 %; measured 0.3 %)
        assert abs(zg / row["zeta_g"] - 1) < 5e-3
        assert abs(zl / row["zeta_l"] - 1) < 5e-3
        assert abs(fl["rho_l"] / fl["rho_g"] / row["rho_ratio"] - 1) < 5e-3
        assert abs(fl["nu_g"] / fl["nu_l"] / row["nu_ratio"] - 1) < 5e-3
        assert abs(zl / zg / row["zeta_ratio"] - 1) < 5e-3


def test_quadrature_reference_sharp_interface_limit():
    """The quadrature reference itself: as W -> 0 the profile tends to the two-layer
    closed form (zeta_l below H/2, zeta_g above): zeta u' = -F (y - y*) with
    y* = [h^2/(2 zeta_l) + (H^2 - h^2)/(2 zeta_g)] / [h/zeta_l + (H - h)/zeta_g], h = H/2,
    u = F/zeta_l (y* y - y^2/2) below and u(H) = 0 from above."""
    from _layered import layered_reference
    H, F, zl, zg = 0.5e-3, 0.36, 8.9e-4, 1.8e-5
    h = H / 2
    y = np.linspace(0.0, H, 201)[1:-1]
    ystar = (h * h / (2 * zl) + (H * H - h * h) / (2 * zg)) / (h / zl + (H - h) / zg)
    below = F / zl * (ystar * y - y * y / 2)
    above = F / zg * ((H * H - y * y) / 2 - ystar * (H - y))
    exact = np.where(y < h, below, above)
    errs = []
    for W in (H / 200, H / 2000, H / 20000):
        u = layered_reference(y, H, W, F, zl, zg, n=2000001)
        errs.append(np.abs(u - exact).max() / exact.max())
    # first order in W (the smeared viscosity jump): 3.2e-2, 3.3e-3, 3.3e-4 measured
    assert errs[2] < 5e-4
    assert 8.0 < errs[0] / errs[1] < 12.0 and 8.0 < errs[1] / errs[2] < 12.0
