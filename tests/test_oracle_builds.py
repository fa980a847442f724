"""Pins of the oracle's long-double and dual-number builds (CPU only).

The FP64 oracle is the definition the GPU path is checked against; the same source
built in long double measures the FP64 rounding floor of long runs, and built with
forward-mode dual numbers gives the reference gradient of the adjoint workload's
loss.  Each build is pinned here to something other than itself: the exact discrete
Poiseuille solution (closed form), the FP64 build, and differences of the FP64
oracle that are exact because the thermal LBE is affine in the heat source and the
wall flux when there is no buoyancy (Sec. 2.2: the momentum LBE does not see g)."""
import numpy as np
import pytest

import oracle
from paper_2302_04120_gb300 import workloads as wl

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
W5 = np.array([1 / 3] + [1 / 6] * 4)


def _run(w, steps, **kw):
    o = oracle.Oracle(w["params"], **kw)
    for bc in w["bcs"]:
        o.set_bc(*bc)
    if w.get("q3") is not None:
        o.set_source(q3=w["q3"])
    o.init(**(w.get("init") or {}))
    o.step(steps)
    return o


def test_extended_build_reaches_exact_poiseuille():
    """Long double: the steady BGK + Guo + half-way-wall channel equals the exact
    discrete solution u_j = F y_j (H - y_j) / (2 rho nu) + (F dx^2/(rho nu))(16 Lam - 3)/24,
    Lam = (tau/dt - 1/2)^2, to 1e-15 of u_max (measured 3.3e-16, the FP64 rounding of
    the closed form itself; the FP64 oracle's steady state sits 2e-14 away)."""
    ny, tau_bar = 5, 0.8
    dx, nu, rho, umax = 1e-3 / 32, 1e-6, 1000.0, 1e-3
    dt = (tau_bar - 0.5) * dx * dx / (3 * nu)
    F = 8 * rho * nu * umax / (ny * dx) ** 2
    o = oracle.Oracle(dict(nx=2, ny=ny, flow=9, flow_op=0, dx=dx, dt=dt, rho0=rho, nu=nu, Fb=(F, 0)),
                      extended=True)
    o.set_bc(2, oracle.BC_WALL)
    o.set_bc(3, oracle.BC_WALL)
    o.init()
    prev = None
    for _ in range(60):
        o.step(2000)
        u = o.moments()["ux"][:, 0]
        if prev is not None and np.max(np.abs(u - prev)) == 0.0:
            break
        prev = u
    y = (np.arange(ny) + 0.5) * dx
    H = ny * dx
    ex = F * y * (H - y) / (2 * rho * nu) + F * dx * dx / (rho * nu) * (16 * (tau_bar - 0.5) ** 2 - 3) / 24
    assert np.max(np.abs(u - ex)) / np.max(ex) < 1e-15


def test_extended_build_agrees_with_fp64_on_short_runs():
    """Same steps in two precisions: after 20 steps of the forced-convection channel
    (every boundary rule, MRT both lattices) the deviations f - w rho0, g - w T0 and
    u differ by FP64 rounding only (< 1e-13 of their magnitude)."""
    w = wl.channel(nx=30, ny=10, steps=20, Re=100 * 10 / 256)
    a, b = _run(w, 20), _run(w, 20, extended=True)
    p = w["params"]
    for name, wts, ref in (("f", W9, p["rho0"]), ("g", W5, p["T0"])):
        da = a.dist(name, post=True) - wts[:, None, None] * ref
        db = b.dist(name, post=True) - wts[:, None, None] * ref
        assert np.max(np.abs(da - db)) < 1e-13 * np.max(np.abs(db))
    ma, mb = a.moments(), b.moments()
    assert np.max(np.abs(ma["ux"] - mb["ux"])) < 1e-13 * np.max(np.abs(mb["ux"]))


def test_dual_build_value_part_is_the_fp64_oracle():
    """The value part of every dual number follows the FP64 oracle bit for bit."""
    w = wl.channel(nx=30, ny=10, steps=25, Re=100 * 10 / 256)
    w["q3"] = wl.smooth_source(30, 10, seed=5, sigma_cells=2.0, scale=1e8)
    a = _run(w, 25)
    o = oracle.Oracle(w["params"], dual=True)
    for bc in w["bcs"]:
        o.set_bc(*bc)
    o.set_source(q3=w["q3"])
    o.seed(dnu=1.0, dq3=np.ones((10, 30)), dqwall=np.ones((2, 30)))
    o.init(**w["init"])
    o.step(25)
    ma, mb = a.moments(), o.moments()
    for k in ("ux", "uy", "T", "rho"):
        assert np.array_equal(ma[k], mb[k]), k


def _small_gradient_case():
    nx, ny, steps = 12, 6, 40
    w = wl.channel(nx=nx, ny=ny, steps=steps, Re=100 * ny / 256)
    w["q3"] = wl.smooth_source(nx, ny, seed=5, sigma_cells=2.0, scale=1e8)
    T_base = _run(w, steps).moments()["T"][:, -1]
    H = ny * w["params"]["dx"]
    y = (np.arange(ny) + 0.5) * w["params"]["dx"]
    return w, steps, T_base + 0.01 * np.sin(np.pi * y / H)


def _with_qwall(w, qw):
    w2 = dict(w)
    w2["bcs"] = [(s, k, uw, rw, tk, qw[s - 2] if s in (2, 3) and tk == oracle.TBC_FLUX else tw)
                 for s, k, uw, rw, tk, tw in w["bcs"]]
    return w2


def test_dual_gradient_elementwise_against_exact_differences():
    """12 x 6 channel, 40 steps: every element of dL/dq''' (72 cells) and dL/dq''
    (2 x 12 wall nodes) from the dual build equals r . (T(x + s e_k) - T(x)) / s with
    r = dL/dT_out, which is exact up to rounding because T is affine in q''' and q''.
    s is large enough that the rounding of T (~6e-14 K) stays far below the
    difference; bound 1e-10 relative to the largest element (measured 2.6e-14)."""
    w, steps, target = _small_gradient_case()
    ny, nx = 6, 12
    L, g3, gw, gnu = oracle.outlet_loss_gradient(w, steps, target)
    T0 = _run(w, steps).moments()["T"][:, -1]
    r = 2.0 * (T0 - target) / ny
    assert L == pytest.approx(np.mean((T0 - target) ** 2), rel=1e-15)
    s3 = 1e13
    ref3 = np.zeros((ny, nx))
    for j in range(ny):
        for i in range(nx):
            w2 = dict(w)
            w2["q3"] = w["q3"].copy()
            w2["q3"][j, i] += s3
            ref3[j, i] = r @ (_run(w2, steps).moments()["T"][:, -1] - T0) / s3
    assert np.max(np.abs(g3 - ref3)) <= 1e-10 * np.max(np.abs(ref3))
    qw = np.full((2, nx), w["qflux"])
    sw = 1e9
    refw = np.zeros((2, nx))
    for side in range(2):
        for i in range(nx):
            q2 = qw.copy()
            q2[side, i] += sw
            refw[side, i] = r @ (_run(_with_qwall(w, q2), steps).moments()["T"][:, -1] - T0) / sw
    assert np.max(np.abs(gw - refw)) <= 1e-10 * np.max(np.abs(refw))


def test_dual_gradient_nu_against_richardson_differences():
    """dL/dnu (nu enters nonlinearly through the MRT rates) against Richardson-
    extrapolated central differences of the FP64 oracle's loss, (4 D(h/2) - D(h))/3
    with relative steps h = 2e-4: truncation O(h^4), rounding ~1e-8 of the result."""
    w, steps, target = _small_gradient_case()
    _, _, _, gnu = oracle.outlet_loss_gradient(w, steps, target, q3=False, qwall=False)
    nu = w["params"]["nu"]

    def loss(v):
        w2 = dict(w)
        w2["params"] = dict(w["params"], nu=v)
        return np.mean((_run(w2, steps).moments()["T"][:, -1] - target) ** 2)

    def D(h):
        return (loss(nu * (1 + h)) - loss(nu * (1 - h))) / (2 * h * nu)

    ref = (4 * D(1e-4) - D(2e-4)) / 3
    assert abs(gnu - ref) <= 1e-6 * abs(ref)
