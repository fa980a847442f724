"""GPU (CUDA, sm_103a) vs CPU oracle: single-phase hot path.

Tolerances (stated by the method's contract, on deviations, reading R25):
  FP64 path:        1e-12 relative max-norm on u (relative to max |u|), on T - T_in and
                    on the post-collision population deviations f - w rho0, g - w T0;
  FP32-deviation:   1e-5 relative L2 on u and T - T_in.
The FP64 comparisons use the oracle's long-double build: the FP64 oracle stores
absolute f ~ w rho0 and T ~ 300 K, and its own rounding on these deviations reaches
1e-12 within a few hundred steps (measured against the long-double build: 2.8e-12 on
T - T_in after 300 steps, 4.9e-12 on u_y after the 20000 Poiseuille steps), while the
GPU stores the deviations themselves.  Populations are compared element by element
after the same number of steps (GPU post-collision buffer vs the oracle's last
post-collision values)."""
import numpy as np
import pytest

from _helpers import W5, W9, deviations, rel_l2, rel_max, run_gpu, run_oracle
from paper_2302_04120_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

lbm = pytest.importorskip("paper_2302_04120_gb300.lbm")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_04120_gb300 import build
    build.build()
    torch.cuda.init()


FP64, FP32 = 0, 1


def _compare_fields(o, s, T_in=None, tol=1e-12, prec=FP64):
    """FP64: u and T - T_in to `tol` relative max-norm (u relative to max |u|).
    FP32 deviation form: `tol` relative L2 on u and T - T_in."""
    mo = o.moments()
    mg = s.moments()
    sp = np.hypot(mo["ux"], mo["uy"])
    norm = rel_max if prec == FP64 else rel_l2
    out = dict(ux=norm(mg["ux"], mo["ux"], sp), uy=norm(mg["uy"], mo["uy"], sp))
    if T_in is not None:
        out["dT"] = norm(mg["T"] - T_in, mo["T"] - T_in)
    for k, v in out.items():
        assert v < tol, (k, v, out)
    return out


def _compare_populations(o, s, w, tol=1e-12):
    """Post-collision deviations f - w_i rho0 and g - w_i T0 element by element,
    relative to their largest magnitude."""
    st = s.state_arrays(deviations=True)
    p = w["params"]
    if p.get("flow", 9):
        assert rel_max(st["f"], deviations(o.dist("f", post=True), W9, p["rho0"])) < tol
    if p.get("thermal", 0):
        wg = W9 if p["thermal"] == 9 else W5
        assert rel_max(st["g"], deviations(o.dist("g", post=True), wg, p.get("T0", 300.0))) < tol


# ---------------------------------------------------------------------------
def test_poiseuille_workload_full():
    """64 x 33 D2Q9 BGK channel, 20000 steps, FP64: GPU = oracle to 1e-12 and the
    steady profile matches the exact discrete half-way bounce-back solution."""
    w = wl.poiseuille()
    o = run_oracle(w, extended=True)
    s = run_gpu(w, FP64)
    # measured 6.2e-14 (u_x), 5.3e-16 (u_y), 8.4e-14 (f - w rho0); the FP64 oracle
    # itself is 1.3e-12 / 4.9e-12 / 5.7e-10 away from the long-double run
    _compare_fields(o, s)
    _compare_populations(o, s, w)
    u = s.moments()["ux"][:, 0]
    p = w["params"]
    dx, nu, rho, F = p["dx"], p["nu"], p["rho0"], w["Fb"]
    y = (np.arange(p["ny"]) + 0.5) * dx
    H = p["ny"] * dx
    ex = F / (2 * rho * nu) * y * (H - y) + F * dx * dx / (rho * nu) * (16 * 0.09 - 3) / 24
    assert np.max(np.abs(u - ex)) / np.max(ex) < 1e-7   # slowest mode decayed to ~1e-8


@pytest.mark.parametrize("flow_op,thermal_op", [(0, 0), (1, 1), (1, 0), (0, 1)])
def test_channel_all_boundaries_fp64(flow_op, thermal_op):
    """Forced-convection channel (BB-velocity inlet, anti-BB outlet, heat-flux walls,
    inlet temperature, thermal outflow) on a ragged 100 x 42 grid (several 64 x 4
    tiles plus partial ones), 300 steps, FP64."""
    w = wl.channel(nx=100, ny=42, steps=300, Re=100 * 42 / 256, flow_op=flow_op, thermal_op=thermal_op)
    o = run_oracle(w, extended=True)
    s = run_gpu(w, FP64)
    _compare_fields(o, s, T_in=w["T_in"])
    _compare_populations(o, s, w)


def test_channel_fp32_deviation():
    """Same channel in FP32-deviation storage: 1e-5 relative L2 on u and T - T_in
    after 2000 steps."""
    w = wl.channel(nx=100, ny=42, steps=2000, Re=100 * 42 / 256)
    o = run_oracle(w)
    s = run_gpu(w, FP32)
    _compare_fields(o, s, T_in=w["T_in"], tol=1e-5, prec=FP32)


@pytest.mark.parametrize("prec,steps", [(FP64, 12), (FP32, 200)])
def test_channel_full_size(prec, steps):
    """The 2048 x 256 forced-convection workload in the launch configuration the
    benchmark times; 12 steps in FP64, 200 in FP32.  FP32: u to 1e-5 relative L2,
    T to 1e-5 relative L2 in K (the contract's measure) and T - T_in to 1e-4
    relative max-norm: after 200 steps the heated layer is two rows of 256, so an
    L2 norm of T - T_in would measure FP32 rounding of the advective g deviations
    (~2e-7 K) over the unheated 99 % of the grid rather than the heated part."""
    w = wl.channel(steps=steps)
    o = run_oracle(w, extended=prec == FP64)
    s = run_gpu(w, prec)
    if prec == FP64:
        _compare_fields(o, s, T_in=w["T_in"], tol=1e-12, prec=FP64)
        _compare_populations(o, s, w)
        return
    mo, mg = o.moments(), s.moments()
    sp = np.hypot(mo["ux"], mo["uy"])
    assert rel_l2(mg["ux"], mo["ux"], sp) < 1e-5
    assert rel_l2(mg["uy"], mo["uy"], sp) < 1e-5
    assert rel_l2(mg["T"], mo["T"]) < 1e-5
    assert rel_max(mg["T"] - w["T_in"], mo["T"] - w["T_in"]) < 1e-4


def test_sources_and_force_fields():
    """Per-cell heat source q''' and force field through lbm_set_source."""
    w = wl.channel(nx=70, ny=36, steps=150, Re=100 * 36 / 256)
    rng = np.random.default_rng(11)
    q3 = 1e7 * rng.standard_normal((36, 70))
    force = 50.0 * rng.standard_normal((2, 36, 70))
    o = run_oracle(w, q3=q3, force=force, extended=True)
    s = run_gpu(w, FP64, q3=q3, force=force)
    _compare_fields(o, s, T_in=w["T_in"])
    _compare_populations(o, s, w)


@pytest.mark.parametrize("op", [0, 1])
def test_thermal_only_gaussian(op):
    """flow = NONE: D2Q5 advection-diffusion of a Gaussian on a periodic 64 x 48
    box with a prescribed velocity."""
    nx, ny, dx = 64, 48, 1e-5
    alpha = 0.6 / (1000 * 4180)
    dt = 0.3 * dx * dx / (3 * alpha)
    u = (2e-4, -1e-4)
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y)
    T0 = 300 + 10 * np.exp(-((X - 3e-4) ** 2 + (Y - 2.4e-4) ** 2) / (2 * (6e-5) ** 2))
    params = dict(nx=nx, ny=ny, flow=0, thermal=5, thermal_op=op, dx=dx, dt=dt, rho0=1000.0, cp=4180.0,
                  k=0.6, T0=300.0, u_prescribed=u)
    w = dict(params=params, bcs=[], init=dict(a=None, ux=np.full((ny, nx), u[0]), uy=np.full((ny, nx), u[1]), b=T0),
             steps=200)
    o = run_oracle(w, extended=True)
    s = run_gpu(w, FP64)
    mo, mg = o.moments(), s.moments()
    assert rel_max(mg["T"] - 300, mo["T"] - 300) < 1e-12
    _compare_populations(o, s, w)


@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 2), (2, 1), (5, 3)])
def test_tiny_and_degenerate_grids(nx, ny):
    """Degenerate sizes: a single periodic node, and grids smaller than one tile
    with walls (every node is a boundary node)."""
    rng = np.random.default_rng(nx * 10 + ny)
    dx, nu = 1e-4, 1e-6
    dt = 0.3 * dx * dx / (3 * nu)
    p = dict(nx=nx, ny=ny, flow=9, flow_op=1, thermal=5, thermal_op=1, dx=dx, dt=dt, rho0=1000.0, nu=nu,
             cp=4180.0, k=0.6, T0=300.0, Fb=(3.0, -1.0))
    bcs = []
    if ny > 1:
        bcs = [(2, 1, np.concatenate([np.full(nx, 1e-4), np.zeros(nx)]), 1000.0, 2, np.full(nx, 310.0)),
               (3, 1, None, 1000.0, 1, np.full(nx, 1e3))]
    init = dict(a=1000 + rng.standard_normal((ny, nx)), ux=1e-3 * rng.standard_normal((ny, nx)),
                uy=1e-3 * rng.standard_normal((ny, nx)), b=300 + rng.standard_normal((ny, nx)))
    w = dict(params=p, bcs=bcs, init=init, steps=40)
    o = run_oracle(w, extended=True)
    s = run_gpu(w, FP64)
    _compare_fields(o, s, T_in=300.0)
    _compare_populations(o, s, w)


def test_zero_steps_returns_initial_fields():
    w = wl.channel(nx=40, ny=12, steps=0, Re=100 * 12 / 256)
    s = run_gpu(w, FP64, steps=0)
    m = s.moments()
    np.testing.assert_allclose(m["T"], w["init"]["b"], rtol=0, atol=1e-12)
    o = run_oracle(w, steps=0)
    assert rel_max(m["ux"], o.moments()["ux"]) < 1e-12


def test_state_roundtrip_device_moments_and_integrals():
    """Checkpoint/restart through lbm_get_state/lbm_set_state; moments into a
    device tensor; FP64 mass integral vs the oracle; a planted NaN is flagged."""
    import torch
    w = wl.channel(nx=64, ny=24, steps=100, Re=100 * 24 / 256)
    s = run_gpu(w, FP64)
    st = s.get_state()
    s.step(50)
    a = s.moments()
    s.set_state(st)
    s.step(50)
    b = s.moments()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    dev = torch.empty((2, 24, 64), dtype=torch.float64, device="cuda")
    lbm.lbm_moments(s.h, lbm.LBM_UX | lbm.LBM_T, dev)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dev[0].cpu().numpy(), b["ux"])
    np.testing.assert_array_equal(dev[1].cpu().numpy(), b["T"])
    o = run_oracle(w, steps=150)
    mass_o = o.moments()["rho"].sum() * w["params"]["dx"] ** 2
    ints = s.integrals()
    assert abs(ints[0] - mass_o) / mass_o < 1e-13
    assert ints[3] == 0 and s.check() == lbm.LBM_OK
    bad = st.view(np.float64).copy()
    bad[5 * 64 * 24 + 7] = np.nan
    s.set_state(bad.view(np.uint8))
    assert s.check() == lbm.LBM_ERR_DIVERGED
    assert "non-finite" in lbm.lbm_last_error(s.h)


def test_autotune_keeps_state_and_results():
    """Autotuning the step's launch neither advances nor changes the solution: bit
    for bit when it keeps the grid launch (the block shape does not enter the
    arithmetic), to FP64 rounding (1e-13) when it picks the TMA-staged kernel."""
    w = wl.channel(nx=100, ny=42, steps=30, Re=100 * 42 / 256)
    a = run_gpu(w, FP64, steps=10)
    blk = a.autotune()
    assert blk[0] * blk[1] % 32 == 0 and a.steps == 10
    kind = a.launch_config()[0]
    a.step(20)
    b = run_gpu(w, FP64, steps=30)
    ma, mb = a.moments(), b.moments()
    for k in ma:
        if kind == lbm.LBM_LAUNCH_GRID:
            assert np.array_equal(ma[k], mb[k]), k
        else:
            assert np.max(np.abs(ma[k] - mb[k])) <= 1e-13 * max(np.max(np.abs(mb[k])), 1e-300), k


@pytest.mark.parametrize("flow_op,thermal_op", [(0, 1), (1, 1)])
def test_buoyancy_cavity_parity(flow_op, thermal_op):
    """Two-way coupling (Boussinesq force of App. D) in the 65 x 65 heated cavity:
    400 steps FP64 vs the oracle (1e-12), FP32 vs the oracle (1e-5 relative L2)."""
    w = wl.natural_convection(steps=400, flow_op=flow_op, thermal_op=thermal_op)
    o = run_oracle(w, extended=True)
    s = run_gpu(w, FP64)
    _compare_fields(o, s, T_in=293.85)
    _compare_populations(o, s, w)
    s32 = run_gpu(w, FP32)
    _compare_fields(o, s32, T_in=293.85, tol=1e-5, prec=FP32)


def test_buoyancy_cavity_nusselt_on_gpu():
    """Steady mean Nusselt number of the Ra ~ 1e4 cavity from the GPU (FP64 and
    FP32 deviation forms) within 1 % of the benchmark 2.243 printed in App. D."""
    from test_oracle_pins import cavity_nusselt
    w = wl.natural_convection(steps=40000)
    for prec in (FP64, FP32):
        s = run_gpu(w, prec)
        nu, spread = cavity_nusselt(s.moments(), w)
        assert abs(nu - 2.243) / 2.243 < 0.01, (prec, nu)
        assert spread < 1e-4


def _cavity_ra1e6(steps):
    """App. D at Ra = 1e6: the same air and dx = dt = 2e-4, walls at 373.85 / 293.15 K
    and a cavity side of 0.060 m (reading R38: the printed 0.60 m gives Ra ~ 1e9, while
    0.060 m gives Ra = 0.995e6 with alpha = k / (rho c_p) of the printed properties):
    300 x 300 nodes."""
    w = wl.natural_convection(L=0.060, T_h=373.85, T_c=293.15, steps=steps)
    assert abs(w["Ra"] - 1e6) / 1e6 < 1e-2 and w["params"]["nx"] == 300
    return w


def test_buoyancy_cavity_ra1e6_parity():
    """The Ra = 1e6 cavity (300 x 300, BGK momentum + D2Q5 MRT thermal), 200 steps:
    FP64 against the oracle's long-double build to 1e-12, FP32 to 1e-5 relative L2."""
    w = _cavity_ra1e6(200)
    o = run_oracle(w, extended=True)
    s = run_gpu(w, FP64)
    _compare_fields(o, s, T_in=293.15)
    _compare_populations(o, s, w)
    _compare_fields(o, run_gpu(w, FP32), T_in=293.15, tol=1e-5, prec=FP32)


def test_buoyancy_cavity_ra1e6_nusselt_on_gpu():
    """Steady mean Nusselt number of the Ra = 1e6 cavity (App. D) from the GPU, FP64
    and FP32 deviation forms, within 1 % of the benchmark 8.800 the paper prints (its
    dimensional LBM: 8.805), with a uniform heat flux through every vertical face."""
    from test_oracle_pins import cavity_nusselt
    w = _cavity_ra1e6(0)
    for prec in (FP64, FP32):
        s = run_gpu(w, prec, steps=0)
        prev = None
        for _ in range(40):
            s.step(20000)
            nu, spread = cavity_nusselt(s.moments(), w)
            if prev is not None and abs(nu - prev) < 1e-6 * nu and spread < 1e-4:
                break
            prev = nu
        s.close()
        assert abs(nu - 8.800) / 8.800 < 0.01, (prec, nu, spread)
        assert spread < 1e-4, (prec, spread)


def _run_launch(w, prec, launch, steps):
    s = lbm.Solver(w["params"], precision=prec)
    s.apply_workload(w)
    s.set_launch(*launch)
    s.step(steps)
    return s


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("nx,ny,block", [(100, 42, (32, 2)), (97, 13, (64, 1)), (33, 9, (32, 4)), (130, 7, (128, 2)),
                                         (3, 5, (32, 1))])
def test_occupancy_launch_equals_grid_launch(prec, nx, ny, block):
    """LBM_LAUNCH_GRID_OCC (the step built for 6 resident blocks per SM) on ragged grids,
    including one without interior nodes, against the default grid launch: the same
    arithmetic, so equal to rounding (1e-13 of the largest deviation in FP64, 1e-6 in
    FP32; the two builds may contract different operations into FMAs), and against the
    oracle."""
    w = wl.channel(nx=nx, ny=ny, steps=0, Re=100 * ny / 256)
    steps = 150
    a = _run_launch(w, prec, (lbm.LBM_LAUNCH_GRID_OCC, *block), steps)
    assert a.launch_config()[0] == lbm.LBM_LAUNCH_GRID_OCC
    b = _run_launch(w, prec, (lbm.LBM_LAUNCH_GRID, 64, 4), steps)
    sa, sb = a.state_arrays(deviations=True), b.state_arrays(deviations=True)
    tol = 1e-13 if prec == FP64 else 1e-6
    for k in sa:
        assert np.max(np.abs(sa[k] - sb[k])) <= tol * np.max(np.abs(sb[k])), k
    o = run_oracle(dict(w, steps=steps), extended=prec == FP64)
    _compare_fields(o, a, T_in=w["T_in"], tol=1e-12 if prec == FP64 else 1e-5, prec=prec)


def test_occupancy_launch_full_size_and_graph_replay():
    """The 2048 x 256 workload with the occupancy build, 200 steps (graph-replayed runs of
    64 steps), FP32: equal to the grid launch to 1e-6 of the largest deviation."""
    w = wl.channel(steps=0)
    a = _run_launch(w, FP32, (lbm.LBM_LAUNCH_GRID_OCC, 32, 2), 200)
    b = _run_launch(w, FP32, (lbm.LBM_LAUNCH_GRID, 32, 2), 200)
    sa, sb = a.state_arrays(deviations=True), b.state_arrays(deviations=True)
    for k in sa:
        assert np.max(np.abs(sa[k] - sb[k])) <= 1e-6 * np.max(np.abs(sb[k])), k
