"""TMA-staged persistent step launch (LBM_LAUNCH_TMA) against the grid launch and
the FP64 oracle.

The staged launch changes only where the pulled values come from (boxes in shared
memory instead of shifted global loads), so on the same inputs it must give the
grid launch's post-collision populations to rounding (the two kernels may contract
different pairs of operations into FMAs); the oracle comparisons use
the single-phase tolerances (FP64 1e-12 relative max-norm against the oracle's
long-double build, FP32 deviation 1e-5 relative L2).  Grids are ragged against the 32 x 4 and 32 x 8 tiles, and the
cases cover walls, velocity inlet, pressure outlet, heat-flux / temperature /
outflow thermal sides, periodic axes, per-cell sources, buoyancy and grids smaller
than one tile."""
import numpy as np
import pytest

from _helpers import rel_l2, rel_max, run_oracle
from paper_2302_04120_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

lbm = pytest.importorskip("paper_2302_04120_gb300.lbm")

FP64, FP32 = 0, 1


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_04120_gb300 import build
    build.build()


def _run(w, prec, launch=None, steps=None, q3=None, force=None):
    s = lbm.Solver(w["params"], precision=prec)
    for bc in w["bcs"]:
        s.set_bc(*bc)
    q = q3 if q3 is not None else w.get("q3")
    if q is not None or force is not None:
        s.set_source(q, force)
    if launch is not None:
        s.set_launch(*launch)
    s.init(**(w.get("init") or {}))
    s.step(w["steps"] if steps is None else steps)
    return s


def _same_state(a, b, prec=FP64):
    """Equal to rounding: 1e-13 (FP64) or 1e-6 (FP32) of each lattice's largest
    stored population (the two kernels inline the same arithmetic in different
    contexts and the compiler may contract a different pair into an FMA)."""
    sa, sb = a.state_arrays(), b.state_arrays()
    tol = 1e-13 if prec == FP64 else 1e-6
    for k in sa:
        assert np.max(np.abs(sa[k] - sb[k])) <= tol * np.max(np.abs(sb[k])), k


def _fields_vs_oracle(o, s, T_in, prec):
    mo, mg = o.moments(), s.moments()
    sp = np.hypot(mo["ux"], mo["uy"])
    if prec == FP64:
        assert rel_max(mg["ux"], mo["ux"], sp) < 1e-12
        assert rel_max(mg["uy"], mo["uy"], sp) < 1e-12
        if T_in is not None:
            assert rel_max(mg["T"] - T_in, mo["T"] - T_in) < 1e-12
    else:
        assert rel_l2(mg["ux"], mo["ux"], sp) < 1e-5
        assert rel_l2(mg["uy"], mo["uy"], sp) < 1e-5
        if T_in is not None:
            assert rel_l2(mg["T"] - T_in, mo["T"] - T_in) < 1e-5


@pytest.mark.parametrize("flow_op,thermal_op", [(0, 0), (1, 1), (1, 0), (0, 1)])
@pytest.mark.parametrize("launch", [(1, 8, 2, 1), (1, 4, 3, 2), (1, 8, 1, 1)])
def test_channel_fp64_tma_equals_grid_launch(flow_op, thermal_op, launch):
    """Ragged 100 x 42 forced-convection channel, 300 steps, FP64: every boundary kind."""
    w = wl.channel(nx=100, ny=42, steps=300, Re=100 * 42 / 256, flow_op=flow_op, thermal_op=thermal_op)
    a = _run(w, FP64, launch)
    assert a.launch_config() == launch
    b = _run(w, FP64)
    _same_state(a, b)
    _fields_vs_oracle(run_oracle(w, extended=True), a, w["T_in"], FP64)


@pytest.mark.parametrize("launch", [(1, 8, 3, 2), (1, 4, 4, 3), (1, 8, 4, 1)])
def test_channel_fp32_tma_equals_grid_launch(launch):
    w = wl.channel(nx=100, ny=42, steps=2000, Re=100 * 42 / 256)
    a = _run(w, FP32, launch)
    b = _run(w, FP32)
    _same_state(a, b, FP32)
    _fields_vs_oracle(run_oracle(w), a, w["T_in"], FP32)


def test_full_size_fp32_tma_against_oracle():
    """The 2048 x 256 workload, 200 steps, FP32 deviation storage, staged launch
    32 x 8 with three stages and two CTAs per SM, and the launch lbm_autotune picks
    (the one the benchmark times)."""
    w = wl.channel(steps=200)
    o = run_oracle(w)
    mo = o.moments()
    sp = np.hypot(mo["ux"], mo["uy"])
    a = _run(w, FP32, (1, 8, 3, 2))
    t = _run(w, FP32, steps=1)
    t.autotune()
    t.step(199)
    for s in (a, t):
        mg = s.moments()
        assert rel_l2(mg["ux"], mo["ux"], sp) < 1e-5
        assert rel_l2(mg["uy"], mo["uy"], sp) < 1e-5
        assert rel_l2(mg["T"], mo["T"]) < 1e-5
        assert rel_max(mg["T"] - w["T_in"], mo["T"] - w["T_in"]) < 1e-4
    _same_state(a, t, FP32)


def test_sources_forces_and_buoyancy_tma():
    """Per-cell q''' and force fields (70 x 36 channel) and the buoyancy-coupled
    65 x 65 cavity (walls on all four sides) through the staged launch."""
    w = wl.channel(nx=70, ny=36, steps=150, Re=100 * 36 / 256)
    rng = np.random.default_rng(11)
    q3 = 1e7 * rng.standard_normal((36, 70))
    force = 50.0 * rng.standard_normal((2, 36, 70))
    a = _run(w, FP64, (1, 8, 2, 1), q3=q3, force=force)
    b = _run(w, FP64, q3=q3, force=force)
    _same_state(a, b)
    _fields_vs_oracle(run_oracle(w, q3=q3, force=force, extended=True), a, w["T_in"], FP64)
    w = wl.natural_convection(steps=400, flow_op=1, thermal_op=1)
    a = _run(w, FP64, (1, 4, 2, 2))
    b = _run(w, FP64)
    _same_state(a, b)
    _fields_vs_oracle(run_oracle(w, extended=True), a, 293.85, FP64)


@pytest.mark.parametrize("op", [0, 1])
def test_thermal_only_periodic_tma(op):
    """flow = NONE (five planes), periodic in x and y: the wrap-around links are
    taken by the edge path, the interior from the staged boxes."""
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
    a = _run(w, FP64, (1, 8, 3, 1))
    b = _run(w, FP64)
    _same_state(a, b)
    assert rel_max(a.moments()["T"] - 300, run_oracle(w, extended=True).moments()["T"] - 300) < 1e-12


@pytest.mark.parametrize("nx,ny", [(1, 1), (5, 3), (33, 9)])
def test_grids_smaller_than_a_tile_tma(nx, ny):
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
    a = _run(w, FP64, (1, 8, 2, 1))
    b = _run(w, FP64)
    _same_state(a, b)
    _fields_vs_oracle(run_oracle(w, extended=True), a, 300.0, FP64)


def test_launch_configuration_errors_and_roundtrip():
    w = wl.channel(nx=40, ny=12, steps=0, Re=100 * 12 / 256)
    s = _run(w, FP64, steps=0)
    assert s.launch_config() == (0, 64, 4, 0)
    for bad in [(1, 6, 2, 1), (1, 8, 0, 1), (1, 8, 5, 1), (1, 8, 2, 0), (1, 8, 2, 99), (0, 48, 4, 0),
                (0, 64, 8, 0), (2, 8, 2, 1)]:
        with pytest.raises(lbm.LbmError):
            s.set_launch(*bad)
    assert s.launch_config() == (0, 64, 4, 0)
    s.set_launch(1, 4, 2, 1)
    assert s.launch_config() == (1, 4, 2, 1)
    s.set_launch(0, 32, 8)
    assert s.launch_config() == (0, 32, 8, 0)
    b = wl.bubble(n=48, ny=40, R_cells=10.0, W_cells=4.0, steps=0)
    m = _run(b, FP64, steps=0)
    with pytest.raises(lbm.LbmError):
        m.set_launch(1, 8, 2, 1)


def test_integrals_report_no_timeout_after_staged_steps():
    w = wl.channel(nx=100, ny=42, steps=50, Re=100 * 42 / 256)
    s = _run(w, FP32, (1, 8, 3, 2))
    assert s.check() == lbm.LBM_OK
    ints = s.integrals()
    assert ints[3] == 0


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_staged_copy_wait_runs_out_and_recovers(prec):
    """Failure detection of the bounded waits: with a 2 ms limit and the expiry
    self-test on, every block of the next TMA-staged step waits on a barrier that
    nothing completes; the wait runs out, the block lets its copies in flight land and
    exits, and lbm_check reports LBM_ERR_TIMEOUT once.  The context stays usable: after
    restoring the saved state the solve continues and equals an undisturbed run bit
    for bit, and the next check is clean."""
    w = wl.channel(nx=100, ny=42, steps=0, Re=100 * 42 / 256)
    ref = _run(w, prec, launch=(lbm.LBM_LAUNCH_TMA, 8, 3, 2), steps=30)
    s = _run(w, prec, launch=(lbm.LBM_LAUNCH_TMA, 8, 3, 2), steps=20)
    saved = s.get_state()
    s.set_wait_limit(2e-3, expire_next=True)
    s.step(1)
    assert s.check() == lbm.LBM_ERR_TIMEOUT
    assert "gave up waiting" in lbm.lbm_last_error(s.h)
    assert s.check() == lbm.LBM_OK          # reported once
    s.set_wait_limit(1.0)
    s.set_state(saved)
    s.step(10)
    assert s.check() == lbm.LBM_OK
    sa, sb = s.state_arrays(deviations=True), ref.state_arrays(deviations=True)
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k


def test_step_health_check_stops_at_a_planted_nan():
    """lbm_step with a check interval of 10: a healthy run passes every check (the last
    good step follows the step count); after a non-finite population is planted
    through lbm_set_state, the next check inside lbm_step returns LBM_ERR_DIVERGED at
    the first multiple of 10 and keeps the step count of the last passed check."""
    w = wl.channel(nx=64, ny=24, steps=0, Re=100 * 24 / 256)
    s = _run(w, FP64, steps=0)
    s.set_check_interval(10)
    assert s.last_good_step == -1
    s.step(25)
    assert s.steps == 25 and s.last_good_step == 20
    st = s.get_state().view(np.float64).copy()
    st[2 * 64 * 24 + 5 * 64 + 9] = np.nan
    s.set_state(st.view(np.uint8))
    with pytest.raises(lbm.LbmError) as err:
        s.step(40)
    assert err.value.status == lbm.LBM_ERR_DIVERGED
    assert s.steps == 30 and s.last_good_step == 20
    assert "last healthy check at step 20" in str(err.value)
    s.set_check_interval(0)
    with pytest.raises(lbm.LbmError):
        s.set_check_interval(-1)
