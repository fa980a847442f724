"""GPU vs FP64 CPU oracle: two-phase solves between resting walls (layered Poiseuille
flow of Sec. 4.4; half-way bounce-back of z and h, mirrored phi in the stencils).

FP64: phi, u (relative to max |u|), p - mean p and the post-collision h, z to 1e-12
relative max-norm.  FP32 deviation storage: the steady layered profile within 1e-4
relative L2 of the oracle's (FP64 recovery of rho, u, p across the interface)."""
import numpy as np
import pytest

from _helpers import rel_l2, rel_max, run_gpu, run_oracle
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


def _air_water(ny, steps, nx=2, z_op=1):
    H = 0.5e-3
    dx = H / ny
    dt = 0.1 * dx * dx / (3.0 * wl.AIR_WATER_25C["nu_l"])
    fl = dict(wl.AIR_WATER_25C, sigma=1e-4)
    return wl.layered_poiseuille(fl, H=H, dx=dx, dt=dt, nx=nx, W=H / 10, steps=steps, z_op=z_op)


def _check_fp64(w):
    o = run_oracle(w)
    s = run_gpu(w, 0)
    mo, mg = o.moments(), s.moments()
    sp = np.hypot(mo["ux"], mo["uy"])
    assert rel_max(mg["phi"], mo["phi"]) < 1e-12
    assert rel_max(mg["ux"], mo["ux"], sp) < 1e-12
    assert rel_max(mg["uy"], mo["uy"], sp) < 1e-12
    assert rel_max(mg["p"], mo["p"], mo["p"] - mo["p"].mean()) < 1e-12
    st = s.state_arrays()
    assert rel_max(st["h"], o.dist("h", post=True)) < 1e-12
    assert rel_max(st["z"], o.dist("z", post=True)) < 1e-12
    s.close()


@pytest.mark.parametrize("z_op", [1, 0])
def test_layered_fp64_short(z_op):
    """37 x 40 layered air-water channel (ragged against the 32 x 8 tile in x, five
    tile rows), walls at y = 0 and y = H, 300 steps."""
    _check_fp64(_air_water(40, 300, nx=37, z_op=z_op))


@pytest.mark.parametrize("z_op", [1, 0])
def test_closed_box_bubble_fp64(z_op):
    """Bubble R = 8 in a 36 x 28 box walled on all four sides (corners), 60 steps."""
    w = wl.bubble(n=36, ny=28, R_cells=8.0, W_cells=4.0, steps=60, z_op=z_op)
    w["bcs"] = [(s, wl.BC_WALL, None, w["params"]["rho_l"], wl.TBC_NONE, None) for s in range(4)]
    _check_fp64(w)


def test_x_walls_only_fp64():
    """Walls at x = 0 and x = L, periodic in y: the layered channel turned sideways."""
    w = _air_water(40, 200, nx=2)
    p = dict(w["params"], nx=w["params"]["ny"], ny=5, Fb=(0.0, w["Fx"]))
    phi = np.repeat(w["init"]["a"][:, :1].T, 5, axis=0)
    rho_l = p["rho_l"]
    w2 = dict(w, params=p, init=dict(a=phi, ux=None, uy=None, b=None),
              bcs=[(0, wl.BC_WALL, None, rho_l, wl.TBC_NONE, None), (1, wl.BC_WALL, None, rho_l, wl.TBC_NONE, None)])
    _check_fp64(w2)


def test_layered_fp32_steady():
    """FP32 deviation storage: the steady 40-row layered profile (60000 steps) within
    1e-4 relative L2 of the FP64 oracle's."""
    w = _air_water(40, 60000)
    uo = run_oracle(w).moments()["ux"]
    s = run_gpu(w, 1)
    ug = s.moments()["ux"]
    s.close()
    assert rel_l2(ug, uo) < 1e-4


def test_two_phase_bc_rejections():
    w = _air_water(40, 0)
    s = lbm.Solver(w["params"], precision=0)
    with pytest.raises(lbm.LbmError):
        s.set_bc(2, wl.BC_VELOCITY, None, 1.0, wl.TBC_NONE, None)
    with pytest.raises(lbm.LbmError):
        s.set_bc(2, wl.BC_WALL, np.full(2 * w["params"]["nx"], 1e-3), 1.0, wl.TBC_NONE, None)
    with pytest.raises(lbm.LbmError):
        s.set_bc(2, wl.BC_WALL, None, 1.0, wl.TBC_FLUX, None)
    s.set_bc(2, wl.BC_WALL, np.zeros(2 * w["params"]["nx"]), 1.0, wl.TBC_NONE, None)
    s.close()
