"""The stationary-bubble workload at its configuration (Sec. 4.3): saturated water at
25 C (density ratio 43349), periodic 512 x 512 box, R = 64 dx, W = 5 dx, dx = 5e-6 m,
dt = 1e-7 s, M = 1e-5 m^2/s, D2Q5 h (BGK), D2Q9 z (MRT), 100000 steps, on the GPU in the
FP32 mixed form (FP64 recovery across the interface) and in FP64.

Against the FP64 oracle's run of the same workload (tests/golden/bubble_512.*, written
by make_bubble_512.py, which calls only the oracle):
  * the Laplace jump dp = P_in - P_out, pressures averaged where phi < 1e-3 and
    phi > 1 - 1e-3 (readings R12, R14), within 1 % of the oracle's;
  * phi and p - mean(p) element by element, and the spurious velocity field, within
    10x the oracle's own spread under a perturbation of phi0 at the form's rounding
    level (1e-15 for FP64, 1e-7 for FP32): the guarded normal of Sec. 2.3 is
    discontinuous where |grad phi| is rounding noise, so rounding differences grow;
  * the largest spurious speed within 1 % of the oracle's plus that spread.
At 100000 steps (10 ms) the bubble in the 2.56 mm box still oscillates: dp swings
between -11 % and +7 % of sigma/R over 50000-step intervals (reading R41), so the
Laplace law is checked in the paper's own set-up instead: the 1 mm x 1 mm box with the
six radii 125 ... 250 um of the Laplace table of Sec. 4.3, run to a steady jump."""
import json
import os

import numpy as np
import pytest

from _helpers import rel_max, run_gpu
from paper_2302_04120_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

lbm = pytest.importorskip("paper_2302_04120_gb300.lbm")
HERE = os.path.dirname(__file__)
GOLDEN_JSON = os.path.join(HERE, "golden", "bubble_512.json")
GOLDEN_NPZ = os.path.join(HERE, "golden", "bubble_512.npz")
FP64, FP32 = 0, 1


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_04120_gb300 import build
    build.build()


def _laplace_jump(m):
    phi, p = m["phi"], m["p"]
    return p[phi < 1e-3].mean() - p[phi > 1 - 1e-3].mean()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_bubble_512_against_oracle(prec):
    if not os.path.exists(GOLDEN_NPZ):
        pytest.skip("oracle fixture not written yet: run tests/golden/make_bubble_512.py")
    with open(GOLDEN_JSON) as fh:
        g = json.load(fh)
    ref = np.load(GOLDEN_NPZ)
    w = wl.bubble()
    assert g["steps"] == w["steps"] == 100000
    s = run_gpu(w, prec)
    m = s.moments()
    ints = s.integrals()
    s.close()
    assert ints[3] == 0
    dp = _laplace_jump(m)
    assert abs(dp - g["dp"]) <= 0.01 * abs(g["dp"]), (dp, g["dp"])
    # phase conservation over the run (sum phi of the initial tanh profile)
    phi0 = w["init"]["a"].sum()
    assert abs(ints[1] - phi0) <= (1e-12 if prec == FP64 else 1e-6) * phi0
    env = g["envelope"].get("1e-15" if prec == FP64 else "1e-07")
    if env is None:
        pytest.skip("the oracle's rounding envelope is not in the fixture yet (make_bubble_512.py)")
    d_phi = rel_max(m["phi"], ref["phi"])
    d_p = rel_max(m["p"] - m["p"].mean(), ref["p"])
    sp_ref = np.hypot(ref["ux"], ref["uy"])
    d_u = rel_max(np.stack([m["ux"], m["uy"]]), np.stack([ref["ux"], ref["uy"]]), sp_ref)
    assert d_phi <= max(1e-12, 10 * env["phi"]), (d_phi, env)
    assert d_p <= max(1e-12, 10 * env["p"]), (d_p, env)
    assert d_u <= max(1e-12, 10 * env["u"]), (d_u, env)
    sp_max = np.hypot(m["ux"], m["uy"]).max()
    assert abs(sp_max - g["u_spurious_max"]) <= (0.01 + 10 * env["u"]) * g["u_spurious_max"]


def _paper_laplace_table():
    with open(os.path.join(HERE, "golden", "paper_numbers.json")) as fh:
        d = json.load(fh)
    return d["laplace_error_percent_sat_water_25C"], d["density_profile_E2_percent_sat_water_25C"]


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_laplace_law_in_the_papers_box(prec):
    """Sec. 4.3 set-up: 1 mm x 1 mm periodic box (200 x 200 nodes), saturated water at
    25 C, R = 250, 225, 200, 175, 150, 125 um (50 ... 25 dx), W = 25 um, 200000 steps
    (dp changes by less than 0.1 % between 100000 and 200000 steps).  Per radius the
    Laplace-law error |dp - sigma/R| / (sigma/R) lies within 0.75 percentage points of
    the error the paper prints for it (4.351 ... 4.996 %) and below 6 %, growing with
    R as in the paper's table; the least-squares slope of dp against 1/R is within 6 %
    of sigma; the density profile's E2 against the tanh profile of Eq. density_prof
    (reading R13) along the horizontal diameter is below 1 % (paper 0.25 ... 0.46 %)."""
    lap, dens = _paper_laplace_table()
    sigma = wl.SAT_WATER_25C["sigma"]
    fl = wl.SAT_WATER_25C
    inv_R, dps, errs = [], [], []
    for R_inv, paper_err in zip(lap["R_inv"], lap["value"]):
        Rc = round(1.0 / R_inv / 5e-6)
        w = wl.bubble(n=200, R_cells=float(Rc), steps=200000)
        s = run_gpu(w, prec)
        m = s.moments()
        assert s.integrals()[3] == 0
        s.close()
        dp = _laplace_jump(m)
        err = 100 * abs(dp - sigma / w["R"]) / (sigma / w["R"])
        assert err < 6.0 and abs(err - paper_err) < 0.75, (Rc, err, paper_err)
        # density along the horizontal line through the centre (the row closest to it)
        dx = w["params"]["dx"]
        j = int(w["yc"] / dx)
        r = np.hypot((np.arange(200) + 0.5) * dx - w["xc"], (j + 0.5) * dx - w["yc"])
        ex = 0.5 * (fl["rho_l"] + fl["rho_g"]) + 0.5 * (fl["rho_l"] - fl["rho_g"]) * np.tanh(2 * (r - w["R"]) / w["W"])
        e2 = 100 * np.sqrt(np.sum((m["rho"][j] - ex) ** 2) / np.sum(ex ** 2))
        assert e2 < 1.0, (Rc, e2)
        inv_R.append(1.0 / w["R"])
        dps.append(dp)
        errs.append(err)
    assert all(a >= b - 0.05 for a, b in zip(errs, errs[1:])), errs   # error grows with R
    slope, _ = np.polyfit(inv_R, dps, 1)
    assert abs(slope - sigma) <= 0.06 * sigma, (slope, sigma)
