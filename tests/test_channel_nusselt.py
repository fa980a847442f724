"""The 2048 x 256 forced-convection workload over its full 50000 steps on the GPU,
against the oracle's run of the same workload in its long-double build (stored in
tests/golden/ by make_channel_nusselt.py, which calls only the oracle):

  * the fields u_x, u_y and T - T_in element by element: FP64 to 1e-12 relative
    max-norm (u relative to max |u|; measured 3.9e-15, 1.4e-15, 6.6e-14), FP32
    deviation storage to 1e-5 relative L2 (measured 5.1e-7, 5.3e-8, 8.1e-6);
  * the local Nusselt number along both walls, Nu(x) = q'' D_h / (k (T_w - T_m)) with
    T_w by half-cell extrapolation and T_m the velocity-weighted bulk temperature
    (reading R22), compared from column 8 on (over the first columns T_w - T_m
    crosses zero next to the fixed-temperature inlet column, where Nu is singular):
    relative L2 1e-12 in FP64 (measured 4.6e-14), 1e-5 in FP32 (measured 4.5e-6).
"""
import json
import os

import numpy as np
import pytest

from _helpers import rel_l2, rel_max, run_gpu
from paper_2302_04120_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

lbm = pytest.importorskip("paper_2302_04120_gb300.lbm")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "channel_nusselt_2048x256.json")
FIELDS = os.path.join(os.path.dirname(__file__), "golden", "channel_2048x256_fields.npz")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not os.path.exists(FIELDS):
        pytest.skip("oracle fixture not written yet: run its script under tests/golden/")
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_04120_gb300 import build
    build.build()


def _local_nusselt(T, u, q, k, dx, H):
    Tm = (u * T).sum(0) / u.sum(0)
    lower = q * 2 * H / (k * (T[0] + q * dx / (2 * k) - Tm))
    upper = q * 2 * H / (k * (T[-1] + q * dx / (2 * k) - Tm))
    return lower, upper


@pytest.mark.parametrize("prec", [lbm.LBM_FP64, lbm.LBM_FP32DEV])
def test_channel_full_run_against_oracle(prec):
    with open(GOLDEN) as fh:
        g = json.load(fh)
    ref = np.load(FIELDS)
    w = wl.channel()
    assert g["steps"] == w["steps"] == 50000
    s = run_gpu(w, prec)
    m = s.moments(lbm.LBM_UX | lbm.LBM_UY | lbm.LBM_T)
    s.close()
    dT = m["T"] - w["T_in"]
    sp = np.hypot(ref["ux"], ref["uy"])
    if prec == lbm.LBM_FP64:
        assert rel_max(m["ux"], ref["ux"], sp) < 1e-12
        assert rel_max(m["uy"], ref["uy"], sp) < 1e-12
        assert rel_max(dT, ref["dT"]) < 1e-12
    else:
        assert rel_l2(m["ux"], ref["ux"], sp) < 1e-5
        assert rel_l2(m["uy"], ref["uy"], sp) < 1e-5
        assert rel_l2(dT, ref["dT"]) < 1e-5
    p = w["params"]
    lower, upper = _local_nusselt(m["T"], m["ux"], w["qflux"], p["k"], p["dx"], w["H"])
    assert np.all(np.isfinite(lower)) and np.all(np.isfinite(upper))
    tol = 1e-12 if prec == lbm.LBM_FP64 else 1e-5
    assert rel_l2(lower[8:], np.array(g["Nu_lower"])[8:]) < tol
    assert rel_l2(upper[8:], np.array(g["Nu_upper"])[8:]) < tol
