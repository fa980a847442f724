"""The 2048 x 256 forced-convection workload over its full 50000 steps on the GPU: the
local Nusselt number along both walls against the FP64 oracle's (stored in
tests/golden/channel_nusselt_2048x256.json by make_channel_nusselt.py, which calls only
the oracle).  Nu(x) = q'' D_h / (k (T_w - T_m)) with T_w by half-cell extrapolation and
T_m the velocity-weighted bulk temperature (reading R22).

Compared from column 8 on: over the first columns T_w - T_m crosses zero next to the
fixed-temperature inlet column, where Nu is singular (-617 to 776 in the oracle's).
Tolerances, relative L2 over x: FP64 1e-8 (50000 steps of rounding on T, amplified by
T / (T_w - T_m) ~ 100 in Nu; 1.1e-10 measured); FP32 deviation storage 1e-4 (4.4e-6
measured)."""
import json
import os

import numpy as np
import pytest

from _helpers import rel_l2, run_gpu
from paper_2302_04120_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

lbm = pytest.importorskip("paper_2302_04120_gb300.lbm")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "channel_nusselt_2048x256.json")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
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


@pytest.mark.parametrize("prec,tol", [(lbm.LBM_FP64, 1e-8), (lbm.LBM_FP32DEV, 1e-4)])
def test_channel_local_nusselt_against_oracle(prec, tol):
    with open(GOLDEN) as fh:
        g = json.load(fh)
    w = wl.channel()
    assert g["steps"] == w["steps"]
    s = run_gpu(w, prec)
    m = s.moments(lbm.LBM_UX | lbm.LBM_T)
    s.close()
    p = w["params"]
    lower, upper = _local_nusselt(m["T"], m["ux"], w["qflux"], p["k"], p["dx"], w["H"])
    assert np.all(np.isfinite(lower)) and np.all(np.isfinite(upper))
    assert rel_l2(lower[8:], np.array(g["Nu_lower"])[8:]) < tol
    assert rel_l2(upper[8:], np.array(g["Nu_upper"])[8:]) < tol
