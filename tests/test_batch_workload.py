"""The batched workload at its configuration: 256 independent forced-convection
channels of uneven size (numpy PCG64 seed 4: Nx ~ U{128..4096}, Ny ~ U{32..512},
Re ~ U(10, 200), Pr in {0.7, 7}; D2Q9 MRT + D2Q5 MRT, water, q'' = 4e4 W m^-2), FP32
deviation storage, one launch per step with the autotuned tile, 5000 steps.

A seeded sample of 16 of the channels (np.random.default_rng(0).choice(256, 16)) is
compared element by element with the FP64 oracle's run of the same channels
(tests/golden/batch_sample_seed4.npz, written by make_batch_sample.py, which calls only
the oracle): u_x, u_y and T - T_in on every 4th row and 8th column and on the whole
outlet column, 1e-5 relative L2 per channel (the FP32 contract), u relative to the
channel's largest speed.  Measured: at most 9.5e-7 (u_x), 4.4e-7 (u_y), 5.7e-6
(T - T_in) over the 16 channels."""
import os

import numpy as np
import pytest

from _helpers import rel_l2
from paper_2302_04120_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

lbm = pytest.importorskip("paper_2302_04120_gb300.lbm")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "batch_sample_seed4.npz")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not os.path.exists(GOLDEN):
        pytest.skip("oracle fixture not written yet: run its script under tests/golden/")
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_04120_gb300 import build
    build.build()


def test_batched_workload_sample_against_oracle():
    ref = np.load(GOLDEN)
    ws = wl.channel_batch(steps=5000)
    assert len(ws) == 256
    b = lbm.Batch([w["params"] for w in ws], precision=lbm.LBM_FP32DEV)
    for ch, w in zip(b.channels, ws):
        for bc in w["bcs"]:
            ch.set_bc(*bc)
        ch.init(**w["init"])
    b.step(10)
    b.autotune()
    b.step(4990)
    sample = np.sort(np.random.default_rng(0).choice(256, 16, replace=False))
    for k in sample:
        m = b.channels[k].moments(lbm.LBM_UX | lbm.LBM_UY | lbm.LBM_T)
        assert b.channels[k].steps == 5000
        got = dict(ux=m["ux"], uy=m["uy"], dT=m["T"] - ws[k]["T_in"])
        sp = np.hypot(ref[f"{k}_ux"], ref[f"{k}_uy"])
        sp_out = np.hypot(ref[f"{k}_ux_outlet"], ref[f"{k}_uy_outlet"])
        for name in ("ux", "uy", "dT"):
            g = got[name]
            r, r_out = ref[f"{k}_{name}"], ref[f"{k}_{name}_outlet"]
            scale, scale_out = (sp, sp_out) if name != "dT" else (r, r_out)
            assert rel_l2(g[::4, ::8], r, scale) < 1e-5, (k, name, rel_l2(g[::4, ::8], r, scale))
            assert rel_l2(g[:, -1], r_out, scale_out) < 1e-5, (k, name)
    for ch in b.channels:
        assert ch.check() == lbm.LBM_OK
    b.close()
