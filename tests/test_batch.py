"""Batched solves (many uneven channels, one launch per step, graph replay,
autotuned tiles) against the same channels stepped one by one and against the
FP64 oracle."""
import numpy as np
import pytest

from _helpers import rel_max, run_oracle
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


def _small_batch(count=7, seed=4):
    """Seeded uneven channels in the workload's recipe, shrunk for the oracle."""
    return wl.channel_batch(count=count, seed=seed, steps=0, nx_range=(20, 260), ny_range=(6, 70))


def _setup(solver, w):
    for bc in w["bcs"]:
        solver.set_bc(*bc)
    solver.init(**w["init"])


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_equals_one_by_one(prec):
    """57 steps (pre-collision first step, parity alignment, graph pairs and a
    trailing single step): every channel equals the same channel stepped alone to
    rounding -- 1e-13 (FP64) or 1e-6 (FP32) of each field's magnitude.  The batched
    and the single-solve kernels inline the same arithmetic in different contexts,
    and the compiler may contract a different pair of operations into an FMA."""
    ws = _small_batch()
    b = lbm.Batch([w["params"] for w in ws], precision=prec)
    for ch, w in zip(b.channels, ws):
        _setup(ch, w)
    b.step(57)
    for k, w in enumerate(ws):
        s = lbm.Solver(w["params"], precision=prec)
        _setup(s, w)
        s.step(57)
        a, r = b.channels[k].moments(), s.moments()
        for key in ("ux", "uy", "T", "rho"):
            # T and rho relative to their absolute values (FP32 holds T ~ 300 K to
            # ~2e-5 K), velocities relative to the largest speed
            scale = np.max(np.hypot(r["ux"], r["uy"])) if key in ("ux", "uy") else np.max(np.abs(r[key]))
            tol = 1e-13 if prec == 0 else 1e-6
            assert np.max(np.abs(a[key] - r[key])) <= tol * scale, (k, key, np.max(np.abs(a[key] - r[key])))
        assert b.channels[k].steps == 57


def test_batch_autotune_keeps_solution_and_matches_oracle():
    ws = _small_batch(count=5, seed=9)
    b = lbm.Batch([w["params"] for w in ws], precision=0)
    for ch, w in zip(b.channels, ws):
        _setup(ch, w)
    b.step(10)
    cfg = b.autotune()
    assert cfg[0] * cfg[1] % 32 == 0 and cfg[2] >= 1
    b.step(30)
    for k in (0, 3):
        o = run_oracle(dict(ws[k], steps=40))
        mo, mg = o.moments(), b.channels[k].moments()
        sp = np.hypot(mo["ux"], mo["uy"])
        assert rel_max(mg["ux"], mo["ux"], sp) < 1e-12
        assert rel_max(mg["T"], mo["T"]) < 1e-12


def test_batch_rejects_mixed_configurations():
    ws = _small_batch(count=2)
    p0 = dict(ws[0]["params"])
    p1 = dict(ws[1]["params"], thermal_op=0)
    with pytest.raises(lbm.LbmError):
        lbm.Batch([p0, p1])
    b = lbm.Batch([p0, dict(ws[1]["params"])])
    _setup(b.channels[0], ws[0])
    with pytest.raises(lbm.LbmError):   # channel 1 not initialised
        b.step(1)
