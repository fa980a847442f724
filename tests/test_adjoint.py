"""Reverse-time adjoint of the fused step (D2Q9 MRT + D2Q5 MRT, FP64).

Checks: every element of the gradient fields against the oracle's reference
gradient (forward-mode dual numbers); the loss equals the FP64 oracle's; directional
derivatives of the loss
with respect to the heat-source field, the wall heat flux and the viscosity
match central finite differences of the ORACLE's loss (relative step 1e-6) to
1e-4 on a small channel with several checkpoint segments, and central
differences of the GPU forward on the full 1024 x 128 workload; the autograd
wrapper returns the same gradients."""
import os

import numpy as np
import pytest

from _helpers import run_oracle
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


def _with(w, q3=None, qwall=None, nu=None):
    """Copy of workload w with a heat source, wall fluxes (2, nx) and viscosity."""
    w2 = dict(w)
    w2["params"] = dict(w["params"])
    if nu is not None:
        w2["params"]["nu"] = nu
    if q3 is not None:
        w2["q3"] = q3
    if qwall is not None:
        bcs = []
        for side, kind, uw, rw, tk, tw in w["bcs"]:
            if side in (2, 3) and tk == 1:
                tw = qwall[side - 2]
            bcs.append((side, kind, uw, rw, tk, tw))
        w2["bcs"] = bcs
    return w2


def _oracle_loss(w, target):
    T = run_oracle(w).moments()["T"][:, -1]
    return np.mean((T - target) ** 2)


def _gpu_loss(w, target):
    from _helpers import run_gpu
    s = run_gpu(w, 0)
    T = s.moments(lbm.LBM_T)["T"][:, -1]
    s.close()
    return np.mean((T - target) ** 2)


def _adjoint(w, steps, K, target):
    s = lbm.Solver(w["params"], precision=0)
    for bc in w["bcs"]:
        s.set_bc(*bc)
    s.set_source(w["q3"], None)
    s.init(**w["init"])
    out = lbm.lbm_adjoint(s.h, steps, K, target, s.nx, s.ny)
    s.close()
    return out


def _setup_small():
    nx, ny, steps = 40, 12, 120
    w = wl.channel(nx=nx, ny=ny, steps=steps, Re=100 * ny / 256)
    w["q3"] = wl.smooth_source(nx, ny, seed=5, sigma_cells=3.0, scale=1e8)
    base = run_oracle(_with(w, q3=np.zeros((ny, nx)))).moments()["T"][:, -1]
    H = ny * w["params"]["dx"]
    y = (np.arange(ny) + 0.5) * w["params"]["dx"]
    target = base + 0.01 * np.sin(np.pi * y / H)   # adjoint workload target recipe
    qw = np.vstack([np.full(nx, w["qflux"]), np.full(nx, w["qflux"])])
    return w, steps, target, qw


def test_adjoint_small_against_oracle_finite_differences():
    w, steps, target, qw = _setup_small()
    nx, ny = w["params"]["nx"], w["params"]["ny"]
    loss, g3, gw, gnu = _adjoint(w, steps, 25, target)        # 4 full segments + 1 partial
    L0 = _oracle_loss(w, target)
    # L is built from T ~ 300 K: a 1e-12 relative agreement of T (3e-10 K) allows
    # |dL| <= 2 sqrt(L) * 3e-10 K, i.e. ~1e-7 of L here
    assert abs(loss - L0) <= 1e-7 * L0
    rng = np.random.default_rng(21)
    # heat source direction
    # L is quadratic in the sources, so central differences are exact up to rounding;
    # the direction's scale only keeps the rounding of L (~1e-15 K^2) far below dL
    v = rng.standard_normal((ny, nx)) * 1e10
    eps = 1e-6
    Lp = _oracle_loss(_with(w, q3=w["q3"] + eps * v), target)
    Lm = _oracle_loss(_with(w, q3=w["q3"] - eps * v), target)
    fd, ad = (Lp - Lm) / (2 * eps), np.sum(g3 * v)
    assert abs(fd - ad) <= 1e-4 * abs(fd), (fd, ad)
    # wall heat flux direction (both walls)
    d = rng.standard_normal((2, nx)) * 4e7
    Lp = _oracle_loss(_with(w, qwall=qw + eps * d), target)
    Lm = _oracle_loss(_with(w, qwall=qw - eps * d), target)
    fd, ad = (Lp - Lm) / (2 * eps), np.sum(gw * d)
    assert abs(fd - ad) <= 1e-4 * abs(fd), (fd, ad)
    # viscosity (nonlinear: enters the MRT rates)
    nu = w["params"]["nu"]
    h = 1e-6 * nu
    Lp = _oracle_loss(_with(w, nu=nu + h), target)
    Lm = _oracle_loss(_with(w, nu=nu - h), target)
    fd = (Lp - Lm) / (2 * h)
    assert abs(fd - gnu) <= 1e-4 * abs(fd), (fd, gnu)


def test_adjoint_small_elementwise_against_oracle_gradient():
    """Every element of the GPU's gradient with respect to the heat source (40 x 12
    cells) and the wall flux (2 x 40 wall nodes), and dL/dnu, against the oracle's
    reference gradient: one forward-mode dual-number run of the oracle per input
    element, exact up to rounding (pinned in test_oracle_builds.py).  Bound 1e-8
    relative max-norm; the loss to 1e-7 (it is built from T ~ 300 K)."""
    import oracle
    from _helpers import rel_max
    w, steps, target, qw = _setup_small()
    loss, g3, gw, gnu = _adjoint(w, steps, 25, target)
    L, r3, rw, rnu = oracle.outlet_loss_gradient(w, steps, target)
    assert abs(loss - L) <= 1e-7 * L
    assert rel_max(g3, r3) < 1e-8
    assert rel_max(gw, rw) < 1e-8
    assert abs(gnu - rnu) <= 1e-8 * abs(rnu)


def test_adjoint_checkpoint_interval_does_not_change_the_gradient():
    w, steps, target, qw = _setup_small()
    a = _adjoint(w, steps, 25, target)
    b = _adjoint(w, steps, 7, target)
    c = _adjoint(w, steps, steps, target)
    for x in (b, c):
        assert np.array_equal(a[1], x[1]) and np.array_equal(a[2], x[2]) and a[3] == x[3] and a[0] == x[0]


def test_adjoint_full_workload_against_gpu_finite_differences():
    """1024 x 128 channel, 2000 steps, checkpoints every 100 (the adjoint workload)."""
    w = wl.adjoint_channel()
    nx, ny, steps = 1024, 128, 2000
    base = _gpu_loss_field(_with(w, q3=np.zeros((ny, nx))))
    H = ny * w["params"]["dx"]
    y = (np.arange(ny) + 0.5) * w["params"]["dx"]
    target = base + 0.01 * np.sin(np.pi * y / H)
    loss, g3, gw, gnu = _adjoint(w, steps, 100, target)
    assert abs(loss - _gpu_loss(w, target)) <= 1e-12 * loss
    rng = np.random.default_rng(22)
    v = rng.standard_normal((ny, nx)) * 1e9
    eps = 1e-6
    fd = (_gpu_loss(_with(w, q3=w["q3"] + eps * v), target) - _gpu_loss(_with(w, q3=w["q3"] - eps * v), target)) / (2 * eps)
    assert abs(fd - np.sum(g3 * v)) <= 1e-4 * abs(fd)
    qw = np.vstack([np.full(nx, w["qflux"])] * 2)
    d = rng.standard_normal((2, nx)) * 4e7
    fd = (_gpu_loss(_with(w, qwall=qw + eps * d), target) - _gpu_loss(_with(w, qwall=qw - eps * d), target)) / (2 * eps)
    assert abs(fd - np.sum(gw * d)) <= 1e-4 * abs(fd)
    nu = w["params"]["nu"]
    h = 1e-6 * nu
    fd = (_gpu_loss(_with(w, nu=nu + h), target) - _gpu_loss(_with(w, nu=nu - h), target)) / (2 * h)
    assert abs(fd - gnu) <= 1e-4 * abs(fd)


def _gpu_loss_field(w):
    from _helpers import run_gpu
    s = run_gpu(w, 0)
    T = s.moments(lbm.LBM_T)["T"][:, -1]
    s.close()
    return T


def test_autograd_function_matches_adjoint():
    import torch
    from paper_2302_04120_gb300.autograd import channel_loss
    w, steps, target, qw = _setup_small()
    q3 = torch.tensor(w["q3"], dtype=torch.float64, requires_grad=True)
    qwall = torch.tensor(qw, dtype=torch.float64, requires_grad=True)
    nu = torch.tensor(w["params"]["nu"], dtype=torch.float64, requires_grad=True)
    L = channel_loss(q3, qwall, nu, w, steps, 25, target)
    (3.0 * L).backward()
    loss, g3, gw, gnu = _adjoint(w, steps, 25, target)
    # forward runs lbm_step, the adjoint its own checkpointed forward: equal to rounding
    assert abs(float(L.detach()) - loss) <= 1e-12 * loss
    np.testing.assert_array_equal(q3.grad.numpy(), 3.0 * g3)
    np.testing.assert_array_equal(qwall.grad.numpy(), 3.0 * gw)
    assert float(nu.grad) == 3.0 * gnu


def test_adjoint_rejects_unsupported_configurations():
    w = wl.channel(nx=20, ny=8, steps=10, Re=100 * 8 / 256, flow_op=0)
    s = lbm.Solver(w["params"], precision=0)
    for bc in w["bcs"]:
        s.set_bc(*bc)
    s.init(**w["init"])
    with pytest.raises(lbm.LbmError):
        lbm.lbm_adjoint(s.h, 10, 5, np.zeros(8), 20, 8)
    w = wl.channel(nx=20, ny=8, steps=10, Re=100 * 8 / 256)
    s = lbm.Solver(w["params"], precision=0)
    for bc in w["bcs"]:
        s.set_bc(*bc)
    s.init(**w["init"])
    s.step(1)
    with pytest.raises(lbm.LbmError):       # not freshly initialised
        lbm.lbm_adjoint(s.h, 10, 5, np.zeros(8), 20, 8)


def test_fp32_adjoint_against_fp64_and_oracle():
    """The adjoint of the FP32 deviation form (forward in FP32 storage, adjoint
    variables in FP32, parameter gradients accumulated in FP64) on the 40 x 12 channel:
    its gradient fields against the FP64 adjoint and the oracle's dual-number gradient,
    relative max-norm within 1e-3 (FP32 rounding of the forward states and of the
    reverse sweep; measured 4.8e-4, 7.0e-4, 5.3e-4), the loss within 2e-3 (L is the
    mean square of T - T_target ~ 0.01 K, and the FP32 forward holds T to a few 1e-6 K:
    7.6e-4 measured)."""
    import oracle
    from _helpers import rel_max
    w, steps, target, qw = _setup_small()
    s = lbm.Solver(w["params"], precision=1)
    for bc in w["bcs"]:
        s.set_bc(*bc)
    s.set_source(w["q3"], None)
    s.init(**w["init"])
    loss, g3, gw, gnu = lbm.lbm_adjoint(s.h, steps, 25, target, s.nx, s.ny)
    s.close()
    L, r3, rw, rnu = oracle.outlet_loss_gradient(w, steps, target)
    d3, dw, dnu = rel_max(g3, r3), rel_max(gw, rw), abs(gnu - rnu) / abs(rnu)
    print(f"FP32 adjoint vs oracle: q3 {d3:.2e}, qwall {dw:.2e}, nu {dnu:.2e}, loss {abs(loss - L) / L:.2e}")
    assert abs(loss - L) <= 2e-3 * L
    assert d3 < 1e-3 and dw < 1e-3 and dnu < 1e-3


ADJ_REF = os.path.join(os.path.dirname(__file__), "golden", "adjoint_reference_1024x128.json")


@pytest.mark.parametrize("prec,tol", [(0, 1e-7), (1, 2e-3)])
def test_adjoint_full_workload_against_oracle_reference(prec, tol):
    """The gradient workload at its configuration (1024 x 128, 2000 steps, checkpoints
    every 100) against exact directional derivatives of the oracle's run of it
    (forward-mode dual numbers, tests/golden/adjoint_reference_1024x128.json, written by
    make_adjoint_reference.py, which calls only the oracle): the loss, dL/dnu, dL/dq'''
    at three sampled cells and along a smooth direction, dL/dq'' at two sampled wall
    nodes.  FP64 within 1e-7 of each value: the oracle stores T ~ 300 K itself, and over
    2000 steps its rounding moves T - T_target (~7e-3 K at the outlet) by ~1e-10 K, i.e.
    ~1e-8 of the derivatives (1.0e-8 measured on dL/dnu; the 40 x 12 test above holds
    1e-8 element by element).  FP32 (its gradient is that of the FP32 forward map, whose
    stored T deviations carry ~1e-6 K of rounding against T - T_target ~ 7e-3 K): the
    loss within 2e-3 (2.1e-4 measured), the loss-wide derivatives (nu and the smooth
    heat-source direction) within 2e-3 (9.3e-4 measured on dL/dnu), the single cells and
    wall nodes within 1.5e-2 of the largest value of their group (cells 6.3e-4, wall
    nodes 3.2e-3 and 8.8e-3 measured; the FP64 kernels on the same device hold 1e-8, so
    the spread is the FP32 arithmetic's, not the adjoint's)."""
    import json
    if not os.path.exists(ADJ_REF):
        pytest.skip("oracle fixture not written yet: run tests/golden/make_adjoint_reference.py")
    with open(ADJ_REF) as fh:
        ref = json.load(fh)
    w = wl.adjoint_channel()
    nx, ny = w["params"]["nx"], w["params"]["ny"]
    assert ref["steps"] == w["steps"] == 2000
    target = np.array(ref["target"])
    s = lbm.Solver(w["params"], precision=prec)
    for bc in w["bcs"]:
        s.set_bc(*bc)
    s.set_source(w["q3"], None)
    s.init(**w["init"])
    loss, g3, gw, gnu = lbm.lbm_adjoint(s.h, 2000, 100, target, nx, ny)
    s.close()
    assert abs(loss - ref["loss"]) <= (1e-7 if prec == 0 else 2e-3) * ref["loss"]
    assert abs(gnu - ref["dL_dnu"]) <= tol * abs(ref["dL_dnu"])
    d = wl.smooth_source(nx, ny, seed=ref["q3_direction"]["seed"], scale=1.0)
    assert abs(np.sum(g3 * d) - ref["q3_direction"]["dL"]) <= tol * abs(ref["q3_direction"]["dL"])
    tol_el = tol if prec == 0 else 1.5e-2
    for group, get in ((ref["q3_cells"], lambda c: g3[c["j"], c["i"]]),
                       (ref["qwall_nodes"], lambda c: gw[c["side"], c["i"]])):
        scale = max(abs(c["dL"]) for c in group) if prec == 1 else None
        for c in group:
            assert abs(get(c) - c["dL"]) <= tol_el * (abs(c["dL"]) if scale is None else scale), (c, get(c))
