"""The allocation-free integrals entry point agrees with lbm_integrals.

lbm_field_integrals_noalloc serves callers that cannot call cudaMalloc (code
inside a memory pool or arena that owns the device, under an allocator that
forbids foreign allocations, or where an allocation's implicit synchronisation
is not allowed).  It reduces macroscopic fields the caller already holds on the
device, through a fixed static scratch array instead of a per-handle buffer.
This file is named so that pytest collects it last."""
import numpy as np
import pytest

from _helpers import run_gpu
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


def _check_pair(ref, got, umax_tol=1e-12):
    # same tolerance as the FP64 parity tests: 1e-12 relative; max |u| of a
    # single-phase FP32 solve is formed from |u|^2 rounded to FP32 (2^-24 relative)
    assert abs(got[0] - ref[0]) <= 1e-12 * abs(ref[0])
    assert abs(got[1] - ref[1]) <= 1e-12 * max(abs(ref[1]), 1.0)
    assert abs(got[2] - ref[2]) <= umax_tol * ref[2]
    assert got[3] == ref[3]


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_lbm_integrals_single_phase(prec):
    """Forced-convection channel (ragged 100 x 42): two calls in a row on device
    fields from lbm_moments give lbm_integrals' mass, max |u| and health count."""
    import torch
    w = wl.channel(nx=100, ny=42, steps=60, Re=100 * 42 / 256)
    s = run_gpu(w, prec)
    ref = s.integrals()
    fields = torch.empty((3, 42, 100), dtype=torch.float64, device="cuda")
    lbm.lbm_moments(s.h, lbm.LBM_RHO | lbm.LBM_UX | lbm.LBM_UY, fields)
    c = s.constants()["c"]
    for call in range(2):
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        st = lbm.lbm_field_integrals_noalloc(fields[0], fields[1], fields[2], None, 100, 42,
                                             w["params"]["dx"], c, out)
        assert st == lbm.LBM_OK, lbm.lbm_last_error(None)
        torch.cuda.synchronize()
        _check_pair(ref, out.cpu().numpy().tolist(), 1e-12 if prec == 0 else 1.2e-7)


def test_noalloc_matches_lbm_integrals_two_phase():
    """Two-phase bubble: phase sum and mass agree too (two calls in a row, with a
    call on a different grid in between to show the shared scratch is rewritten)."""
    import torch
    w = wl.bubble(n=48, ny=40, R_cells=10.0, W_cells=4.0, steps=20)
    s = run_gpu(w, 0)
    ref = s.integrals()
    m = torch.empty((4, 40, 48), dtype=torch.float64, device="cuda")
    lbm.lbm_moments(s.h, lbm.LBM_RHO | lbm.LBM_UX | lbm.LBM_UY | lbm.LBM_PHI, m)
    c = s.constants()["c"]
    other = torch.ones((3, 5000, 9), dtype=torch.float64, device="cuda")
    for call in range(2):
        out = torch.zeros(4, dtype=torch.float64, device="cuda")
        assert lbm.lbm_field_integrals_noalloc(m[0], m[1], m[2], m[3], 48, 40, w["params"]["dx"], c, out) == 0
        torch.cuda.synchronize()
        _check_pair(ref, out.cpu().numpy().tolist())
        junk = torch.zeros(4, dtype=torch.float64, device="cuda")
        assert lbm.lbm_field_integrals_noalloc(other[0], other[1], other[2], None, 9, 5000, 1.0, 10.0, junk) == 0
        torch.cuda.synchronize()
        assert junk.cpu().numpy().tolist() == [45000.0, 0.0, np.sqrt(2.0), 0.0]


def test_noalloc_rejects_oversize_grid():
    """Grids beyond the static scratch limit are refused before any launch."""
    import ctypes as C
    big_nx, big_ny = 4096, 2049          # 8,392,704 > 4096 * 2048 cells
    fake = C.c_void_p(16)                 # never dereferenced: the size check comes first
    st = lbm.lib().lbm_field_integrals_noalloc(fake, fake, fake, None, big_nx, big_ny, 1.0, 1.0, fake, None)
    assert st == lbm.LBM_ERR_ARG
    assert "static scratch limit" in lbm.lbm_last_error(None)


@pytest.mark.parametrize("two_phase", [False, True])
def test_bad_cell_excluded_everywhere(two_phase):
    """One non-finite population planted through lbm_set_state: lbm_integrals counts
    the cell and leaves it out of the mass and the phase sum; the allocation-free call
    on the moments of the same state gives the same four values (to rounding), and the
    mass equals the sum over the healthy cells of the moments."""
    import torch
    if two_phase:
        w = wl.bubble(n=48, ny=40, R_cells=10.0, W_cells=4.0, steps=20)
    else:
        w = wl.channel(nx=64, ny=24, steps=20, Re=100 * 24 / 256)
    nx, ny = w["params"]["nx"], w["params"]["ny"]
    s = run_gpu(w, 0)
    st = s.get_state().view(np.float64).copy()
    st[5 * nx * ny + 3 * nx + 7] = np.nan          # plane 5, node (7, 3)
    s.set_state(st.view(np.uint8))
    ref = s.integrals()
    assert ref[3] == 1 and np.all(np.isfinite(ref[:3]))
    m = torch.empty((4, ny, nx), dtype=torch.float64, device="cuda")
    lbm.lbm_moments(s.h, lbm.LBM_RHO | lbm.LBM_UX | lbm.LBM_UY | lbm.LBM_PHI, m)
    host = m.cpu().numpy()
    healthy = np.isfinite(host[0]) & np.isfinite(host[1]) & np.isfinite(host[2])
    assert healthy.sum() == nx * ny - 1
    dx = w["params"]["dx"]
    assert abs(ref[0] - host[0][healthy].sum() * dx * dx) <= 1e-12 * ref[0]
    if two_phase:
        assert abs(ref[1] - host[3][healthy].sum()) <= 1e-12 * ref[1]
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    phi = m[3] if two_phase else None
    assert lbm.lbm_field_integrals_noalloc(m[0], m[1], m[2], phi, nx, ny, dx, s.constants()["c"], out) == 0
    torch.cuda.synchronize()
    _check_pair(ref, out.cpu().numpy().tolist())
