"""The C-ABI library loads and exports every symbol that include/*.h declares;
host-side argument validation works without a GPU (no compute call is made)."""
import ctypes as C
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2302_04120_gb300 import build
    return build.build()


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(lbm_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_core_entry_points():
    names = _declared_functions()
    for req in ("lbm_create", "lbm_set_source", "lbm_set_bc", "lbm_step", "lbm_moments", "lbm_destroy",
                "lbm_init_fields", "lbm_integrals"):
        assert req in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [n for n in _declared_functions() if n not in exported]
    assert not missing, missing
    lib = C.CDLL(built)
    for n in _declared_functions():
        assert hasattr(lib, n)


def test_params_struct_layout_matches_header(built, tmp_path):
    """ctypes mirror of lbm_params has the C layout (sizeof and offsets)."""
    from paper_2302_04120_gb300 import lbm
    src = tmp_path / "layout.c"
    fields = [f[0] for f in lbm.lbm_params._fields_]
    body = "\n".join(f'printf("{f} %zu\\n", offsetof(lbm_params, {f}));' for f in fields)
    src.write_text(f'#include <stdio.h>\n#include <stddef.h>\n#include "lbm.h"\nint main(void){{'
                   f'printf("sizeof %zu\\n", sizeof(lbm_params));{body}return 0;}}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    rows = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    assert int(rows["sizeof"]) == C.sizeof(lbm.lbm_params)
    for f in fields:
        assert int(rows[f]) == getattr(lbm.lbm_params, f).offset, f


def test_create_rejects_bad_parameters_without_gpu(built):
    """Validation happens before any CUDA call, so these run on a CPU-only host."""
    from paper_2302_04120_gb300 import lbm
    L = lbm.lib()
    h = C.c_void_p()

    def create(**kw):
        p = lbm.lbm_params_default()
        p.nx, p.ny, p.dx, p.dt = 8, 8, 1e-5, 1e-6
        for k, v in kw.items():
            setattr(p, k, v)
        return L.lbm_create(C.byref(p), None, C.byref(h))

    assert create(nx=0) == lbm.LBM_ERR_ARG
    assert b"nx" in L.lbm_last_error(None)
    assert create(dt=-1.0) == lbm.LBM_ERR_ARG
    assert create(nu=0.0) == lbm.LBM_ERR_UNSTABLE_TAU
    assert create(nu=-1e-6) == lbm.LBM_ERR_UNSTABLE_TAU
    assert create(flow=7) == lbm.LBM_ERR_ARG
    assert create(precision=5) == lbm.LBM_ERR_ARG
    assert create(flow=0, thermal=0) == lbm.LBM_ERR_ARG
    assert create(phase=5) == lbm.LBM_ERR_ARG           # two-phase without properties
    assert create(omega_e_dt=2.5) == lbm.LBM_ERR_ARG
    assert create(thermal=5, k=0.0) == lbm.LBM_ERR_UNSTABLE_TAU
    assert h.value is None
    assert L.lbm_create(None, None, C.byref(h)) == lbm.LBM_ERR_ARG


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2302_04120_gb300 import lbm
    monkeypatch.setattr(lbm, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(lbm, "_lib", None)
    with pytest.raises(RuntimeError):
        lbm.lib()


def test_noalloc_binding_checks_arguments_without_gpu():
    """The binding of lbm_field_integrals_noalloc refuses tensors the kernel would read
    past (wrong dtype, strided, too short, out4 too short) or that are not on a CUDA
    device, before any C call: these run on a CPU-only host."""
    torch = pytest.importorskip("torch")
    from paper_2302_04120_gb300 import lbm
    nx, ny = 6, 5
    good = torch.zeros(nx * ny, dtype=torch.float64)
    out = torch.zeros(4, dtype=torch.float64)
    cases = [
        ((good.float(), good, good, None, out), "float64"),
        ((good, torch.zeros(2 * nx * ny, dtype=torch.float64)[::2], good, None, out), "contiguous"),
        ((good, good, good[:-1], None, out), "values"),
        ((good, good, good, good[:3], out), "values"),
        ((good, good, good, None, out[:3]), "values"),
        ((good, good, good, None, [0.0] * 4), "torch tensor"),
        ((good, good, good, None, out), "CUDA"),
    ]
    for (rho, ux, uy, phi, o), msg in cases:
        with pytest.raises(ValueError, match=msg):
            lbm.lbm_field_integrals_noalloc(rho, ux, uy, phi, nx, ny, 1e-6, 1.0, o)
    with pytest.raises(ValueError):
        lbm.lbm_field_integrals_noalloc(good, good, good, None, 0, ny, 1e-6, 1.0, out)
