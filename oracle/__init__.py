"""ctypes wrapper of the plain FP64 CPU oracle (``oracle/lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers.  The CUDA library never imports this package and this package never
imports the CUDA library; the two share only the seeded input generators of
``paper_2302_04120_gb300.workloads`` (which hold none of the method's
arithmetic).

Paper: Martins, Alvarino & Cabezas-Gomez, arXiv:2302.04120.  Each function of
the C file cites the section/equation it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

BC_PERIODIC, BC_WALL, BC_VELOCITY, BC_PRESSURE, BC_SYMMETRY = 0, 1, 2, 3, 4
TBC_NONE, TBC_FLUX, TBC_TEMP, TBC_OUTFLOW, TBC_SYMMETRY, TBC_WETNODE = 0, 1, 2, 3, 4, 5


class OrcParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("flow", C.c_int), ("flow_op", C.c_int),
        ("thermal", C.c_int), ("thermal_op", C.c_int), ("phase", C.c_int), ("z_op", C.c_int),
        ("nu_rule", C.c_int), ("literal", C.c_int),
        ("dx", C.c_double), ("dt", C.c_double),
        ("rho0", C.c_double), ("nu", C.c_double), ("cp", C.c_double), ("k", C.c_double),
        ("T0", C.c_double),
        ("rho_l", C.c_double), ("rho_g", C.c_double), ("nu_l", C.c_double), ("nu_g", C.c_double),
        ("sigma", C.c_double), ("W", C.c_double), ("mobility", C.c_double),
        ("omega_e_dt", C.c_double), ("omega_eps_dt", C.c_double),
        ("Fb", C.c_double * 2), ("u_prescribed", C.c_double * 2),
        ("conv_coef", C.c_double), ("T_inf", C.c_double),
        ("gravity", C.c_double * 2), ("beta_exp", C.c_double), ("T_ref", C.c_double), ("rho_ref", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP over cells)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
               _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d = C.POINTER(C.c_double)
        _lib.orc_create.restype = C.c_void_p
        _lib.orc_create.argtypes = [C.POINTER(OrcParams)]
        _lib.orc_destroy.argtypes = [C.c_void_p]
        _lib.orc_constants.argtypes = [C.c_void_p, d]
        _lib.orc_matrix.argtypes = [C.c_void_p, C.c_int, d]
        _lib.orc_set_bc.argtypes = [C.c_void_p, C.c_int, C.c_int, d, C.c_double, C.c_int, d]
        _lib.orc_set_source.argtypes = [C.c_void_p, d, d]
        _lib.orc_init.argtypes = [C.c_void_p, d, d, d, d]
        _lib.orc_step.argtypes = [C.c_void_p, C.c_long]
        _lib.orc_moments.argtypes = [C.c_void_p, d, d, d, d, d, d]
        _lib.orc_get_dist.argtypes = [C.c_void_p, C.c_int, C.c_int, d]
        _lib.orc_set_dist.argtypes = [C.c_void_p, C.c_int, d]
        _lib.orc_steps.restype = C.c_long
        _lib.orc_steps.argtypes = [C.c_void_p]
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _arr(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None:
        assert a.size == n, (a.size, n)
    return a


_PARAM_KEYS = [f[0] for f in OrcParams._fields_]
_DEFAULTS = dict(flow=9, flow_op=0, thermal=0, thermal_op=0, phase=0, z_op=1, nu_rule=0,
                 literal=0, rho0=1000.0, nu=1e-6, cp=4180.0, k=0.6, T0=300.0, rho_l=0.0,
                 rho_g=0.0, nu_l=0.0, nu_g=0.0, sigma=0.0, W=1.0, mobility=0.0,
                 omega_e_dt=1.0, omega_eps_dt=1.0, Fb=(0.0, 0.0), u_prescribed=(0.0, 0.0),
                 conv_coef=0.0, T_inf=0.0, gravity=(0.0, 0.0), beta_exp=0.0, T_ref=0.0, rho_ref=0.0)


class Oracle:
    """One oracle solve.  ``params`` is a dict of SI quantities (see ``OrcParams``).

    Grid fields are numpy arrays of shape (ny, nx) (row j = y index).
    Distributions come back as (q, ny, nx).
    """

    def __init__(self, params: dict):
        full = dict(_DEFAULTS)
        full.update({k: v for k, v in params.items() if k in _PARAM_KEYS})
        self.p = full
        s = OrcParams()
        for k in _PARAM_KEYS:
            v = full[k]
            if k in ("Fb", "u_prescribed", "gravity"):
                getattr(s, k)[0] = float(v[0])
                getattr(s, k)[1] = float(v[1])
            else:
                setattr(s, k, v)
        self._s = s
        self.nx, self.ny = int(full["nx"]), int(full["ny"])
        self.h = lib().orc_create(C.byref(s))
        if not self.h:
            raise MemoryError("oracle allocation failed")

    def close(self):
        if self.h:
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- set-up -----------------------------------------------------------
    def constants(self):
        out = np.zeros(5)
        lib().orc_constants(self.h, _ptr(out))
        return dict(c=out[0], cs2=out[1], tau=out[2], tauT=out[3], tauphi=out[4])

    def matrix(self, which: int):
        n = 81 if which in (0, 1, 4) else 25
        out = np.zeros(n)
        lib().orc_matrix(self.h, which, _ptr(out))
        m = int(round(np.sqrt(n)))
        return out.reshape(m, m)

    def set_bc(self, side, kind, uw=None, rho_w=None, tkind=TBC_NONE, tw=None):
        ln = self.ny if side < 2 else self.nx
        uw = _arr(uw, 2 * ln)
        tw = _arr(tw, ln)
        rw = self.p["rho0"] if rho_w is None else rho_w
        lib().orc_set_bc(self.h, side, kind, _ptr(uw), float(rw), tkind, _ptr(tw))

    def set_source(self, q3=None, force=None):
        n = self.nx * self.ny
        self._q3 = _arr(q3, n)
        self._force = _arr(force, 2 * n)
        lib().orc_set_source(self.h, _ptr(self._q3), _ptr(self._force))

    def init(self, a=None, ux=None, uy=None, b=None):
        n = self.nx * self.ny
        lib().orc_init(self.h, _ptr(_arr(a, n)), _ptr(_arr(ux, n)), _ptr(_arr(uy, n)),
                       _ptr(_arr(b, n)))

    # --- stepping and output ----------------------------------------------
    def step(self, n: int):
        lib().orc_step(self.h, int(n))

    @property
    def steps(self):
        return lib().orc_steps(self.h)

    def moments(self):
        shp = (self.ny, self.nx)
        out = {k: np.zeros(shp) for k in ("rho", "ux", "uy", "T", "p", "phi")}
        lib().orc_moments(self.h, *[_ptr(out[k]) for k in ("rho", "ux", "uy", "T", "p", "phi")])
        return out

    def dist(self, which: str, post: bool = False):
        w = {"f": 0, "g": 1, "h": 2, "z": 3}[which]
        q = 9 if w in (0, 3) or (w == 1 and int(self.p["thermal"]) == 9) else 5
        out = np.zeros((q, self.ny, self.nx))
        lib().orc_get_dist(self.h, w, int(post), _ptr(out))
        return out

    def set_dist(self, which: str, arr):
        w = {"f": 0, "g": 1, "h": 2, "z": 3}[which]
        q = 9 if w in (0, 3) or (w == 1 and int(self.p["thermal"]) == 9) else 5
        a = _arr(arr, q * self.nx * self.ny)
        lib().orc_set_dist(self.h, w, _ptr(a))


def e2_percent(ref, num):
    """Relative L2 error norm E2 in percent, Eq. error_norm_2 (Sec. 4)."""
    ref = np.asarray(ref, dtype=np.float64)
    num = np.asarray(num, dtype=np.float64)
    return 100.0 * np.sqrt(np.sum((ref - num) ** 2) / np.sum(ref ** 2))
