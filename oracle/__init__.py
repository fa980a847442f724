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
# the same source built with -DORACLE_EXTENDED: every step in long double (80-bit
# extended on x86-64, binary128 on AArch64), to measure the FP64 rounding floor
_LIB_EXT = os.path.join(_HERE, "liboracle_ext.so")
# the same source built as C++ with -DORACLE_DUAL: every step in forward-mode dual
# numbers (oracle/dual.h), giving exact directional derivatives of the forward map
_LIB_DUAL = os.path.join(_HERE, "liboracle_dual.so")
_DUAL_H = os.path.join(_HERE, "dual.h")

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


def build(force: bool = False, extended: bool = False, dual: bool = False) -> str:
    """Compile the oracle (no FMA contraction, OpenMP over cells): FP64 with gcc, long
    double with ``extended``, or forward-mode dual numbers (g++) with ``dual``."""
    out = _LIB_DUAL if dual else _LIB_EXT if extended else _LIB
    src_time = max(os.path.getmtime(_SRC), os.path.getmtime(_DUAL_H))
    if force or not os.path.exists(out) or os.path.getmtime(out) < src_time:
        if dual:
            cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                   "-x", "c++", "-DORACLE_DUAL", "-I", _HERE, _SRC, "-o", out + ".tmp", "-lm"]
        else:
            cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                   *(["-DORACLE_EXTENDED"] if extended else []), _SRC, "-o", out + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)
    return out


_libs = {}


def lib(extended: bool = False, dual: bool = False):
    key = "dual" if dual else "ext" if extended else "fp64"
    if key not in _libs:
        L = C.CDLL(build(extended=extended, dual=dual))
        d = C.POINTER(C.c_double)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(OrcParams)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_constants.argtypes = [C.c_void_p, d]
        L.orc_matrix.argtypes = [C.c_void_p, C.c_int, d]
        L.orc_set_bc.argtypes = [C.c_void_p, C.c_int, C.c_int, d, C.c_double, C.c_int, d]
        L.orc_set_source.argtypes = [C.c_void_p, d, d]
        L.orc_init.argtypes = [C.c_void_p, d, d, d, d]
        L.orc_step.argtypes = [C.c_void_p, C.c_long]
        L.orc_moments.argtypes = [C.c_void_p, d, d, d, d, d, d]
        L.orc_get_dist.argtypes = [C.c_void_p, C.c_int, C.c_int, d]
        L.orc_set_dist.argtypes = [C.c_void_p, C.c_int, d]
        L.orc_steps.restype = C.c_long
        L.orc_steps.argtypes = [C.c_void_p]
        if dual:
            L.orc_seed.argtypes = [C.c_void_p, C.c_double, d, d]
            L.orc_tangent.argtypes = [C.c_void_p, d, d, d]
        _libs[key] = L
    return _libs[key]


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
    Distributions come back as (q, ny, nx).  ``extended=True`` runs the same steps
    in long double; ``dual=True`` in forward-mode dual numbers (``seed`` and
    ``tangent``); inputs and outputs stay FP64 in every build.
    """

    def __init__(self, params: dict, extended: bool = False, dual: bool = False):
        self._L = lib(extended, dual)
        self.extended, self.dual = extended, dual
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
        self.h = self._L.orc_create(C.byref(s))
        if not self.h:
            raise MemoryError("oracle allocation failed")

    def close(self):
        if self.h:
            self._L.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- set-up -----------------------------------------------------------
    def constants(self):
        out = np.zeros(5)
        self._L.orc_constants(self.h, _ptr(out))
        return dict(c=out[0], cs2=out[1], tau=out[2], tauT=out[3], tauphi=out[4])

    def matrix(self, which: int):
        n = 81 if which in (0, 1, 4) else 25
        out = np.zeros(n)
        self._L.orc_matrix(self.h, which, _ptr(out))
        m = int(round(np.sqrt(n)))
        return out.reshape(m, m)

    def set_bc(self, side, kind, uw=None, rho_w=None, tkind=TBC_NONE, tw=None):
        ln = self.ny if side < 2 else self.nx
        uw = _arr(uw, 2 * ln)
        tw = _arr(tw, ln)
        rw = self.p["rho0"] if rho_w is None else rho_w
        self._L.orc_set_bc(self.h, side, kind, _ptr(uw), float(rw), tkind, _ptr(tw))

    def set_source(self, q3=None, force=None):
        n = self.nx * self.ny
        self._q3 = _arr(q3, n)
        self._force = _arr(force, 2 * n)
        self._L.orc_set_source(self.h, _ptr(self._q3), _ptr(self._force))

    def init(self, a=None, ux=None, uy=None, b=None):
        n = self.nx * self.ny
        self._L.orc_init(self.h, _ptr(_arr(a, n)), _ptr(_arr(ux, n)), _ptr(_arr(uy, n)),
                       _ptr(_arr(b, n)))

    # --- stepping and output ----------------------------------------------
    def step(self, n: int):
        self._L.orc_step(self.h, int(n))

    @property
    def steps(self):
        return self._L.orc_steps(self.h)

    def moments(self):
        shp = (self.ny, self.nx)
        out = {k: np.zeros(shp) for k in ("rho", "ux", "uy", "T", "p", "phi")}
        self._L.orc_moments(self.h, *[_ptr(out[k]) for k in ("rho", "ux", "uy", "T", "p", "phi")])
        return out

    def dist(self, which: str, post: bool = False):
        w = {"f": 0, "g": 1, "h": 2, "z": 3}[which]
        q = 9 if w in (0, 3) or (w == 1 and int(self.p["thermal"]) == 9) else 5
        out = np.zeros((q, self.ny, self.nx))
        self._L.orc_get_dist(self.h, w, int(post), _ptr(out))
        return out

    def seed(self, dnu=0.0, dq3=None, dqwall=None):
        """Direction of one derivative (dual build): d nu, a direction of the heat-source
        field (ny, nx) and one of the wall flux (2, nx) for the y- and y+ sides.  Call
        after set_bc / set_source and before step."""
        assert self.dual
        n = self.nx * self.ny
        self._dq3 = _arr(dq3, n)
        self._dqw = _arr(dqwall, 2 * self.nx)
        self._L.orc_seed(self.h, float(dnu), _ptr(self._dq3), _ptr(self._dqw))

    def tangent(self):
        """Derivatives of u_x, u_y and T along the seeded direction (dual build)."""
        assert self.dual
        shp = (self.ny, self.nx)
        out = {k: np.zeros(shp) for k in ("ux", "uy", "T")}
        self._L.orc_tangent(self.h, *[_ptr(out[k]) for k in ("ux", "uy", "T")])
        return out

    def set_dist(self, which: str, arr):
        w = {"f": 0, "g": 1, "h": 2, "z": 3}[which]
        q = 9 if w in (0, 3) or (w == 1 and int(self.p["thermal"]) == 9) else 5
        a = _arr(arr, q * self.nx * self.ny)
        self._L.orc_set_dist(self.h, w, _ptr(a))


def e2_percent(ref, num):
    """Relative L2 error norm E2 in percent, Eq. error_norm_2 (Sec. 4)."""
    ref = np.asarray(ref, dtype=np.float64)
    num = np.asarray(num, dtype=np.float64)
    return 100.0 * np.sqrt(np.sum((ref - num) ** 2) / np.sum(ref ** 2))


def outlet_loss_jvp(w, steps, T_target, dnu=0.0, dq3=None, dqwall=None):
    """The outlet-temperature loss L = mean_j (T(nx - 1, j; steps) - T_target[j])^2 of a
    single-phase thermal solve (workload dict w: params, bcs, init, q3) and its exact
    directional derivative along (dnu, dq3 (ny, nx), dqwall (2, nx)), from one run of
    the oracle's forward-mode dual-number build.  Returns (L, dL)."""
    p = w["params"]
    ny = int(p["ny"])
    T_target = np.asarray(T_target, dtype=np.float64)
    o = Oracle(p, dual=True)
    for bc in w["bcs"]:
        o.set_bc(*bc)
    if w.get("q3") is not None:
        o.set_source(q3=w["q3"])
    o.seed(dnu=dnu, dq3=dq3, dqwall=dqwall)
    o.init(**(w.get("init") or {}))
    o.step(steps)
    T = o.moments()["T"][:, -1]
    dT = o.tangent()["T"][:, -1]
    o.close()
    e = T - T_target
    return float(np.mean(e ** 2)), float((2.0 * e / ny) @ dT)


def outlet_loss_gradient(w, steps, T_target, q3=True, qwall=True, nu=True):
    """Reference gradient of the outlet-temperature loss
    L = mean_j (T(nx - 1, j; steps) - T_target[j])^2 of a single-phase thermal solve
    (workload dict w: params, bcs, init, q3), by forward-mode dual numbers: one
    directional derivative of the whole run per input element, each exact to
    rounding.  Inputs: the heat-source field (Eq. forcing_term_g via
    qdot = q3/(rho c_p)), the heat flux of the y- and y+ walls (Eq. BB_T) and the
    kinematic viscosity (Eq. eq_kinematic_viscosity).  Returns (L, dL/dq3 (ny, nx),
    dL/dqwall (2, nx), dL/dnu); the parts not asked for are None."""
    p = w["params"]
    nx, ny = int(p["nx"]), int(p["ny"])
    loss, _ = outlet_loss_jvp(w, steps, T_target)
    g3 = gw = gnu = None
    if q3:
        g3 = np.zeros((ny, nx))
        for j in range(ny):
            for i in range(nx):
                e = np.zeros((ny, nx))
                e[j, i] = 1.0
                g3[j, i] = outlet_loss_jvp(w, steps, T_target, dq3=e)[1]
    if qwall:
        gw = np.zeros((2, nx))
        for s in range(2):
            for i in range(nx):
                e = np.zeros((2, nx))
                e[s, i] = 1.0
                gw[s, i] = outlet_loss_jvp(w, steps, T_target, dqwall=e)[1]
    if nu:
        gnu = outlet_loss_jvp(w, steps, T_target, dnu=1.0)[1]
    return loss, g3, gw, gnu
