"""Thin Python binding of the C ABI in ``include/lbm.h`` (ctypes).

Argument marshalling only: every step of the solver runs in the CUDA kernels of
``liblbm.so``.  Functions carry the C names; ``Solver`` wraps a handle for
convenience.  Host arrays are numpy float64 arrays of shape (ny, nx); device
arrays may be torch CUDA float64 tensors (their data pointer is passed with
``on_device=1``).  There is no CPU fallback: if the library is missing this
module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbm.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_UNSTABLE_TAU, LBM_ERR_NOMEM = 0, -1, -2, -3
LBM_ERR_CUDA, LBM_ERR_DIVERGED, LBM_ERR_TIMEOUT, LBM_ERR_STATE = -4, -5, -6, -7
LBM_NONE, LBM_D2Q5, LBM_D2Q9 = 0, 5, 9
LBM_BGK, LBM_MRT = 0, 1
LBM_FP64, LBM_FP32DEV = 0, 1
LBM_BC_PERIODIC, LBM_BC_WALL, LBM_BC_VELOCITY, LBM_BC_PRESSURE, LBM_BC_SYMMETRY = 0, 1, 2, 3, 4
LBM_TBC_NONE, LBM_TBC_FLUX, LBM_TBC_TEMP, LBM_TBC_OUTFLOW, LBM_TBC_SYMMETRY, LBM_TBC_WETNODE = 0, 1, 2, 3, 4, 5
LBM_RHO, LBM_UX, LBM_UY, LBM_T, LBM_P, LBM_PHI = 1, 2, 4, 8, 16, 32
LBM_LAUNCH_GRID, LBM_LAUNCH_TMA, LBM_LAUNCH_GRID_OCC = 0, 1, 2
_MOMENT_BITS = [("rho", 1), ("ux", 2), ("uy", 4), ("T", 8), ("p", 16), ("phi", 32)]


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"lbm status {status}: {msg}")
        self.status = status


class lbm_params(C.Structure):
    _fields_ = [
        ("flow", C.c_int), ("flow_op", C.c_int), ("thermal", C.c_int), ("thermal_op", C.c_int),
        ("phase", C.c_int), ("z_op", C.c_int), ("nu_rule", C.c_int), ("literal", C.c_int),
        ("precision", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
        ("dx", C.c_double), ("dt", C.c_double),
        ("rho0", C.c_double), ("nu", C.c_double), ("cp", C.c_double), ("k", C.c_double),
        ("T0", C.c_double),
        ("rho_l", C.c_double), ("rho_g", C.c_double), ("nu_l", C.c_double), ("nu_g", C.c_double),
        ("sigma", C.c_double), ("W", C.c_double), ("mobility", C.c_double),
        ("omega_e_dt", C.c_double), ("omega_eps_dt", C.c_double),
        ("body_force", C.c_double * 2), ("u_prescribed", C.c_double * 2),
        ("gravity", C.c_double * 2), ("beta_exp", C.c_double), ("T_ref", C.c_double), ("rho_ref", C.c_double),
    ]


_lib = None
_dp = C.POINTER(C.c_double)


def lib():
    """Load liblbm.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2302_04120_gb300.build.build() first")
        L = C.CDLL(LIB_PATH)
        L.lbm_params_default.argtypes = [C.POINTER(lbm_params)]
        L.lbm_params_default.restype = None
        L.lbm_create.argtypes = [C.POINTER(lbm_params), C.c_void_p, C.POINTER(C.c_void_p)]
        L.lbm_set_bc.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_double, C.c_int, C.c_void_p]
        L.lbm_set_source.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.lbm_set_lagged_sink.argtypes = [C.c_void_p, C.c_double, C.c_double]
        L.lbm_init_fields.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.lbm_step.argtypes = [C.c_void_p, C.c_long]
        L.lbm_steps_done.argtypes = [C.c_void_p]
        L.lbm_steps_done.restype = C.c_long
        L.lbm_moments.argtypes = [C.c_void_p, C.c_uint, C.c_void_p, C.c_int]
        L.lbm_integrals.argtypes = [C.c_void_p, _dp]
        L.lbm_check.argtypes = [C.c_void_p]
        L.lbm_state_bytes.argtypes = [C.c_void_p]
        L.lbm_state_bytes.restype = C.c_size_t
        L.lbm_get_state.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t]
        L.lbm_set_state.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t]
        L.lbm_constants.argtypes = [C.c_void_p, _dp]
        L.lbm_synchronize.argtypes = [C.c_void_p]
        L.lbm_last_error.argtypes = [C.c_void_p]
        L.lbm_last_error.restype = C.c_char_p
        L.lbm_destroy.argtypes = [C.c_void_p]
        L.lbm_destroy.restype = None
        for name in ("lbm_create", "lbm_set_bc", "lbm_set_source", "lbm_set_lagged_sink", "lbm_init_fields", "lbm_step",
                     "lbm_moments", "lbm_integrals", "lbm_check", "lbm_get_state", "lbm_set_state",
                     "lbm_constants", "lbm_synchronize"):
            getattr(L, name).restype = C.c_int
        _extra_signatures(L)
        _lib = L
    return _lib


def _extra_signatures(L):
    """Signatures of the allocation-free, batched and adjoint entry points."""
    L.lbm_field_integrals_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                              C.c_double, C.c_double, C.c_void_p, C.c_void_p]
    L.lbm_field_integrals_noalloc.restype = C.c_int
    L.lbm_batch_create.argtypes = [C.POINTER(lbm_params), C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]
    L.lbm_batch_create.restype = C.c_int
    L.lbm_batch_channel.argtypes = [C.c_void_p, C.c_int]
    L.lbm_batch_channel.restype = C.c_void_p
    L.lbm_batch_size.argtypes = [C.c_void_p]
    L.lbm_batch_size.restype = C.c_int
    L.lbm_batch_step.argtypes = [C.c_void_p, C.c_long]
    L.lbm_batch_step.restype = C.c_int
    L.lbm_batch_autotune.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
    L.lbm_batch_autotune.restype = C.c_int
    L.lbm_batch_config.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
    L.lbm_batch_config.restype = C.c_int
    L.lbm_batch_last_error.argtypes = [C.c_void_p]
    L.lbm_batch_last_error.restype = C.c_char_p
    L.lbm_batch_destroy.argtypes = [C.c_void_p]
    L.lbm_batch_destroy.restype = None
    L.lbm_autotune.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
    L.lbm_autotune.restype = C.c_int
    L.lbm_probe_fma_rate.argtypes = [C.c_int, _dp]
    L.lbm_probe_fma_rate.restype = C.c_int
    L.lbm_set_launch.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
    L.lbm_set_launch.restype = C.c_int
    L.lbm_launch_config.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
    L.lbm_launch_config.restype = C.c_int
    L.lbm_adjoint.argtypes = [C.c_void_p, C.c_long, C.c_int, C.c_void_p, _dp, C.c_void_p, C.c_void_p, _dp]
    L.lbm_adjoint.restype = C.c_int
    L.lbm_set_check_interval.argtypes = [C.c_void_p, C.c_long]
    L.lbm_set_check_interval.restype = C.c_int
    L.lbm_last_good_step.argtypes = [C.c_void_p]
    L.lbm_last_good_step.restype = C.c_long
    L.lbm_set_wait_limit.argtypes = [C.c_void_p, C.c_double, C.c_int]
    L.lbm_set_wait_limit.restype = C.c_int


def _check(h, st):
    if st != LBM_OK:
        msg = lib().lbm_last_error(h)
        raise LbmError(st, msg.decode() if msg else "")


def _host(a, n=None):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and arr.size != n:
        raise ValueError(f"expected {n} values, got {arr.size}")
    return arr, arr.ctypes.data_as(C.c_void_p)


def _ptr(a, n=None):
    """(keepalive, pointer, on_device) for a numpy array or a torch CUDA tensor."""
    if a is None:
        return None, None, 0
    if hasattr(a, "is_cuda") and a.is_cuda:
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("device arrays must be contiguous float64 tensors")
        if n is not None and a.numel() != n:
            raise ValueError(f"expected {n} values, got {a.numel()}")
        return a, C.c_void_p(a.data_ptr()), 1
    arr, p = _host(a, n)
    return arr, p, 0


# --- C-named functions ------------------------------------------------------
def lbm_params_default():
    p = lbm_params()
    lib().lbm_params_default(C.byref(p))
    return p


def lbm_create(params: lbm_params, stream=None):
    h = C.c_void_p()
    st = lib().lbm_create(C.byref(params), stream, C.byref(h))
    _check(None, st)
    return h


def lbm_set_bc(h, side, kind, uw=None, rho_w=0.0, tkind=LBM_TBC_NONE, tw=None):
    a, pa = _host(uw)
    b, pb = _host(tw)
    _check(h, lib().lbm_set_bc(h, side, kind, pa, float(rho_w), tkind, pb))


def lbm_set_source(h, q3=None, force=None, n=None):
    a, pa, da = _ptr(q3, n)
    b, pb, db = _ptr(force, None if n is None else 2 * n)
    on_dev = da or db
    if (q3 is not None and force is not None) and da != db:
        raise ValueError("q3 and force must both be host or both be device arrays")
    _check(h, lib().lbm_set_source(h, pa, pb, on_dev))


def lbm_set_lagged_sink(h, conv_coef, T_inf):
    _check(h, lib().lbm_set_lagged_sink(h, float(conv_coef), float(T_inf)))


def lbm_init_fields(h, a=None, ux=None, uy=None, b=None, n=None):
    keep = [_ptr(x, n) for x in (a, ux, uy, b)]
    devs = {k[2] for k in keep if k[0] is not None}
    if len(devs) > 1:
        raise ValueError("fields must all be host or all be device arrays")
    on_dev = devs.pop() if devs else 0
    _check(h, lib().lbm_init_fields(h, keep[0][1], keep[1][1], keep[2][1], keep[3][1], on_dev))


def lbm_step(h, n):
    _check(h, lib().lbm_step(h, int(n)))


def lbm_steps_done(h):
    return lib().lbm_steps_done(h)


def lbm_moments(h, mask, out, on_device=None):
    if hasattr(out, "is_cuda") and out.is_cuda:
        _check(h, lib().lbm_moments(h, mask, C.c_void_p(out.data_ptr()), 1))
    else:
        assert out.dtype == np.float64 and out.flags["C_CONTIGUOUS"]
        _check(h, lib().lbm_moments(h, mask, out.ctypes.data_as(C.c_void_p), 0))
    return out


def lbm_integrals(h):
    out = (C.c_double * 4)()
    _check(h, lib().lbm_integrals(h, out))
    return [out[i] for i in range(4)]


def lbm_check(h):
    return lib().lbm_check(h)


def lbm_state_bytes(h):
    return lib().lbm_state_bytes(h)


def lbm_get_state(h):
    nb = lbm_state_bytes(h)
    buf = np.empty(nb, dtype=np.uint8)
    _check(h, lib().lbm_get_state(h, buf.ctypes.data_as(C.c_void_p), nb))
    return buf


def lbm_set_state(h, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(h, lib().lbm_set_state(h, buf.ctypes.data_as(C.c_void_p), buf.size))


def lbm_constants(h):
    out = (C.c_double * 5)()
    _check(h, lib().lbm_constants(h, out))
    return dict(c=out[0], cs2=out[1], tau=out[2], tauT=out[3], tauphi=out[4])


def lbm_synchronize(h):
    _check(h, lib().lbm_synchronize(h))


def lbm_last_error(h=None):
    m = lib().lbm_last_error(h)
    return m.decode() if m else ""


def lbm_destroy(h):
    lib().lbm_destroy(h)


def lbm_probe_fma_rate(precision):
    """GFLOP/s of dependent-chain FMAs on the current device (LBM_FP64 or LBM_FP32DEV)."""
    out = C.c_double(0.0)
    _check(None, lib().lbm_probe_fma_rate(int(precision), C.byref(out)))
    return out.value


def lbm_set_check_interval(h, every):
    _check(h, lib().lbm_set_check_interval(h, int(every)))


def lbm_last_good_step(h):
    return lib().lbm_last_good_step(h)


def lbm_set_wait_limit(h, seconds, expire_next=False):
    _check(h, lib().lbm_set_wait_limit(h, float(seconds), int(bool(expire_next))))


def lbm_set_launch(h, cfg):
    """Single-phase step launch: cfg = (kind, a, b, c), see include/lbm.h."""
    arr = (C.c_int * 4)(*[int(v) for v in cfg])
    _check(h, lib().lbm_set_launch(h, arr))


def lbm_launch_config(h):
    arr = (C.c_int * 4)()
    _check(h, lib().lbm_launch_config(h, arr))
    return tuple(arr)


def lbm_adjoint(h, steps, ckpt_every, T_target, nx, ny, want_q3=True, want_qwall=True, want_nu=True):
    """Forward run + reverse-time adjoint: returns (loss, dL/dq3 (ny, nx), dL/dq_wall (2, nx), dL/dnu)."""
    tt = np.ascontiguousarray(np.asarray(T_target, dtype=np.float64))
    assert tt.size == ny
    loss = C.c_double()
    g3 = np.zeros((ny, nx)) if want_q3 else None
    gw = np.zeros((2, nx)) if want_qwall else None
    gn = C.c_double()
    _check(h, lib().lbm_adjoint(h, int(steps), int(ckpt_every), tt.ctypes.data_as(C.c_void_p), C.byref(loss),
                                None if g3 is None else g3.ctypes.data_as(C.c_void_p),
                                None if gw is None else gw.ctypes.data_as(C.c_void_p),
                                C.byref(gn) if want_nu else None))
    return loss.value, g3, gw, (gn.value if want_nu else None)


def _noalloc_arg(name, t, n):
    """Check one tensor argument of lbm_field_integrals_noalloc before its address goes
    to the kernel, which reads n doubles from it (or writes them, for out4)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a torch tensor")
    if t.dtype != torch.float64:
        raise ValueError(f"{name} must be float64, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < n:
        raise ValueError(f"{name} holds {t.numel()} values, the call needs {n}")
    return t


def lbm_field_integrals_noalloc(rho, ux, uy, phi, nx, ny, dx, c, out4, stream=None):
    """Allocation-free integrals of device fields into the device array out4; returns
    the status code.  rho, ux, uy (and phi, or None) are contiguous float64 CUDA
    tensors of at least nx*ny values, out4 one of at least 4, all on one device;
    anything else raises ValueError before the C call."""
    nx, ny = int(nx), int(ny)
    if nx < 1 or ny < 1:
        raise ValueError("nx and ny must be >= 1")
    n = nx * ny
    named = [("rho", rho, n), ("ux", ux, n), ("uy", uy, n), ("phi", phi, n), ("out4", out4, 4)]
    ts = [None if t is None and k == "phi" else _noalloc_arg(k, t, m) for k, t, m in named]
    for (k, _, _), t in zip(named, ts):
        if t is not None and not t.is_cuda:
            raise ValueError(f"{k} must be a CUDA tensor")
    if len({t.device for t in ts if t is not None}) != 1:
        raise ValueError("all tensors must be on one device")
    ptr = [None if t is None else C.c_void_p(t.data_ptr()) for t in ts]
    return lib().lbm_field_integrals_noalloc(ptr[0], ptr[1], ptr[2], ptr[3], nx, ny, float(dx), float(c), ptr[4],
                                             stream)


# --- convenience wrapper -----------------------------------------------------
_PARAM_NAMES = [f[0] for f in lbm_params._fields_]


def make_params(d: dict, precision=LBM_FP64) -> lbm_params:
    """lbm_params from an SI dict (workload keys; Fb -> body_force)."""
    p = lbm_params_default()
    for k, v in d.items():
        if k == "Fb":
            p.body_force[0], p.body_force[1] = float(v[0]), float(v[1])
        elif k == "u_prescribed":
            p.u_prescribed[0], p.u_prescribed[1] = float(v[0]), float(v[1])
        elif k == "gravity":
            p.gravity[0], p.gravity[1] = float(v[0]), float(v[1])
        elif k in _PARAM_NAMES and k not in ("body_force",):
            setattr(p, k, v)
    if d.get("flow", 9) == 0:
        p.flow = LBM_NONE
    p.precision = precision
    return p


class Solver:
    """One solve on the GPU.  ``params`` is an SI dict as produced by
    ``paper_2302_04120_gb300.workloads``."""

    def __init__(self, params: dict, precision=LBM_FP64, stream=None, handle=None):
        self.params = dict(params)
        self.nx, self.ny = int(params["nx"]), int(params["ny"])
        self.n = self.nx * self.ny
        self.precision = precision
        self._owned = handle is None
        self.h = lbm_create(make_params(params, precision), stream) if handle is None else handle

    def close(self):
        if self._owned and self.h is not None and self.h.value:
            lbm_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_bc(self, side, kind, uw=None, rho_w=None, tkind=LBM_TBC_NONE, tw=None):
        rw = self.params.get("rho0", 1000.0) if rho_w is None else rho_w
        lbm_set_bc(self.h, side, kind, uw, rw, tkind, tw)

    def apply_workload(self, w):
        for bc in w["bcs"]:
            self.set_bc(*bc)
        if w.get("q3") is not None:
            lbm_set_source(self.h, q3=w["q3"], n=self.n)
        init = w.get("init") or {}
        self.init(**init)

    def set_source(self, q3=None, force=None):
        lbm_set_source(self.h, q3, force, n=self.n)

    def set_lagged_sink(self, conv_coef, T_inf):
        lbm_set_lagged_sink(self.h, conv_coef, T_inf)

    def init(self, a=None, ux=None, uy=None, b=None):
        lbm_init_fields(self.h, a, ux, uy, b, n=self.n)

    def step(self, n):
        lbm_step(self.h, n)

    @property
    def steps(self):
        return lbm_steps_done(self.h)

    def moments(self, mask=63):
        sel = [name for name, bit in _MOMENT_BITS if mask & bit]
        out = np.empty((len(sel), self.ny, self.nx))
        lbm_moments(self.h, mask, out)
        return {k: out[i] for i, k in enumerate(sel)}

    def integrals(self):
        return lbm_integrals(self.h)

    def autotune(self):
        blk = (C.c_int * 2)()
        _check(self.h, lib().lbm_autotune(self.h, blk))
        return blk[0], blk[1]

    def set_launch(self, kind, a, b, c=0):
        """(LBM_LAUNCH_GRID or LBM_LAUNCH_GRID_OCC, block_x, block_y) or (LBM_LAUNCH_TMA, tile_height, stages,
        ctas_per_sm)."""
        lbm_set_launch(self.h, (kind, a, b, c))

    def launch_config(self):
        return lbm_launch_config(self.h)

    def check(self):
        return lbm_check(self.h)

    def set_check_interval(self, every):
        lbm_set_check_interval(self.h, every)

    @property
    def last_good_step(self):
        return lbm_last_good_step(self.h)

    def set_wait_limit(self, seconds, expire_next=False):
        lbm_set_wait_limit(self.h, seconds, expire_next)

    def constants(self):
        return lbm_constants(self.h)

    def get_state(self):
        return lbm_get_state(self.h)

    def set_state(self, buf):
        lbm_set_state(self.h, buf)

    def state_arrays(self, deviations=False):
        """Post-collision populations (q, ny, nx) as float64.  Single-phase solves store
        deviations from the rest equilibrium; they are returned as stored with
        ``deviations=True`` (f - w_i rho0, g - w_i T0), else with w_i rho0 and w_i T0
        added back."""
        raw = self.get_state()
        dt = np.float64 if self.precision == LBM_FP64 else np.float32
        a = raw.view(dt).astype(np.float64).reshape(-1, self.ny, self.nx)
        p = self.params
        if p.get("phase", 0):
            return dict(z=a[0:9], h=a[9:14], phiu=a[14:16])
        out = {}
        k = 0
        keep = 0.0 if deviations else 1.0
        if p.get("flow", 9):
            w9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
            out["f"] = a[0:9] + keep * w9[:, None, None] * p.get("rho0", 1000.0)
            k = 9
        if p.get("thermal", 0) == 9:
            w9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
            out["g"] = a[k:k + 9] + keep * w9[:, None, None] * p.get("T0", 300.0)
        elif p.get("thermal", 0):
            w5 = np.array([1 / 3] + [1 / 6] * 4)
            out["g"] = a[k:k + 5] + keep * w5[:, None, None] * p.get("T0", 300.0)
        return out


def _bcheck(b, st):
    if st != LBM_OK:
        msg = lib().lbm_batch_last_error(b)
        raise LbmError(st, msg.decode() if msg else "")


class Batch:
    """Many independent single-phase channels advanced by one launch per step.
    ``channels[k]`` is a Solver view of channel k (boundaries, sources, init,
    moments); advance only with ``step``."""

    def __init__(self, params_list, precision=LBM_FP64, stream=None):
        arr = (lbm_params * len(params_list))(*[make_params(p, precision) for p in params_list])
        h = C.c_void_p()
        _bcheck(None, lib().lbm_batch_create(arr, len(params_list), stream, C.byref(h)))
        self.h = h
        self.channels = [Solver(p, precision, handle=C.c_void_p(lib().lbm_batch_channel(h, k)))
                         for k, p in enumerate(params_list)]

    def step(self, n):
        _bcheck(self.h, lib().lbm_batch_step(self.h, int(n)))

    def autotune(self):
        cfg = (C.c_int * 3)()
        _bcheck(self.h, lib().lbm_batch_autotune(self.h, cfg))
        return tuple(cfg)

    def config(self, bx, by, grid):
        _bcheck(self.h, lib().lbm_batch_config(self.h, bx, by, grid))

    def close(self):
        if self.h is not None and self.h.value:
            for c in self.channels:
                c.h = None
            lib().lbm_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
