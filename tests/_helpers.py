"""Shared runners for the GPU-vs-oracle parity tests.

Both sides receive the same seeded inputs from ``paper_2302_04120_gb300.workloads``;
the oracle is the FP64 CPU program under ``oracle/``; the GPU path is called
through the C ABI (``paper_2302_04120_gb300.lbm``)."""
import numpy as np

import oracle

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
W5 = np.array([1 / 3] + [1 / 6] * 4)


def run_oracle(w, steps=None, q3=None, force=None, extended=False):
    """The oracle on workload w; ``extended`` runs it in long double, whose rounding
    is far below the 1e-12 bar (the FP64 oracle's own floor on populations, T - T_in
    and long runs is at or above it)."""
    o = oracle.Oracle(w["params"], extended=extended)
    for bc in w["bcs"]:
        o.set_bc(*bc)
    if q3 is not None or force is not None or w.get("q3") is not None:
        o.set_source(q3=q3 if q3 is not None else w.get("q3"), force=force)
    o.init(**(w.get("init") or {}))
    o.step(w["steps"] if steps is None else steps)
    return o


def run_gpu(w, precision, steps=None, q3=None, force=None):
    from paper_2302_04120_gb300 import lbm
    s = lbm.Solver(w["params"], precision=precision)
    for bc in w["bcs"]:
        s.set_bc(*bc)
    q = q3 if q3 is not None else w.get("q3")
    if q is not None or force is not None:
        s.set_source(q, force)
    s.init(**(w.get("init") or {}))
    s.step(w["steps"] if steps is None else steps)
    return s


def rel_max(a, b, ref=None):
    """||a - b||_inf / ||ref||_inf (ref defaults to b): relative max-norm on a
    deviation field (velocity, T - T_in, p - mean p, phi)."""
    ref = b if ref is None else ref
    den = np.max(np.abs(ref))
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / (den if den > 0 else 1.0)


def rel_l2(a, b, ref=None):
    ref = b if ref is None else ref
    den = np.sqrt(np.sum(np.asarray(ref) ** 2))
    return np.sqrt(np.sum((np.asarray(a) - np.asarray(b)) ** 2)) / (den if den > 0 else 1.0)


def deviations(a, w9_or_w5, ref_value):
    """Populations minus the rest equilibrium w_i * ref (rho0 for f, T0 for g)."""
    return np.asarray(a) - np.asarray(w9_or_w5)[:, None, None] * ref_value
