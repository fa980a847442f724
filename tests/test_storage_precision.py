"""Evaluation of the storage format of the populations (FP32 deviations, FP16
evaluated): the FP64 oracle is stepped with its stored populations rounded, after every
step, to FP32 or FP16 deviations from the rest equilibrium (f - w_i rho0, g - w_i T0),
and its fields are compared with the unrounded run.  This isolates the storage rounding
(the GPU's FP32 path also rounds its arithmetic and stores post- rather than
pre-collision populations; its own parity tests bound that).

On the 128 x 24 forced-convection channel after 1000 steps (relative L2 against FP64):
FP32 u 3.3e-8, T - T_in 6.3e-7; FP16 u 7.7e-4, T - T_in 2.7e-2, rho - mean 1.5e-2.
On the 2048 x 256 workload after 500 steps: FP32 u 1.1e-6, T - T_in 7.7e-5 (the heated
layer is still thin; see the full-size parity test); FP16 u 7.7e-3, T - T_in 0.31,
rho - mean 0.98.  FP16 storage misses the 1e-5 bar by orders of magnitude (an 11-bit
mantissa on deviations of several kg m^-3 or K loses the per-step increments), so only
the FP32 form is built."""
import numpy as np

import oracle
from paper_2302_04120_gb300 import workloads as wl

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
W5 = np.array([1 / 3] + [1 / 6] * 4)[:, None, None]


def _run(w, steps, dtype):
    o = oracle.Oracle(w["params"])
    for bc in w["bcs"]:
        o.set_bc(*bc)
    o.init(**w["init"])
    rho0, T0 = w["params"]["rho0"], w["params"]["T0"]
    for _ in range(steps):
        o.step(1)
        if dtype is not None:
            f, g = o.dist("f"), o.dist("g")
            o.set_dist("f", (f - W9 * rho0).astype(dtype).astype(np.float64) + W9 * rho0)
            o.set_dist("g", (g - W5 * T0).astype(dtype).astype(np.float64) + W5 * T0)
    return o.moments()


def _errors(m, ref, T_in):
    eu = np.sqrt(np.sum((m["ux"] - ref["ux"]) ** 2 + (m["uy"] - ref["uy"]) ** 2)
                 / np.sum(ref["ux"] ** 2 + ref["uy"] ** 2))
    eT = np.sqrt(np.sum((m["T"] - ref["T"]) ** 2) / np.sum((ref["T"] - T_in) ** 2))
    return eu, eT


def test_fp32_deviation_storage_meets_the_bar_and_fp16_does_not():
    w = wl.channel(nx=128, ny=24, steps=0, Re=100.0 * 24 / 256)
    ref = _run(w, 1000, None)
    eu32, eT32 = _errors(_run(w, 1000, np.float32), ref, w["T_in"])
    eu16, eT16 = _errors(_run(w, 1000, np.float16), ref, w["T_in"])
    assert eu32 < 1e-6 and eT32 < 1e-5
    assert eu16 > 1e-4 and eT16 > 1e-3
