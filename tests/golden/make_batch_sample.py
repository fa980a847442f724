"""Writes batch_sample_seed4.npz: the FP64 oracle's fields for a seeded sample of 16 of
the 256 channels of the batched forced-convection workload (numpy PCG64 seed 4 for the
channels: Nx ~ U{128..4096}, Ny ~ U{32..512}, Re ~ U(10, 200), Pr in {0.7, 7}; D2Q9 MRT
+ D2Q5 MRT, water, q'' = 4e4 W m^-2 on both walls) after their 5000 steps.

The sample is np.random.default_rng(0).choice(256, 16, replace=False), sorted.  For each
sampled channel k the file holds, under keys "<k>_<field>", the fields u_x, u_y and
T - T_in on every 4th row and every 8th column (rows 0, 4, ..., columns 0, 8, ...) and
the full outlet column (i = Nx - 1) of each, so the GPU's batched fields are compared
element by element on about 260 000 nodes.  Calls only the oracle and the seeded input
generators.

    python tests/golden/make_batch_sample.py          (about 2.5 h on 8 cores)
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2302_04120_gb300 import workloads as wl  # noqa: E402

NPZ = os.path.join(HERE, "batch_sample_seed4.npz")
STEPS = 5000
ROW_STRIDE, COL_STRIDE = 4, 8


def sample_indices():
    return np.sort(np.random.default_rng(0).choice(256, 16, replace=False))


def main():
    specs = wl.channel_batch_specs()
    out = {}
    if os.path.exists(NPZ):
        out = dict(np.load(NPZ))
    t_all = time.time()
    for k in sample_indices():
        if f"{k}_ux" in out:
            continue
        w = wl.channel_from_spec(specs[k], steps=STEPS)
        o = oracle.Oracle(w["params"])
        for bc in w["bcs"]:
            o.set_bc(*bc)
        o.init(**w["init"])
        t0 = time.time()
        o.step(STEPS)
        m = o.moments()
        o.close()
        fields = dict(ux=m["ux"], uy=m["uy"], dT=m["T"] - w["T_in"])
        for name, f in fields.items():
            out[f"{k}_{name}"] = f[::ROW_STRIDE, ::COL_STRIDE].copy()
            out[f"{k}_{name}_outlet"] = f[:, -1].copy()
        np.savez_compressed(NPZ, **out)
        print(f"channel {k} ({w['params']['nx']} x {w['params']['ny']}) in {time.time() - t0:.0f} s",
              flush=True)
    print(f"done in {time.time() - t_all:.0f} s")


if __name__ == "__main__":
    main()
