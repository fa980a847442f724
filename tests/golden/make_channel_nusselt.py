"""Writes channel_nusselt_2048x256.json and channel_2048x256_fields.npz: the FP64
oracle's local Nusselt number along both walls, and its u_x, u_y and T - T_in fields
(compressed, FP64), for the 2048 x 256 forced-convection workload (D2Q9 MRT + D2Q5 MRT, water,
Re = 100, Pr = 7, q'' = 4e4 W m^-2 on both walls) after its 50000 steps, with
Nu(x) = q'' D_h / (k (T_w - T_m)), D_h = 2H, T_w from the wall row by the half-cell
extrapolation T + q'' dx / (2k) and T_m the velocity-weighted bulk temperature (reading
R22).  Calls only the oracle and the seeded input generators.

The oracle runs in its long-double build: over 50000 steps the FP64 oracle's own
rounding (absolute T ~ 300 K and f ~ w rho0 are stored) reaches the 1e-12 level on
u and beyond it on T - T_in, so the FP64 GPU path is compared with a reference
whose rounding is ~2000 times finer.

    python tests/golden/make_channel_nusselt.py        (about 2 h on 8 x86-64 cores)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2302_04120_gb300 import workloads as wl  # noqa: E402


def local_nusselt(T, u, q, k, dx, H):
    """Nu(x) at the lower (row 0) and upper (row ny - 1) walls."""
    Tm = (u * T).sum(0) / u.sum(0)
    lower = q * 2 * H / (k * (T[0] + q * dx / (2 * k) - Tm))
    upper = q * 2 * H / (k * (T[-1] + q * dx / (2 * k) - Tm))
    return lower, upper, Tm


def main():
    w = wl.channel()
    o = oracle.Oracle(w["params"], extended=True)
    for bc in w["bcs"]:
        o.set_bc(*bc)
    o.init(**w["init"])
    t0 = time.time()
    o.step(w["steps"])
    m = o.moments()
    p = w["params"]
    lower, upper, Tm = local_nusselt(m["T"], m["ux"], w["qflux"], p["k"], p["dx"], w["H"])
    out = dict(workload=w["name"], steps=w["steps"], Nu_lower=[float(x) for x in lower],
               Nu_upper=[float(x) for x in upper], T_bulk=[float(x) for x in Tm],
               oracle_seconds=round(time.time() - t0, 1),
               command="python tests/golden/make_channel_nusselt.py")
    with open(os.path.join(HERE, "channel_nusselt_2048x256.json"), "w") as fh:
        json.dump(out, fh)
    np.savez_compressed(os.path.join(HERE, "channel_2048x256_fields.npz"), ux=m["ux"], uy=m["uy"],
                        dT=m["T"] - w["T_in"])
    print("written", w["steps"], "steps in", out["oracle_seconds"], "s")


if __name__ == "__main__":
    main()
