"""Writes adjoint_reference_1024x128.json: exact directional derivatives of the
outlet-temperature loss of the gradient workload (1024 x 128 channel, D2Q9 MRT + D2Q5
MRT, water, Re = 50, Gaussian-filtered heat-source field of seed 5, 2000 steps) from the
oracle's forward-mode dual-number build, one oracle run per derivative:

  * the loss L = mean_j (T(nx - 1, j) - T_target[j])^2 with T_target the outlet
    temperature of the same run without heat source plus 0.01 K sin(pi y / H)
    (reading R26), and dL/dnu;
  * dL/dq''' at three cells drawn with numpy PCG64 seed 0 among the last 12 columns
    (in the 1.25 ms of 2000 steps the flow, u_m = 0.079 m/s, carries heat 40 to 60
    columns, so the outlet loss barely sees cells further upstream: 93 columns upstream
    the derivative is below 1e-28), and along one
    smooth direction (the workload's filter applied to seed 7);
  * dL/dq'' at two wall nodes drawn with the same generator among the last 12 columns.

Calls only the oracle and the seeded input generators.

    python tests/golden/make_adjoint_reference.py      (about 10 min on 16 cores)
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

OUT = os.path.join(HERE, "adjoint_reference_1024x128.json")


def target_profile(w, steps):
    """Outlet T of the run without heat source + 0.01 K sin(pi y / H) (reading R26)."""
    p = w["params"]
    o = oracle.Oracle(p)
    for bc in w["bcs"]:
        o.set_bc(*bc)
    o.init(**w["init"])
    o.step(steps)
    base = o.moments()["T"][:, -1]
    o.close()
    ny, dx = p["ny"], p["dx"]
    y = (np.arange(ny) + 0.5) * dx
    return base + 0.01 * np.sin(np.pi * y / (ny * dx))


def main():
    t0 = time.time()
    w = wl.adjoint_channel()
    nx, ny, steps = w["params"]["nx"], w["params"]["ny"], w["steps"]
    target = target_profile(w, steps)
    rng = np.random.default_rng(0)
    cells = [(int(rng.integers(0, ny)), int(rng.integers(nx - 12, nx))) for _ in range(3)]
    walls = [(int(rng.integers(0, 2)), int(rng.integers(nx - 12, nx))) for _ in range(2)]
    direction = wl.smooth_source(nx, ny, seed=7, scale=1.0)
    L, dnu = oracle.outlet_loss_jvp(w, steps, target, dnu=1.0)
    out = dict(workload="channel_adjoint_1024x128_2000steps", steps=steps, target=[float(v) for v in target],
               loss=L, dL_dnu=dnu, q3_cells=[], qwall_nodes=[],
               q3_direction=dict(seed=7, dL=oracle.outlet_loss_jvp(w, steps, target, dq3=direction)[1]))
    for j, i in cells:
        e = np.zeros((ny, nx))
        e[j, i] = 1.0
        out["q3_cells"].append(dict(j=j, i=i, dL=oracle.outlet_loss_jvp(w, steps, target, dq3=e)[1]))
    for side, i in walls:
        e = np.zeros((2, nx))
        e[side, i] = 1.0
        out["qwall_nodes"].append(dict(side=side, i=i, dL=oracle.outlet_loss_jvp(w, steps, target, dqwall=e)[1]))
    out["oracle_seconds"] = round(time.time() - t0, 1)
    out["command"] = "python tests/golden/make_adjoint_reference.py"
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
    print("written in", out["oracle_seconds"], "s")


if __name__ == "__main__":
    main()
