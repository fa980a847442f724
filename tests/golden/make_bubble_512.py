"""Writes bubble_512.json and bubble_512.npz: the FP64 oracle's stationary bubble of the
two-phase workload (Sec. 4.3: saturated water at 25 C, rho_l/rho_g = 43349, periodic
512 x 512 box, R = 64 dx, W = 5 dx, dx = 5e-6 m, dt = 1e-7 s, M = 1e-5 m^2/s, D2Q5 h with
BGK, D2Q9 z with MRT) after its 100000 steps.

Stored:
  * the Laplace pressure jump dp = P_in - P_out (reading R12) with the pressures averaged
    where phi < 1e-3 (gas) and phi > 1 - 1e-3 (liquid) (reading R14), and the geometric
    averages r < R - 2W, r > R + 2W;
  * the largest spurious speed max |u| and sum(phi);
  * the fields phi, p - mean(p), u_x, u_y (compressed .npz, FP64);
  * the oracle's own rounding envelope: the relative max-norm spread of phi, p - mean(p)
    and u between the unperturbed run and runs whose phi0 is multiplied by
    (1 + eps N(0,1)) (numpy PCG64 seed 0) for eps = 1e-15 (FP64 level) and 1e-7 (FP32
    level).  The guarded interface normal is discontinuous where |grad phi| is rounding
    noise, so rounding-level differences grow with time; a GPU result is compared
    against this spread.

Calls only the oracle and the seeded input generators.

    python tests/golden/make_bubble_512.py           (about 5 h on 8 cores: three runs)
    python tests/golden/make_bubble_512.py --base    (the unperturbed run only, ~1.5 h)
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

JSON = os.path.join(HERE, "bubble_512.json")
NPZ = os.path.join(HERE, "bubble_512.npz")


def laplace_jump(m, r, R, W):
    phi, p = m["phi"], m["p"]
    dp = p[phi < 1e-3].mean() - p[phi > 1 - 1e-3].mean()
    dp_geo = p[r < R - 2 * W].mean() - p[r > R + 2 * W].mean()
    return float(dp), float(dp_geo)


def run(w, eps):
    o = oracle.Oracle(w["params"])
    phi0 = w["init"]["a"]
    if eps:
        phi0 = phi0 * (1 + eps * np.random.default_rng(0).standard_normal(phi0.shape))
    o.init(a=phi0)
    t0 = time.time()
    o.step(w["steps"])
    m = o.moments()
    o.close()
    return m, time.time() - t0


def rel_max(a, b, ref):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(ref)))


def main():
    base_only = "--base" in sys.argv
    w = wl.bubble()
    out = {}
    if os.path.exists(JSON):
        with open(JSON) as fh:
            out = json.load(fh)
    if not os.path.exists(NPZ) or out.get("steps") != w["steps"]:
        m, sec = run(w, 0.0)
        dp, dp_geo = laplace_jump(m, w["r"], w["R"], w["W"])
        sp = np.hypot(m["ux"], m["uy"])
        out = dict(workload=w["name"], steps=w["steps"], R=w["R"], W=w["W"],
                   sigma=w["params"]["sigma"], dp=dp, dp_geometric=dp_geo,
                   sigma_over_R=w["params"]["sigma"] / w["R"], u_spurious_max=float(sp.max()),
                   phi_sum=float(m["phi"].sum()), oracle_seconds=round(sec, 1),
                   command="python tests/golden/make_bubble_512.py", envelope={})
        np.savez_compressed(NPZ, phi=m["phi"], p=m["p"] - m["p"].mean(), ux=m["ux"], uy=m["uy"])
        with open(JSON, "w") as fh:
            json.dump(out, fh, indent=1)
        print("base run written:", out["dp"], out["u_spurious_max"], sec, "s", flush=True)
    if base_only:
        return
    ref = np.load(NPZ)
    sp = np.hypot(ref["ux"], ref["uy"])
    for eps in (1e-7, 1e-15):
        key = f"{eps:g}"
        if key in out["envelope"]:
            continue
        m, sec = run(w, eps)
        pm = m["p"] - m["p"].mean()
        out["envelope"][key] = dict(phi=rel_max(m["phi"], ref["phi"], ref["phi"]),
                                    p=rel_max(pm, ref["p"], ref["p"]),
                                    u=rel_max(np.stack([m["ux"], m["uy"]]), np.stack([ref["ux"], ref["uy"]]), sp),
                                    dp=laplace_jump(m, w["r"], w["R"], w["W"])[0],
                                    oracle_seconds=round(sec, 1))
        with open(JSON, "w") as fh:
            json.dump(out, fh, indent=1)
        print("envelope", key, out["envelope"][key], flush=True)


if __name__ == "__main__":
    main()
