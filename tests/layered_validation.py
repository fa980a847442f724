"""Layered two-phase Poiseuille flow of Sec. 4.4 on the GPU against the quadrature of
its steady equation (tests/_layered.py): the four fluid systems and the refinement
study, FP64, several solves at once on separate CUDA streams.

Not collected by pytest (tens of millions of steps per solve: minutes of GPU time).
Run from the repository root, e.g.

    python tests/layered_validation.py --cases paper --out layered.jsonl --max-secs 900

Each case is stepped in chunks of --chunk steps until the profile changes by less than
1e-6 (relative max-norm) over a chunk, or until --max-steps / --max-secs; one JSON
line per case reports E2 (Eq. error_norm_2, in %) and the last chunk's change.  The
flow is x-invariant, so 2 columns give the paper's 10-column result.  --state-dir
saves each solve's state after every chunk and resumes from it.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

from _layered import e2, reference_for  # noqa: E402
from paper_2302_04120_gb300 import workloads as wl  # noqa: E402

# (system, dx [m], dt [s], z operator): the four systems at the finest grid of the
# refinement study, the BGK-z air-water variant, and the two coarser grids of the
# refinement study (saturated water at 100 C).
PAPER_CASES = [("air_water_25C", 1.25e-6, 1.25e-8, 1), ("air_water_25C", 1.25e-6, 1.25e-8, 0),
               ("sat_water_100C", 1.25e-6, 1.25e-8, 1), ("sat_water_80C", 1.25e-6, 1.25e-8, 1),
               ("sat_water_25C", 1.25e-6, 1.25e-8, 1), ("sat_water_100C", 5e-6, 1e-7, 1),
               ("sat_water_100C", 2.5e-6, 2.5e-8, 1)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cases", default="paper", help="'paper' or system:dx:dt:z_op;...")
    ap.add_argument("--chunk", type=float, default=2e6)
    ap.add_argument("--max-steps", type=float, default=4e8)
    ap.add_argument("--max-secs", type=float, default=900)
    ap.add_argument("--state-dir", default=None)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    import torch
    from paper_2302_04120_gb300 import build, lbm
    build.build()
    cases = PAPER_CASES if a.cases == "paper" else [
        (f[0], float(f[1]), float(f[2]), int(f[3])) for f in (c.split(":") for c in a.cases.split(";"))]
    chunk = int(a.chunk) // 3200 * 3200
    runs = []
    for name, dx, dt, z_op in cases:
        w = wl.layered_poiseuille(name, dx=dx, dt=dt, nx=2, z_op=z_op)
        st = torch.cuda.Stream()
        s = lbm.Solver(w["params"], precision=lbm.LBM_FP64, stream=st.cuda_stream)
        for bc in w["bcs"]:
            s.set_bc(*bc)
        s.init(**w["init"])
        tag = f"{name}_{dx:g}_{dt:g}_z{z_op}"
        n0 = 0
        if a.state_dir and os.path.exists(os.path.join(a.state_dir, tag + ".json")):
            s.set_state(np.fromfile(os.path.join(a.state_dir, tag + ".bin"), dtype=np.uint8))
            n0 = json.load(open(os.path.join(a.state_dir, tag + ".json")))["steps"]
        runs.append(dict(case=(name, dx, dt, z_op), tag=tag, w=w, s=s, st=st, ref=reference_for(w), n=n0,
                         prev=None, done=False))
    with open(os.path.join(HERE, "golden", "paper_numbers.json")) as fh:
        printed = json.load(fh)["layered_poiseuille_E2_percent"]
    out = open(a.out, "a") if a.out else None
    t0 = time.time()
    while not all(r["done"] for r in runs):
        for _ in range(chunk // 3200):  # interleave the solves' streams
            for r in runs:
                if not r["done"]:
                    r["s"].step(3200)
        for r in runs:
            if r["done"]:
                continue
            r["n"] += chunk
            u = r["s"].moments()["ux"].mean(axis=1)
            ok = bool(np.all(np.isfinite(u)))
            ch = None if r["prev"] is None or not ok else float(np.abs(u - r["prev"]).max() / np.abs(u).max())
            r["prev"] = u
            name, dx, dt, z_op = r["case"]
            rec = dict(system=name, dx=dx, dt=dt, z_op=z_op, ny=r["w"]["params"]["ny"], steps=r["n"],
                       E2_pct=100 * e2(u, r["ref"]) if ok else None, change=ch, secs=round(time.time() - t0, 1))
            if ok and a.state_dir:
                os.makedirs(a.state_dir, exist_ok=True)
                r["s"].get_state().tofile(os.path.join(a.state_dir, r["tag"] + ".bin"))
                json.dump(dict(steps=r["n"]), open(os.path.join(a.state_dir, r["tag"] + ".json"), "w"))
            if abs(dx - 1.25e-6) < 1e-12 and name in printed:
                rec["paper_E2_pct"] = printed[name]
            elif name == "sat_water_100C":
                rec["paper_E2_pct"] = printed["refinement_sat_water_100C"].get(f"dx_{dx:g}_dt_{dt:g}")
            stop = (not ok or (ch is not None and ch < 1e-6) or r["n"] >= a.max_steps
                    or time.time() - t0 > a.max_secs)
            if stop:
                r["done"] = True
                rec["converged"] = bool(ok and ch is not None and ch < 1e-6)
                print(json.dumps(rec), flush=True)
                if out:
                    out.write(json.dumps(rec) + "\n")
                    out.flush()
    for r in runs:
        r["s"].close()


if __name__ == "__main__":
    main()
