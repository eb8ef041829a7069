"""Write the FP64 oracle's trajectory of the 1024x128 droplet-migration
channel (walls with adhesion, velocity inlet with the alpha correction,
convective outlet with the chi correction; Sec. III C) to
channel_1024x128_trajectory.json.

Calls only the oracle and the seeded input generator.  Every 1000 steps it
records lambda (Eq. 21) and chi (Eq. 23) for the next step, the inlet and
outlet mass fluxes, the component masses, and the droplet (nodes with
rho_1 > rho_2): its area A, the area-equivalent diameter D = 2 sqrt(A/pi),
its centroid and its extent along x.  Run:
    python tests/golden/make_channel_trajectory.py [--steps 30000] [--threads 8]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2512_12934_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "channel_1024x128_trajectory.json")


def droplet_stats(rho, solid):
    """Droplet of component 1: nodes where rho_1 > rho_2."""
    drop = (rho[0] > rho[1]) & (solid == 0)
    ys, xs = np.nonzero(drop)
    A = int(drop.sum())
    return {"area": A, "diameter": float(2.0 * np.sqrt(A / np.pi)),
            "xc": float(xs.mean()) if A else -1.0, "yc": float(ys.mean()) if A else -1.0,
            "xmin": int(xs.min()) if A else -1, "xmax": int(xs.max()) if A else -1}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=30000)
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    w = W.channel()
    o = O.Oracle2D(w.cfg, w.solid, w.rho, w.u, threads=a.threads)
    m0 = o.scalars()["mass"].tolist()
    recs = []
    t0 = time.time()
    for k in range(a.steps // a.every):
        o.step(a.every)
        s = o.scalars()
        rho, _, _ = o.macros()
        rec = {"step": s["step"], "lambda": s["lambda"], "chi": s["chi"], "Qin": s["Qin"], "Qout": s["Qout"],
               "mass": s["mass"].tolist()}
        rec.update(droplet_stats(rho, w.solid))
        recs.append(rec)
        print(rec["step"], "%.0f s" % (time.time() - t0), flush=True)
    json.dump({"workload": "channel_1024x128_droplet_migration", "G12": w.cfg["G12"], "mass0": m0,
               "generator": "tests/golden/make_channel_trajectory.py (FP64 oracle)", "records": recs},
              open(OUT, "w"), indent=1)


if __name__ == "__main__":
    main()
