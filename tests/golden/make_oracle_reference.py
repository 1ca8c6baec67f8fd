"""Write per-step FP64 oracle results for a named workload (calls only oracle/).

    python tests/golden/make_oracle_reference.py ising3d_chi16 [--steps N] [--out PATH]

Output: tests/golden/<name>.jsonl (or PATH), one JSON object per coarse-graining
step, appended as each step finishes (a partial file is a valid prefix).
"""

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import hotrg_oracle as o  # noqa: E402

WORKLOADS = {
    # 3D Ising, chi = 16, near the critical coupling, h = 0, cycling z, x, y
    "ising3d_chi16": dict(d=3, beta=0.2216544, h=0.0, chi=16, steps=30, first=2),
    # 2D Ising, chi = 8, critical coupling, alternating x, y
    "ising2d_chi8": dict(d=2, beta=0.4406868, h=0.0, chi=8, steps=20, first=0),
    # 4D Ising, chi = 6, cycling x, y, z, w
    "ising4d_chi6": dict(d=4, beta=0.15, h=0.0, chi=6, steps=12, first=0),
    # 2D Ising, chi = 24, beta = 0.3 (ordered phase), alternating x, y: near-null
    # environments (about 530 of 576 eigenvalues below 1e-15 lambda_1)
    "ising2d_chi24_b03": dict(d=2, beta=0.3, h=0.0, chi=24, steps=20, first=0),
    # 3D Ising, chi = 20, through step 7 (a steady step costs ~4e14 flop on the CPU: ~35 min)
    "ising3d_chi20": dict(d=3, beta=0.2216544, h=0.0, chi=20, steps=7, first=2),
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=sorted(WORKLOADS))
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--out", default=None, help="output path (default: tests/golden/<name>.jsonl)")
    args = ap.parse_args()
    w = WORKLOADS[args.name]
    steps = args.steps or w["steps"]
    path = args.out or os.path.join(os.path.dirname(os.path.abspath(__file__)), args.name + ".jsonl")
    run = o.HotrgRun(w["d"], w["beta"], w["h"])
    with open(path, "w") as f:
        head = dict(kind="header", workload=args.name, **{k: w[k] for k in ("d", "beta", "h", "chi")},
                    ln_z0=run.ln_z, source="oracle/hotrg_oracle.py (FP64 CPU)")
        f.write(json.dumps(head) + "\n")
        f.flush()
        for a in o.cyclic_axes(w["d"], steps, first=w["first"]):
            t0 = time.time()
            rec = run.step(a, w["chi"])
            legs = [dict(axis=l.axis, eps=l.eps, eps_prime=l.eps_prime, chose_prime=l.chose_prime,
                         gap=None if l.gap_at_cut == float("inf") else l.gap_at_cut,
                         lam=[float(x) for x in l.lam[:24]],
                         lam_prime=[float(x) for x in l.lam_prime[:24]]) for l in rec.legs]
            f.write(json.dumps(dict(kind="step", step=rec.step, axis=a, chis=list(rec.chis),
                                    ln_z_per_site=rec.ln_z_per_site, trace=rec.trace,
                                    gu_wen_x=rec.gu_wen_x, legs=legs,
                                    seconds=round(time.time() - t0, 1))) + "\n")
            f.flush()
            print(f"step {rec.step} axis {a} chis {rec.chis} lnZ/V {rec.ln_z_per_site:.15f} "
                  f"{time.time() - t0:.0f}s", flush=True)


if __name__ == "__main__":
    main()
