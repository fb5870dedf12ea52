"""Writes oracle_counts_16x256.json: the FP64 CPU oracle's iteration counts of the two-step
BiCGStab with the order-2 weak-coupling preconditioner, plain and with Euler's S_{2k/3,k/3}
acceleration, on the 16^3 x 256 workload, seed 0, tol 1e-10.  bench.py scales its bounded
CPU-baseline sample (a few oracle iterations) by them.  Runs already stored are kept.

Calls only oracle/ and the seeded input generator.  Takes tens of minutes on one core:
    python tests/golden/make_oracle_counts_16x256.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1008_3647_gb300.inputs import field_and_source  # noqa: E402


def main(nx=16, ntau=256, seed=0, tol=1e-10):
    lat = O.Lattice(nx, ntau, 0.05, 5.0)
    sigma, b = field_and_source(nx, ntau, seed)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_counts_16x256.json")
    out = {"nx": nx, "ntau": ntau, "tau": 0.05, "g": 5.0, "tol": tol, "seed": seed, "runs": {}}
    if os.path.exists(path):
        with open(path) as f:
            out["runs"] = json.load(f)["runs"]
    for name, pc in [("bicg_wce2", {"kind": "wce", "order": 2}),
                     ("bicg_wce2_euler23", {"kind": "wce", "order": 2, "euler": "euler23"})]:
        if name in out["runs"]:
            continue
        t0 = time.time()
        _, info = O.solve_bicgstab_two_step(lat, sigma, b, tol, 20000, pc)
        out["runs"][name] = {"iterations": info["iterations"], "steps": info["iterations_step"],
                             "converged": info["converged"], "seconds": time.time() - t0}
        print(name, out["runs"][name], flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
