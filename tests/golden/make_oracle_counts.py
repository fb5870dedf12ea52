"""Writes oracle_counts_8x64.json: iteration counts of the FP64 CPU oracle's solvers on the
8^3 x 64 workload (tau = 0.05, g = 5, sigma ~ U[-pi, pi], b ~ N(0, 1), seeds 0..2, tol 1e-10).

Calls only oracle/ and the seeded input generator.  Run from the repository root:
    python tests/golden/make_oracle_counts.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1008_3647_gb300.inputs import field_and_source  # noqa: E402

METHODS = {
    "cg_none": ("cg", None),
    "cg_cheb8": ("cg", {"kind": "cheb", "degree": 8}),
    "cg_cheb16": ("cg", {"kind": "cheb", "degree": 16}),
    "cg_cheb32": ("cg", {"kind": "cheb", "degree": 32}),
    "cg_sca2": ("cg", {"kind": "sca", "alpha": 2.0}),
    "bicg_none": ("bicg", None),
    "bicg_wce0": ("bicg", {"kind": "wce", "order": 0}),
    "bicg_wce1": ("bicg", {"kind": "wce", "order": 1}),
    "bicg_wce2": ("bicg", {"kind": "wce", "order": 2}),
    "bicg_wce4": ("bicg", {"kind": "wce", "order": 4}),
    "bicg_wce2_euler": ("bicg", {"kind": "wce", "order": 2, "euler": True}),
    "bicg_wce4_euler": ("bicg", {"kind": "wce", "order": 4, "euler": True}),
}


def main(seeds=(0, 1, 2), nx=8, ntau=64, tol=1e-10):
    lat = O.Lattice(nx, ntau, 0.05, 5.0)
    out = {"nx": nx, "ntau": ntau, "tau": 0.05, "g": 5.0, "tol": tol, "runs": {}}
    for seed in seeds:
        sigma, b = field_and_source(nx, ntau, seed)
        for name, (kind, pc) in METHODS.items():
            fn = O.solve_cg_normal if kind == "cg" else O.solve_bicgstab_two_step
            O.bicgstab.last_restarts = 0
            _, info = fn(lat, sigma, b, tol, 20000, pc)
            out["runs"]["%s/%d" % (name, seed)] = {
                "iterations": info["iterations"], "steps": info.get("iterations_step"),
                "converged": info["converged"], "restarts": info.get("restarts", 0)}
            print(name, seed, info["iterations"], info.get("iterations_step"), flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_counts_8x64.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
