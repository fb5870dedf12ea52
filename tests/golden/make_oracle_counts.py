"""Writes oracle_counts_8x64.json: iteration counts of the FP64 CPU oracle's solvers on the
8^3 x 64 workload (tau = 0.05, g = 5, sigma ~ U[-pi, pi], b ~ N(0, 1), seeds 0..9 -- ten random
configurations as in Sec. 5 -- tol 1e-10), for every method of Tables 1 and 2 plus the
strong-coupling parameter scan alpha in {1, 1.5, 2, 3, 4}.

Calls only oracle/ and the seeded input generator.  Run from the repository root:
    python tests/golden/make_oracle_counts.py
(one process per core; about ten minutes on eight cores).
"""
import json
import multiprocessing as mp
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
    "cg_wce0": ("cg", {"kind": "wce", "order": 0}),
    "cg_wce2": ("cg", {"kind": "wce", "order": 2}),
    "cg_wce2_euler23": ("cg", {"kind": "wce", "order": 2, "euler": "euler23"}),
    "cg_scacheb8": ("cg", {"kind": "sca_cheb", "alpha": 2.0, "degree": 8}),
    "cg_scacheb16": ("cg", {"kind": "sca_cheb", "alpha": 2.0, "degree": 16}),
    "cg_sca1": ("cg", {"kind": "sca", "alpha": 1.0}),
    "cg_sca1.5": ("cg", {"kind": "sca", "alpha": 1.5}),
    "cg_sca2": ("cg", {"kind": "sca", "alpha": 2.0}),
    "cg_sca3": ("cg", {"kind": "sca", "alpha": 3.0}),
    "cg_sca4": ("cg", {"kind": "sca", "alpha": 4.0}),
    "bicg_none": ("bicg", None),
    "bicg_wce0": ("bicg", {"kind": "wce", "order": 0}),
    "bicg_wce1": ("bicg", {"kind": "wce", "order": 1}),
    "bicg_wce2": ("bicg", {"kind": "wce", "order": 2}),
    "bicg_wce4": ("bicg", {"kind": "wce", "order": 4}),
    "bicg_wce2_euler": ("bicg", {"kind": "wce", "order": 2, "euler": True}),
    "bicg_wce4_euler": ("bicg", {"kind": "wce", "order": 4, "euler": True}),
    "bicg_wce2_euler23": ("bicg", {"kind": "wce", "order": 2, "euler": "euler23"}),
    "bicg_wce4_euler23": ("bicg", {"kind": "wce", "order": 4, "euler": "euler23"}),
    "bicg_wce2_vanw": ("bicg", {"kind": "wce", "order": 2, "euler": "vanw", "s": 1.0}),
    "bicg_wce4_vanw": ("bicg", {"kind": "wce", "order": 4, "euler": "vanw", "s": 1.0}),
}
NX, NTAU, TOL, SEEDS = 8, 64, 1e-10, tuple(range(10))


def run(job):
    name, seed = job
    kind, pc = METHODS[name]
    lat = O.Lattice(NX, NTAU, 0.05, 5.0)
    sigma, b = field_and_source(NX, NTAU, seed)
    fn = O.solve_cg_normal if kind == "cg" else O.solve_bicgstab_two_step
    O.bicgstab.last_restarts = 0
    _, info = fn(lat, sigma, b, TOL, 20000, pc)
    return "%s/%d" % (name, seed), {
        "iterations": info["iterations"], "steps": info.get("iterations_step"),
        "converged": info["converged"], "restarts": info.get("restarts", 0)}


def main():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_counts_8x64.json")
    out = {"nx": NX, "ntau": NTAU, "tau": 0.05, "g": 5.0, "tol": TOL, "seeds": list(SEEDS),
           "runs": {}}
    if os.path.exists(path):  # keep the runs already stored (same workload), add the missing ones
        with open(path) as f:
            old = json.load(f)
        if (old.get("nx"), old.get("ntau"), old.get("tol")) == (NX, NTAU, TOL):
            out["runs"] = old["runs"]
    jobs = [(name, seed) for seed in SEEDS for name in METHODS
            if "%s/%d" % (name, seed) not in out["runs"]]
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        for key, res in pool.imap_unordered(run, jobs):
            out["runs"][key] = res
            print(key, res["iterations"], res["steps"], flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
