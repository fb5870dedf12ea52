"""Paths selected by environment switches, each in a fresh process (the switches are read once):
UFG_NO_MOMENTUM=1 keeps batched WCE solves in the position basis, where the BiCGStab direction
update rides on the TMA forward transform; UFG_PDL=1 launches every kernel with programmatic
dependent launch; UFG_NO_FUSED_Q=1 applies Q = M^T M as two launches.  The solutions must still
reach the 1e-10 residual recomputed by the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np, torch
import oracle as O
from paper_1008_3647_gb300 import ufg
from paper_1008_3647_gb300.inputs import field_and_source
shapes = [(16, 48, 14), (16, 64, 11)]
probs, host = [], []
for nx, nt, seed in shapes:
    sg, b = field_and_source(nx, nt, seed)
    host.append((nx, nt, sg, b))
    probs.append({"nx": nx, "ntau": nt, "sigma": torch.from_numpy(sg).cuda(),
                  "b": torch.from_numpy(b).cuda(),
                  "x": torch.zeros(nt, nx, nx, nx, dtype=torch.float64, device="cuda")})
for prec in (ufg.UFG_MIXED, ufg.UFG_FP64):
    st = ufg.ufg_solve_batch(probs, "wce", {"order": 2}, tol=1e-10, precision=prec)
    for (nx, nt, sg, b), pr, s in zip(host, probs, st):
        assert s["status"] == ufg.UFG_OK, s
        r = b - O.apply_Q(O.Lattice(nx, nt), sg, pr["x"].cpu().numpy())
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
print("env path ok")
"""


@pytest.mark.parametrize("env", [{"UFG_NO_MOMENTUM": "1"}, {"UFG_PDL": "1"}])
def test_batched_solve_under_switch(env):
    e = dict(os.environ)
    e.update(env)
    e["PYTHONPATH"] = ROOT + os.pathsep + e.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=e, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and "env path ok" in r.stdout, (r.stdout[-2000:], r.stderr[-2000:])


SCRIPT_CG = r"""
import numpy as np, torch
import oracle as O
from paper_1008_3647_gb300 import ufg
from paper_1008_3647_gb300.inputs import field_and_source
nx, nt = 16, 48
sg, b = field_and_source(nx, nt, 21)
lat = ufg.Lattice(nx, nt)
field = ufg.Field(lat, torch.from_numpy(sg).cuda())
solver = ufg.Solver(lat)
solver.ufg_set_preconditioner("cheb", degree=16)
for prec in (ufg.UFG_MIXED, ufg.UFG_FP64):
    x, st = solver.ufg_solve_cg_normal(field, torch.from_numpy(b).cuda(), tol=1e-10,
                                       precision=prec)
    assert st["status"] == ufg.UFG_OK, st
    r = b - O.apply_Q(O.Lattice(nx, nt), sg, x.cpu().numpy())
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
print("env path ok")
"""


@pytest.mark.parametrize("env", [{}, {"UFG_NO_FUSED_Q": "1"}])
def test_cg_chebyshev_with_and_without_fused_q(env):
    e = dict(os.environ)
    e.update(env)
    e["PYTHONPATH"] = ROOT + os.pathsep + e.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", SCRIPT_CG], cwd=ROOT, env=e, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and "env path ok" in r.stdout, (r.stdout[-2000:], r.stderr[-2000:])
