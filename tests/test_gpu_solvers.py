"""GPU solvers through the C ABI: every solve reaches ||b - M^T M x|| / ||b|| <= 1e-10 recomputed
by the FP64 oracle, and FP64 iteration counts agree with the oracle's (stored by
tests/golden/make_oracle_counts.py) to within 2 % or 2 iterations."""
import json
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_3647_gb300.inputs import field_and_source

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_counts_8x64.json")


@pytest.fixture(scope="module")
def ufg():
    from paper_1008_3647_gb300 import ufg as u
    u.load()
    return u


def _true_rel(olat, sigma, b, x):
    r = b - O.apply_Q(olat, sigma, x)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def _counts_close(a, b):
    return abs(a - b) <= max(2, 0.02 * b)


def test_plain_fp64_cg_4x16(ufg):
    nx, ntau = 4, 16
    sigma, b = field_and_source(nx, ntau, 0)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    x, st = solver.ufg_solve_cg_normal(field, torch.from_numpy(b).cuda(), tol=1e-10)
    olat = O.Lattice(nx, ntau)
    assert st["status"] == ufg.UFG_OK, st
    assert _true_rel(olat, sigma, b, x.cpu().numpy()) <= 1e-10
    _, info = O.solve_cg_normal(olat, sigma, b, 1e-10)
    assert _counts_close(st["iterations"], info["iterations"]), (st["iterations"], info)
    assert st["n_M"] >= st["iterations"] and st["mv_paper"] == 2 * st["iterations"]


METHODS = {
    "cg_none": ("cg", "none", {}),
    "cg_cheb8": ("cg", "cheb", {"degree": 8}),
    "cg_cheb16": ("cg", "cheb", {"degree": 16}),
    "cg_cheb32": ("cg", "cheb", {"degree": 32}),
    "cg_sca2": ("cg", "sca", {"alpha": 2.0}),
    "bicg_none": ("bicg", "none", {}),
    "bicg_wce0": ("bicg", "wce", {"order": 0}),
    "bicg_wce1": ("bicg", "wce", {"order": 1}),
    "bicg_wce2": ("bicg", "wce", {"order": 2}),
    "bicg_wce4": ("bicg", "wce", {"order": 4}),
    "bicg_wce2_euler": ("bicg", "wce", {"order": 2, "euler": True}),
    "bicg_wce4_euler": ("bicg", "wce", {"order": 4, "euler": True}),
    "bicg_wce2_euler23": ("bicg", "wce", {"order": 2, "euler": "euler23"}),
    "bicg_wce4_euler23": ("bicg", "wce", {"order": 4, "euler": "euler23"}),
    "bicg_wce2_vanw": ("bicg", "wce", {"order": 2, "euler": "vanw", "s": 1.0}),
    "bicg_wce4_vanw": ("bicg", "wce", {"order": 4, "euler": "vanw", "s": 1.0}),
    "cg_wce0": ("cg", "wce", {"order": 0}),
    "cg_wce2": ("cg", "wce", {"order": 2}),
    "cg_wce2_euler23": ("cg", "wce", {"order": 2, "euler": "euler23"}),
    "cg_scacheb8": ("cg", "sca_cheb", {"alpha": 2.0, "degree": 8}),
    "cg_scacheb16": ("cg", "sca_cheb", {"alpha": 2.0, "degree": 16}),
    "cg_sca1.5": ("cg", "sca", {"alpha": 1.5}),
    "cg_sca3": ("cg", "sca", {"alpha": 3.0}),
    "cg_sca4": ("cg", "sca", {"alpha": 4.0}),
}
# the ten seeded configurations of the stored oracle counts for the cheap methods, three for the
# slow ones (thousands of iterations)
SLOW = {"cg_none", "bicg_none", "cg_sca1.5", "cg_sca2", "cg_sca3", "cg_sca4", "cg_wce0", "cg_wce2",
        "cg_wce2_euler23"}
CASES = [(m, sd) for m in METHODS for sd in (range(3) if m in SLOW else range(10))]


@pytest.mark.parametrize("method,seed", CASES)
def test_8x64_fp64_matches_oracle(ufg, method, seed):
    gold = json.load(open(GOLD))
    ref = gold["runs"]["%s/%d" % (method, seed)]
    nx, ntau = gold["nx"], gold["ntau"]
    sigma, b = field_and_source(nx, ntau, seed)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    kind, pc, kw = METHODS[method]
    solver.ufg_set_preconditioner(pc, **kw)
    fn = solver.ufg_solve_cg_normal if kind == "cg" else solver.ufg_solve_bicgstab_two_step
    x, st = fn(field, torch.from_numpy(b).cuda(), tol=1e-10)
    if not ref["converged"] or method == "bicg_none":
        # unpreconditioned BiCGStab on M breaks down again and again; whether the restart budget
        # runs out first depends on rounding (the oracle and the GPU may end either way)
        assert st["status"] in (ufg.UFG_OK, ufg.UFG_BREAKDOWN, ufg.UFG_NOT_CONVERGED), st
        if st["status"] != ufg.UFG_OK:
            return
    else:
        assert st["status"] == ufg.UFG_OK, st
    rel = _true_rel(O.Lattice(nx, ntau), sigma, b, x.cpu().numpy())
    assert rel <= 1e-10
    if ref["converged"] and ref.get("restarts", 0) == 0 and st["restarts"] == 0:
        # without near-breakdown restarts the counts agree; after one they depend on rounding
        assert _counts_close(st["iterations"], ref["iterations"]), (st["iterations"], ref)


@pytest.mark.parametrize("kind,pc,kw", [("cg", "cheb", {"degree": 16}), ("bicg", "wce", {"order": 2})])
def test_mixed_precision_16x256(ufg, kind, pc, kw):
    nx, ntau = 16, 256
    sigma, b = field_and_source(nx, ntau, 0)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    solver.ufg_set_preconditioner(pc, **kw)
    fn = solver.ufg_solve_cg_normal if kind == "cg" else solver.ufg_solve_bicgstab_two_step
    bd = torch.from_numpy(b).cuda()
    x, st = fn(field, bd, tol=1e-10, precision=ufg.UFG_MIXED, inner_tol=1e-5)
    assert st["status"] == ufg.UFG_OK, st
    assert st["outer_iterations"] >= 1
    assert _true_rel(O.Lattice(nx, ntau), sigma, b, x.cpu().numpy()) <= 1e-10
    x64, st64 = fn(field, bd, tol=1e-10)
    assert st64["status"] == ufg.UFG_OK
    err = float((x - x64).norm() / x64.norm())
    assert err < 1e-6  # both solutions within the 1e-10 residual ball of the same system


@pytest.mark.parametrize("kind,pc,kw", [("cg", "sca", {"alpha": 2.0}), ("bicg", "wce", {"order": 2})])
def test_mixed_inner_tolerance_autotuned(ufg, kind, pc, kw):
    nx, ntau = 8, 32
    sigma, b = field_and_source(nx, ntau, 4)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    solver.ufg_set_preconditioner(pc, **kw)
    fn = solver.ufg_solve_cg_normal if kind == "cg" else solver.ufg_solve_bicgstab_two_step
    bd = torch.from_numpy(b).cuda()
    x, st = fn(field, bd, tol=1e-10, precision=ufg.UFG_MIXED, inner_tol=-1.0)
    assert st["status"] == ufg.UFG_OK, st
    assert st["inner_tol"] in (1e-3, 1e-4, 1e-5, 1e-6)
    assert _true_rel(O.Lattice(nx, ntau), sigma, b, x.cpu().numpy()) <= 1e-10
    # the choice is kept; an initial guess given with the first tuned call of a method survives
    # the tuning trials (warm start from the solution: the solve that takes x0 - CG, or the
    # second BiCGStab step - needs almost no iterations)
    x2, st2 = fn(field, bd, tol=1e-10, precision=ufg.UFG_MIXED, inner_tol=-1.0)
    assert st2["inner_tol"] == st["inner_tol"]
    fresh = ufg.Solver(lat)
    fresh.ufg_set_preconditioner(pc, **kw)
    fn2 = fresh.ufg_solve_cg_normal if kind == "cg" else fresh.ufg_solve_bicgstab_two_step
    x3, st3 = fn2(field, bd, x.clone(), tol=1e-10, precision=ufg.UFG_MIXED, inner_tol=-1.0,
                  x0_given=True)
    assert st3["status"] == ufg.UFG_OK
    assert st3["iterations_step"][1 if kind == "bicg" else 0] <= 2, st3
    fixed = fn(field, bd, tol=1e-10, precision=ufg.UFG_MIXED, inner_tol=1e-4)[1]
    assert fixed["inner_tol"] == 1e-4


def test_host_buffers_match_device_buffers(ufg):
    nx, ntau = 8, 16
    sigma, b = field_and_source(nx, ntau, 9)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    solver.ufg_set_preconditioner("wce", order=2)
    xd, st = solver.ufg_solve_bicgstab_two_step(field, torch.from_numpy(b).cuda(), tol=1e-10)
    bh = torch.from_numpy(b.copy())
    xh = torch.zeros_like(bh)
    xh, sth = solver.ufg_solve_bicgstab_two_step(field, bh, xh, tol=1e-10)
    assert sth["status"] == ufg.UFG_OK
    assert torch.equal(xh, xd.cpu())  # same kernels, same order: bit-identical


def test_initial_guess_is_used(ufg):
    nx, ntau = 6, 12
    sigma, b = field_and_source(nx, ntau, 2)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    bd = torch.from_numpy(b).cuda()
    x, st = solver.ufg_solve_cg_normal(field, bd, tol=1e-10)
    x2, st2 = solver.ufg_solve_cg_normal(field, bd, x.clone(), tol=1e-10, x0_given=True)
    assert st2["status"] == ufg.UFG_OK and st2["iterations"] <= 1


def test_maxit_reports_not_converged(ufg):
    nx, ntau = 8, 32
    sigma, b = field_and_source(nx, ntau, 1)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    x, st = solver.ufg_solve_cg_normal(field, torch.from_numpy(b).cuda(), tol=1e-10, maxit=5)
    assert st["status"] == ufg.UFG_NOT_CONVERGED
    assert st["iterations"] == 5


def test_nonfinite_rhs_reports_nonfinite(ufg):
    nx, ntau = 4, 8
    sigma, b = field_and_source(nx, ntau, 1)
    b[2, 1, 1, 1] = np.nan  # the failure is made on the host
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    for fn in (solver.ufg_solve_cg_normal, solver.ufg_solve_bicgstab_two_step):
        x, st = fn(field, torch.from_numpy(b).cuda(), tol=1e-10)
        assert st["status"] == ufg.UFG_NONFINITE


def test_zero_rhs_gives_zero(ufg):
    lat = ufg.Lattice(4, 8)
    sigma, _ = field_and_source(4, 8, 0)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    b = torch.zeros(lat.shape, dtype=torch.float64, device="cuda")
    for fn in (solver.ufg_solve_cg_normal, solver.ufg_solve_bicgstab_two_step):
        x, st = fn(field, b, tol=1e-10)
        assert st["status"] == ufg.UFG_OK and float(x.abs().max()) == 0.0


def test_wrong_preconditioner_for_solver_rejected(ufg):
    lat = ufg.Lattice(4, 8)
    sigma, b = field_and_source(4, 8, 0)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    solver.ufg_set_preconditioner("cheb", degree=8)
    with pytest.raises(ufg.UfgError):  # Chebyshev and SCA precondition M^T M, not M
        solver.ufg_solve_bicgstab_two_step(field, torch.from_numpy(b).cuda())
    with pytest.raises(ufg.UfgError):
        solver.ufg_set_preconditioner("cheb", degree=7)
