"""Failure statuses through the C ABI, made without a GPU fault.

* UFG_TIMEOUT: the library's bounded device waits (TMA copies into shared memory) raise a flag of
  the lattice when they run out.  ufg_test_expire_waits makes the next slice launches run one extra
  bounded wait on a barrier whose bytes never arrive, so that wait runs out after a few hundred
  polling rounds; the kernel returns, its own copies having completed, and the call (or the
  lattice check after an apply) must report UFG_TIMEOUT, with the flag cleared afterwards.
* UFG_BREAKDOWN: unpreconditioned BiCGStab on M near-breaks down again and again (its spectrum
  circles around 1), so the restart budget runs out -- as it does in the oracle on the same input.
* UFG_NOT_CONVERGED at g = 10: the weak-coupling series diverges once A > 1, and the paper reports
  that the g = 10 solves fail within 15,000 MV operations (Sec. 5, before Table 3).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_3647_gb300.inputs import field_and_source

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ufg():
    from paper_1008_3647_gb300 import ufg as u
    u.load()
    yield u
    u.ufg_test_expire_waits(0)


@pytest.mark.parametrize("nx,ntau,dtype", [(32, 8, torch.float32), (16, 12, torch.float32),
                                           (16, 12, torch.float64), (8, 10, torch.float64)])
def test_expired_wait_is_reported_after_apply(ufg, nx, ntau, dtype):
    lat = ufg.Lattice(nx, ntau)
    sigma, x = field_and_source(nx, ntau, 3)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    xd = torch.from_numpy(x).cuda().to(dtype)
    clean = ufg.ufg_apply_M(field, xd)
    lat.ufg_lattice_check()  # nothing ran out
    ufg.ufg_test_expire_waits(1)
    y = ufg.ufg_apply_M(field, xd)
    with pytest.raises(ufg.UfgError) as e:
        lat.ufg_lattice_check()
    assert e.value.status == ufg.UFG_TIMEOUT
    assert "bounded device wait" in str(e.value)
    lat.ufg_lattice_check()  # the flag was cleared by the check
    # the expired wait was an extra one: the kernel's own copies completed, the result stands
    assert torch.equal(y, clean)


def test_expired_wait_turns_solve_into_timeout(ufg):
    nx, ntau = 16, 64
    sigma, b = field_and_source(nx, ntau, 11)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    solver.ufg_set_preconditioner("wce", order=2)
    bd = torch.from_numpy(b).cuda()
    ufg.ufg_test_expire_waits(1)
    with pytest.raises(ufg.UfgError) as e:
        solver.ufg_solve_bicgstab_two_step(field, bd, tol=1e-10)
    assert e.value.status == ufg.UFG_TIMEOUT
    x, st = solver.ufg_solve_bicgstab_two_step(field, bd, tol=1e-10)  # the next call is clean
    assert st["status"] == ufg.UFG_OK
    r = b - O.apply_Q(O.Lattice(nx, ntau), sigma, x.cpu().numpy())
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)


def test_expired_wait_turns_batch_into_timeout(ufg):
    shapes = [(16, 16, 1), (8, 24, 2)]
    probs = []
    for nx, nt, seed in shapes:
        sg, b = field_and_source(nx, nt, seed)
        probs.append({"nx": nx, "ntau": nt, "sigma": torch.from_numpy(sg).cuda(),
                      "b": torch.from_numpy(b).cuda(),
                      "x": torch.zeros(nt, nx, nx, nx, dtype=torch.float64, device="cuda")})
    ufg.ufg_test_expire_waits(1)
    with pytest.raises(ufg.UfgError) as e:
        ufg.ufg_solve_batch(probs, "wce", {"order": 2}, tol=1e-10, precision=ufg.UFG_MIXED)
    assert e.value.status == ufg.UFG_TIMEOUT
    stats = ufg.ufg_solve_batch(probs, "wce", {"order": 2}, tol=1e-10, precision=ufg.UFG_MIXED)
    assert all(st["status"] == ufg.UFG_OK for st in stats)


def test_unpreconditioned_bicgstab_reports_breakdown(ufg):
    # 8^3 x 64, seed 0: the oracle's BiCGStab exhausts its 100 restarts in both steps
    # (tests/golden/oracle_counts_8x64.json, bicg_none/0)
    nx, ntau = 8, 64
    sigma, b = field_and_source(nx, ntau, 0)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    x, st = solver.ufg_solve_bicgstab_two_step(field, torch.from_numpy(b).cuda(), tol=1e-10,
                                               maxit=20000)
    assert st["status"] == ufg.UFG_BREAKDOWN, st
    assert st["restarts"] >= 100
    assert np.isfinite(x.cpu().numpy()).all()


def test_strong_coupling_g10_does_not_converge_within_paper_budget(ufg):
    # g = 10 (A = 1.139): BiCGStab + WCE2 costs 2 (d + 1) 3 = 18 MV per iteration, so 15,000 MV
    # allow 833 iterations per step
    nx, ntau = 8, 50
    sigma, b = field_and_source(nx, ntau, 0)
    lat = ufg.Lattice(nx, ntau, 0.05, 10.0)
    assert lat.A > 1.0
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    solver.ufg_set_preconditioner("wce", order=2)
    x, st = solver.ufg_solve_bicgstab_two_step(field, torch.from_numpy(b).cuda(), tol=1e-10,
                                               maxit=833)
    assert st["status"] in (ufg.UFG_NOT_CONVERGED, ufg.UFG_BREAKDOWN, ufg.UFG_NONFINITE), st
    assert st["true_residual"] > 1e-10 or not np.isfinite(st["true_residual"])


def test_force_finishes_a_broken_down_solve_with_cg(ufg):
    # the same system as the breakdown test above, through the force: BiCGStab breaks down and
    # CG on M^T M (Chebyshev 16) finishes the solve, so the force and the action are still those
    # of Q^{-1} phi
    nx, ntau = 8, 64
    sigma, b = field_and_source(nx, ntau, 0)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    dS, X, S, st = solver.ufg_hmc_force(field, torch.from_numpy(b).cuda(), tol=1e-10)
    assert st["status"] == ufg.UFG_OK, st
    olat = O.Lattice(nx, ntau)
    Xh = X.cpu().numpy()
    r = b - O.apply_Q(olat, sigma, Xh)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    ref = O.force_dS_dsigma(olat, sigma, Xh)
    # (1e-11: this unpreconditioned solution spans a wide range, so the force entries do too)
    assert float(np.abs(dS.cpu().numpy() - ref).max() / np.abs(ref).max()) < 1e-11
    assert S == pytest.approx(float(np.dot(b.ravel(), Xh.ravel())), rel=1e-12)
