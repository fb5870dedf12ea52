"""HMC trajectories through the C ABI (the phi-algorithm of Sec. 1): the library's trajectory
against the oracle's on the same random numbers, acceptance and rejection, and a mixed-precision
trajectory on a larger lattice."""
import math

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
    return u


def _inputs(nx, ntau, seed):
    sigma, eta = field_and_source(nx, ntau, seed)
    pi0 = np.random.default_rng(seed + 100).standard_normal(sigma.shape)
    return sigma, eta, pi0


@pytest.mark.parametrize("nx,ntau,n_steps,dt,pc", [(4, 8, 5, 0.05, "wce"), (6, 10, 4, 0.04, "none"),
                                                   (8, 12, 3, 0.05, "wce")])
def test_trajectory_matches_oracle(ufg, nx, ntau, n_steps, dt, pc):
    sigma, eta, pi0 = _inputs(nx, ntau, 7)
    olat = O.Lattice(nx, ntau)
    s_ref, p_ref, info = O.hmc_trajectory(olat, sigma, eta, pi0, 0.5, n_steps, dt)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    if pc == "wce":
        solver.ufg_set_preconditioner("wce", order=2)
    s, p, st = solver.ufg_hmc_trajectory(field, torch.from_numpy(eta).cuda(),
                                         torch.from_numpy(pi0).cuda(), 0.5, n_steps, dt, tol=1e-12)
    assert st["status"] == ufg.UFG_OK, st
    assert st["md_steps"] == n_steps and st["force_solves"] == n_steps + 1
    assert st["accepted"] == int(info["accepted"])
    assert st["H_old"] == pytest.approx(info["H_old"], rel=1e-10)
    assert st["H_new"] == pytest.approx(info["H_new"], rel=1e-10)
    assert abs(st["dH"] - info["dH"]) < 1e-7
    assert st["action_old"] == pytest.approx(float(np.sum(eta * eta)), rel=1e-9)
    assert float(np.abs(s.cpu().numpy() - s_ref).max()) < 1e-8
    assert float(np.abs(p.cpu().numpy() - p_ref).max()) < 1e-8


def test_rejection_restores_the_field(ufg):
    nx, ntau = 4, 8
    sigma, eta, pi0 = _inputs(nx, ntau, 8)
    big = 2.0 * pi0  # a coarse step with large momenta: dH > 0
    olat = O.Lattice(nx, ntau)
    _, _, info = O.hmc_trajectory(olat, sigma, eta, big, 0.0, 3, 0.2)
    assert info["dH"] > 0
    u_rej = min(0.999999, 1.001 * math.exp(-info["dH"]))
    lat = ufg.Lattice(nx, ntau)
    sd = torch.from_numpy(sigma).cuda()
    field = ufg.Field(lat, sd)
    solver = ufg.Solver(lat)
    solver.ufg_set_preconditioner("wce", order=2)
    x = torch.from_numpy(eta).cuda()
    s, _, st = solver.ufg_hmc_trajectory(field, x, torch.from_numpy(big).cuda(), u_rej, 3, 0.2,
                                         tol=1e-12)
    assert st["accepted"] == 0 and st["dH"] > 0
    assert torch.equal(s, sd)  # the old configuration, bit for bit
    fresh = ufg.Field(lat, sd)
    assert torch.equal(ufg.ufg_apply_M(field, x), ufg.ufg_apply_M(fresh, x))
    # and accepted just below exp(-dH): the field then holds the new configuration
    s2, _, st2 = solver.ufg_hmc_trajectory(field, x, torch.from_numpy(big).cuda(),
                                           0.999 * math.exp(-info["dH"]), 3, 0.2, tol=1e-12)
    assert st2["accepted"] == 1 and not torch.equal(s2, sd)
    assert torch.equal(ufg.ufg_apply_M(field, x), ufg.ufg_apply_M(ufg.Field(lat, s2), x))


def test_mixed_precision_trajectory_16cubed(ufg):
    nx, ntau = 16, 12
    sigma, eta, pi0 = _inputs(nx, ntau, 9)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    solver.ufg_set_preconditioner("wce", order=2, euler="euler23")
    s, p, st = solver.ufg_hmc_trajectory(field, torch.from_numpy(eta).cuda(),
                                         torch.from_numpy(pi0).cuda(), 0.3, 3, 0.02, tol=1e-11,
                                         precision=ufg.UFG_MIXED)
    assert st["status"] == ufg.UFG_OK and st["force_solves"] == 4
    # the energy error grows with the volume (49,152 sites here); the end point, H and dH
    # against the oracle's trajectory from the same random numbers
    olat = O.Lattice(nx, ntau)
    s_ref, p_ref, info = O.hmc_trajectory(olat, sigma, eta, pi0, 0.3, 3, 0.02, tol=1e-12)
    assert st["accepted"] == int(info["accepted"])
    assert st["H_old"] == pytest.approx(info["H_old"], rel=1e-10)
    assert abs(st["dH"] - info["dH"]) < 1e-4, (st["dH"], info["dH"])
    assert float(np.abs(s.cpu().numpy() - s_ref).max()) < 1e-7
    assert float(np.abs(p.cpu().numpy() - p_ref).max()) < 1e-7
