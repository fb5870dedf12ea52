"""Pins of the oracle's HMC trajectory (the phi-algorithm of Sec. 1): the free case, time
reversibility of the leapfrog integrator, the second-order energy error, and the Metropolis rule."""
import math

import numpy as np

import oracle as O
from paper_1008_3647_gb300.inputs import field_and_source


def _inputs(nx, ntau, seed):
    sigma, eta = field_and_source(nx, ntau, seed)
    pi0 = np.random.default_rng(seed + 100).standard_normal(sigma.shape)
    return sigma, eta, pi0


def test_free_field_moves_in_straight_lines():
    # g = 0: A = 0, so M does not depend on sigma, the force vanishes and H is conserved exactly
    lat = O.Lattice(2, 4, 0.05, 0.0)
    sigma, eta, pi0 = _inputs(2, 4, 1)
    s1, p1, info = O.hmc_trajectory(lat, sigma, eta, pi0, 0.5, 5, 0.1)
    assert np.allclose(s1, sigma + 5 * 0.1 * pi0, atol=1e-13)
    assert np.allclose(p1, pi0, atol=1e-13)
    assert abs(info["dH"]) < 1e-10 and info["accepted"]
    assert math.isclose(info["action_old"], float(np.sum(eta * eta)), rel_tol=1e-10)


def test_leapfrog_is_time_reversible():
    lat = O.Lattice(2, 6, 0.05, 5.0)
    sigma, eta, pi0 = _inputs(2, 6, 2)
    phi = O.apply_Mdag(lat, sigma, eta)
    s1, p1, _, _ = O.leapfrog(lat, sigma, pi0, phi, 6, 0.05)
    s2, p2, _, _ = O.leapfrog(lat, s1, -p1, phi, 6, 0.05)
    assert np.allclose(s2, sigma, atol=1e-9)
    assert np.allclose(p2, -pi0, atol=1e-9)


def test_energy_error_is_second_order():
    # fixed trajectory length, dt halved: the leapfrog energy error drops by about 4
    lat = O.Lattice(2, 6, 0.05, 5.0)
    sigma, eta, pi0 = _inputs(2, 6, 3)
    dH = []
    for n, dt in ((4, 0.1), (8, 0.05), (16, 0.025)):
        _, _, info = O.hmc_trajectory(lat, sigma, eta, pi0, 0.0, n, dt)
        dH.append(abs(info["dH"]))
    assert 0.15 < dH[1] / dH[0] < 0.4 and 0.15 < dH[2] / dH[1] < 0.4, dH


def test_metropolis_rule():
    lat = O.Lattice(2, 6, 0.05, 5.0)
    sigma, eta, pi0 = _inputs(2, 6, 4)
    _, _, info = O.hmc_trajectory(lat, sigma, eta, 2.0 * pi0, 0.0, 3, 0.2)
    dH = info["dH"]
    assert dH > 0  # a coarse step with large momenta loses energy conservation upward
    p = math.exp(-dH)
    s_acc, _, a = O.hmc_trajectory(lat, sigma, eta, 2.0 * pi0, 0.999 * p, 3, 0.2)
    s_rej, _, r = O.hmc_trajectory(lat, sigma, eta, 2.0 * pi0, min(0.999999, 1.001 * p), 3, 0.2)
    assert a["accepted"] and not r["accepted"]
    assert np.array_equal(s_rej, sigma) and not np.allclose(s_acc, sigma)
