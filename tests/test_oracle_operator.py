"""Pins of the oracle's operator layer against values and identities the paper and the
mathematics fix (no GPU).  Each test names the passage it follows."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1008_3647_gb300.inputs import field_and_source


def _tiny(nx=4, ntau=6, seed=0, g=5.0, dispersion=0):
    lat = O.Lattice(nx, ntau, 0.05, g, dispersion)
    sigma, b = field_and_source(nx, ntau, seed)
    return lat, sigma, b


def test_coupling_A_matches_paper_printed_values(golden_dir):
    # Sec. 5: A ~ 0.52 / 0.75 / 0.95 for g = 2.5 / 5 / 7.5 and ~1.14 for g = 10 at tau = 0.05.
    rows = [l.split() for l in open(os.path.join(golden_dir, "coupling_A.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for tau, g, a in rows:
        assert round(O.coupling_A(float(tau), float(g)), 2) == pytest.approx(float(a), abs=1e-12)


def test_momentum_range_is_paper_range():
    # Sec. 1: k_i = 2 pi n_i / N_x with n_i = -N_x/2 .. N_x/2 - 1.
    for nx in (4, 6, 8):
        n = np.sort(np.round(O.momentum_1d(nx) * nx / (2 * np.pi)).astype(int))
        assert list(n) == list(range(-nx // 2, nx // 2))


@pytest.mark.parametrize("dispersion", [0, 1])
def test_kinetic_plane_wave_eigenvalues(dispersion):
    # K is diagonal in momentum space with E(k) = k^2/2 (Sec. 1): cos(k.r) is an eigenvector of
    # exp(-tau K) with eigenvalue exp(-tau E(k)); the constant (k = 0) is unchanged.
    nx, tau = 6, 0.05
    lat = O.Lattice(nx, 2, tau, 5.0, dispersion)
    z, y, x = np.meshgrid(np.arange(nx), np.arange(nx), np.arange(nx), indexing="ij")
    for n in [(0, 0, 0), (1, 0, 0), (0, 2, 1), (3, 3, -3), (-2, 1, 3)]:
        k = [2 * np.pi * ni / nx for ni in n]
        u = np.cos(k[0] * x + k[1] * y + k[2] * z)
        if dispersion == 0:
            e = 0.5 * sum(ki * ki for ki in k)
        else:
            e = sum(1 - math.cos(ki) for ki in k)
        out = O.kinetic(lat, np.stack([u, u]))
        assert np.allclose(out, math.exp(-tau * e) * np.stack([u, u]), atol=1e-13)


def test_kinetic_dense_is_symmetric_contraction():
    lat = O.Lattice(4, 1 + 1, 0.05, 5.0)
    Kd = O.dense_from_apply(lambda u: O.kinetic(lat, u[None])[0], (4, 4, 4))
    assert np.allclose(Kd, Kd.T, atol=1e-14)
    ev = np.linalg.eigvalsh(Kd)
    assert ev.max() <= 1 + 1e-14 and ev.min() > 0  # ||exp(-tau K)|| = 1


def _dense_blocks(lat, sigma):
    Kd = O.dense_from_apply(lambda u: O.kinetic(lat, u[None])[0], (lat.nx,) * 3)
    w = 1 + lat.A * np.sin(sigma.reshape(lat.ntau, -1))
    return [Kd @ np.diag(w[t]) for t in range(lat.ntau)]


def test_dense_M_matches_block_definition():
    # Eq. (MatrixM): 1 on the diagonal, -B_j below it, +B_{N_tau} in the top-right corner.
    lat, sigma, _ = _tiny(4, 5)
    V = lat.volume
    Bs = _dense_blocks(lat, sigma)
    Md = np.eye(V * lat.ntau)
    for t in range(lat.ntau - 1):
        Md[(t + 1) * V:(t + 2) * V, t * V:(t + 1) * V] = -Bs[t]
    Md[0:V, (lat.ntau - 1) * V:] = Bs[-1]
    Mo = O.dense_from_apply(lambda u: O.apply_M(lat, sigma, u), lat.shape)
    assert np.allclose(Mo, Md, atol=1e-13)


def test_det_M_equals_det_one_plus_transfer_product():
    # det M[sigma] = det(1 + B_{N_tau} ... B_1), the determinant behind Eq. (HSZ).
    lat, sigma, _ = _tiny(4, 6, seed=3)
    Mo = O.dense_from_apply(lambda u: O.apply_M(lat, sigma, u), lat.shape)
    Bs = _dense_blocks(lat, sigma)
    P = np.eye(lat.volume)
    for B in Bs:
        P = B @ P
    s1, l1 = np.linalg.slogdet(Mo)
    s2, l2 = np.linalg.slogdet(np.eye(lat.volume) + P)
    assert s1 == s2 and l1 == pytest.approx(l2, rel=1e-11, abs=1e-11)


@pytest.mark.parametrize("nx,ntau", [(4, 6), (4, 8), (2, 10)])
def test_free_gas_determinant(nx, ntau):
    # sigma = 0: M = M0 and det M0 = prod_k (1 + exp(-beta E(k))), beta = tau N_tau (free Fermi gas,
    # antiperiodic time); a periodic corner would give prod (1 - exp(-beta E)) instead.
    lat = O.Lattice(nx, ntau, 0.05, 5.0)
    sigma = np.zeros(lat.shape)
    Mo = O.dense_from_apply(lambda u: O.apply_M(lat, sigma, u), lat.shape)
    sign, logdet = np.linalg.slogdet(Mo)
    expect = np.sum(np.log1p(np.exp(-lat.beta * lat.E)))
    assert sign > 0 and logdet == pytest.approx(expect, rel=1e-12)


def test_adjoint_identity_and_dense_transpose():
    lat, sigma, b = _tiny(4, 6, seed=1)
    rng = np.random.default_rng(7)
    u = rng.standard_normal(lat.shape)
    v = rng.standard_normal(lat.shape)
    lhs = np.vdot(u, O.apply_M(lat, sigma, v))
    rhs = np.vdot(O.apply_Mdag(lat, sigma, u), v)
    assert lhs == pytest.approx(rhs, rel=1e-13)
    Md = O.dense_from_apply(lambda x: O.apply_M(lat, sigma, x), lat.shape)
    Mt = O.dense_from_apply(lambda x: O.apply_Mdag(lat, sigma, x), lat.shape)
    assert np.allclose(Mt, Md.T, atol=1e-14)
    M1 = O.dense_from_apply(lambda x: O.apply_M1(lat, sigma, x), lat.shape)
    M1t = O.dense_from_apply(lambda x: O.apply_M1T(lat, sigma, x), lat.shape)
    assert np.allclose(M1t, M1.T, atol=1e-14)


def test_weak_coupling_split_M_equals_M0_plus_A_M1():
    # Sec. 3: M = M0 + A M1 with C_j = exp(-tau K) sin sigma_j (Eq. MatrixM_1).
    lat, sigma, b = _tiny(4, 6, seed=2)
    zero = np.zeros(lat.shape)
    lhs = O.apply_M(lat, sigma, b)
    rhs = O.apply_M(lat, zero, b) + lat.A * O.apply_M1(lat, sigma, b)
    assert np.allclose(lhs, rhs, atol=1e-13)


@pytest.mark.parametrize("nx,ntau", [(4, 6), (6, 5)])
def test_M0_inverse_fourier_acceleration(nx, ntau):
    # Sec. 3: M0^{-1} diagonal in (omega, k) with omega = (2n+1) pi / N_tau; must invert M[0].
    lat = O.Lattice(nx, ntau, 0.05, 5.0)
    zero = np.zeros(lat.shape)
    v = np.random.default_rng(4).standard_normal(lat.shape)
    assert np.allclose(O.apply_M(lat, zero, O.apply_M0inv(lat, v)), v, atol=1e-12)
    assert np.allclose(O.apply_Mdag(lat, zero, O.apply_M0invT(lat, v)), v, atol=1e-12)
    if nx == 4:
        M0 = O.dense_from_apply(lambda x: O.apply_M(lat, zero, x), lat.shape)
        Mi = O.dense_from_apply(lambda x: O.apply_M0inv(lat, x), lat.shape)
        assert np.allclose(Mi, np.linalg.inv(M0), atol=1e-12)


def test_Q_is_symmetric_positive_definite():
    lat, sigma, _ = _tiny(4, 4, seed=5)
    Qd = O.dense_from_apply(lambda x: O.apply_Q(lat, sigma, x), lat.shape)
    assert np.allclose(Qd, Qd.T, atol=1e-13)
    assert np.linalg.eigvalsh(Qd).min() > 0
