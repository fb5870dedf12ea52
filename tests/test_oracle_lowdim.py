"""Pins of the oracle on lower-dimensional lattices (N_x^dim x N_tau, dim = 1, 2), to which the
methods carry over unchanged (Sec. 6): only the kinetic factor's dimension changes.  Each pin is
fixed by a closed form or a construction independent of the oracle's FFT path (no GPU)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1008_3647_gb300.inputs import field_and_source


def _circulant_1d(nx, tau, dispersion):
    """exp(-tau K) on one axis summed directly: T_ij = (1/N) sum_k exp(-tau E(k)) cos(k (i - j))
    over k = 2 pi n / N, n = -N/2 .. N/2 - 1 (Sec. 1)."""
    n = np.arange(-nx // 2, nx // 2)
    k = 2 * np.pi * n / nx
    e = 0.5 * k ** 2 if dispersion == 0 else 1.0 - np.cos(k)
    d = np.arange(nx)[:, None] - np.arange(nx)[None, :]
    return np.einsum("k,kij->ij", np.exp(-tau * e), np.cos(k[:, None, None] * d[None])) / nx


@pytest.mark.parametrize("dispersion", [0, 1])
@pytest.mark.parametrize("dim", [1, 2])
def test_kinetic_is_the_direct_sum_circulant(dim, dispersion):
    # Sec. 1 (K diagonal in momentum space) on dim axes: the dense kinetic operator is the
    # direct-sum circulant T in 1-D and its Kronecker square T (x) T in 2-D
    nx, tau = 6, 0.05
    lat = O.Lattice(nx, 2, tau, 5.0, dispersion, dim)
    Kd = O.dense_from_apply(lambda u: O.kinetic(lat, u[None])[0], (nx,) * dim)
    T = _circulant_1d(nx, tau, dispersion)
    ref = T if dim == 1 else np.kron(T, T)
    assert np.allclose(Kd, ref, atol=1e-14)


@pytest.mark.parametrize("dim", [1, 2])
def test_plane_wave_eigenvalues(dim):
    nx, tau = 8, 0.05
    lat = O.Lattice(nx, 2, tau, 5.0, 0, dim)
    grids = np.meshgrid(*([np.arange(nx)] * dim), indexing="ij")
    for n in [(0, 0), (1, 0), (3, -2), (-4, 1)]:
        k = [2 * np.pi * ni / nx for ni in n[:dim]]
        u = np.cos(sum(ki * g for ki, g in zip(k, grids)))
        out = O.kinetic(lat, np.stack([u, u]))
        e = 0.5 * sum(ki * ki for ki in k)
        assert np.allclose(out, math.exp(-tau * e) * np.stack([u, u]), atol=1e-13)


@pytest.mark.parametrize("dim,nx,ntau", [(1, 8, 6), (1, 4, 10), (2, 4, 6), (2, 6, 4)])
def test_free_gas_determinant(dim, nx, ntau):
    # sigma = 0: det M0 = prod_k (1 + exp(-beta E(k))) (free fermions, antiperiodic time)
    lat = O.Lattice(nx, ntau, 0.05, 5.0, 0, dim)
    Mo = O.dense_from_apply(lambda u: O.apply_M(lat, np.zeros(lat.shape), u), lat.shape)
    sign, logdet = np.linalg.slogdet(Mo)
    k = 2 * np.pi * np.arange(-nx // 2, nx // 2) / nx
    e1 = 0.5 * k ** 2
    E = e1 if dim == 1 else (e1[:, None] + e1[None, :]).ravel()
    assert sign > 0 and logdet == pytest.approx(np.sum(np.log1p(np.exp(-lat.beta * E))),
                                                rel=1e-12)


@pytest.mark.parametrize("dim", [1, 2])
def test_dense_M_matches_block_definition(dim):
    # Eq. (MatrixM): 1 on the diagonal, -B_j below it, +B_{N_tau} in the corner, with
    # B_j = T (x) ... (x) T diag(1 + A sin sigma_j) built from the direct-sum circulant
    nx, ntau = 4, 5
    lat = O.Lattice(nx, ntau, 0.05, 5.0, 0, dim)
    sigma, _ = field_and_source(nx, ntau, 2, dim)
    T = _circulant_1d(nx, 0.05, 0)
    K = T if dim == 1 else np.kron(T, T)
    V = lat.volume
    w = 1 + lat.A * np.sin(sigma.reshape(ntau, V))
    Md = np.eye(V * ntau)
    for t in range(ntau - 1):
        Md[(t + 1) * V:(t + 2) * V, t * V:(t + 1) * V] = -K @ np.diag(w[t])
    Md[0:V, (ntau - 1) * V:] = K @ np.diag(w[-1])
    Mo = O.dense_from_apply(lambda u: O.apply_M(lat, sigma, u), lat.shape)
    assert np.allclose(Mo, Md, atol=1e-13)
    Mt = O.dense_from_apply(lambda u: O.apply_Mdag(lat, sigma, u), lat.shape)
    assert np.allclose(Mt, Md.T, atol=1e-13)
    Qd = O.dense_from_apply(lambda u: O.apply_Q(lat, sigma, u), lat.shape)
    assert np.allclose(Qd, Md.T @ Md, atol=1e-12)


@pytest.mark.parametrize("dim", [1, 2])
def test_M0inv_inverts_M0(dim):
    # Sec. 3: M0^{-1} (Fourier acceleration) is the exact inverse of M at sigma = 0
    lat = O.Lattice(6, 8, 0.05, 5.0, 0, dim)
    _, y = field_and_source(6, 8, 4, dim)
    zero = np.zeros(lat.shape)
    assert np.allclose(O.apply_M(lat, zero, O.apply_M0inv(lat, y)), y, atol=1e-12)
    assert np.allclose(O.apply_Mdag(lat, zero, O.apply_M0invT(lat, y)), y, atol=1e-12)


@pytest.mark.parametrize("dim", [1, 2])
def test_solvers_reach_the_dense_solution(dim):
    # Eq. (1) / Eq. (2): CG on Q and two-step BiCGStab with the paper's preconditioners solve the
    # same system as a dense solve
    nx, ntau = 4, 6
    lat = O.Lattice(nx, ntau, 0.05, 5.0, 0, dim)
    sigma, b = field_and_source(nx, ntau, 9, dim)
    Qd = O.dense_from_apply(lambda u: O.apply_Q(lat, sigma, u), lat.shape)
    ref = np.linalg.solve(Qd, b.ravel()).reshape(lat.shape)
    for pc in ({"kind": "cheb", "degree": 8}, {"kind": "sca", "alpha": 2.0}):
        x, info = O.solve_cg_normal(lat, sigma, b, 1e-12, 5000, pc)
        assert info["converged"] and np.allclose(x, ref, rtol=1e-8, atol=1e-9)
    x, info = O.solve_bicgstab_two_step(lat, sigma, b, 1e-12, 5000,
                                        {"kind": "wce", "order": 2, "euler": "euler23"})
    assert info["converged"] and np.allclose(x, ref, rtol=1e-8, atol=1e-9)
