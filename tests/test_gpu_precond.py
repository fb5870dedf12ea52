"""GPU parity of the three preconditioners (through the C ABI) against the FP64 oracle.

FP64 tolerances: SCA 1e-12 (a recurrence of O(N_tau) rounding steps); weak coupling 1e-11 (d+1
exact inverses of O(N_tau + 3N) steps each); Chebyshev 1e-9 relative (degree-d polynomial in Q
whose factors are individually far from 1, amplifying rounding by the factors' spread).
FP32: 1e-4 for the recurrences, 2e-3 for the Chebyshev polynomial (same amplification at
FP32 unit roundoff)."""
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


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _setup(ufg, nx, ntau, seed, dtype=torch.float64):
    sigma, r = field_and_source(nx, ntau, seed)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    rd = torch.from_numpy(r).to("cuda", dtype)
    return lat, field, solver, sigma, rd, rd.double().cpu().numpy(), O.Lattice(nx, ntau)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-4)])
@pytest.mark.parametrize("nx,ntau,alpha", [(4, 16, 2.0), (8, 64, 2.0), (6, 7, 1.5), (16, 33, 3.0)])
def test_sca_parity(ufg, nx, ntau, alpha, dtype, tol):
    lat, field, solver, sigma, rd, r, olat = _setup(ufg, nx, ntau, 3, dtype)
    solver.ufg_set_preconditioner("sca", alpha=alpha)
    z = solver.ufg_apply_preconditioner(field, rd).double().cpu().numpy()
    D, L = O.sca_factors(olat, sigma, alpha)
    assert _rel(z, O.sca_apply(D, L, r)) < tol


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-11), (torch.float32, 1e-4)])
@pytest.mark.parametrize("order,euler", [(0, False), (1, False), (2, False), (4, False), (2, True),
                                         (4, True)])
@pytest.mark.parametrize("transpose", [False, True])
def test_wce_parity(ufg, order, euler, transpose, dtype, tol):
    nx, ntau = 8, 24
    lat, field, solver, sigma, rd, r, olat = _setup(ufg, nx, ntau, 4, dtype)
    solver.ufg_set_preconditioner("wce", order=order, euler=euler)
    z = solver.ufg_apply_preconditioner(field, rd, transpose=transpose).double().cpu().numpy()
    fn = O.wce_apply_T if transpose else O.wce_apply
    assert _rel(z, fn(olat, sigma, r, order, euler)) < tol


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-11), (torch.float32, 1e-4)])
@pytest.mark.parametrize("nx,ntau", [(4, 16), (10, 12), (16, 20), (16, 9), (32, 6)])
def test_wce_parity_shapes(ufg, nx, ntau, dtype, tol):
    # N_x = 8 and 16 run the momentum-space M1 term as one fused kernel per slice
    lat, field, solver, sigma, rd, r, olat = _setup(ufg, nx, ntau, 5, dtype)
    solver.ufg_set_preconditioner("wce", order=2)
    for tr, fn in [(False, O.wce_apply), (True, O.wce_apply_T)]:
        z = solver.ufg_apply_preconditioner(field, rd, transpose=tr).double().cpu().numpy()
        assert _rel(z, fn(olat, sigma, r, 2)) < tol


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-9), (torch.float32, 2e-3)])
@pytest.mark.parametrize("degree", [8, 16, 32])
def test_chebyshev_parity(ufg, degree, dtype, tol):
    nx, ntau = 8, 16
    lat, field, solver, sigma, rd, r, olat = _setup(ufg, nx, ntau, 6, dtype)
    solver.ufg_set_preconditioner("cheb", degree=degree)
    z = solver.ufg_apply_preconditioner(field, rd).double().cpu().numpy()
    s, eps = O.cheb_scale_eps(olat, sigma)
    ref = O.cheb_apply(lambda u: O.apply_Q(olat, sigma, u), r, degree, eps, s)
    assert _rel(z, ref) < tol


def test_chebyshev_explicit_scale_and_eps(ufg):
    lat, field, solver, sigma, rd, r, olat = _setup(ufg, 6, 10, 7)
    solver.ufg_set_preconditioner("cheb", degree=16, eps=0.01, scale=9.5)
    z = solver.ufg_apply_preconditioner(field, rd).cpu().numpy()
    ref = O.cheb_apply(lambda u: O.apply_Q(olat, sigma, u), r, 16, 0.01, 9.5)
    assert _rel(z, ref) < 1e-9
