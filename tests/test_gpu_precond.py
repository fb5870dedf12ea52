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
@pytest.mark.parametrize("order,accel,p,s", [(2, "euler23", 0.5, 1.0), (4, "euler23", 0.5, 1.0),
                                             (6, "euler23", 0.4, 1.0), (2, "vanw", 0.5, 1.0),
                                             (4, "vanw", 0.5, 2.0), (4, "vanw", 0.3, 0.5),
                                             (3, "euler", 0.35, 1.0)])
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("nx,ntau", [(8, 24), (16, 12)])
def test_wce_accelerated_parity(ufg, order, accel, p, s, transpose, nx, ntau, dtype, tol):
    # the Euler S_{2k/3,k/3} variant and the special van Wijngaarden transformation (Sec. 3.1):
    # the library's host-side weights (its own recursion and quadrature) against the oracle's
    lat, field, solver, sigma, rd, r, olat = _setup(ufg, nx, ntau, 8, dtype)
    solver.ufg_set_preconditioner("wce", order=order, euler=accel, p=p, s=s)
    z = solver.ufg_apply_preconditioner(field, rd, transpose=transpose).double().cpu().numpy()
    fn = O.wce_apply_T if transpose else O.wce_apply
    assert _rel(z, fn(olat, sigma, r, order, accel, None, p, s)) < tol


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-11), (torch.float32, 1e-4)])
@pytest.mark.parametrize("order,accel", [(0, "none"), (2, "none"), (2, "euler23"), (4, "vanw")])
@pytest.mark.parametrize("nx,ntau", [(8, 24), (16, 12), (6, 10)])
def test_two_sided_wce_for_cg_parity(ufg, order, accel, nx, ntau, dtype, tol):
    # the CG form P_d P_d^T of the weak-coupling preconditioner (ufg_apply_preconditioner with
    # transpose = 2) against the oracle's
    lat, field, solver, sigma, rd, r, olat = _setup(ufg, nx, ntau, 9, dtype)
    solver.ufg_set_preconditioner("wce", order=order, euler=accel)
    z = solver.ufg_apply_preconditioner(field, rd, transpose=2).double().cpu().numpy()
    ref = O.make_preconditioner(olat, sigma, {"kind": "wce", "order": order, "euler": accel},
                                normal=True)(r)
    assert _rel(z, ref) < tol


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-10), (torch.float32, 2e-3)])
@pytest.mark.parametrize("degree,eps", [(8, 0.01), (16, 1e-3)])
@pytest.mark.parametrize("nx,ntau", [(8, 16), (6, 10)])
def test_sca_chebyshev_parity(ufg, degree, eps, nx, ntau, dtype, tol):
    # SCA with the Chebyshev polynomial as a secondary filter, explicit scale and eps
    lat, field, solver, sigma, rd, r, olat = _setup(ufg, nx, ntau, 10, dtype)
    s = O.sca_cheb_scale(olat, sigma, 2.0)
    solver.ufg_set_preconditioner("sca_cheb", alpha=2.0, degree=degree, eps=eps, scale=s)
    z = solver.ufg_apply_preconditioner(field, rd, transpose=2).double().cpu().numpy()
    ref = O.sca_cheb_apply(olat, sigma, r, 2.0, degree, eps, s)
    assert _rel(z, ref) < tol


def test_sca_chebyshev_default_scale_matches_oracle_estimate(ufg):
    # the library's own power-method estimate of the spectral scale (FP64, same start vector)
    lat, field, solver, sigma, rd, r, olat = _setup(ufg, 8, 16, 11)
    solver.ufg_set_preconditioner("sca_cheb", alpha=2.0, degree=8)
    z = solver.ufg_apply_preconditioner(field, rd, transpose=2).cpu().numpy()
    ref = O.sca_cheb_apply(olat, sigma, r, 2.0, 8)
    assert _rel(z, ref) < 1e-9


def test_wce_rejects_bad_acceleration(ufg):
    lat = ufg.Lattice(4, 8)
    solver = ufg.Solver(lat)
    for kw in ({"euler": 4}, {"euler": "vanw", "s": -1.0}, {"euler": "euler", "p": 1.5}):
        with pytest.raises(ufg.UfgError):
            solver.ufg_set_preconditioner("wce", order=2, **kw)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-11), (torch.float32, 1e-4)])
@pytest.mark.parametrize("nx,ntau", [(4, 16), (10, 12), (16, 20), (16, 9), (32, 6)])
def test_wce_parity_shapes(ufg, nx, ntau, dtype, tol):
    # N_x = 8 and 16 run the momentum-space M1 term as one fused kernel per slice
    lat, field, solver, sigma, rd, r, olat = _setup(ufg, nx, ntau, 5, dtype)
    solver.ufg_set_preconditioner("wce", order=2)
    for tr, fn in [(False, O.wce_apply), (True, O.wce_apply_T)]:
        z = solver.ufg_apply_preconditioner(field, rd, transpose=tr).double().cpu().numpy()
        assert _rel(z, fn(olat, sigma, r, 2)) < tol


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-11), (torch.float32, 1e-4)])
@pytest.mark.parametrize("order,euler", [(2, False), (4, "euler23")])
@pytest.mark.parametrize("nx,ntau", [(4, 200), (6, 131)])
def test_wce_parity_long_time_extents(ufg, nx, ntau, order, euler, dtype, tol):
    # per-thread recurrence chunks of N_tau / 8 = 17 and 25 elements: several load groups of the
    # writing, assigning and accumulating recurrences plus a ragged tail, in both directions
    lat, field, solver, sigma, rd, r, olat = _setup(ufg, nx, ntau, 6, dtype)
    solver.ufg_set_preconditioner("wce", order=order, euler=euler)
    for tr, fn in [(False, O.wce_apply), (True, O.wce_apply_T)]:
        z = solver.ufg_apply_preconditioner(field, rd, transpose=tr).double().cpu().numpy()
        err = _rel(z, fn(olat, sigma, r, order, euler))
        assert err < tol, (tr, err)


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
