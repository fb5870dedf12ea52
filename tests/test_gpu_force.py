"""HMC force dS/dsigma of S = phi^T (M^T M)^{-1} phi on the GPU: kernel parity with the oracle's
force formula for the same X (1e-12), agreement with central finite differences of S computed by
GPU solves (relative 1e-6), the heat-bath identity S = |eta|^2, and the autograd wrapper."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_3647_gb300.inputs import field_and_source, sample_sites

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ufg():
    from paper_1008_3647_gb300 import ufg as u
    u.load()
    return u


@pytest.mark.parametrize("nx,ntau", [(4, 8), (8, 32), (32, 6)])
def test_force_kernel_parity(ufg, nx, ntau):
    sigma, X = field_and_source(nx, ntau, 31)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    solver = ufg.Solver(lat)
    dS = solver.ufg_force_from_solution(field, torch.from_numpy(X).cuda()).cpu().numpy()
    ref = O.force_dS_dsigma(O.Lattice(nx, ntau), sigma, X)
    assert float(np.abs(dS - ref).max() / np.abs(ref).max()) < 1e-12


def _action(ufg, lat, solver, sigma, phi):
    field = ufg.Field(lat, sigma)
    S, X, st = solver.ufg_pseudofermion_action(field, phi, tol=1e-13)
    assert st["status"] == ufg.UFG_OK, st
    return S, X


@pytest.mark.parametrize("nx,ntau,nsites", [(8, 32, 64)])
def test_force_matches_central_differences(ufg, nx, ntau, nsites):
    sigma, eta = field_and_source(nx, ntau, 41)
    lat = ufg.Lattice(nx, ntau)
    solver = ufg.Solver(lat)
    solver.ufg_set_preconditioner("wce", order=2)
    sig = torch.from_numpy(sigma).cuda()
    field = ufg.Field(lat, sig)
    phi = ufg.ufg_apply_Mdag(field, torch.from_numpy(eta).cuda())
    dS, X, S0, st = solver.ufg_hmc_force(field, phi, tol=1e-13)
    assert st["status"] == ufg.UFG_OK
    assert S0 == pytest.approx(float(np.sum(eta * eta)), rel=1e-9)  # phi = M^T eta => S = |eta|^2
    h = 1e-4
    dS = dS.cpu().numpy().ravel()
    for i in sample_sites(lat.shape, nsites, 5):
        sp = sig.clone().view(-1)
        sp[i] += h
        sm = sig.clone().view(-1)
        sm[i] -= h
        Sp, _ = _action(ufg, lat, solver, sp.view(lat.shape), phi)
        Sm, _ = _action(ufg, lat, solver, sm.view(lat.shape), phi)
        fd = (Sp - Sm) / (2 * h)
        assert dS[i] == pytest.approx(fd, rel=1e-6, abs=1e-8 * abs(S0))


def test_force_matches_oracle_gradient_8cubed(ufg):
    # GPU solve + GPU force against the oracle's solve + oracle force on an 8^3 lattice
    nx, ntau = 8, 16
    sigma, eta = field_and_source(nx, ntau, 43)
    olat = O.Lattice(nx, ntau)
    phi = O.apply_Mdag(olat, sigma, eta)
    Xo, _ = O.solve_cg_normal(olat, sigma, phi, tol=1e-13)
    ref = O.force_dS_dsigma(olat, sigma, Xo)
    lat = ufg.Lattice(nx, ntau)
    solver = ufg.Solver(lat)
    solver.ufg_set_preconditioner("wce", order=2)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    dS, X, S, st = solver.ufg_hmc_force(field, torch.from_numpy(phi).cuda(), tol=1e-12)
    assert float(np.abs(dS.cpu().numpy() - ref).max() / np.abs(ref).max()) < 1e-8


def test_force_full_size_32cubed_x512(ufg):
    # the HMC force workload itself (32^3 x 512, 16.8M sites): mixed-precision solve of
    # M^T M X = phi with phi = M^T eta, then the force kernel; the oracle recomputes the solve's
    # true residual and the force formula from the same X
    nx, ntau = 32, 512
    sigma, eta = field_and_source(nx, ntau, 51)
    olat = O.Lattice(nx, ntau)
    lat = ufg.Lattice(nx, ntau)
    solver = ufg.Solver(lat)
    solver.ufg_set_preconditioner("wce", order=2)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    phi = ufg.ufg_apply_Mdag(field, torch.from_numpy(eta).cuda())
    dS, X, S0, st = solver.ufg_hmc_force(field, phi, tol=1e-10, precision=ufg.UFG_MIXED)
    assert st["status"] == ufg.UFG_OK, st
    assert S0 == pytest.approx(float(np.sum(eta * eta)), rel=1e-8)  # S = |eta|^2
    Xh, ph = X.cpu().numpy(), phi.cpu().numpy()
    r = ph - O.apply_Q(olat, sigma, Xh)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(ph)
    ref = O.force_dS_dsigma(olat, sigma, Xh)
    assert float(np.abs(dS.cpu().numpy() - ref).max() / np.abs(ref).max()) < 1e-12


def test_force_full_size_central_differences(ufg):
    # Config 5 in full: dS/dsigma on 64 seeded sites of the 32^3 x 512 lattice against central
    # differences [S(sigma + h e_i) - S(sigma - h e_i)] / 2h of S = phi^T Q^{-1} phi.  S itself is
    # extensive (|eta|^2 ~ 1.7e7), so the difference of two separately solved actions cancels
    # ~10 digits; it is evaluated instead as the exact identity
    #   S+ - S- = phi^T (Q+^{-1} - Q-^{-1}) phi = X+^T (Q- - Q+) X-,   X+- = Q+-^{-1} phi,
    # with M+ = M- + D, D x = -sgn K(dw x_t(r) e_r) on slice t+1 (+ at the antiperiodic wrap),
    # dw = A (sin(sigma+h) - sin(sigma-h)) = 2 A cos(sigma) sin(h):
    #   X+^T (Q- - Q+) X- = -[(M- X+).(D X-) + (D X+).(M- X-) + (D X+).(D X-)],
    # every term a product with the localised vector D X, so nothing cancels.
    nx, ntau = 32, 512
    V = nx ** 3
    sigma, eta = field_and_source(nx, ntau, 51)
    lat = ufg.Lattice(nx, ntau)
    solver = ufg.Solver(lat)
    solver.ufg_set_preconditioner("wce", order=2)
    sig = torch.from_numpy(sigma).cuda()
    field = ufg.Field(lat, sig)
    phi = ufg.ufg_apply_Mdag(field, torch.from_numpy(eta).cuda())
    kw = {"tol": 1e-12, "precision": ufg.UFG_MIXED}
    dS, _, _, st = solver.ufg_hmc_force(field, phi, **kw)
    assert st["status"] == ufg.UFG_OK, st
    dS = dS.view(-1)
    h = 1e-4  # central-difference truncation ~h^2/6 relative
    fp, fm = ufg.Field(lat, sig), ufg.Field(lat, sig)
    zero = torch.zeros(lat.shape, dtype=torch.float64, device="cuda")

    def D(X, t, r, dw):
        u = zero.clone()
        u.view(ntau, V)[t, r] = dw * X.view(ntau, V)[t, r]
        Ku = ufg.ufg_apply_kinetic(field, u).view(ntau, V)
        out = zero.clone().view(ntau, V)
        out[(t + 1) % ntau] = (-1.0 if t < ntau - 1 else 1.0) * Ku[t]
        return out.view(lat.shape)

    worst = 0.0
    for i in sample_sites(lat.shape, 64, 7):
        t, r = divmod(int(i), V)
        sp, sm = sig.clone().view(-1), sig.clone().view(-1)
        sp[i] += h
        sm[i] -= h
        fp.update(sp.view(lat.shape))
        fm.update(sm.view(lat.shape))
        _, Xp, s1 = solver.ufg_pseudofermion_action(fp, phi, **kw)
        _, Xm, s2 = solver.ufg_pseudofermion_action(fm, phi, **kw)
        assert s1["status"] == ufg.UFG_OK and s2["status"] == ufg.UFG_OK
        dw = 2.0 * lat.A * np.cos(float(sigma.reshape(-1)[i])) * np.sin(h)
        DXp, DXm = D(Xp, t, r, dw), D(Xm, t, r, dw)
        MXp, MXm = ufg.ufg_apply_M(fm, Xp), ufg.ufg_apply_M(fm, Xm)
        delta = -float((MXp * DXm).sum() + (DXp * MXm).sum() + (DXp * DXm).sum())
        fd = delta / (2 * h)
        err = abs(float(dS[i]) - fd) / max(abs(fd), 1e-3 * float(dS.abs().max()))
        worst = max(worst, err)
    assert worst < 1e-6, worst


def test_autograd_backward_is_force(ufg):
    nx, ntau = 6, 10
    sigma, eta = field_and_source(nx, ntau, 44)
    lat = ufg.Lattice(nx, ntau)
    solver = ufg.Solver(lat)
    solver.ufg_set_preconditioner("wce", order=1)
    sig = torch.from_numpy(sigma).cuda().requires_grad_(True)
    field = ufg.Field(lat, sig.detach())
    phi = ufg.ufg_apply_Mdag(field, torch.from_numpy(eta).cuda())
    S = ufg.PseudofermionAction.apply(sig, phi, solver, {"tol": 1e-12})
    S.backward()
    dS, _, S2, _ = solver.ufg_hmc_force(field, phi, tol=1e-12)
    assert float(S.detach()) == pytest.approx(S2, rel=1e-10)
    assert torch.allclose(sig.grad, dS, rtol=1e-8, atol=1e-10 * float(dS.abs().max()))
