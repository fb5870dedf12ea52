"""Pins of the oracle's solvers (Eq. 1-3) and of the MV accounting of Sec. 5, and of the force."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1008_3647_gb300.inputs import field_and_source


def _dense(lat, sigma, op):
    return O.dense_from_apply(lambda x: op(lat, sigma, x), lat.shape)


def test_cg_normal_matches_dense_solve():
    lat = O.Lattice(4, 6, 0.05, 5.0)
    sigma, b = field_and_source(4, 6, 0)
    x, info = O.solve_cg_normal(lat, sigma, b, tol=1e-12)
    ref = np.linalg.solve(_dense(lat, sigma, O.apply_Q), b.ravel())
    assert info["converged"]
    assert np.allclose(x.ravel(), ref, rtol=1e-8, atol=1e-8 * np.abs(ref).max())


@pytest.mark.parametrize("pc", [None, {"kind": "cheb", "degree": 8}, {"kind": "sca", "alpha": 2.0}])
def test_preconditioned_cg_reaches_true_residual(pc):
    lat = O.Lattice(4, 8, 0.05, 5.0)
    sigma, b = field_and_source(4, 8, 2)
    x, info = O.solve_cg_normal(lat, sigma, b, tol=1e-10, pc=pc)
    r = b - O.apply_Q(lat, sigma, x)
    assert info["converged"]
    assert np.linalg.norm(r) <= 2e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("pc", [None, {"kind": "wce", "order": 0}, {"kind": "wce", "order": 2},
                                {"kind": "wce", "order": 2, "euler": True}])
def test_two_step_bicgstab_composite_residual(pc):
    lat = O.Lattice(4, 8, 0.05, 5.0)
    sigma, b = field_and_source(4, 8, 3)
    x, info = O.solve_bicgstab_two_step(lat, sigma, b, tol=1e-10, pc=pc)
    r = b - O.apply_Q(lat, sigma, x)
    assert info["converged"]
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)


def test_bicgstab_matches_dense_solve():
    lat = O.Lattice(4, 4, 0.05, 5.0)
    sigma, b = field_and_source(4, 4, 8)
    Md = _dense(lat, sigma, O.apply_M)
    x, it, ok = O.bicgstab(lambda u: O.apply_M(lat, sigma, u), b, 1e-13, 500)
    assert ok and np.allclose(x.ravel(), np.linalg.solve(Md, b.ravel()), atol=1e-10)


def test_wce_preconditioner_cuts_iterations():
    # Sec. 5: WCE preconditioning lowers the BiCGStab iteration count (Table 1's trend).
    lat = O.Lattice(4, 16, 0.05, 5.0)
    sigma, b = field_and_source(4, 16, 0)
    its = [O.solve_bicgstab_two_step(lat, sigma, b, 1e-10, pc=pc)[1]["iterations"]
           for pc in (None, {"kind": "wce", "order": 0}, {"kind": "wce", "order": 2})]
    assert its[1] < its[0] and its[2] <= its[1]


def test_mv_formula_reproduces_table2_from_table1(golden_dir):
    # Sec. 5: Table 2 = Table 1 x per-iteration MV cost; exact for Chebyshev and WCE, ~3 for SCA.
    rows = {}
    for line in open(os.path.join(golden_dir, "paper_tables_1_2.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows[(f[0], int(f[1]), int(f[2]))] = [None if v == "-" else int(v) for v in f[3:]]
    n = 0
    for (tab, nx, nt), t1 in rows.items():
        if tab != "T1":
            continue
        t2 = rows[("T2", nx, nt)]
        for col, (kind, d) in enumerate([("cheb", 8), ("cheb", 16), ("cheb", 32)]):
            if t1[col] is not None:
                assert O.mv_formula(kind, t1[col], d) == t2[col]
                n += 1
        for j, d in enumerate((0, 1, 2)):
            if t1[4 + j] is not None:
                assert O.mv_formula("wce", t1[4 + j], d) == t2[4 + j]
                n += 1
        if t1[3] is not None:
            assert abs(t2[3] / O.mv_formula("sca", t1[3]) - 1) < 1e-3
            n += 1
    assert n == 9 * 7 - 3  # three entries are '-' in Table 1


def test_pseudofermion_action_of_heatbath_source():
    # phi = M^dagger eta gives Q^{-1} phi = M^{-1} eta and S = phi^T Q^{-1} phi = |eta|^2.
    lat = O.Lattice(4, 6, 0.05, 5.0)
    sigma, eta = field_and_source(4, 6, 12)
    phi = O.apply_Mdag(lat, sigma, eta)
    S, X = O.pseudofermion_action(lat, sigma, phi, tol=1e-13)
    assert S == pytest.approx(float(np.sum(eta * eta)), rel=1e-9)


def test_force_matches_central_finite_differences():
    # dS/dsigma of S = phi^T Q^{-1} phi (the paper's fermion force with a minus sign, Sec. 1),
    # against central differences of S computed with dense solves.
    lat = O.Lattice(2, 5, 0.05, 5.0)
    sigma, eta = field_and_source(2, 5, 21)
    phi = O.apply_Mdag(lat, sigma, eta)

    def S(sig):
        Q = _dense(lat, sig, O.apply_Q)
        return float(phi.ravel() @ np.linalg.solve(Q, phi.ravel()))
    Q = _dense(lat, sigma, O.apply_Q)
    X = np.linalg.solve(Q, phi.ravel()).reshape(lat.shape)
    F = O.force_dS_dsigma(lat, sigma, X)
    h = 1e-5
    for idx in [0, 3, 7, 11, 17, 22, 39]:
        sp = sigma.copy().ravel(); sp[idx] += h
        sm = sigma.copy().ravel(); sm[idx] -= h
        fd = (S(sp.reshape(lat.shape)) - S(sm.reshape(lat.shape))) / (2 * h)
        assert F.ravel()[idx] == pytest.approx(fd, rel=1e-6, abs=1e-7)
