"""Pins of the oracle's preconditioners: Chebyshev (Sec. 2), weak coupling + Euler (Sec. 3),
strong coupling (Sec. 4)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1008_3647_gb300.inputs import field_and_source


@pytest.mark.parametrize("n", [4, 8, 16])
@pytest.mark.parametrize("eps", [1e-2, 1e-3])
def test_chebyshev_error_bound(n, eps):
    # Sec. 2: |R| = |(P(z) - 1/z) z| <= 2 ((1 - sqrt eps)/(1 + sqrt eps))^(2n+1) on [eps, 1].
    z = np.linspace(eps, 1.0, 4001)
    R = np.abs(O.cheb_scalar(z, n, eps) * z - 1.0)
    bound = 2 * ((1 - math.sqrt(eps)) / (1 + math.sqrt(eps))) ** (2 * n + 1)
    assert R.max() <= bound * (1 + 1e-9)
    # the bound is nearly attained (the polynomial is the minimax one, not something smaller)
    assert R.max() >= 0.5 * bound


def test_chebyshev_real_quadratic_pairing_equals_root_product():
    for n, eps in [(4, 0.01), (8, 0.003), (16, 0.02)]:
        a, b, norm = O.cheb_quadratic_factors(n, eps)
        z0 = 0.5 * (1 + eps)
        z = np.linspace(0.0, 1.2, 97)
        p = np.ones_like(z)
        for k in range(n):
            p *= ((z - a[k]) ** 2 + b[k] ** 2) / norm[k]
        assert np.allclose(p / z0, O.cheb_scalar(z, n, eps), rtol=1e-10, atol=1e-12)


def test_bit_reversed_order_is_a_permutation():
    assert O.bit_reversed(4) == [0, 2, 1, 3]
    assert O.bit_reversed(8) == [0, 4, 2, 6, 1, 5, 3, 7]
    for n in (1, 3, 5, 16):
        assert sorted(O.bit_reversed(n)) == list(range(n))


def test_chebyshev_apply_is_matrix_function_of_Q():
    # P(Q/s)/s computed factor by factor equals the matrix function through the eigensystem.
    lat = O.Lattice(4, 4, 0.05, 5.0)
    sigma, v = field_and_source(4, 4, 11)
    s, eps = O.cheb_scale_eps(lat, sigma)
    Qd = O.dense_from_apply(lambda x: O.apply_Q(lat, sigma, x), lat.shape)
    lam, U = np.linalg.eigh(Qd)
    assert lam.max() <= s  # the scale bounds the spectrum
    for d in (8, 16):
        ref = U @ (O.cheb_scalar(lam / s, d // 2, eps) / s * (U.T @ v.ravel()))
        out = O.cheb_apply(lambda x: O.apply_Q(lat, sigma, x), v, d, eps, s)
        assert np.allclose(out.ravel(), ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def test_euler_transform_geometric_closed_form():
    # Eq. (Euler) with p applied d times to the partial sums of sum (-x)^n has the closed form
    # [1 + x (p - (1-p) x)^d] / (1 + x) (binomial theorem).
    for x in (0.3, 0.9, 1.5):
        for d in (1, 2, 4, 7):
            for p in (0.5, 0.3):
                S = np.cumsum([(-x) ** n for n in range(d + 1)])
                got = O.euler_transform(S, p)
                assert got == pytest.approx((1 + x * (p - (1 - p) * x) ** d) / (1 + x), rel=1e-13)


def test_euler_accelerates_log2_series():
    S = np.cumsum([(-1) ** n / (n + 1) for n in range(12)])
    assert abs(O.euler_transform(S) - math.log(2)) < 1e-3 * abs(S[-1] - math.log(2))


def test_euler_weights_order2():
    # d = 2, p = 1/2: the weights of the three series terms are (1, 3/4, 1/4).
    assert np.allclose(O.euler_weights(2, True), [1.0, 0.75, 0.25])
    assert np.allclose(O.euler_weights(3, False), [1, 1, 1, 1])


def test_euler_table_geometric_closed_form():
    # Eq. (Euler) on the partial sums L (1 - (-x)^(k+1)) of sum (-x)^n, L = 1/(1+x): one step maps
    # (-x)^(k+1) to (-x)^(k+1) (p - (1-p) x), so S_{j,k} = L (1 - (-x)^(k+1) (p - (1-p) x)^j).
    for x in (0.3, 0.9, 1.5):
        for d in (2, 4, 6):
            S = np.cumsum([(-x) ** n for n in range(d + 1)])
            for p in (0.5, 0.3):
                for j in range(d + 1):
                    for k in range(d - j + 1):
                        ref = (1 - (-x) ** (k + 1) * (p - (1 - p) * x) ** j) / (1 + x)
                        assert O.euler_table(S, j, k, p) == pytest.approx(ref, rel=1e-12, abs=1e-14)
    with pytest.raises(ValueError):
        O.euler_table(np.ones(3), 2, 1)


def test_euler_23_level_reading():
    # S_{2 kmax/3, kmax/3}: exact where 3 divides kmax, otherwise the nearest level, k = kmax - j
    assert [O.euler_23_level(d) for d in (3, 6, 9, 12)] == [2, 4, 6, 8]
    assert [O.euler_23_level(d) for d in (1, 2, 4, 5, 7)] == [1, 1, 3, 3, 5]
    # order 2: S_{1,1} = (S_{0,1} + S_{0,2}) / 2, weights (1, 1, 1/2)
    assert np.allclose(O.euler_weights(2, "euler23"), [1.0, 1.0, 0.5])
    # the weights reproduce the table entry on any series
    t = np.array([1.0, -0.7, 0.45, -0.3, 0.2])
    for d, j in ((4, 3), (3, 2)):
        assert O.euler_weights(d, "euler23") @ t[:d + 1] == pytest.approx(
            O.euler_table(np.cumsum(t[:d + 1]), j, d - j), rel=1e-14)


def test_vanwijngaarden_unit_lambda_mu_is_classical_euler_series():
    # lambda_k = 1 with phi = delta(t - 1) gives mu_k = 1, and the estimate is the truncated
    # classical Euler series sum_{n<=d} b_n; on sum (-x)^n, b_n = (1-p) (p - (1-p) x)^n.
    for x in (0.4, 1.2):
        for p in (0.5, 0.35):
            for d in (0, 3, 8):
                c = O.vanwijngaarden_weights(d, np.ones(d + 1), np.ones(d + 1), p)
                r = p - (1 - p) * x
                ref = (1 - p) * (1 - r ** (d + 1)) / (1 - r)
                assert c @ np.array([(-x) ** n for n in range(d + 1)]) == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("s", [0.5, 1.0, 2.0])
def test_special_vanwijngaarden_mu_closed_form(s):
    # p = 1/2: t^k / ((1+t)/2)^(k+1) = 2^(k+1) sum_i C(k,i) (-1)^i (1+t)^-(i+1) and
    # int_0^inf s e^(-st) (1+t)^-m dt = s e^s E_m(s), E_m the exponential integral.
    from scipy.special import expn
    lam, mu = O.special_vw_lambda_mu(6, s, 0.5)
    for k in range(7):
        ref = 2 ** (k + 1) * s * math.exp(s) * sum(
            math.comb(k, i) * (-1) ** i * expn(i + 1, s) for i in range(k + 1))
        assert mu[k] == pytest.approx(ref, rel=1e-8)
        # the defining moment relation of lambda and phi: 1/lambda_k = int phi(t) t^k dt = k!/s^k
        assert lam[k] == pytest.approx(s ** k / math.factorial(k), rel=1e-15)


def test_special_vanwijngaarden_sums_divergent_geometric_series():
    # sum (-1.5)^n diverges; its Borel (and analytic-continuation) value is 1/(1+1.5) = 0.4, which
    # the special transformation keeps.  The truncated estimate approaches it as d grows.
    x, ref = 1.5, 0.4
    errs = []
    for d in (4, 8, 16):
        c = O.euler_weights(d, "vanw", 0.5, 2.0)
        errs.append(abs(c @ np.array([(-x) ** n for n in range(d + 1)]) - ref))
    assert errs[2] < errs[1] < errs[0] and errs[2] < 1e-4
    # and the plain partial sums run away
    assert abs(np.sum([(-x) ** n for n in range(17)]) - ref) > 100


def test_accelerated_wce_weights_sum_the_same_series():
    # every acceleration of Eq. (WCE) is sum_n c_n t_n over the same terms: the preconditioner
    # applied through the weights equals the one built from the accelerated partial sums
    lat = O.Lattice(4, 6, 0.05, 5.0)
    sigma, v = field_and_source(4, 6, 2)
    terms = [O.apply_M0inv(lat, v)]
    for _ in range(4):
        terms.append(-lat.A * O.apply_M0inv(lat, O.apply_M1(lat, sigma, terms[-1])))
    for mode in ("euler", "euler23", "vanw"):
        c = O.euler_weights(4, mode, 0.5, 1.0)
        ref = sum(cn * t for cn, t in zip(c, terms))
        assert np.allclose(O.wce_apply(lat, sigma, v, 4, mode), ref, rtol=1e-12, atol=1e-13)
    # Euler-2/3 by hand: S_{3,1} from the partial sums
    S = np.cumsum(np.array(terms), axis=0)
    assert np.allclose(O.wce_apply(lat, sigma, v, 4, "euler23"), O.euler_table(S, 3, 1),
                       rtol=1e-13, atol=1e-14)


def test_two_sided_wce_for_cg_is_spd_and_exact_at_zero_field():
    # CG on M^T M with the series on both sides: P = P_d P_d^T is symmetric positive definite
    lat = O.Lattice(4, 4, 0.05, 5.0)
    sigma, b = field_and_source(4, 4, 12)
    pc = O.make_preconditioner(lat, sigma, {"kind": "wce", "order": 2}, normal=True)
    P = O.dense_from_apply(pc, lat.shape)
    assert np.allclose(P, P.T, atol=1e-12)
    assert np.linalg.eigvalsh(0.5 * (P + P.T)).min() > 0
    # at sigma = 0 every order is exact (M1 = 0, P_d = M0^{-1} = M^{-1}): one CG iteration
    zero = np.zeros(lat.shape)
    x, info = O.solve_cg_normal(lat, zero, b, 1e-10, 50, {"kind": "wce", "order": 2})
    assert info["converged"] and info["iterations"] <= 1
    assert np.allclose(O.apply_Q(lat, zero, x), b, atol=1e-9)


def test_sca_chebyshev_filter_is_spd_and_maps_the_spectrum():
    # P = P(G/s)/s P_S with G = P_S Q: P Q = P(G/s) G / s is similar to a function of G, so its
    # eigenvalues are z P(z) at z = lambda(G)/s, and |z P(z) - 1| obeys the Chebyshev bound of
    # Sec. 2 wherever z lies in [eps, 1]
    lat = O.Lattice(2, 6, 0.05, 5.0)
    sigma, _ = field_and_source(2, 6, 13)
    alpha, degree, eps = 2.0, 8, 0.05
    D, L = O.sca_factors(lat, sigma, alpha)
    Q = O.dense_from_apply(lambda u: O.apply_Q(lat, sigma, u), lat.shape)
    PS = O.dense_from_apply(lambda u: O.sca_apply(D, L, u), lat.shape)
    lamG = np.sort(np.linalg.eigvals(PS @ Q).real)
    s = O.sca_cheb_scale(lat, sigma, alpha)
    assert lamG.max() <= s <= 1.2 * lamG.max()  # the power estimate bounds the spectrum
    P = O.dense_from_apply(lambda u: O.sca_cheb_apply(lat, sigma, u, alpha, degree, eps, s),
                           lat.shape)
    assert np.allclose(P, P.T, atol=1e-10 * np.abs(P).max())
    assert np.linalg.eigvalsh(0.5 * (P + P.T)).min() > 0
    mu = np.sort(np.linalg.eigvals(P @ Q).real)
    z = lamG / s
    assert np.allclose(mu, np.sort(z * O.cheb_scalar(z, degree // 2, eps)), rtol=1e-8, atol=1e-10)
    inside = (z >= eps) & (z <= 1)
    bound = 2 * ((1 - math.sqrt(eps)) / (1 + math.sqrt(eps))) ** (degree + 1)
    assert np.all(np.abs(z[inside] * O.cheb_scalar(z[inside], degree // 2, eps) - 1) <= bound)


def test_wce_exact_at_zero_field():
    # sin(0) = 0 so M1 = 0 and every order of Eq. (WCE) is exactly M0^{-1} = M^{-1}.
    lat = O.Lattice(4, 6, 0.05, 5.0)
    zero = np.zeros(lat.shape)
    v = np.random.default_rng(0).standard_normal(lat.shape)
    for d in (0, 2):
        out = O.wce_apply(lat, zero, v, d)
        assert np.allclose(O.apply_M(lat, zero, out), v, atol=1e-12)


@pytest.mark.parametrize("d", [0, 1, 2, 4])
def test_wce_telescoping_identity(d):
    # M = M0 (1 + A X) gives M P_d v = v - M0 (-A X)^{d+1} M0^{-1} v.
    lat = O.Lattice(4, 6, 0.05, 5.0)
    sigma, v = field_and_source(4, 6, 3)
    w = O.apply_M0inv(lat, v)
    for _ in range(d + 1):
        w = -lat.A * O.apply_M0inv(lat, O.apply_M1(lat, sigma, w))
    rhs = v - O.apply_M(lat, np.zeros(lat.shape), w)
    lhs = O.apply_M(lat, sigma, O.wce_apply(lat, sigma, v, d))
    assert np.allclose(lhs, rhs, atol=1e-11)


def test_wce_transpose_is_transpose():
    lat = O.Lattice(4, 4, 0.05, 5.0)
    sigma, _ = field_and_source(4, 4, 9)
    for d, eu in [(1, False), (2, True), (4, "euler23"), (3, "vanw")]:
        P = O.dense_from_apply(lambda x: O.wce_apply(lat, sigma, x, d, eu), lat.shape)
        PT = O.dense_from_apply(lambda x: O.wce_apply_T(lat, sigma, x, d, eu), lat.shape)
        assert np.allclose(PT, P.T, atol=1e-12)


def test_wce_converges_to_inverse_at_small_coupling():
    lat = O.Lattice(4, 6, 0.05, 0.2)  # A ~ 0.14
    sigma, v = field_and_source(4, 6, 1)
    Mv = O.apply_M(lat, sigma, v)
    errs = [np.linalg.norm(O.wce_apply(lat, sigma, Mv, d) - v) for d in (0, 1, 2, 3)]
    assert all(errs[i + 1] < 0.3 * errs[i] for i in range(3))


def _dense_sca(D, L, site):
    nt = D.shape[0]
    Dv = D.reshape(nt, -1)[:, site]
    Lv = L.reshape(nt, -1)[:, site]
    Ld = np.eye(nt)  # L^dagger: -L_j below the diagonal, +L_N at (N, 1)
    for t in range(nt - 1):
        Ld[t + 1, t] = -Lv[t]
    Ld[nt - 1, 0] += Lv[nt - 1]
    return Ld, np.diag(Dv)


@pytest.mark.parametrize("alpha", [1.0, 2.0])
def test_sca_factorisation_structure(alpha):
    # Sec. 4: L^dagger D L reproduces M~^dagger M~ (B_j -> 1 + A sin sigma_j) with the diagonal
    # 1 replaced by alpha, except the fill-in -B_{0,N} B_{0,1} / D_1 at (N, 2) and (2, N).
    lat = O.Lattice(2, 7, 0.05, 5.0)
    sigma, _ = field_and_source(2, 7, 4)
    D, L = O.sca_factors(lat, sigma, alpha)
    w = 1 + lat.A * np.sin(sigma.reshape(7, -1))
    nt = 7
    for site in range(8):
        Ld, Dd = _dense_sca(D, L, site)
        prod = Ld @ Dd @ Ld.T
        Mt = np.eye(nt)
        for t in range(nt - 1):
            Mt[t + 1, t] = -w[t, site]
        Mt[0, nt - 1] = w[nt - 1, site]
        target = Mt.T @ Mt + (alpha - 1.0) * np.eye(nt)
        fill = -w[nt - 1, site] * w[0, site] / D.reshape(nt, -1)[0, site]
        target[nt - 1, 1] += fill
        target[1, nt - 1] += fill
        assert np.allclose(prod, target, atol=1e-12)


def test_sca_apply_is_exact_inverse_of_factorisation():
    lat = O.Lattice(2, 9, 0.05, 5.0)
    sigma, y = field_and_source(2, 9, 6)
    D, L = O.sca_factors(lat, sigma, 2.0)
    z = O.sca_apply(D, L, y)
    for site in range(8):
        Ld, Dd = _dense_sca(D, L, site)
        ref = np.linalg.solve(Ld @ Dd @ Ld.T, y.reshape(9, -1)[:, site])
        assert np.allclose(z.reshape(9, -1)[:, site], ref, rtol=1e-12, atol=1e-12)
