"""Plain FP64 CPU oracle of the unitary-Fermi-gas fermion matrix, its solvers and preconditioners.

TEST INFRASTRUCTURE ONLY.  This module is the independent reference that the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (CPU-baseline and
reference legs) may import it; the library's product path never does, and the two share no
code, no tables and no constant generators.

Everything is numpy float64, written for readability, not speed.  The kinetic factor is applied
literally as "K is diagonal in momentum space": a 3-D discrete Fourier transform (numpy's FFT
as a library step), a multiplication by exp(-tau E(k)) on the momentum grid of Sec. 1, and the
inverse transform.  The GPU path instead uses a real separable circulant contraction.

Conventions (readings of the paper where it leaves a choice open):
  * arrays are shaped [N_tau, N_x, N_x, N_x] = [t][z][y][x] (lower-dimensional lattices, which
    the methods carry over to (Sec. 6): [N_tau, N_x, N_x] or [N_tau, N_x]); slice t (0-based) is the paper's
    time index j = t + 1, so B_t uses sigma_t and the corner block of Eq. (MatrixM) is
    B_{N_tau-1} mapping slice N_tau-1 onto slice 0;
  * hbar = m = lattice spacing = 1, so E(k) = |k|^2 / 2 (dispersion 0).  dispersion 1 is the
    Hubbard-type lattice dispersion E(k) = sum_i (1 - cos k_i) (Sec. 6, other dispersions);
  * the fermion matrix is real, so M^dagger = M^T (Sec. 1, after Eq. (MatrixM)).

Parity status: every function below is pinned by the tests in tests/test_oracle_*.py except
the iteration counts of the solvers against the paper's Tables 1-3 (parity unpinned: the
paper's stopping rule, preconditioning side and units are not fully specified).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Lattice", "coupling_A", "momentum_1d", "energy_grid", "kinetic",
    "potentials", "apply_M", "apply_Mdag", "apply_Q", "apply_M1", "apply_M1T",
    "apply_M0inv", "apply_M0invT", "dense_from_apply", "sca_factors", "sca_apply",
    "cheb_roots", "cheb_quadratic_factors", "bit_reversed", "cheb_scale_eps",
    "cheb_apply", "cheb_scalar", "sca_cheb_scale", "sca_cheb_apply", "euler_transform", "euler_table", "euler_23_level",
    "special_vw_lambda_mu", "vanwijngaarden_weights", "euler_weights", "wce_apply",
    "wce_apply_T", "make_preconditioner", "cg", "bicgstab", "solve_cg_normal", "solve_bicgstab_two_step",
    "pseudofermion_action", "force_dS_dsigma", "leapfrog", "hmc_trajectory", "mv_formula", "Counter",
]


# ----------------------------------------------------------------------------------------
# Lattice, coupling, dispersion (Sec. 1: B_j, A, K_{k,k'}, k_i = 2 pi n_i / N_x)
# ----------------------------------------------------------------------------------------

def coupling_A(tau: float, g: float) -> float:
    """A = sqrt(2) sqrt(exp(tau g) - 1), the coupling of the continuous HST (Sec. 1)."""
    return math.sqrt(2.0) * math.sqrt(math.exp(tau * g) - 1.0)


def momentum_1d(nx: int) -> np.ndarray:
    """k_i = 2 pi n_i / N_x for n_i = -N_x/2 .. N_x/2 - 1, listed in numpy FFT order.

    numpy's FFT index m carries frequency m (mod N_x); the representative in the paper's
    range is n = m for m < N_x/2 and n = m - N_x otherwise (so n = -N_x/2 appears, +N_x/2 not).
    """
    if nx % 2:
        raise ValueError("N_x must be even for the momentum range n = -N_x/2..N_x/2-1")
    m = np.arange(nx)
    n = np.where(m < nx // 2, m, m - nx)
    return 2.0 * np.pi * n / nx


def energy_grid(nx: int, dispersion: int = 0, dim: int = 3) -> np.ndarray:
    """E(k) on the dim-dimensional momentum grid ([kz][ky][kx] for dim 3, numpy FFT order).

    dispersion 0: E = hbar^2 k^2 / 2m with hbar = m = 1 (Sec. 1).
    dispersion 1: E = sum_i (1 - cos k_i), a Hubbard-type lattice dispersion (Sec. 6).
    """
    if dim not in (1, 2, 3):
        raise ValueError("dim must be 1, 2 or 3")
    k = momentum_1d(nx)
    ks = np.meshgrid(*([k] * dim), indexing="ij")
    if dispersion == 0:
        return sum(0.5 * ki ** 2 for ki in ks)
    if dispersion == 1:
        return sum(1.0 - np.cos(ki) for ki in ks)
    raise ValueError("unknown dispersion")


@dataclass
class Lattice:
    """N_x^dim x N_tau lattice with imaginary time step tau and coupling g (Sec. 1, Sec. 5;
    dim = 3 is the paper's problem, 1 and 2 the lower dimensions of Sec. 6)."""
    nx: int
    ntau: int
    tau: float = 0.05
    g: float = 5.0
    dispersion: int = 0
    dim: int = 3
    A: float = field(init=False)
    E: np.ndarray = field(init=False, repr=False)

    def __post_init__(self):
        if (self.nx < 2 or self.nx % 2 or self.ntau < 2 or self.tau <= 0 or self.g < 0
                or self.dim not in (1, 2, 3)):
            raise ValueError("invalid lattice")
        self.A = coupling_A(self.tau, self.g)
        self.E = energy_grid(self.nx, self.dispersion, self.dim)

    @property
    def shape(self):
        return (self.ntau,) + (self.nx,) * self.dim

    @property
    def volume(self):
        return self.nx ** self.dim

    @property
    def space_axes(self):
        return tuple(range(-self.dim, 0))

    @property
    def beta(self):
        return self.tau * self.ntau


def kinetic(lat: Lattice, u: np.ndarray) -> np.ndarray:
    """exp(-tau K) u on every time slice: K is diagonal in momentum space with entries E(k)."""
    uh = np.fft.fftn(u, axes=lat.space_axes)
    uh *= np.exp(-lat.tau * lat.E)
    return np.fft.ifftn(uh, axes=lat.space_axes).real


def potentials(lat: Lattice, sigma: np.ndarray):
    """Per-site diagonal factors: w = 1 + A sin(sigma) (B_j), s = sin(sigma) (C_j, Eq. MatrixM_1)
    and c = A cos(sigma) = dw/dsigma (force)."""
    s = np.sin(sigma)
    return 1.0 + lat.A * s, s, lat.A * np.cos(sigma)


# ----------------------------------------------------------------------------------------
# The fermion matrix M[sigma] (Eq. MatrixM), its transpose, and M = M0 + A M1 (Eq. MatrixM_1)
# ----------------------------------------------------------------------------------------

def _shift_blocks(lat, x, diag):
    """Returns z with z[t+1] = -e^{-tau K}(diag_t x_t) for t < N_tau-1 and
    z[0] = +e^{-tau K}(diag_{N_tau-1} x_{N_tau-1}): the off-diagonal blocks of Eq. (MatrixM)."""
    kin = kinetic(lat, diag * x)
    z = np.empty_like(x)
    z[1:] = -kin[:-1]
    z[0] = kin[-1]
    return z


def _shift_blocks_T(lat, y, diag):
    """Transpose of _shift_blocks: z[t] = -diag_t e^{-tau K} y_{t+1} (t < N_tau-1) and
    z[N_tau-1] = +diag_{N_tau-1} e^{-tau K} y_0 (K is real symmetric)."""
    kin = kinetic(lat, y)
    z = np.empty_like(y)
    z[:-1] = -diag[:-1] * kin[1:]
    z[-1] = diag[-1] * kin[0]
    return z


def apply_M(lat, sigma, x):
    """M[sigma] x with B_j = exp(-tau K)(1 + A sin sigma_j) (Eq. MatrixM and the B_j definition)."""
    w, _, _ = potentials(lat, sigma)
    return x + _shift_blocks(lat, x, w)


def apply_Mdag(lat, sigma, y):
    """M^dagger y = M^T y (M is real, Sec. 1)."""
    w, _, _ = potentials(lat, sigma)
    return y + _shift_blocks_T(lat, y, w)


def apply_Q(lat, sigma, x):
    """Q x = M^dagger M x, the normal-equation operator of Eq. (1)."""
    return apply_Mdag(lat, sigma, apply_M(lat, sigma, x))


def apply_M1(lat, sigma, x):
    """M1 x with blocks C_j = exp(-tau K) sin sigma_j (Eq. MatrixM_1)."""
    _, s, _ = potentials(lat, sigma)
    return _shift_blocks(lat, x, s)


def apply_M1T(lat, sigma, y):
    """M1^T y."""
    _, s, _ = potentials(lat, sigma)
    return _shift_blocks_T(lat, y, s)


def _antiperiodic_phases(ntau):
    """omega = (2 n_tau + 1) pi / N_tau (Sec. 3, Fourier acceleration): an antiperiodic temporal
    transform is an ordinary DFT of x_t e^{-i pi t / N_tau}."""
    t = np.arange(ntau)
    return np.exp(-1j * np.pi * t / ntau)


def apply_M0inv(lat, y):
    """M0^{-1} y by Fourier acceleration (Sec. 3): in frequency-momentum space M0^{-1} is
    diagonal with entries [1 - exp(-i omega - tau E(k))]^{-1}, omega antiperiodic.

    With the transform x_t = sum_omega e^{i omega t} x~_omega the normalisation constant is 1.
    """
    tshape = (lat.ntau,) + (1,) * lat.dim
    ph = _antiperiodic_phases(lat.ntau).reshape(tshape)
    axes = tuple(range(lat.dim + 1))
    yh = np.fft.fftn(y * ph, axes=axes)
    m = np.arange(lat.ntau)
    omega = ((2 * m + 1) * np.pi / lat.ntau).reshape(tshape)
    denom = 1.0 - np.exp(-1j * omega - lat.tau * lat.E[None])
    xh = yh / denom
    return (np.fft.ifftn(xh, axes=axes) / ph).real


def apply_M0invT(lat, y):
    """(M0^T)^{-1} y: the transposed diagonal [1 - exp(+i omega - tau E(k))]^{-1}."""
    tshape = (lat.ntau,) + (1,) * lat.dim
    ph = _antiperiodic_phases(lat.ntau).reshape(tshape)
    axes = tuple(range(lat.dim + 1))
    yh = np.fft.fftn(y * ph, axes=axes)
    m = np.arange(lat.ntau)
    omega = ((2 * m + 1) * np.pi / lat.ntau).reshape(tshape)
    denom = 1.0 - np.exp(+1j * omega - lat.tau * lat.E[None])
    xh = yh / denom
    return (np.fft.ifftn(xh, axes=axes) / ph).real


def dense_from_apply(op, shape):
    """Dense matrix of a linear operator (tiny lattices only), column by column."""
    n = int(np.prod(shape))
    out = np.empty((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        out[:, j] = op(e.reshape(shape)).ravel()
        e[j] = 0.0
    return out


# ----------------------------------------------------------------------------------------
# Strong-coupling approximation (Sec. 4): L^dagger D L factorisation of M~^dagger M~
# ----------------------------------------------------------------------------------------

def sca_factors(lat, sigma, alpha):
    """D_t and L_t of Sec. 4 per site, with B_{0,t} = 1 + A sin sigma_t.

    The paper's 1-based recurrences are used with j = t + 1:
      D_1 = alpha + B_{0,1}^2 (no predecessor),
      D_j = alpha + B_{0,j}^2 - B_{0,j-1}^2 / D_{j-1}           (2 <= j <= N_tau - 1),
      D_N = alpha + B_{0,N}^2 - B_{0,N-1}^2 / D_{N-1} - B_{0,N}^2 / D_1,
      L_j = B_{0,j} / D_j (j <= N_tau - 1),  L_N = B_{0,N} / D_1.
    Returned arrays are [N_tau][z][y][x] with index t = j - 1.
    """
    w, _, _ = potentials(lat, sigma)
    nt = lat.ntau
    D = np.empty_like(w)
    L = np.empty_like(w)
    D[0] = alpha + w[0] ** 2
    for t in range(1, nt - 1):
        D[t] = alpha + w[t] ** 2 - w[t - 1] ** 2 / D[t - 1]
    D[nt - 1] = alpha + w[nt - 1] ** 2 - w[nt - 2] ** 2 / D[nt - 2] - w[nt - 1] ** 2 / D[0]
    for t in range(nt - 1):
        L[t] = w[t] / D[t]
    L[nt - 1] = w[nt - 1] / D[0]
    return D, L


def sca_apply(D, L, y):
    """(L^dagger D L)^{-1} y = L^{-1} D^{-1} L^{dagger -1} y (Sec. 4).

    L^dagger^{-1}: the forward recursion printed in Sec. 4; D^{-1}: pointwise; L^{-1}: the
    backward substitution of the transposed (upper) matrix, read off from the same structure.
    """
    nt = y.shape[0]
    x = np.empty_like(y)
    x[0] = y[0]
    for t in range(1, nt):
        x[t] = y[t] + L[t - 1] * x[t - 1]
    x[nt - 1] = x[nt - 1] - L[nt - 1] * x[0]
    u = x / D
    z = np.empty_like(y)
    z[nt - 1] = u[nt - 1]
    for t in range(nt - 2, 0, -1):
        z[t] = u[t] + L[t] * z[t + 1]
    z[0] = u[0] + L[0] * z[1] - L[nt - 1] * z[nt - 1] if nt > 1 else u[0]
    return z


# ----------------------------------------------------------------------------------------
# Chebyshev preconditioner (Sec. 2, Eq. ChebInv and the roots/coefficient equations)
# ----------------------------------------------------------------------------------------

def cheb_roots(n: int, eps: float) -> np.ndarray:
    """z_{2n,k} = (1+eps)/2 [1 - cos(2 pi k/(2n+1))] - i sqrt(eps) sin(2 pi k/(2n+1)), k=1..2n."""
    k = np.arange(1, 2 * n + 1)
    th = 2.0 * np.pi * k / (2 * n + 1)
    return 0.5 * (1 + eps) * (1 - np.cos(th)) - 1j * np.sqrt(eps) * np.sin(th)


def cheb_scalar(z, n: int, eps: float):
    """P(z) = c_{2n} prod_k (z - z_{2n,k}) with c_{2n}^{-1} = (1+eps)/2 prod_k ((1+eps)/2 - z_k)."""
    roots = cheb_roots(n, eps)
    z0 = 0.5 * (1 + eps)
    cinv = z0 * np.prod(z0 - roots)
    z = np.asarray(z, dtype=complex)
    p = np.ones_like(z)
    for r in roots:
        p = p * (z - r)
    return (p / cinv).real


def cheb_quadratic_factors(n: int, eps: float):
    """Pairs the conjugate roots z_k, z_{2n+1-k} (k = 1..n) into real quadratics
    (z - a_k)^2 + b_k^2 and returns (a_k, b_k, norm_k) with norm_k = (z0 - a_k)^2 + b_k^2, so that
    P(z) = (1/z0) prod_k [(z - a_k)^2 + b_k^2] / norm_k exactly equals c_{2n} prod (z - z_k)."""
    roots = cheb_roots(n, eps)[:n]
    z0 = 0.5 * (1 + eps)
    a = roots.real
    b = -roots.imag
    norm = (z0 - a) ** 2 + b ** 2
    return a, b, norm


def bit_reversed(n: int):
    """Order of the n quadratic factors: factor index k-1 taken in bit-reversed order over
    ceil(log2 n) bits (reading of the 'bit-reversal ordering' named in Sec. 2); indices that
    reverse to >= n are skipped."""
    bits = max(1, (n - 1).bit_length())
    out = []
    for i in range(1 << bits):
        r = int(format(i, "0%db" % bits)[::-1], 2)
        if r < n:
            out.append(r)
    return out


def cheb_scale_eps(lat, sigma, eps=None):
    """Spectrum normalisation of M^dagger M to [eps, 1] (Sec. 2): scale s = (2 + A)^2 bounds
    ||M||^2 because ||exp(-tau K)|| = 1 and |1 + A sin sigma| <= 1 + A; default eps = free-gas
    lowest eigenvalue (2 - 2 cos(pi/N_tau)) / s."""
    s = (2.0 + lat.A) ** 2
    if eps is None:
        eps = (2.0 - 2.0 * math.cos(math.pi / lat.ntau)) / s
    return s, eps


def cheb_apply(qop, v, degree: int, eps: float, scale: float, counter=None):
    """z = P(Q/scale) v / scale ~ Q^{-1} v with P of degree 2n = degree, applied factor by factor
    (each real quadratic = two applications of Q) in bit-reversed order."""
    n = degree // 2
    a, b, norm = cheb_quadratic_factors(n, eps)
    z0 = 0.5 * (1 + eps)
    out = v.copy()
    for k in bit_reversed(n):
        u = qop(out) / scale - a[k] * out
        out = (qop(u) / scale - a[k] * u + b[k] ** 2 * out) / norm[k]
        if counter is not None:
            counter.add("Q", 2)
    return out / (z0 * scale)


def sca_cheb_scale(lat, sigma, alpha, steps=30, safety=1.1):
    """Spectral scale s of G = (L^T D L)^{-1} Q for the combined preconditioner: the power method
    v <- G v / |v| from v = w = 1 + A sin(sigma) (deterministic: no random start vector), whose
    ratio |G v| / |v| approaches lambda_max(G) from below, times a safety factor."""
    D, L = sca_factors(lat, sigma, alpha)
    v = potentials(lat, sigma)[0].copy()
    vn = float(np.linalg.norm(v))
    lam = 0.0
    for _ in range(steps):
        g = sca_apply(D, L, apply_Q(lat, sigma, v)) / vn
        lam = float(np.linalg.norm(g))
        v, vn = g, lam
    return safety * lam


def sca_cheb_apply(lat, sigma, r, alpha, degree, eps=None, scale=None, counter=None):
    """The strong-coupling preconditioner with the Chebyshev polynomial as a secondary filter (end
    of Sec. 4): z = P(G/s)/s P_S r with P_S = (L^T D L)^{-1} (Sec. 4) and G = P_S Q, P the
    polynomial of Sec. 2 (cheb_apply with G as its operator).  Defaults: eps = 1e-3, s from
    sca_cheb_scale."""
    D, L = sca_factors(lat, sigma, alpha)
    s = scale if scale else sca_cheb_scale(lat, sigma, alpha)
    e = eps if eps else 1e-3

    def gop(u):
        if counter is not None:
            counter.add("SCA", 1)
        return sca_apply(D, L, apply_Q(lat, sigma, u))
    if counter is not None:
        counter.add("SCA", 1)
    return cheb_apply(gop, sca_apply(D, L, r), degree, e, s, counter)


# ----------------------------------------------------------------------------------------
# Weak-coupling expansion (Sec. 3, Eq. WCE) and Euler acceleration (Eq. Euler)
# ----------------------------------------------------------------------------------------

def euler_transform(partial_sums, p=0.5):
    """Repeated application of S_{j+1,k} = p S_{j,k} + (1-p) S_{j,k+1} until one term is left:
    returns S_{kmax,0} (Sec. 3.1).  Works on scalars or arrays."""
    S = list(partial_sums)
    while len(S) > 1:
        S = [p * S[k] + (1 - p) * S[k + 1] for k in range(len(S) - 1)]
    return S[0]


def euler_table(partial_sums, j: int, k: int, p=0.5):
    """S_{j,k} of Eq. (Euler): the recursion applied j times to the partial sums S_{0,0..kmax},
    entry k of the resulting sequence (needs j + k <= kmax)."""
    S = list(partial_sums)
    if not 0 <= k <= len(S) - 1 - j:
        raise ValueError("S_{j,k} needs j + k <= kmax")
    for _ in range(j):
        S = [p * S[i] + (1 - p) * S[i + 1] for i in range(len(S) - 1)]
    return S[k]


def euler_23_level(d: int) -> int:
    """Level j of the variant S_{2 kmax/3, kmax/3} (Sec. 3.1) for kmax = d: the paper leaves the
    rounding open; j is the integer nearest 2d/3 and k = d - j, so the entry still uses every
    term of the series."""
    return (2 * d + 1) // 3


def special_vw_lambda_mu(d: int, s: float = 1.0, p: float = 0.5):
    """The special van Wijngaarden transformation (Sec. 3.1): lambda_k = s^k / k!, phi(t) =
    s exp(-s t), and mu_k = int_0^inf phi(t) t^k / (1 - p + p t)^(k+1) dt for k = 0..d (the
    integral by scipy's adaptive quadrature as a library step)."""
    from scipy import integrate
    lam = np.array([s ** k / math.factorial(k) for k in range(d + 1)])
    mu = np.empty(d + 1)
    for k in range(d + 1):
        f = lambda t, k=k: s * math.exp(-s * t) * t ** k / (1.0 - p + p * t) ** (k + 1)  # noqa: E731
        mu[k] = integrate.quad(f, 0.0, np.inf, epsabs=1e-16, epsrel=1e-13, limit=400)[0]
    return lam, mu


def vanwijngaarden_weights(d: int, lam, mu, p: float = 0.5):
    """Weights c_j with sum_j c_j t_j = sum_{n=0}^{d} mu_n b_n, the van Wijngaarden estimate
    truncated at order d (Sec. 3.1): the terms t_j = (-1)^j a_j are multiplied by lambda_j, Euler
    transformed, b_n = sum_{j<=n} C(n, j) p^(n-j) (1-p)^(j+1) lambda_j t_j, and summed with the
    weights mu_n."""
    c = np.zeros(d + 1)
    for j in range(d + 1):
        acc = 0.0
        for n in range(j, d + 1):
            acc += math.comb(n, j) * p ** (n - j) * mu[n]
        c[j] = lam[j] * (1.0 - p) ** (j + 1) * acc
    return c


ACCEL = {False: 0, True: 1, 0: 0, 1: 1, 2: 2, 3: 3, "none": 0, "euler": 1, "euler23": 2,
         "vanw": 3}


def euler_weights(d: int, euler=True, p: float = 0.5, s: float = 1.0):
    """Weights c_n of the accelerated order-d sum sum_n c_n t_n, t_n the n-th term of the series.
    euler: 0/False/"none" plain partial sum S_{0,d}; 1/True/"euler" S_{d,0}; 2/"euler23"
    S_{j,d-j} with j = euler_23_level(d); 3/"vanw" the special van Wijngaarden transformation with
    parameter s.  The Euler weights come from running the recursion on unit series (so they
    follow Eq. Euler, not a closed form)."""
    mode = ACCEL[euler]
    if mode == 0 or d == 0 and mode != 3:
        return np.ones(d + 1)
    if mode == 3:
        lam, mu = special_vw_lambda_mu(d, s, p)
        return vanwijngaarden_weights(d, lam, mu, p)
    j = d if mode == 1 else euler_23_level(d)
    c = np.empty(d + 1)
    for n in range(d + 1):
        terms = np.zeros(d + 1)
        terms[n] = 1.0
        c[n] = euler_table(np.cumsum(terms), j, d - j, p)
    return c


def _accelerated_sum(terms, d, euler, p, s):
    mode = ACCEL[euler]
    if mode == 0:
        return np.sum(terms, axis=0)
    if mode in (1, 2):
        j = d if mode == 1 else euler_23_level(d)
        return euler_table(np.cumsum(np.array(terms), axis=0), j, d - j, p)
    c = euler_weights(d, 3, p, s)
    return sum(cn * t for cn, t in zip(c, terms))


def wce_apply(lat, sigma, v, d: int, euler=False, counter=None, p=0.5, s=1.0):
    """P_d v = sum_{n=0}^{d} (-A X)^n M0^{-1} v with X = M0^{-1} M1 (Eq. WCE), optionally
    accelerated over the partial sums (euler: see euler_weights)."""
    terms = []
    w = apply_M0inv(lat, v)
    if counter is not None:
        counter.add("M0inv", 1)
    terms.append(w)
    for _ in range(d):
        w = -lat.A * apply_M0inv(lat, apply_M1(lat, sigma, w))
        if counter is not None:
            counter.add("M1", 1)
            counter.add("M0inv", 1)
        terms.append(w)
    return _accelerated_sum(terms, d, euler, p, s)


def wce_apply_T(lat, sigma, v, d: int, euler=False, counter=None, p=0.5, s=1.0):
    """P_d^T v = sum_n (-A)^n M0^{-T} (M1^T M0^{-T})^n v: the exact transpose of P_d, the
    weak-coupling preconditioner of M^dagger (same acceleration as wce_apply)."""
    terms = []
    w = apply_M0invT(lat, v)
    if counter is not None:
        counter.add("M0invT", 1)
    terms.append(w)
    for _ in range(d):
        w = -lat.A * apply_M0invT(lat, apply_M1T(lat, sigma, w))
        if counter is not None:
            counter.add("M1T", 1)
            counter.add("M0invT", 1)
        terms.append(w)
    return _accelerated_sum(terms, d, euler, p, s)


# ----------------------------------------------------------------------------------------
# Krylov solvers (Eq. 1-3; textbook forms: PCG as Saad Alg. 9.1, BiCGStab as van der Vorst 1992
# with right preconditioning)
# ----------------------------------------------------------------------------------------

class Counter(dict):
    def add(self, k, n=1):
        self[k] = self.get(k, 0) + n


def _dot(a, b):
    return float(np.dot(a.ravel(), b.ravel()))


def cg(aop, b, tol, maxit, precond=None, x0=None):
    """Preconditioned CG on an SPD operator; stops when the recursive residual satisfies
    ||r|| <= tol ||b||.  Returns (x, iterations, converged)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - aop(x) if x0 is not None else b.copy()
    z = precond(r) if precond else r
    p = z.copy()
    rz = _dot(r, z)
    bn = math.sqrt(_dot(b, b))
    if bn == 0.0:
        return x, 0, True
    if math.sqrt(_dot(r, r)) <= tol * bn:
        return x, 0, True
    for it in range(1, maxit + 1):
        q = aop(p)
        alpha = rz / _dot(p, q)
        x = x + alpha * p
        r = r - alpha * q
        if math.sqrt(_dot(r, r)) <= tol * bn:
            return x, it, True
        z = precond(r) if precond else r
        rz_new = _dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, False


def bicgstab(aop, b, tol, maxit, precond=None, x0=None, restart_cos=1e-12, max_restarts=100):
    """Right-preconditioned BiCGStab (van der Vorst 1992); stops when ||r|| <= tol ||b||.

    Near-breakdown of rho = (rhat, r) (|rho| <= restart_cos ||rhat|| ||r||) or omega = 0 restarts
    the method from the current iterate with the true residual r = b - A x as the new shadow
    vector (the usual remedy; the paper does not discuss breakdown).
    Returns (x, iterations, converged); the restart count is in bicgstab.last_restarts.
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - aop(x) if x0 is not None else b.copy()
    bn = math.sqrt(_dot(b, b))
    bicgstab.last_restarts = 0
    if bn == 0.0:
        return x, 0, True
    if math.sqrt(_dot(r, r)) <= tol * bn:
        return x, 0, True
    K = precond if precond else (lambda u: u)
    restarts = 0

    def fresh(r):
        return r.copy(), 1.0, 1.0, 1.0, np.zeros_like(b), np.zeros_like(b)
    rhat, rho_old, alpha, omega, v, p = fresh(r)
    it = 0
    while it < maxit:
        it += 1
        rho = _dot(rhat, r)
        if abs(rho) <= restart_cos * math.sqrt(_dot(rhat, rhat) * _dot(r, r)):
            if restarts >= max_restarts:
                return x, it, False
            restarts += 1
            bicgstab.last_restarts = restarts
            r = b - aop(x)
            rhat, rho_old, alpha, omega, v, p = fresh(r)
            rho = _dot(rhat, r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        y = K(p)
        v = aop(y)
        alpha = rho / _dot(rhat, v)
        s = r - alpha * v
        if math.sqrt(_dot(s, s)) <= tol * bn:
            return x + alpha * y, it, True
        z = K(s)
        t = aop(z)
        tt = _dot(t, t)
        omega = _dot(t, s) / tt if tt > 0 else 0.0
        x = x + alpha * y + omega * z
        r = s - omega * t
        if math.sqrt(_dot(r, r)) <= tol * bn:
            return x, it, True
        rho_old = rho
        if omega == 0.0:  # stagnation: restart from the true residual
            if restarts >= max_restarts:
                return x, it, False
            restarts += 1
            bicgstab.last_restarts = restarts
            r = b - aop(x)
            rhat, rho_old, alpha, omega, v, p = fresh(r)
    return x, maxit, False


def _make_pc(lat, sigma, pc, counter, transpose=False, normal=False):
    """Preconditioner closure.  normal=True: for CG on M^dagger M, where the weak-coupling series
    is used from both sides, P_d P_d^dagger ~ M^{-1} M^{-dagger} (M0^{-dagger} on the left and
    M0^{-1} on the right, end of Sec. 5)."""
    kind = pc.get("kind", "none") if pc else "none"
    if kind == "wce" and normal:
        args = (pc["order"], pc.get("euler", False))
        kw = {"p": pc.get("p", 0.5), "s": pc.get("s", 1.0)}
        return lambda r: wce_apply(lat, sigma, wce_apply_T(lat, sigma, r, *args, counter, **kw),
                                   *args, counter, **kw)
    if kind == "none":
        return None
    if kind == "cheb":
        s, eps = cheb_scale_eps(lat, sigma, pc.get("eps"))
        if pc.get("scale"):
            s = pc["scale"]
        qop = lambda u: apply_Q(lat, sigma, u)  # noqa: E731
        return lambda r: cheb_apply(qop, r, pc["degree"], eps, s, counter)
    if kind == "sca_cheb":
        alpha, degree = pc.get("alpha", 2.0), pc["degree"]
        s = pc.get("scale") or sca_cheb_scale(lat, sigma, alpha)
        return lambda r: sca_cheb_apply(lat, sigma, r, alpha, degree, pc.get("eps"), s, counter)
    if kind == "sca":
        D, L = sca_factors(lat, sigma, pc.get("alpha", 2.0))

        def f(r):
            counter.add("SCA", 1)
            return sca_apply(D, L, r)
        return f
    if kind == "wce":
        fn = wce_apply_T if transpose else wce_apply
        return lambda r: fn(lat, sigma, r, pc["order"], pc.get("euler", False), counter,
                            pc.get("p", 0.5), pc.get("s", 1.0))
    raise ValueError(kind)


def make_preconditioner(lat, sigma, pc, transpose=False, normal=False):
    """The preconditioner the solvers use for a settings dict (see _make_pc); None for none."""
    return _make_pc(lat, sigma, pc, Counter(), transpose, normal)


def solve_cg_normal(lat, sigma, b, tol=1e-10, maxit=20000, pc=None):
    """CG on M^dagger M x = b (Eq. 1) with an SPD preconditioner (Chebyshev, SCA, or the
    weak-coupling series from both sides)."""
    counter = Counter()

    def qop(u):
        counter.add("M")
        counter.add("Mdag")
        return apply_Q(lat, sigma, u)
    x, it, ok = cg(qop, b, tol, maxit, _make_pc(lat, sigma, pc, counter, normal=True))
    return x, {"iterations": it, "converged": ok, "counts": dict(counter)}


def solve_bicgstab_two_step(lat, sigma, b, tol=1e-10, maxit=20000, pc=None):
    """M^dagger y = b then M x = y (Eq. 2) with right-preconditioned BiCGStab.

    Tolerance split: step 1 to tol/2; step 2 to tol ||b|| / (2 (2 + A) ||y||), since
    ||b - M^dagger M x|| <= ||r_1|| + ||M^dagger|| ||r_2|| and ||M^dagger|| <= 2 + A.
    """
    counter = Counter()

    def mdag(u):
        counter.add("Mdag")
        return apply_Mdag(lat, sigma, u)

    def m(u):
        counter.add("M")
        return apply_M(lat, sigma, u)
    y, it1, ok1 = bicgstab(mdag, b, 0.5 * tol, maxit, _make_pc(lat, sigma, pc, counter, True))
    r1 = bicgstab.last_restarts
    tol2 = tol * math.sqrt(_dot(b, b)) / (2.0 * (2.0 + lat.A) * math.sqrt(_dot(y, y)))
    x, it2, ok2 = bicgstab(m, y, tol2, maxit, _make_pc(lat, sigma, pc, counter, False))
    return x, {"iterations": it1 + it2, "iterations_step": (it1, it2),
               "converged": ok1 and ok2, "counts": dict(counter),
               "restarts": r1 + bicgstab.last_restarts}


def mv_formula(method: str, iterations: int, d: int = 0, beta: float = 1.0) -> float:
    """MV-operation accounting of Sec. 5: CG + Chebyshev of degree d costs 2(d+1) per iteration,
    BiCGStab + WCE of order d costs 2(d+1)(1+2 beta), CG + SCA about 3, unpreconditioned CG and
    BiCGStab 2."""
    if method == "cheb":
        return iterations * 2 * (d + 1)
    if method == "wce":
        return iterations * 2 * (d + 1) * (1 + 2 * beta)
    if method == "sca":
        return iterations * 3
    if method == "none":
        return iterations * 2
    raise ValueError(method)


# ----------------------------------------------------------------------------------------
# Pseudofermion action and HMC fermion force (Sec. 1)
# ----------------------------------------------------------------------------------------

def pseudofermion_action(lat, sigma, phi, x=None, tol=1e-13):
    """S_p = phi^T Q^{-1} phi with Q = M^dagger M; returns (S, X = Q^{-1} phi)."""
    if x is None:
        x, _ = solve_cg_normal(lat, sigma, phi, tol=tol)
    return _dot(phi, x), x


def leapfrog(lat, sigma, pi, phi, n_steps, dt, tol=1e-13):
    """Molecular dynamics of the phi-algorithm (Sec. 1): H = sum pi^2/2 + S_p(sigma) with phi held
    fixed, integrated by leapfrog (half step in pi, n_steps steps in sigma with full pi steps
    between them, final half step).  Returns (sigma, pi, S_p at the start, S_p at the end)."""
    sigma, pi = sigma.copy(), pi.copy()
    S0, X = pseudofermion_action(lat, sigma, phi, tol=tol)
    pi -= 0.5 * dt * force_dS_dsigma(lat, sigma, X)
    S1 = S0
    for k in range(1, n_steps + 1):
        sigma += dt * pi
        S1, X = pseudofermion_action(lat, sigma, phi, tol=tol)
        pi -= (0.5 if k == n_steps else 1.0) * dt * force_dS_dsigma(lat, sigma, X)
    return sigma, pi, S0, S1


def hmc_trajectory(lat, sigma0, eta, pi0, u, n_steps, dt, tol=1e-13):
    """One trajectory: pseudofermion heat bath phi = M^dagger eta (so S_p = |eta|^2), leapfrog,
    Metropolis accept with probability min(1, exp(-dH)) against the uniform number u (Sec. 1).
    Returns (sigma, pi, info)."""
    phi = apply_Mdag(lat, sigma0, eta)
    sigma, pi, S0, S1 = leapfrog(lat, sigma0, pi0, phi, n_steps, dt, tol)
    H0 = 0.5 * _dot(pi0, pi0) + S0
    H1 = 0.5 * _dot(pi, pi) + S1
    dH = H1 - H0
    accepted = dH <= 0 or u < math.exp(-dH)
    return (sigma if accepted else sigma0.copy()), pi, {
        "H_old": H0, "H_new": H1, "dH": dH, "accepted": accepted, "action_old": S0,
        "action_new": S1}


def force_dS_dsigma(lat, sigma, X):
    """dS_p/dsigma for S_p = phi^T Q^{-1} phi, given X = Q^{-1} phi.

    The paper's fermion force is F = phi^T Q^{-1} (dQ/dsigma) Q^{-1} phi = X^T (dQ/dsigma) X and
    dS/dsigma = -F.  With Y = M X and dQ = dM^T M + M^T dM, X^T dQ X = 2 Y^T (dM X), where the
    only sigma_t(r)-dependent block is -B_t at (t+1, t) (+B at the corner) with
    dB_t/dsigma_t(r) = exp(-tau K) e_r A cos sigma_t(r) e_r^T.
    """
    _, _, c = potentials(lat, sigma)
    Y = apply_M(lat, sigma, X)
    # Y~_{t+1}: the slice that multiplies block (t+1, t), with the antiperiodic corner sign.
    Yn = np.empty_like(Y)
    Yn[:-1] = -Y[1:]
    Yn[-1] = Y[0]
    KY = kinetic(lat, Yn)  # exp(-tau K) is symmetric
    F = 2.0 * c * X * KY   # = X^T (dQ/dsigma) X
    return -F
