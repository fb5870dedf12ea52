"""The momentum-basis form of the fermion matrix that the batched solver iterates on (Sec. 3,
Fourier acceleration), checked on the oracle's M without a GPU.

With F the orthonormal real Fourier basis of one slice (the eigenbasis of exp(-tau K), Sec. 1)
and b its eigenvalues, F M F^T is, slice by slice,
  (M x^)_t   = x^_t - sgn_t     b .* F( w_{t-1} .* F^T x^_{t-1} )
  (M^T x^)_t = x^_t - sgn_{t+1}      F( w_t .* F^T( b .* x^_{t+1} ) )
with sgn = +1 except at the antiperiodic wrap (-1) and w = 1 + A sin(sigma).  The basis here is
written from its definition (cosines, sines, the constant and the alternating vector); nothing is
shared with the library's transforms."""
import numpy as np

import oracle as O
from paper_1008_3647_gb300.inputs import field_and_source


def _basis_1d(n):
    """Rows: orthonormal real Fourier vectors of a periodic line of n sites (n even) and the
    momentum of each row."""
    x = np.arange(n)
    rows, ks = [np.full(n, 1.0 / np.sqrt(n))], [0.0]
    for k in range(1, n // 2):
        rows.append(np.sqrt(2.0 / n) * np.cos(2 * np.pi * k * x / n))
        ks.append(2 * np.pi * k / n)
    rows.append((-1.0) ** x / np.sqrt(n))
    ks.append(np.pi)
    for k in range(1, n // 2):
        rows.append(np.sqrt(2.0 / n) * np.sin(2 * np.pi * k * x / n))
        ks.append(2 * np.pi * k / n)
    return np.array(rows), np.array(ks)


def _basis_3d(lat):
    F1, k1 = _basis_1d(lat.nx)
    F = np.kron(np.kron(F1, F1), F1)  # [z][y][x] flattening, x fastest
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    b = np.exp(-lat.tau * 0.5 * (kx ** 2 + ky ** 2 + kz ** 2)).ravel()
    return F, b


def _fwd(F, v):
    return (v.reshape(v.shape[0], -1) @ F.T).reshape(v.shape)


def _inv(F, v):
    return (v.reshape(v.shape[0], -1) @ F).reshape(v.shape)


def test_basis_is_orthonormal_and_diagonalises_the_kinetic_factor():
    lat = O.Lattice(4, 3)
    F, b = _basis_3d(lat)
    assert np.abs(F @ F.T - np.eye(F.shape[0])).max() < 1e-13
    _, x = field_and_source(4, 3, 1)
    kx = O.kinetic(lat, x)
    xh = _fwd(F, x).reshape(x.shape[0], -1)
    assert np.abs(_inv(F, (b * xh).reshape(x.shape)) - kx).max() < 1e-13


def test_momentum_form_of_M_and_MT():
    nx, ntau = 4, 5
    lat = O.Lattice(nx, ntau)
    sigma, x = field_and_source(nx, ntau, 3)
    F, b = _basis_3d(lat)
    w = (1.0 + lat.A * np.sin(sigma)).reshape(ntau, -1)
    xh = _fwd(F, x).reshape(ntau, -1)
    sgn = np.ones(ntau)
    sgn[0] = -1.0  # (M x)_0 = x_0 + B x_{N-1}
    ref = _fwd(F, O.apply_M(lat, sigma, x)).reshape(ntau, -1)
    got = np.empty_like(xh)
    for t in range(ntau):
        tp = (t - 1) % ntau
        got[t] = xh[t] - sgn[t] * b * (F @ (w[tp] * (F.T @ xh[tp])))
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
    sgnT = np.ones(ntau)
    sgnT[-1] = -1.0  # (M^T y)_{N-1} = y_{N-1} + B^T y_0
    refT = _fwd(F, O.apply_Mdag(lat, sigma, x)).reshape(ntau, -1)
    for t in range(ntau):
        tn = (t + 1) % ntau
        got[t] = xh[t] - sgnT[t] * (F @ (w[t] * (F.T @ (b * xh[tn]))))
    assert np.abs(got - refT).max() < 1e-13 * np.abs(refT).max()
