"""The momentum basis of the fused kernels (Sec. 3, Fourier acceleration) through the C ABI.

ufg_fourier is pinned by what makes it the right basis, not by its slot order: it is orthogonal
(norms kept, the inverse undoes it) and it diagonalises the oracle's kinetic factor, whose
eigenvalues exp(-tau E(k)) it must reproduce.  ufg_apply_M_momentum is then compared with the
oracle's M and M^T conjugated by that basis.  Tolerances as the position-space applies."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_3647_gb300.inputs import field_and_source

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 2e-5}


@pytest.fixture(scope="module")
def ufg():
    from paper_1008_3647_gb300 import ufg as u
    u.load()
    return u


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _field(ufg, nx, ntau, seed):
    sigma, x = field_and_source(nx, ntau, seed)
    lat = ufg.Lattice(nx, ntau, 0.05, 5.0)
    return sigma, x, lat, ufg.Field(lat, torch.from_numpy(sigma).cuda())


@pytest.mark.parametrize("nx", [8, 12, 16])
def test_fourier_is_orthogonal_and_diagonalises_the_kinetic_factor(ufg, nx):
    ntau = 4
    sigma, x, lat, field = _field(ufg, nx, ntau, 40 + nx)
    xd = torch.from_numpy(x).cuda()
    xh = ufg.ufg_fourier(field, xd)
    assert float(xh.norm() / xd.norm()) == pytest.approx(1.0, abs=1e-13)
    back = ufg.ufg_fourier(field, xh, inverse=True)
    assert _rel(back.cpu().numpy(), x) < 1e-13
    # F exp(-tau K) x = b .* F x with one factor per mode, the same on every slice and vector
    olat = O.Lattice(nx, ntau, 0.05, 5.0)
    kx = torch.from_numpy(O.kinetic(olat, x)).cuda()
    ratio = (ufg.ufg_fourier(field, kx) / xh).cpu().numpy().reshape(ntau, -1)
    assert np.abs(ratio - ratio[0]).max() < 1e-11
    expect = np.sort(np.exp(-0.05 * O.energy_grid(nx)).ravel())
    assert np.abs(np.sort(ratio[0]) - expect).max() < 1e-11


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nx,ntau", [(16, 12), (16, 5), (8, 9)])
def test_momentum_M_matches_oracle(ufg, nx, ntau, dtype):
    if dtype == torch.float32 and nx != 16:
        pytest.skip("FP32 momentum-space kernel built for N_x = 16")
    sigma, x, lat, field = _field(ufg, nx, ntau, 7 + ntau)
    olat = O.Lattice(nx, ntau, 0.05, 5.0)
    xd = torch.from_numpy(x).to("cuda", dtype)
    xin = xd.double().cpu().numpy()
    xh = ufg.ufg_fourier(field, xd)
    for transpose, ref_fn in ((False, O.apply_M), (True, O.apply_Mdag)):
        yh = ufg.ufg_apply_M_momentum(field, xh, transpose=transpose)
        y = ufg.ufg_fourier(field, yh, inverse=True)
        err = _rel(y.double().cpu().numpy(), ref_fn(olat, sigma, xin))
        assert err < TOL[dtype], (transpose, err)


@pytest.mark.parametrize("nx,ntau", [(16, 12), (16, 5), (8, 9)])
def test_momentum_M_emulated_fp64_matches_oracle(ufg, nx, ntau):
    # double-float arithmetic on the FP32 pipe (about 46 bits) on FP64 vectors: against the oracle
    # at the FP64 tolerance, and against the FP64-pipe kernel
    sigma, x, lat, field = _field(ufg, nx, ntau, 21 + ntau)
    olat = O.Lattice(nx, ntau, 0.05, 5.0)
    xh = ufg.ufg_fourier(field, torch.from_numpy(x).cuda())
    for transpose, ref_fn in ((False, O.apply_M), (True, O.apply_Mdag)):
        ye = ufg.ufg_apply_M_momentum(field, xh, transpose=transpose, emulated=True)
        yd = ufg.ufg_apply_M_momentum(field, xh, transpose=transpose)
        assert float((ye - yd).abs().max() / yd.abs().max()) < 1e-12
        y = ufg.ufg_fourier(field, ye, inverse=True)
        assert _rel(y.cpu().numpy(), ref_fn(olat, sigma, x)) < 1e-12


def test_momentum_M_rejects_unbuilt_extent(ufg):
    _, x, lat, field = _field(ufg, 12, 4, 3)
    with pytest.raises(ufg.UfgError):
        ufg.ufg_apply_M_momentum(field, torch.from_numpy(x).cuda())
