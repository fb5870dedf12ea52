"""GPU parity of the operator applies (through the C ABI) against the FP64 oracle.

Tolerances: FP64 applies within 1e-12 of the oracle in max-norm relative to max|ref| (the
bound asked of the library); FP32 applies within 2e-5 (FP32 unit roundoff 6e-8 times the
~3 N + 10 rounding steps a value passes through at N <= 32, with margin)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_3647_gb300.inputs import field_and_source

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 2e-5}
# (N_x, N_tau): the 4^3x16 and 8^3x64 workloads, every built N_x, odd and tiny N_tau
# the long time extents give the M0^{-1} recurrence per-thread chunks (N_tau / 8 elements) of
# several load groups plus a ragged tail
SHAPES = [(4, 16), (8, 64), (6, 7), (10, 5), (12, 9), (16, 12), (32, 5), (4, 3), (4, 200),
          (8, 131)]


@pytest.fixture(scope="module")
def ufg():
    from paper_1008_3647_gb300 import ufg as u
    u.load()
    return u


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


OPS = {
    "M": ("ufg_apply_M", O.apply_M),
    "Mdag": ("ufg_apply_Mdag", O.apply_Mdag),
    "Q": ("ufg_apply_Q", O.apply_Q),
    "M1": ("ufg_apply_M1", O.apply_M1),
    "M1T": ("ufg_apply_M1T", O.apply_M1T),
    "kin": ("ufg_apply_kinetic", lambda lat, s, x: O.kinetic(lat, x)),
    "M0inv": ("ufg_apply_M0inv", lambda lat, s, x: O.apply_M0inv(lat, x)),
    "M0invT": ("ufg_apply_M0invT", lambda lat, s, x: O.apply_M0invT(lat, x)),
}


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nx,ntau", SHAPES)
def test_apply_parity(ufg, nx, ntau, dtype):
    sigma, x = field_and_source(nx, ntau, 100 + nx + ntau)
    lat = ufg.Lattice(nx, ntau, 0.05, 5.0)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    olat = O.Lattice(nx, ntau, 0.05, 5.0)
    xd = torch.from_numpy(x).to("cuda", dtype)
    xin = xd.double().cpu().numpy()  # the FP32 case compares on the rounded input
    for name, (fn, ref_fn) in OPS.items():
        y = getattr(ufg, fn)(field, xd)
        torch.cuda.synchronize()
        ref = ref_fn(olat, sigma, xin)
        err = _rel(y.double().cpu().numpy(), ref)
        assert err < TOL[dtype], "%s N_x=%d N_tau=%d %s: %g" % (name, nx, ntau, dtype, err)


@pytest.mark.parametrize("dispersion", [1])
def test_apply_parity_lattice_dispersion(ufg, dispersion):
    nx, ntau = 8, 6
    sigma, x = field_and_source(nx, ntau, 5)
    lat = ufg.Lattice(nx, ntau, 0.05, 5.0, dispersion)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    olat = O.Lattice(nx, ntau, 0.05, 5.0, dispersion)
    y = ufg.ufg_apply_M(field, torch.from_numpy(x).cuda()).cpu().numpy()
    assert _rel(y, O.apply_M(olat, sigma, x)) < 1e-12


def test_adjoint_identity_gpu(ufg):
    nx, ntau = 16, 20
    sigma, u = field_and_source(nx, ntau, 1)
    _, v = field_and_source(nx, ntau, 2)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    ud, vd = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
    a = float((ud * ufg.ufg_apply_M(field, vd)).sum())
    b = float((ufg.ufg_apply_Mdag(field, ud) * vd).sum())
    assert a == pytest.approx(b, rel=1e-12)


def test_M0inv_inverts_free_M_gpu(ufg):
    nx, ntau = 8, 40
    _, v = field_and_source(nx, ntau, 3)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.zeros(lat.shape, dtype=torch.float64, device="cuda"))
    vd = torch.from_numpy(v).cuda()
    back = ufg.ufg_apply_M(field, ufg.ufg_apply_M0inv(field, vd))
    assert _rel(back.cpu().numpy(), v) < 1e-12


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_apply_full_size_32cubed_x512(ufg, dtype):
    # the 32^3 x 512 workload (16.8M sites) in the launch configuration the bench times
    nx, ntau = 32, 512
    sigma, x = field_and_source(nx, ntau, 7)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    olat = O.Lattice(nx, ntau)
    xd = torch.from_numpy(x).to("cuda", dtype)
    xin = xd.double().cpu().numpy()
    for fn, ref_fn in [("ufg_apply_M", O.apply_M), ("ufg_apply_Mdag", O.apply_Mdag)]:
        y = getattr(ufg, fn)(field, xd).double().cpu().numpy()
        assert _rel(y, ref_fn(olat, sigma, xin)) < TOL[dtype], fn


def test_invalid_arguments_rejected(ufg):
    with pytest.raises(ufg.UfgError) as e:
        ufg.Lattice(5, 8)
    assert e.value.status == ufg.UFG_INVALID_ARG
    with pytest.raises(ufg.UfgError) as e:
        ufg.Lattice(14, 8)
    assert e.value.status == ufg.UFG_UNSUPPORTED
    with pytest.raises(ufg.UfgError):
        ufg.Lattice(8, 2)
    lat = ufg.Lattice(4, 8)
    field = ufg.Field(lat, torch.zeros(lat.shape, dtype=torch.float64, device="cuda"))
    x = torch.zeros(lat.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(ufg.UfgError) as e:  # in place (x aliases y) is rejected
        ufg.ufg_apply_M(field, x, x)
    assert e.value.status == ufg.UFG_INVALID_ARG


@pytest.mark.parametrize("nx,ntau", [(8, 64), (16, 40), (32, 8)])
def test_autotuned_launch_shape_keeps_parity(ufg, nx, ntau):
    lat = ufg.Lattice(nx, ntau)
    shapes = lat.ufg_lattice_autotune()
    for prec, (C, spc) in shapes.items():
        assert C in (0, 1, 2, 4) and spc in (1, 2, 4, 8)
    sigma, x = field_and_source(nx, ntau, 77)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    olat = O.Lattice(nx, ntau)
    for dtype in (torch.float64, torch.float32):
        xd = torch.from_numpy(x).to("cuda", dtype)
        for fn, ref_fn in [("ufg_apply_M", O.apply_M), ("ufg_apply_Mdag", O.apply_Mdag)]:
            y = getattr(ufg, fn)(field, xd).double().cpu().numpy()
            assert _rel(y, ref_fn(olat, sigma, xd.double().cpu().numpy())) < TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("ntau", [3, 4, 17])
def test_fused_Q_16cubed_short_lattices(ufg, ntau, dtype):
    """Q on 16^3 runs as one kernel per output slice (x at t-1, t, t+1): the shortest lattice
    where the three slices differ, N_tau = 4 and an odd N_tau, against the oracle's M^T M."""
    nx = 16
    sigma, x = field_and_source(nx, ntau, 40 + ntau)
    lat = ufg.Lattice(nx, ntau)
    field = ufg.Field(lat, torch.from_numpy(sigma).cuda())
    y = ufg.ufg_apply_Q(field, torch.from_numpy(x).cuda().to(dtype))
    ref = O.apply_Q(O.Lattice(nx, ntau), sigma, x)
    assert _rel(y.double().cpu().numpy(), ref) < TOL[dtype]
