"""The allocation-free Q apply (for callers that cannot call cudaMalloc where they need the
operator) against the regular field-based ufg_apply_Q, through the C ABI.  Collected last so that
a run stopping at its first failure has run everything else already; it also passes alone in a
fresh process."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_3647_gb300.inputs import field_and_source

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 apply tolerance used throughout the GPU tests


@pytest.fixture(scope="module")
def ufg():
    from paper_1008_3647_gb300 import ufg as u
    u.load()
    return u


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("nx,ntau", [(8, 16), (16, 20), (32, 6), (6, 7)])
def test_noalloc_Q_matches_field_Q_twice(ufg, nx, ntau):
    lat = ufg.Lattice(nx, ntau, 0.05, 5.0)
    for call, seed in enumerate((11, 12)):  # two calls in a row, different inputs each time
        sigma, x = field_and_source(nx, ntau, seed)
        sd, xd = torch.from_numpy(sigma).cuda(), torch.from_numpy(x).cuda()
        field = ufg.Field(lat, sd)
        ref = ufg.ufg_apply_Q(field, xd)
        y = torch.full_like(xd, float("nan"))
        ufg.ufg_apply_Q_noalloc(nx, ntau, 0.05, 5.0, sd, xd, y)
        torch.cuda.synchronize()
        assert _rel(y, ref) < TOL, (call, _rel(y, ref))
        # and against the oracle's M^T M directly
        oref = torch.from_numpy(O.apply_Q(O.Lattice(nx, ntau, 0.05, 5.0), sigma, x))
        assert _rel(y.cpu(), oref) < TOL, (call, _rel(y.cpu(), oref))


def test_noalloc_rejects_lattice_beyond_static_limit(ufg):
    nx, ntau = 32, 40  # 1,310,720 sites > 2^20
    z = torch.zeros(ntau, nx, nx, nx, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(z)
    with pytest.raises(ufg.UfgError) as e:
        ufg.ufg_apply_Q_noalloc(nx, ntau, 0.05, 5.0, z, z, y)
    assert e.value.status == ufg.UFG_INVALID_ARG
    assert "static scratch limit" in str(e.value)
