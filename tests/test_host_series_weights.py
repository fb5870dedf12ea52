"""The library's host-side weights of the accelerated weak-coupling series (Sec. 3.1: Euler
S_{d,0}, Euler S_{2d/3,d/3}, the special van Wijngaarden transformation) against the oracle's,
which are pinned in test_oracle_precond.py; and the argument checks.  Host only (no GPU): the
library computes the weights on the CPU."""
import os

import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def ufg():
    from paper_1008_3647_gb300 import build as B
    from paper_1008_3647_gb300 import ufg as u
    if not os.path.exists(B.LIB):
        B.build()
    u.load()
    return u


@pytest.mark.parametrize("order", [0, 1, 2, 3, 4, 6, 9, 16])
@pytest.mark.parametrize("accel", ["none", "euler", "euler23"])
@pytest.mark.parametrize("p", [0.5, 0.3, 0.8])
def test_euler_weights_match_the_oracle(ufg, order, accel, p):
    w = ufg.ufg_wce_series_weights(order, accel, p)
    ref = O.euler_weights(order, accel, p)
    assert np.allclose(w, ref, rtol=1e-13, atol=1e-15), (w, ref)


@pytest.mark.parametrize("order", [0, 1, 2, 4, 8])
@pytest.mark.parametrize("p,s", [(0.5, 1.0), (0.5, 2.0), (0.3, 0.5), (0.7, 3.0)])
def test_van_wijngaarden_weights_match_the_oracle(ufg, order, p, s):
    # the library integrates mu_n by Gauss-Legendre panels, the oracle by adaptive quadrature
    w = ufg.ufg_wce_series_weights(order, "vanw", p, s)
    ref = O.euler_weights(order, "vanw", p, s)
    assert np.allclose(w, ref, rtol=1e-10, atol=1e-14), (w, ref)


def test_defaults_are_the_papers(ufg):
    # p = 0 selects 1/2, s = 0 selects 1
    assert ufg.ufg_wce_series_weights(4, "euler23") == ufg.ufg_wce_series_weights(4, "euler23", 0.5)
    assert ufg.ufg_wce_series_weights(3, "vanw") == ufg.ufg_wce_series_weights(3, "vanw", 0.5, 1.0)


@pytest.mark.parametrize("args", [(17, "euler", 0.5, 1.0), (-1, "none", 0.5, 1.0),
                                  (2, "euler", 1.5, 1.0), (2, "vanw", 0.5, -2.0)])
def test_invalid_arguments_are_refused(ufg, args):
    with pytest.raises(ufg.UfgError) as e:
        ufg.ufg_wce_series_weights(*args)
    assert e.value.status == ufg.UFG_INVALID_ARG
