"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module draws random numbers only; it holds none of the method's arithmetic.  Recipe:
the auxiliary field sigma is i.i.d. uniform on [-pi, pi] (the random configurations of the
paper's Sec. 5), right-hand sides and pseudofermion sources are i.i.d. N(0, 1).  One numpy
PCG64 generator per seed draws, in this order: sigma with shape [N_tau, N_x, N_x, N_x]
(C order; [N_tau, N_x, N_x] or [N_tau, N_x] on lower-dimensional lattices), then the vector of
the same shape.
"""
from __future__ import annotations

import numpy as np


def field_and_source(nx: int, ntau: int, seed: int, dim: int = 3):
    """(sigma, b): sigma ~ U[-pi, pi], b ~ N(0, 1), both float64 [N_tau][N_x]^dim."""
    rng = np.random.default_rng(seed)
    shape = (ntau,) + (nx,) * dim
    sigma = rng.uniform(-np.pi, np.pi, size=shape)
    b = rng.standard_normal(shape)
    return sigma, b


def batch_shapes(n: int = 96, seed: int = 0, nxs=(6, 8, 10, 12), ntaus=(40, 80, 120, 160)):
    """Uneven batch: n (N_x, N_tau) pairs drawn uniformly from nxs x ntaus with one generator;
    problem i then uses seed i + 1 for its own sigma and b."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nx = int(rng.choice(nxs))
        ntau = int(rng.choice(ntaus))
        out.append((nx, ntau, i + 1))
    return out


def sample_sites(shape, count: int, seed: int):
    """count distinct flat site indices drawn uniformly (for finite-difference checks)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(int(np.prod(shape)), size=count, replace=False))
