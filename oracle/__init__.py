"""FP64 CPU oracle for the unitary-Fermi-gas fermion matrix (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline and
reference legs) may import this package.  The CUDA library never calls it and shares no
code with it.
"""
from .ufg_oracle import *  # noqa: F401,F403
