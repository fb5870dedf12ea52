"""GB300 (sm_103a) library for the unitary-Fermi-gas fermion matrix of arXiv:1008.3647.

The product is libufg.so (C ABI in include/ufg.h); ``paper_1008_3647_gb300.ufg`` is its thin
ctypes binding and ``paper_1008_3647_gb300.build`` compiles it in-tree.
"""
