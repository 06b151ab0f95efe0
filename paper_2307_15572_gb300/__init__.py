"""GB300-native randomized low-rank decomposition (arXiv:2307.15572).

The compute path is the C-ABI library built from ``csrc/`` (see
``include/rsvd.h``); ``rsvd`` is its Python binding and ``synth`` the seeded
input generators used by tests and benchmarks.
"""
