"""GB300 (sm_103a) blocked Cholesky and pivot-free LU with step s, after
Camarero, arXiv:1812.02056, Sec. 2 (Algorithms 1 and 2).

The computation lives in the CUDA shared library ``libgbchol.so`` (C ABI in
``include/gbchol.h``); ``binding`` marshals arguments to it.  ``inputs``
holds the seeded synthetic workloads.
"""
__all__ = ["binding", "inputs"]
