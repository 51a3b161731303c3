"""GB300 (sm_103a) single-spin Metropolis sweep of the classical anisotropic
Heisenberg model (arXiv 2106.11286), behind a small C ABI (include/hs.h).

Modules: ``hs`` (ctypes binding, loaded on first use), ``build`` (in-tree
nvcc build of libhs.so), ``inputs`` (seeded synthetic inputs).
"""
__all__ = ["hs", "build", "inputs"]
