"""GB300-native (sm_103a) lattice Boltzmann method on generalized polynomials
for Fermi-Dirac electrons (Coelho, Ilha, Doria, arXiv:1510.07328).

The compute path is the C-ABI shared library ``liblbm_gb300.so`` (CUDA kernels
in ``csrc/``); ``lbm`` is its thin ctypes binding.  ``inputs`` holds the seeded
synthetic workloads.  Importing this package does not load the library.
"""

__all__ = ["inputs", "lbm", "build"]
