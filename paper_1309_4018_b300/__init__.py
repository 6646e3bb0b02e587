"""B300-native treecode boundary-element Poisson-Boltzmann solver.

The compute path is the CUDA library ``libpbbem.so`` (sources in ``csrc/``,
C-ABI in ``include/pbbem.h``, built by ``build.py``); ``pbbem`` is its ctypes
binding.  Importing the package itself needs no GPU.
"""
