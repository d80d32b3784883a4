"""GB300-native D2Q37 thermal lattice-Boltzmann step (arXiv:1703.04594).

The compute path is a C-ABI shared library of hand-written sm_103a CUDA kernels
(``csrc/``, declared in ``include/lbm_d2q37.h``); ``paper_1703_04594_gb300.lbm`` is the
thin ctypes binding over it.  Importing this package does not load the library;
the first call into ``lbm`` does, and raises if the library has not been built.
"""
__all__ = ["inputs", "lbm"]
