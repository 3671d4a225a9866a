"""GB300-native multiplicative vertex-patch smoother for matrix-free Q_k
finite elements, inside geometric multigrid and conjugate gradients
(Wichrowski, Munch, Kronbichler, Kanschat, arXiv 2407.02100).

The compute path is the CUDA library ``libgmg.so`` (C ABI in
``include/gmg.h``); ``gmg`` is its ctypes binding.  Importing the package
does not load the library; the first call does, and fails loudly if it has
not been built.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "gmg", "build"]
