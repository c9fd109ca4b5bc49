"""GB300 algebraic two-level Schwarz preconditioner (arXiv 2201.02250) behind a C ABI.

The compute path is libA2LS.so (hand-written CUDA for sm_103a, declared in
include/a2ls.h); ``a2ls`` is its ctypes binding.  Importing this package
does not load the library; ``a2ls.lib()`` does, and raises if it is absent.
"""
from . import a2ls  # noqa: F401

__all__ = ["a2ls"]
