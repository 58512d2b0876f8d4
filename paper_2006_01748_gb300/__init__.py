"""GB300-native explicit finite-volume step of the anisotropic,
heterogeneous Gatenby-Gawlinski system (arXiv 2006.01748).

The computation lives in ``libgg.so`` (CUDA C++ for sm_103a, C ABI in
``include/gg.h``); ``gg`` is its ctypes binding, ``autograd`` wraps the
adjoint as a ``torch.autograd.Function``, ``inputs`` draws seeded synthetic
workloads.  Importing the package loads nothing; ``build()`` compiles the
library in-tree.
"""
from ._build import build  # noqa: F401

__all__ = ["build", "gg", "inputs"]
