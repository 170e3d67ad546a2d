"""GB300-native PSLR preconditioner (arXiv 2002.00917): hand-written sm_103a CUDA
kernels behind the C ABI of include/pslr.h, with a thin ctypes binding.

Importing the package does not load the CUDA library; ``pslr.load()`` (or the
first :class:`pslr.Pslr`) does, and raises if ``libpslr.so`` has not been built.
"""
from . import build, pslr  # noqa: F401
from .pslr import Pslr, PslrError  # noqa: F401
