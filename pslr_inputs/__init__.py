"""Seeded synthetic inputs shared by the oracle and the CUDA path.

Nothing in this package implements the PSLR method: it generates matrices,
right-hand sides and workload parameters only.
"""
from . import generators, configs  # noqa: F401
