"""GB300-native modal DG right-hand side for driven isothermal turbulence.

``Solver`` (solver.py) drives the CUDA library libdg.so through its C ABI
(include/dg.h); ``inputs`` produces seeded synthetic states.
"""
from .solver import Solver, nmodes  # noqa: F401
