"""GB300-native modal DG right-hand side for driven isothermal turbulence.

``Solver`` (solver.py) drives the CUDA library libdg.so through its C ABI
(include/dg.h); ``AdiabaticSolver`` (adiabatic.py) does the same for the
five-variable adiabatic system; ``inputs`` produces seeded synthetic states.
"""
from .adiabatic import AdiabaticSolver  # noqa: F401
from .solver import Solver, nmodes  # noqa: F401
