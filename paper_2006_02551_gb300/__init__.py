"""GB300 library for nodal DGTD Maxwell solves with a weight-adjusted,
smoothly varying stretched-coordinate PML.

The compute path is the C-ABI shared library built from ``csrc/`` (CUDA
kernels for sm_103a); ``wadg`` is its ctypes binding.
"""
from .wadg import (Group, Solver, WadgError, load, make_profile, reference_operator,  # noqa: F401
                   exported_symbols)
