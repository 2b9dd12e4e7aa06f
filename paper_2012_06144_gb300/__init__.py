"""GB300 (sm_103a) conservative Allen-Cahn multiphase lattice Boltzmann solver.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/lbm.h``); ``lbm`` is its ctypes binding.  See ``lbm.Simulation`` for the
PyTorch-backed convenience wrapper.
"""
from . import lbm  # noqa: F401
from ._build import build  # noqa: F401
