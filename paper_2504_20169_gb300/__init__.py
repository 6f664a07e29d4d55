"""GB300-native PML + outer-boundary thermal lattice Boltzmann step (arXiv 2504.20169).

The compute path is liblbm.so (hand-written sm_103a CUDA behind the C ABI of include/lbm.h);
this package only marshals arguments to it.
"""
from ._lib import LBMError, lib  # noqa: F401
from .solver import Solver, estimate_bytes, lattice_info, peak_fma  # noqa: F401
