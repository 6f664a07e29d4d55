"""Plain, slow, FP64 CPU oracle of the PML + outer-BC lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY. Only the tests, the package smoke check and the CPU-baseline leg of
the benchmark may import this package. The CUDA product path never routes through it and
shares no code with it (no common tables, helpers or constant generators).

Everything here follows the paper (Klass, Gabbana, Bartel, "Perfectly Matched Layers and
Characteristic Boundaries in Lattice Boltzmann: Accuracy vs. Cost", arXiv 2504.20169):

* stencil.py         Sec. 2 "Velocity stencils": D2Q9 / D2Q17 / D2Q37 Gauss-Hermite rules.
* equilibrium.py     Eq. (macro), Eqs. (feq-2), (feq-3), (feq-4); BGK of Eq. (lbe).
* pml.py             Eqs. (decomp-NJ), (PMLCOLL), (PML_ramp), (PMLQ) with the trapezoidal rule,
                     (FD-dx-bw), (FD-dx-center).
* characteristic.py  Eqs. (NSF-CHAR), (PNR), (thermal_CBC_macro_evo),
                     (thermal_LODI_macro_evo), (CBC-Relax); non-equilibrium extrapolation.
* solver.py          the time step of Sec. 2 (collide, stream, BC) on the PML-extended grid,
                     zero-gradient BC Eq. (zg-bc), periodic reference mode (Sec. 5).
* metrics.py         e_Z and pointwise errors of Sec. 5, normwise relative L2, totals.

Readings taken where the paper is silent or garbled are listed in the docstrings of the
functions that take them (R1..R18 style notes are spelled out in place).
"""
from .stencil import Lattice, lattice  # noqa: F401
from .solver import OracleLBM  # noqa: F401
