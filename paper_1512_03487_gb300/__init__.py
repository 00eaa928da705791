"""GB300-native Wilson / domain-wall Dirac operators, CG and fermion force.

The compute path is the CUDA library ``liblqcd.so`` (sources in ``csrc/``,
C ABI in ``include/lqcd.h``); this package is its Python binding. Importing it
fails with ImportError when the library has not been built: there is no CPU
fallback.
"""
from .api import *  # noqa: F401,F403
from .api import LqcdError, hmc_params, lattice, lib, mg_params, operator, solver_params  # noqa: F401

__all__ = [n for n in dir() if n.startswith("lqcd_") or n.startswith("LQCD_")] + [
    "LqcdError", "lattice", "operator", "solver_params", "hmc_params", "mg_params", "lib"]
