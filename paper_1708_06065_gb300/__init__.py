"""GB300 (sm_103a) implementation of lAIR: AMG with local approximate ideal restriction.

``lair`` is the ctypes binding of the CUDA library ``liblair.so`` (C ABI in
include/lair.h); ``autograd.solve`` is the differentiable solve. Importing the
package loads the library and fails if it has not been built.
"""
from .lair import (CF_AUTO, CF_PMIS, CF_RS, CF_USER, FGMRES, FP64, MIXED, P_LAIP, P_ONEPOINT, RELAX_FCF, RELAX_FF,
                   RELAX_FFC, STATIONARY, Hierarchy, LairError, Report, lib, options)

__all__ = ["Hierarchy", "LairError", "Report", "lib", "options", "CF_AUTO", "CF_PMIS", "CF_RS", "CF_USER", "FGMRES",
           "FP64", "MIXED", "P_LAIP", "P_ONEPOINT", "RELAX_FCF", "RELAX_FF", "RELAX_FFC", "STATIONARY"]
