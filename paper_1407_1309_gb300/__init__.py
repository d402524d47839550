"""GB300-native MPDATA step (libmpdata++ 0.1 paper, arXiv 1407.1309).

Hand-written sm_103a CUDA kernels behind a C ABI (include/mpdata.h); this
package holds the kernels' sources (csrc/), their build script, the ctypes
binding (capi), a torch-tensor handle wrapper (solver), the autograd
function, and the seeded input generators (workloads).  Importing the package
does not load the CUDA library; the first call that needs it does, and fails
loudly if it is missing.
"""
from . import capi  # noqa: F401
from .capi import (FCT, TOT, IGA, NUG, KAHAN, RHS_EULER_A, RHS_EULER_B, F32, F64,  # noqa: F401
                   MpdataError)

__all__ = ["capi", "Mpdata", "FCT", "TOT", "IGA", "NUG", "KAHAN", "RHS_EULER_A", "RHS_EULER_B",
           "F32", "F64", "MpdataError"]


def __getattr__(name):
    if name == "Mpdata":
        from .solver import Mpdata
        return Mpdata
    if name == "MPDATAFunction":
        from .autograd import MPDATAFunction
        return MPDATAFunction
    raise AttributeError(name)
