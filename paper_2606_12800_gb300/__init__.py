"""GB300-native flow routing and drainage-area determination.

The data-parallel hot path of W. Bangerth, "Massively parallel flow routing
and drainage area determination": local flow routing (D8 / MFD receivers),
exact global flow routing (w = A^{-1} r), its adjoint, a batched form and a
mass-balance check, as hand-written sm_103a CUDA behind the C ABI of
``include/fr.h`` (``libfr.so``).  This package is the thin Python layer over
that ABI; see ``api`` for the tensor-level functions and ``_lib`` for the raw
ctypes binding with the C names.
"""
from ._lib import (FR_CHECK_FINITE, FR_D4, FR_DINF, FR_D8_LOWEST, FR_D8_STEEPEST, FR_EDGE_ROUTE, FR_EDGE_SINK,
                   FR_SINK, FrError)

__all__ = ["api", "inputs", "FR_CHECK_FINITE", "FR_D4", "FR_DINF", "FR_D8_LOWEST", "FR_D8_STEEPEST", "FR_EDGE_ROUTE",
           "FR_EDGE_SINK", "FR_SINK", "FrError"]


def __getattr__(name):
    if name in ("api", "inputs"):
        import importlib
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
