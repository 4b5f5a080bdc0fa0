"""GB300-native periodizing operator for 2D doubly periodic Laplace, modified
Helmholtz, Stokes and modified Stokes kernels, with the singly periodic
variant and the Stokes pressure (Pei, Askham, Greengard & Jiang, "Periodic
Fast Multipole Method", arXiv 2111.01083).

The computation lives in the CUDA library ``libpfmm.so`` (C ABI in
``include/pfmm.h``); this package only marshals arguments.  Importing the
package does not load the library; the first call does, and raises if it is
missing (there is no CPU fallback).
"""
from .periodic import BatchOp, PeriodicOp, StokesPressure, autotune_batch, periodic, tune_batch, tuned_batch  # noqa: F401
from . import _lib  # noqa: F401

__all__ = ["PeriodicOp", "BatchOp", "StokesPressure", "autotune_batch", "periodic", "tune_batch", "tuned_batch"]
