"""GB300 (sm_103a) distillation low-mode averaging (arXiv:2201.09729).

The compute lives in libdlma.so (C ABI, include/dlma.h); this package is the
thin Python binding: ``Context`` (context.py) and the raw ctypes handle
(_lib.py), plus the autograd wrapper of the solve (autograd.py).
"""
from ._lib import FP16S, FP32, FP64, MEM_DEVICE, MEM_HOST, SOLVER_BICGSTAB, SOLVER_CGNE, DlmaError, load  # noqa: F401
from .context import Context  # noqa: F401

__all__ = ["Context", "DlmaError", "load", "FP64", "FP32", "FP16S", "MEM_HOST", "MEM_DEVICE", "SOLVER_CGNE",
           "SOLVER_BICGSTAB"]
