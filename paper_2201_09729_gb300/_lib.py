"""ctypes binding of the dlma C ABI (include/dlma.h): argument marshalling only.

Every computation runs in libdlma.so; nothing here has a CPU fallback.  If the
library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdlma.so")

DLMA_OK, DLMA_ERR_INVALID_ARG, DLMA_ERR_NOT_CONVERGED, DLMA_ERR_NONFINITE = 0, 1, 2, 3
DLMA_ERR_SINGULAR, DLMA_ERR_OOM, DLMA_ERR_CUDA, DLMA_ERR_TIMEOUT, DLMA_ERR_STATE = 4, 5, 6, 7, 8
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "NOT_CONVERGED", 3: "NONFINITE", 4: "SINGULAR",
                5: "OOM", 6: "CUDA", 7: "TIMEOUT", 8: "STATE"}
FP64, FP32, FP16S = 0, 1, 2
MEM_HOST, MEM_DEVICE = 0, 1
SOLVER_CGNE, SOLVER_BICGSTAB = 0, 1


class Lattice(C.Structure):
    _fields_ = [("L", C.c_int), ("T", C.c_int), ("bc_t", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iters_inner", C.c_int), ("iters_outer", C.c_int),
                ("true_resid", C.c_double), ("converged", C.c_int)]


_P = C.c_void_p
_D = C.c_double
_I = C.c_int
_ST = C.c_int

# name -> (restype, argtypes): the full set of entry points of dlma.h
SIGNATURES = {
    "dlma_create": (_ST, [C.POINTER(Lattice), _I, _P, C.POINTER(_P)]),
    "dlma_destroy": (_ST, [_P]),
    "dlma_last_error": (C.c_char_p, [_P]),
    "dlma_set_memory_cap": (_ST, [_P, C.c_uint64]),
    "dlma_release_workspace": (_ST, [_P]),
    "dlma_set_gauge": (_ST, [_P, _P, _I]),
    "dlma_set_params": (_ST, [_P, _D, _D]),
    "dlma_apply_Dw": (_ST, [_P, _P, _P, _I, _I, _I]),
    "dlma_apply_schur": (_ST, [_P, _P, _P, _I, _I, _I, _I]),
    "dlma_apply_schur_noalloc": (_ST, [_P, _P, _P, _I, _I]),
    "dlma_solve": (_ST, [_P, _P, _P, _I, _D, _I, _P, _I]),
    "dlma_set_solver": (_ST, [_P, _I]),
    "dlma_apply_laplacian": (_ST, [_P, _P, _P, _I, _I]),
    "dlma_laplacian_eigs": (_ST, [_P, _I, _I, _D, _P, _P, _I]),
    "dlma_make_sources": (_ST, [_P, _I, _I, _P, _I, _P, _P, _I]),
    "dlma_project": (_ST, [_P, _I, _P, _I, _P, _I, _P, _I]),
    "dlma_contract": (_ST, [_P, _I, _I, _P, _I, _P, _P, _P, _P, _P, _P, _I]),
    "dlma_correlators": (_ST, [_P, _I, _I, _I, _P, _D, _I, _P, _P, _P, _P, _P, _P, _I]),
    "dlma_correlators_diluted": (_ST, [_P, _I, _I, _I, _P, _D, _I, _P, _P, _P, _P, _P, _P, _I]),
    "dlma_correlators_plain": (_ST, [_P, _I, _I, _P, _I, _D, _I, _P, _P, _I]),
    "dlma_solve_adjoint": (_ST, [_P, _P, _P, _I, _D, _I, _P, _I]),
    "dlma_real_dot": (_ST, [_P, _P, _P, C.c_uint64, _P, _I]),
    "dlma_dirac_eigs": (_ST, [_P, _I, _D, _P, _P, _I]),
    "dlma_dirac_project": (_ST, [_P, _P, _P, _I, _I, _I]),
    "dlma_set_checkpoint": (_ST, [_P, _I]),
    "dlma_checkpoint_serial": (C.c_uint64, [_P]),
    "dlma_correlators_backward": (_ST, [_P, _I, _I, _I, _P, _D, _I, _P, _P, _P, _I]),
    "dlma_index_tables": (_ST, [_P, _P, _P]),
    "dlma_kernel_launches": (C.c_uint64, [_P]),
    "dlma_last_timing": (_ST, [_P, _P, _I]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libdlma.so and attach the signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libdlma.so not found at {path}: build it with paper_2201_09729_gb300.build")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class DlmaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
