"""The C-ABI library builds, loads and exports every entry point declared in
include/dlma.h, and the binding declares a signature for each (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dlma.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dlma_[a-zA-Z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2201_09729_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("dlma_create", "dlma_set_gauge", "dlma_set_params", "dlma_apply_Dw", "dlma_solve",
              "dlma_laplacian_eigs", "dlma_project", "dlma_contract"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2201_09729_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _declared()


def test_create_without_gpu_fails_cleanly(lib):
    # no GPU in this container: dlma_create must return an error status, not crash
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2201_09729_gb300 import _lib
    L = _lib.load()
    h = ctypes.c_void_p()
    lat = _lib.Lattice(4, 4, 0)
    st = L.dlma_create(ctypes.byref(lat), 0, None, ctypes.byref(h))
    assert st != 0
    bad = _lib.Lattice(3, 4, 0)
    assert L.dlma_create(ctypes.byref(bad), 0, None, ctypes.byref(h)) == _lib.DLMA_ERR_INVALID_ARG
