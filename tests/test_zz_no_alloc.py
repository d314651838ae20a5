"""dlma_apply_schur_noalloc: the Schur operator for callers that cannot
allocate device memory (a framework that owns every byte of device memory
through its own pool, or a caller that cannot take the synchronisation a
cudaMalloc may cause).  Its work space is a fixed array in the library's
device memory.  Called through the C ABI on device buffers, it must give the
same result as dlma_apply_schur, on two calls in a row, and reject batches
that do not fit its work space.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_09729_gb300 as dl
    return dl


def test_noalloc_schur_matches_allocating_entry_point(dl):
    import torch

    L, T = 6, 4
    U = synth.gauge_field(L, T, 0.25, 901)
    ctx = dl.Context(L, T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(0.1, 1.2)
    lib = dl.load()
    Vh = L ** 3 * T // 2
    for call, (dagger, seed) in enumerate(((0, 902), (1, 903))):
        host = synth.gaussian_spinors(3, Vh, seed)
        want = ctx.dlma_apply_schur(host, dagger, dl.FP64)
        d_in = torch.from_numpy(host).cuda()
        d_out = torch.full_like(d_in, float("nan"))
        torch.cuda.synchronize()
        st = lib.dlma_apply_schur_noalloc(ctx.h, ctypes.c_void_p(d_in.data_ptr()),
                                          ctypes.c_void_p(d_out.data_ptr()), 3, dagger)
        assert st == 0, lib.dlma_last_error(ctx.h).decode()
        got = d_out.cpu().numpy()
        rel = np.linalg.norm((got - want).ravel()) / np.linalg.norm(want.ravel())
        assert rel < 1e-13, (call, rel)


def test_noalloc_rejects_oversized_batch(dl):
    import torch

    L, T = 16, 32
    U = synth.gauge_field(L, T, 0.2, 904)
    ctx = dl.Context(L, T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(0.08, 1.0)
    lib = dl.load()
    Vh = L ** 3 * T // 2
    # 3 fields x 192 B x Vh x nrhs > 64 MiB for nrhs = 2 at this size
    d = torch.zeros((2, Vh, 4, 3), dtype=torch.complex128, device="cuda")
    st = lib.dlma_apply_schur_noalloc(ctx.h, ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(d.data_ptr()), 2, 0)
    assert st == 1
    assert "work space" in lib.dlma_last_error(ctx.h).decode()
