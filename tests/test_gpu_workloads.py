"""The batched (24^3 x 48, four source timeslices) and full-size (32^3 x 64)
workloads end to end on the GPU.  The oracle cannot run these pipelines, so it
checks what holds at any size: every solve's FP64 true residual, a sampled
solution's residual under the oracle's own operator, sampled eigenpair
residuals under the oracle's Laplacian, and C_dist^PS = tr[tau tau^dag] > 0."""
import numpy as np
import pytest

import synth
from oracle import dirac
from oracle import laplacian as lap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_09729_gb300 as dl
    return dl


def _modes_check(U, L, lam, V, ts, ks):
    # V stays on the device (9.7 GB at 32^3 x 64): copy only the sampled modes
    for t in ts:
        Ut = lap.timeslice_links(U, L, t)
        for k in ks:
            v = V[t, k].cpu().numpy()
            r = -lap.lap_apply(Ut, L, v) - lam[t, k] * v
            assert np.linalg.norm(r) <= 1e-10 * max(1.0, lam[t, k])


def _run(dl, name, inner):
    import torch

    wl = synth.WORKLOADS[name]
    U, eta = synth.workload_inputs(wl)
    ctx = dl.Context(wl.L, wl.T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(wl.m0, wl.csw)
    lam, V = ctx.dlma_laplacian_eigs(-1, wl.n_modes, 1e-10, device_out=True)
    _modes_check(U, wl.L, lam, V, (0, wl.T // 2, wl.T - 1), (0, wl.n_modes - 1))
    del V
    torch.cuda.empty_cache()
    results = []
    for i, tp in enumerate(wl.t_src):
        r = ctx.dlma_correlators(tp, wl.n_modes, torch.from_numpy(np.ascontiguousarray(eta[i])).cuda(), wl.tol,
                                 getattr(dl, inner))
        assert len(r["info"]) == 4 * wl.n_modes + 5 * wl.n_noise
        assert all(x["converged"] and x["true_resid"] <= wl.tol for x in r["info"])
        assert np.all(r["C_dist"][0].real > 0)
        assert np.abs(r["C_dist"][0].imag).max() < 1e-8 * np.abs(r["C_dist"][0].real).max()
        results.append(r)
    # one noise source solved alone, its residual checked by the oracle's operator
    b = np.zeros((1, wl.volume, 4, 3), dtype=np.complex128)
    tp = wl.t_src[0]
    b[0, tp * wl.vol_s:(tp + 1) * wl.vol_s] = eta[0, 0]
    x, info = ctx.dlma_solve(b, wl.tol, getattr(dl, inner))
    eo = dirac.EvenOdd(U, wl.L, wl.T, wl.m0, wl.csw)
    res = np.linalg.norm((b[0] - eo.apply_full(x[0])).ravel()) / np.linalg.norm(b[0].ravel())
    assert res <= wl.tol, res
    ctx.close()
    return results


def test_batched_workload_four_source_timeslices(dl):
    res = _run(dl, "batched_24c48", "FP32")
    # the same noise statistics at every source timeslice: the correlators decay
    # away from the source, C_PS(t' + 1) < C_PS(t') in every case
    wl = synth.WORKLOADS["batched_24c48"]
    for r, tp in zip(res, wl.t_src):
        c = r["C"][0].real
        assert c[(tp + 1) % wl.T] < c[tp]


def test_full_pipeline_workload(dl):
    _run(dl, "full_32c64", "FP16S")
