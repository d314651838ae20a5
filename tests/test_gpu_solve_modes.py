"""The persistent-graph solve (one CUDA graph per batch with a device-side WHILE
loop) and the same passes launched from the host (DLMA_SOLVE_GRAPH=0 in the
environment of a solve, the form kernel profilers can see into) run the same
kernels in the same order: their solutions agree bit for bit, and both pass the
oracle's residual check."""
import numpy as np
import pytest

import synth
from oracle import dirac

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_09729_gb300 as dl
    return dl


@pytest.mark.parametrize("prec,solver", [("FP32", "SOLVER_BICGSTAB"), ("FP32", "SOLVER_CGNE"), ("FP16S", "SOLVER_CGNE")])
def test_graph_and_host_passes_agree(dl, prec, solver, monkeypatch):
    L, T, m0, csw = 6, 8, 0.08, 1.1
    U = synth.gauge_field(L, T, 0.2, 621)
    eo = dirac.EvenOdd(U, L, T, m0, csw)
    b = synth.gaussian_spinors(5, L ** 3 * T, 622)
    # one context (the autotuned stencil shape and batch size, which set the order of
    # the inner-product partial sums, are shared), the switch read at every solve
    ctx = dl.Context(L, T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(m0, csw)
    ctx.dlma_set_solver(getattr(dl, solver))
    out = {}
    for flag in ("1", "0", "1"):
        monkeypatch.setenv("DLMA_SOLVE_GRAPH", flag)
        x, info = ctx.dlma_solve(b, 1e-10, getattr(dl, prec))
        for j in range(5):
            r = np.linalg.norm((b[j] - eo.apply_full(x[j])).ravel()) / np.linalg.norm(b[j].ravel())
            assert r <= 1e-10 and info[j]["converged"], (flag, j, r)
        if flag in out:    # the first graph solve tuned the context: compare from here on
            out[flag] = (x, [i["iters_inner"] for i in info])
        out.setdefault(flag, (x, [i["iters_inner"] for i in info]))
    ctx.close()
    assert out["1"][1] == out["0"][1]
    assert np.array_equal(out["1"][0], out["0"][0])
