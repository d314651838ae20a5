"""GPU parity of the diluted-wall-source correlators (Sec. 3: colour x even-odd
dilution, spin-explicit one-end insertion) against the FP64 oracle, through the
C ABI."""
import numpy as np
import pytest

import synth
from oracle import dilution, dirac, dlma
from oracle import laplacian as lap
from oracle import solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_09729_gb300 as dl
    return dl


@pytest.mark.parametrize("prec,tol,ctol", [("FP64", 1e-12, 1e-10), ("FP32", 1e-10, 1e-8)])
def test_diluted_pipeline_plain_workload(dl, prec, tol, ctol):
    # the 4^3 x 8 workload with two wall noises at t' = 3: GPU modes, diluted
    # sources, 4N + 96 solves and contractions against the oracle with LU solves
    wl = synth.WORKLOADS["plain_4c8"]
    U, _ = synth.workload_inputs(wl)
    tp, nn = 3, 2
    eta = synth.wall_noise(nn, wl.vol_s, synth.NOISE_SEED_BASE + 100 + wl.cfg)
    ctx = dl.Context(wl.L, wl.T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(wl.m0, wl.csw)
    ctx.dlma_laplacian_eigs(-1, wl.n_modes, 1e-13, want_vecs=False)
    res = ctx.dlma_correlators_diluted(tp, wl.n_modes, eta, tol, getattr(dl, prec))
    assert len(res["info"]) == 4 * wl.n_modes + 48 * nn
    assert all(i["converged"] and i["true_resid"] <= tol for i in res["info"])
    eo = dirac.EvenOdd(U, wl.L, wl.T, wl.m0, wl.csw)
    V_all = np.stack([lap.lap_modes(lap.timeslice_links(U, wl.L, t), wl.L, wl.n_modes)[1] for t in range(wl.T)])
    ref = dilution.diluted_correlators(solve.lu_solver(eo), V_all, eta, wl.L, wl.T, tp)
    scale = np.abs(ref["C"]).max(axis=1)
    ref["C_mixed_src"] = dlma.mixed_src(V_all, ref["phi_dist"], wl.L, wl.T)
    for key in ("C_dist", "C_rest", "C_mixed", "C_mixed_src", "C"):
        err = np.abs(res[key] - ref[key]).max(axis=1) / scale
        assert np.all(err <= ctol), (key, err)
    assert np.all(res["C_dist"][0].real > 0)


def test_diluted_batches_with_memory_cap(dl):
    # a memory cap forces one noise vector (48 solves) per batch and a ragged
    # lattice (6^3 x 4: V/2 = 432); results equal the uncapped run
    L, T, N, nn = 6, 4, 4, 3
    U = synth.gauge_field(L, T, 0.2, 405)
    ctx = dl.Context(L, T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(1 / 0.24 - 4, 1.0)
    ctx.dlma_laplacian_eigs(-1, N, 1e-10, want_vecs=False)
    eta = synth.wall_noise(nn, L ** 3, 406)
    full = ctx.dlma_correlators_diluted(1, N, eta, 1e-11, dl.FP64)
    V, Vh = L ** 3 * T, L ** 3 * T // 2
    per_rhs = V * 12 * 16 * 2 + Vh * 12 * 16 * 7 + Vh * 6 * 16 * 8
    ctx.dlma_set_memory_cap(int(50 * per_rhs))
    capped = ctx.dlma_correlators_diluted(1, N, eta, 1e-11, dl.FP64)
    assert all(i["converged"] for i in capped["info"])
    for key in ("C_dist", "C_rest", "C_mixed"):
        assert np.abs(capped[key] - full[key]).max() <= 1e-9 * np.abs(full["C"]).max()
