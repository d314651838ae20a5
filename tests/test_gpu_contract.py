"""GPU parity of the distillation sources, the V^dag psi projections, the
C_rest / C_mixed / C_dist contractions (Eqs. 2-4) and the whole per-source
pipeline against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import dirac, dlma
from oracle import laplacian as lap
from oracle import solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_09729_gb300 as dl
    return dl


def _setup(dl, L, T, eps, kappa, csw, N, nn, seed):
    U = synth.gauge_field(L, T, eps, seed)
    m0 = 1 / (2 * kappa) - 4
    ctx = dl.Context(L, T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(m0, csw)
    eo = dirac.EvenOdd(U, L, T, m0, csw)
    V_all = np.stack([lap.lap_modes(lap.timeslice_links(U, L, t), L, N)[1] for t in range(T)])
    eta = synth.z2z2_noise(nn, L ** 3, seed + 1)
    return ctx, eo, U, V_all, eta


def _close(got, want, scale, tol):
    return np.all(np.abs(got - want) <= tol * scale)


def test_sources_and_projection(dl):
    L, T, N, nn = 6, 4, 6, 3
    ctx, eo, U, V_all, eta = _setup(dl, L, T, 0.2, 0.12, 1.0, N, nn, 301)
    tp = 1
    b = ctx.dlma_make_sources(tp, np.ascontiguousarray(V_all[tp]), eta)
    want = np.concatenate([dlma.distillation_sources(V_all[tp], L, T, tp),
                           dlma.noise_sources(eta, V_all[tp], L, T, tp).reshape(5 * nn, L ** 3 * T, 4, 3)])
    assert np.abs(b - want).max() < 1e-14
    psi = synth.gaussian_spinors(5, L ** 3 * T, 302)
    c_all = ctx.dlma_project(-1, np.ascontiguousarray(V_all), psi)          # [5, T, 4, N]
    for t in range(T):
        w = dlma.coeffs(V_all[t], dlma.timeslice(psi, L, t))               # [5, k, alpha]
        assert np.abs(c_all[:, t] - np.transpose(w, (0, 2, 1))).max() < 1e-12
    c1 = ctx.dlma_project(2, np.ascontiguousarray(V_all[2]), psi)
    assert np.abs(c1[:, 0] - c_all[:, 2]).max() < 1e-13


def test_contract_vs_oracle(dl):
    L, T, N, nn = 4, 8, 5, 3
    ctx, eo, U, V_all, eta = _setup(dl, L, T, 0.2, 0.12, 1.0, N, nn, 303)
    lu = solve.lu_solver(eo)
    r = dlma.dlma_correlators(lu, V_all, eta, L, T, 0)
    phi = np.concatenate([r["phi_dist"], r["phi_noise"].reshape(5 * nn, L ** 3 * T, 4, 3)])
    got = ctx.dlma_contract(0, np.ascontiguousarray(V_all), np.ascontiguousarray(phi), nn)
    scale = np.abs(r["C"]).max(axis=1, keepdims=True)
    for key in ("C_dist", "C_rest", "C_mixed", "C"):
        assert _close(got[key], r[key], scale, 1e-12), key
    # the exact source-side mixed term from the distillation solutions
    assert _close(got["C_mixed_src"], dlma.mixed_src(V_all, r["phi_dist"], L, T), scale, 1e-12)


@pytest.mark.parametrize("prec,tol,ctol", [("FP64", 1e-12, 1e-10), ("FP32", 1e-10, 1e-8), ("FP16S", 1e-10, 1e-8)])
def test_pipeline_plain_workload(dl, prec, tol, ctol):
    # the 4^3 x 8 workload end to end: GPU modes, sources, solves, contractions
    wl = synth.WORKLOADS["plain_4c8"]
    U, eta = synth.workload_inputs(wl)
    ctx = dl.Context(wl.L, wl.T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(wl.m0, wl.csw)
    lam, _ = ctx.dlma_laplacian_eigs(-1, wl.n_modes, 1e-13, want_vecs=False)
    res = ctx.dlma_correlators(0, wl.n_modes, eta[0], tol, getattr(dl, prec))
    assert all(i["converged"] and i["true_resid"] <= tol for i in res["info"])
    assert len(res["info"]) == 4 * wl.n_modes + 5 * wl.n_noise
    eo = dirac.EvenOdd(U, wl.L, wl.T, wl.m0, wl.csw)
    V_all = np.stack([lap.lap_modes(lap.timeslice_links(U, wl.L, t), wl.L, wl.n_modes)[1] for t in range(wl.T)])
    ref = dlma.dlma_correlators(solve.lu_solver(eo), V_all, eta[0], wl.L, wl.T, 0)
    scale = np.abs(ref["C"]).max(axis=1, keepdims=True)
    ref["C_mixed_src"] = dlma.mixed_src(V_all, ref["phi_dist"], wl.L, wl.T)
    for key in ("C_dist", "C_rest", "C_mixed", "C_mixed_src", "C"):
        err = np.abs(res[key] - ref[key]).max(axis=1) / scale[:, 0]
        assert np.all(err <= ctol), (key, err)
    # pseudoscalar C_dist is tr[tau tau^dag]: real and positive
    assert np.all(res["C_dist"][0].real > 0)
    # the total is the library's own C_rest + 2 C_mixed + C_dist
    assert np.abs(res["C"] - (res["C_rest"] + 2 * res["C_mixed"] + res["C_dist"])).max() <= 1e-14 * scale.max()


def test_pipeline_ragged_batches_with_memory_cap(dl):
    # a memory cap forces several solve batches; results must equal the uncapped run
    L, T, N, nn = 6, 8, 6, 3
    U = synth.gauge_field(L, T, 0.2, 305)
    ctx = dl.Context(L, T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(1 / 0.24 - 4, 1.0)
    ctx.dlma_laplacian_eigs(-1, N, 1e-12, want_vecs=False)
    eta = synth.z2z2_noise(nn, L ** 3, 306)
    full = ctx.dlma_correlators(0, N, eta, 1e-11, dl.FP64)
    V = L ** 3 * T
    ctx.dlma_set_memory_cap(int(7 * V * 12 * 16 * 6))
    capped = ctx.dlma_correlators(0, N, eta, 1e-11, dl.FP64)
    for key in ("C_dist", "C_rest", "C_mixed", "C_mixed_src", "C"):
        assert np.abs(capped[key] - full[key]).max() <= 1e-9 * np.abs(full["C"]).max()


@pytest.mark.parametrize("prec,tol,ctol", [("FP64", 1e-12, 1e-10), ("FP32", 1e-10, 1e-8)])
def test_plain_estimator_vs_oracle(dl, prec, tol, ctol):
    # the plain stochastic estimator (no distillation, the comparison of Fig. 1):
    # undiluted noise (4 solves per noise vector) and diluted wall sources (24 per
    # noise vector) against the oracle with LU solves on the 4^3 x 8 workload
    from oracle import dilution
    wl = synth.WORKLOADS["plain_4c8"]
    U, eta = synth.workload_inputs(wl)
    ctx = dl.Context(wl.L, wl.T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(wl.m0, wl.csw)
    eo = dirac.EvenOdd(U, wl.L, wl.T, wl.m0, wl.csw)
    lu = solve.lu_solver(eo)
    tp = 2
    res = ctx.dlma_correlators_plain(tp, eta[0], tol, getattr(dl, prec))
    assert len(res["info"]) == 4 * wl.n_noise and all(i["converged"] for i in res["info"])
    nn = wl.n_noise
    x = lu(dlma.plain_sources(eta[0], wl.L, wl.T, tp).reshape(4 * nn, wl.volume, 4, 3)).reshape(nn, 4, wl.volume, 4, 3)
    want = dlma.plain_estimator(x[:, 0], x[:, 1:4], wl.L, wl.T)
    err = np.abs(res["C"] - want).max(axis=1) / np.abs(want).max(axis=1)
    assert np.all(err <= ctol), err
    ew = synth.wall_noise(2, wl.vol_s, synth.NOISE_SEED_BASE + 200 + wl.cfg)
    rd = ctx.dlma_correlators_plain(tp, ew, tol, getattr(dl, prec))
    assert len(rd["info"]) == 48
    want_d, _ = dilution.plain_diluted_correlators(lu, ew, wl.L, wl.T, tp)
    err = np.abs(rd["C"] - want_d).max(axis=1) / np.abs(want_d).max(axis=1)
    assert np.all(err <= ctol), err


@pytest.mark.parametrize("L,T,N,nrhs", [(6, 4, 6, 5), (8, 4, 40, 37)])
def test_tensor_core_projection_vs_fp64_and_oracle(dl, monkeypatch, L, T, N, nrhs):
    # the split-precision tensor-core projection (default) and the FP64 CUDA-core
    # kernel agree with the oracle to 1e-12 of the largest coefficient; magnitudes
    # spread over five decades along the contraction, a mode count above one
    # 32-mode block (N = 40) and a ragged row count (4 x 37 rows = 1.16 tiles of 128)
    U = synth.gauge_field(L, T, 0.2, 311)
    ctx = dl.Context(L, T, 0, 0)
    ctx.dlma_set_gauge(U)
    V_all = np.stack([lap.lap_modes(lap.timeslice_links(U, L, t), L, N)[1] for t in range(T)])
    psi = synth.gaussian_spinors(nrhs, L ** 3 * T, 312)
    psi[:, ::7] *= 1e-5
    got_tc = ctx.dlma_project(-1, np.ascontiguousarray(V_all), psi)
    monkeypatch.setenv("DLMA_PROJECT_FP64", "1")
    got_64 = ctx.dlma_project(-1, np.ascontiguousarray(V_all), psi)
    for t in range(T):
        w = np.transpose(dlma.coeffs(V_all[t], dlma.timeslice(psi, L, t)), (0, 2, 1))
        scale = np.abs(w).max()
        assert np.abs(got_tc[:, t] - w).max() <= 1e-12 * scale, (t, np.abs(got_tc[:, t] - w).max() / scale)
        assert np.abs(got_64[:, t] - w).max() <= 1e-12 * scale
