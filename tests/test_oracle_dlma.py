"""Pins of the oracle's distillation-LMA contractions (Eqs. 2-4) against the
exact (LU) propagator decomposition and the unbiasedness of the one-end
estimators (no GPU)."""
import numpy as np
import pytest

import synth
from oracle import dirac, dlma
from oracle import laplacian as lap
from oracle import solve


def _setup(L, T, eps, kappa, csw, n_modes, seed):
    U = synth.gauge_field(L, T, eps, seed)
    m0 = 1.0 / (2 * kappa) - 4.0
    eo = dirac.EvenOdd(U, L, T, m0, csw)
    V_all = np.stack([lap.lap_modes(lap.timeslice_links(U, L, t), L, n_modes)[1] for t in range(T)])
    lu = solve.lu_solver(eo)
    S = lu(dlma.point_sources(L, T, 0).reshape(-1, L ** 3 * T, 4, 3)).reshape(L ** 3, 4, 3, L ** 3 * T, 4, 3)
    return U, eo, V_all, lu, S


@pytest.fixture(scope="module")
def small():
    return _setup(4, 4, 0.2, 0.12, 1.0, 5, 41)


def test_projector_properties(small):
    _, _, V_all, _, _ = small
    Vt = V_all[2]
    psi = synth.gaussian_spinors(1, 64, 42)[0]
    b1 = dlma.box(Vt, psi)
    assert np.abs(dlma.box(Vt, b1) - b1).max() < 1e-13                 # idempotent
    chi = synth.gaussian_spinors(1, 64, 43)[0]
    assert abs(np.vdot(chi.ravel(), b1.ravel()) - np.vdot(dlma.box(Vt, chi).ravel(), psi.ravel())) < 1e-12
    ph = np.exp(1j * np.arange(Vt.shape[0]))[:, None, None]
    assert np.abs(dlma.box(Vt * ph, psi) - b1).max() < 1e-13           # phase free


def test_exact_decomposition_identity(small):
    _, _, V_all, _, S = small
    ex = dlma.exact_parts(S, V_all, 4, 4, 0)
    tot = ex["rest"] + ex["mixed_snk"] + ex["mixed_src"] + ex["dist"]
    assert np.abs(tot - ex["full"]).max() < 1e-12 * np.abs(ex["full"]).max()
    # exact pseudoscalar correlator = sum |S|^2 over the sink timeslice: real, positive
    for t in range(4):
        want = np.sum(np.abs(S[:, :, :, t * 64:(t + 1) * 64]) ** 2)
        assert abs(ex["full"][0, t] - want) < 1e-12 * want


def test_cdist_from_perambulator_equals_exact(small):
    _, _, V_all, lu, S = small
    ex = dlma.exact_parts(S, V_all, 4, 4, 0)
    eta = synth.z2z2_noise(2, 64, 44)
    r = dlma.dlma_correlators(lu, V_all, eta, 4, 4, 0)
    scale = np.abs(ex["full"]).max(axis=1, keepdims=True)
    assert np.all(np.abs(r["C_dist"] - ex["dist"]) < 1e-12 * scale)
    # Box at both ends commutes with the channel matrices: the PS C_dist is tr[tau tau^dag] >= 0
    assert np.all(r["C_dist"][0].real > 0) and np.abs(r["C_dist"][0].imag).max() < 1e-12 * scale[0]


def test_noise_estimators_unbiased():
    # the mean over many noises converges to the exact rest / mixed terms
    L, T = 2, 4
    _, _, V_all, lu, S = _setup(L, T, 0.4, 0.12, 1.0, 3, 45)
    ex = dlma.exact_parts(S, V_all, L, T, 0)
    n = 4000
    eta = synth.z2z2_noise(n, L ** 3, 46)
    bn = dlma.noise_sources(eta, V_all[0], L, T, 0)
    phin = lu(bn.reshape(n * 5, L ** 3 * T, 4, 3)).reshape(n, 5, L ** 3 * T, 4, 3)
    samples_r, samples_m = [], []
    for i in range(0, n, 200):
        sl = slice(i, i + 200)
        r, m = dlma.noise_parts(V_all, phin[sl, 0], phin[sl, 1], phin[sl, 2:5], L, T)
        samples_r.append(r)
        samples_m.append(m)
    for samples, exact in ((samples_r, ex["rest"]), (samples_m, ex["mixed_snk"])):
        s = np.array(samples)                               # [batches, 4, T]
        mean = s.mean(axis=0)
        err = s.std(axis=0, ddof=1) / np.sqrt(s.shape[0])
        dev = np.abs(mean - exact)
        assert np.all(dev <= 4.5 * np.abs(err) + 1e-12), (dev / err).max()


def test_planted_mistake_is_caught(small):
    # a dropped (1 - Box') on the source side makes the rest estimator biased:
    # the exact identity no longer closes; this guards the test above.
    _, _, V_all, lu, S = small
    ex = dlma.exact_parts(S, V_all, 4, 4, 0)
    eta = synth.z2z2_noise(400, 64, 47)
    bn = dlma.noise_sources(eta, V_all[0], 4, 4, 0)
    phin = lu(bn.reshape(-1, 256, 4, 3)).reshape(400, 5, 256, 4, 3)
    _, m_ok = dlma.noise_parts(V_all, phin[:, 0], phin[:, 1], phin[:, 2:5], 4, 4)
    _, m_bad = dlma.noise_parts(V_all, phin[:, 0], phin[:, 0], phin[:, 2:5], 4, 4)
    gap_ok = np.abs(m_ok[0] - ex["mixed_snk"][0]).max()
    gap_bad = np.abs(m_bad[0] - ex["mixed_snk"][0]).max()
    assert gap_bad > 3 * gap_ok


def test_ps_loss_adjoint_matches_finite_differences():
    # the oracle's adjoint gradients of L = sum_t w(t) Re C_PS(t) against central
    # differences of L itself (in m0 and along a random complex direction of eta)
    L_, T, N, nn, csw, m0 = 4, 4, 3, 2, 1.0, 0.12
    U = synth.gauge_field(L_, T, 0.2, 48)
    V_all = np.stack([lap.lap_modes(lap.timeslice_links(U, L_, t), L_, N)[1] for t in range(T)])
    eta = synth.z2z2_noise(nn, L_ ** 3, 49)
    w = synth.loss_weights(T, 50)

    def solvers(m):
        eo = dirac.EvenOdd(U, L_, T, m, csw)
        return solve.lu_solver(eo), solve.lu_solver_dag(eo)

    s, sd = solvers(m0)
    loss, dm0, deta = dlma.ps_loss_grads(s, sd, V_all, eta, w, L_, T, 0)
    h = 1e-4
    lp = dlma.ps_loss(solvers(m0 + h)[0], V_all, eta, w, L_, T, 0)[0]
    lm = dlma.ps_loss(solvers(m0 - h)[0], V_all, eta, w, L_, T, 0)[0]
    assert abs((lp - lm) / (2 * h) - dm0) < 1e-6 * abs(dm0)
    d = synth.gaussian_spinors(nn, L_ ** 3, 51)
    lp = dlma.ps_loss(s, V_all, eta + h * d, w, L_, T, 0)[0]
    lm = dlma.ps_loss(s, V_all, eta - h * d, w, L_, T, 0)[0]
    want = np.vdot(deta.ravel(), d.ravel()).real
    assert abs((lp - lm) / (2 * h) - want) < 1e-6 * abs(want)
