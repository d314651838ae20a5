"""Pins of the oracle's correlator contractions against what the mathematics
fixes independently of them (no GPU):

* free field: the exact correlator of every channel (PS, V1, V2, V3) equals the
  closed form built from the momentum-space propagator, evaluated at x and at
  -x (no gamma_5-hermiticity, no adjoint used), for periodic and antiperiodic
  time;
* a random gauge transformation leaves every exact part of Eq. 2 and the
  perambulator's C_dist unchanged (modes recomputed from the transformed
  field, so the projector is compared through the physics, not through V);
* the source-side mixed term from the distillation solutions equals the exact
  (dense propagator) one;
* the plain estimator (no distillation) is unbiased for the exact correlator,
  and with complete dilution it is exact; dropping its vector-channel solve is
  caught;
* with a projector on Dirac low modes (conventional LMA) the mixed propagator
  block vanishes to rounding, with the Laplacian projector it does not.
"""
import numpy as np
import pytest

import synth
from oracle import dilution, dirac, dlma
from oracle import gamma as g
from oracle import laplacian as lap
from oracle import lattice as lat
from oracle import solve


def _modes(U, L, T, n):
    return np.stack([lap.lap_modes(lap.timeslice_links(U, L, t), L, n)[1] for t in range(T)])


def _exact(U, L, T, m0, csw, n_modes, tp=0, bc_t=0):
    eo = dirac.EvenOdd(U, L, T, m0, csw, bc_t)
    lu = solve.lu_solver(eo)
    S = lu(dlma.point_sources(L, T, tp).reshape(-1, L ** 3 * T, 4, 3)).reshape(L ** 3, 4, 3, L ** 3 * T, 4, 3)
    V_all = _modes(U, L, T, n_modes)
    return eo, lu, S, V_all


def _free_propagator(L, T, m0, bc_t, sign):
    """S0(sign * x) [T, L, L, L, 4, 4] (index t, z, y, x) from the closed form
    S(p) = [M - i sum gamma sin p] / [M^2 + sum sin^2 p], M = m0 + sum (1 - cos p),
    p_t = (2 n + bc_t) pi / T: S0(s x) = 1/V sum_p e^{i p x} S(s p)."""
    kt, kz, ky, kx = np.meshgrid(np.arange(T), np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    p = [(2 * np.pi * kt + np.pi * bc_t) / T, 2 * np.pi * kx / L, 2 * np.pi * ky / L, 2 * np.pi * kz / L]
    M = m0 + sum(1 - np.cos(pm) for pm in p)
    den = M ** 2 + sum(np.sin(pm) ** 2 for pm in p)
    num = M[..., None, None] * np.eye(4) - 1j * sign * sum(np.sin(p[mu])[..., None, None] * g.GAMMA[mu]
                                                            for mu in range(4))
    Sp = num / den[..., None, None]
    Sx = np.fft.ifftn(Sp, axes=(0, 1, 2, 3))
    t = np.arange(T)
    return Sx * np.exp(1j * np.pi * bc_t * t / T)[:, None, None, None, None, None]


@pytest.mark.parametrize("bc_t", [0, 1])
def test_free_field_correlators_closed_form(bc_t):
    L, T, m0 = 4, 6, 0.3
    U = synth.unit_gauge(L, T)
    _, _, S, V_all = _exact(U, L, T, m0, 1.0, 3, bc_t=bc_t)
    ex = dlma.exact_parts(S, V_all, L, T, 0)
    Sp = _free_propagator(L, T, m0, bc_t, +1)       # S0(x), x relative to the source
    Sm = _free_propagator(L, T, m0, bc_t, -1)       # S0(-x)
    for ch, G in enumerate(g.CHANNELS):
        # C(t) = sum_{x in t, y in t'} tr[G S(x, y) G S(y, x)], S(x, y) = S0(x - y) (x) 1_colour:
        # translation invariance gives L^3 identical source sites, the colour trace a factor 3
        want = 3 * L ** 3 * np.einsum("ab,tzyxbc,cd,tzyxda->t", G, Sp, G, Sm)
        assert np.abs(ex["full"][ch] - want).max() < 1e-12 * np.abs(want).max(), ch
    # pseudoscalar: sum |S|^2 > 0; the free correlators are real
    assert np.all(ex["full"][0].real > 0)
    assert np.abs(ex["full"].imag).max() < 1e-12 * np.abs(ex["full"]).max()


def test_gauge_invariance_of_exact_parts_and_cdist():
    L, T, m0, csw = 4, 4, 1.0 / (2 * 0.12) - 4.0, 1.0
    U = synth.gauge_field(L, T, 0.25, 71)
    G = synth.random_su3(L ** 3 * T, 72)
    fwd, _ = lat.neighbours(L, T)
    UG = np.stack([G @ U[:, mu] @ np.conj(np.swapaxes(G[fwd[mu]], -1, -2)) for mu in range(4)], axis=1)
    tp = 1
    _, lu, S, V_all = _exact(U, L, T, m0, csw, 5, tp=tp)
    _, luG, SG, VG = _exact(UG, L, T, m0, csw, 5, tp=tp)
    ex, exG = dlma.exact_parts(S, V_all, L, T, tp), dlma.exact_parts(SG, VG, L, T, tp)
    scale = np.abs(ex["full"]).max()
    for key in ("full", "rest", "mixed_snk", "mixed_src", "dist"):
        assert np.abs(ex[key] - exG[key]).max() < 1e-11 * scale, key
    # the estimator's C_dist and, with the transformed noise, its rest / mixed parts
    eta = synth.z2z2_noise(2, L ** 3, 73)
    Gt = G[tp * L ** 3:(tp + 1) * L ** 3]
    etaG = np.einsum("mab,rmsb->rmsa", Gt, eta)
    r = dlma.dlma_correlators(lu, V_all, eta, L, T, tp)
    rG = dlma.dlma_correlators(luG, VG, etaG, L, T, tp)
    for key in ("C_dist", "C_rest", "C_mixed"):
        assert np.abs(r[key] - rG[key]).max() < 1e-11 * scale, key


def test_mixed_src_from_distillation_solutions_is_exact():
    L, T = 4, 4
    U = synth.gauge_field(L, T, 0.2, 74)
    _, lu, S, V_all = _exact(U, L, T, 1.0 / (2 * 0.12) - 4.0, 1.0, 4, tp=2)
    ex = dlma.exact_parts(S, V_all, L, T, 2)
    phid = lu(dlma.distillation_sources(V_all[2], L, T, 2))
    got = dlma.mixed_src(V_all, phid, L, T)
    scale = np.abs(ex["full"]).max(axis=1, keepdims=True)
    assert np.all(np.abs(got - ex["mixed_src"]) < 1e-12 * scale)
    # the source-side and sink-side mixed terms differ on one configuration (the
    # paper merges them by time reversal, which holds on average only)
    assert np.abs(ex["mixed_src"] - ex["mixed_snk"]).max() > 1e-6 * np.abs(ex["mixed_snk"]).max()


def test_plain_estimator_unbiased_and_planted_mistake():
    L, T = 2, 4
    U = synth.gauge_field(L, T, 0.4, 75)
    _, lu, S, V_all = _exact(U, L, T, 1.0 / (2 * 0.12) - 4.0, 1.0, 3)
    ex = dlma.exact_parts(S, V_all, L, T, 0)
    n = 4000
    eta = synth.z2z2_noise(n, L ** 3, 76)
    b = dlma.plain_sources(eta, L, T, 0)
    x = lu(b.reshape(n * 4, L ** 3 * T, 4, 3)).reshape(n, 4, L ** 3 * T, 4, 3)
    good, bad = [], []
    for i in range(0, n, 200):
        sl = slice(i, i + 200)
        good.append(dlma.plain_estimator(x[sl, 0], x[sl, 1:4], L, T))
        # planted mistake: the vector channel's left vector taken as phi instead of D^-1 g5 g_k eta
        bad.append(dlma.plain_estimator(x[sl, 0], np.repeat(x[sl, 0:1], 3, axis=1), L, T))
    for samples, ok in ((good, True), (bad, False)):
        s = np.array(samples)
        mean, err = s.mean(axis=0), s.std(axis=0, ddof=1) / np.sqrt(s.shape[0])
        dev = np.abs(mean - ex["full"])
        if ok:
            assert np.all(dev <= 4.5 * np.abs(err) + 1e-12), (dev / err).max()
        else:
            assert np.any(dev[1:] > 10 * np.abs(err[1:]) + 1e-12)


def test_plain_diluted_with_complete_dilution_is_exact():
    # one "noise vector" whose pieces are every unit vector (site, colour) of t':
    # sum_d eta_d eta_d^dag = 1 exactly, so the estimator is the exact correlator
    L, T, tp = 2, 4, 1
    U = synth.gauge_field(L, T, 0.3, 77)
    _, _, S, V_all = _exact(U, L, T, 1.0 / (2 * 0.12) - 4.0, 1.0, 3, tp=tp)
    ex = dlma.exact_parts(S, V_all, L, T, tp)
    Vs = L ** 3
    # phi_{d = (m, c), beta} = D^-1 (e_{m, c} (x) e_beta) = S[m, beta, c]
    phi = np.transpose(S, (0, 2, 1, 3, 4, 5)).reshape(1, Vs * 3, 4, L ** 3 * T, 4, 3)
    got = dilution.plain_diluted(phi, L, T)
    assert np.abs(got - ex["full"]).max() < 1e-12 * np.abs(ex["full"]).max()


def test_dirac_low_modes_make_the_mixed_block_vanish():
    # Sec. 1 / after Eq. 2: with Box built from Dirac eigenmodes, Box and the propagator
    # commute and C_mixed = 0.  Qhat = g5 Dhat is hermitian; P from its n smallest |lambda|
    # gives P Dhat^-1 (1 - g5 P g5) = 0 to rounding, the Laplacian Box does not.
    from oracle import lma
    L, T = 2, 4
    U = synth.gauge_field(L, T, 0.3, 78)
    eo = dirac.EvenOdd(U, L, T, 1.0 / (2 * 0.12) - 4.0, 1.0)
    Dh = lma.schur_matrix(eo)
    # the dense Schur matrix is the oracle's own stencil
    v = synth.gaussian_spinors(1, L ** 3 * T // 2, 79)[0]
    assert np.abs(Dh @ v.ravel() - eo.schur(v).ravel()).max() < 1e-12
    lam, u = lma.dirac_low_modes(eo, 6)
    for i in range(6):
        qu = dirac.apply_gamma5(eo.schur(u[i]))
        assert np.linalg.norm(qu - lam[i] * u[i]) < 1e-11
    Dinv = np.linalg.inv(Dh)
    n = Dh.shape[0]
    Uc = u.reshape(6, n).T
    P = Uc @ np.conj(Uc.T)
    G5 = lma.gamma5_matrix(n // 12)
    mixed = P @ Dinv @ (np.eye(n) - G5 @ P @ G5)
    assert np.abs(mixed).max() < 1e-12 * np.abs(Dinv).max()
    # the Laplacian projector on the even sites of a timeslice does not commute
    V_all = _modes(U, L, T, 2)
    t = 1
    even = eo.even
    # Box restricted to the even sites of timeslice t, written out
    Vt = V_all[t]
    idx = [i for i, s in enumerate(even) if s // L ** 3 == t]
    m_of = {i: even[i] % L ** 3 for i in idx}
    Bx = np.zeros((n, n), dtype=np.complex128)
    for i in idx:
        for j in idx:
            blk = np.einsum("kc,kd->cd", Vt[:, m_of[i], :], np.conj(Vt[:, m_of[j], :]))
            for a in range(4):
                Bx[12 * i + 3 * a:12 * i + 3 * a + 3, 12 * j + 3 * a:12 * j + 3 * a + 3] = blk
    mixed_lap = Bx @ Dinv @ (np.eye(n) - Bx)
    assert np.abs(mixed_lap).max() > 1e-3 * np.abs(Dinv).max()
    # the projector helper of the oracle applies the same P (and g5 P g5)
    w = synth.gaussian_spinors(1, n // 12, 80)[0]
    assert np.abs(lma.project(u, w).ravel() - P @ w.ravel()).max() < 1e-13
    assert np.abs(lma.project(u, w, True).ravel() - G5 @ P @ G5 @ w.ravel()).max() < 1e-13
