"""Pins of the oracle CGNE solve and Laplacian eigensolve (no GPU)."""
import numpy as np
import pytest

import synth
from oracle import dirac
from oracle import gamma as g
from oracle import laplacian as lap
from oracle import lattice as lat
from oracle import solve


def test_cgne_matches_lu_plain_workload():
    wl = synth.WORKLOADS["plain_4c8"]
    U, _ = synth.workload_inputs(wl)
    eo = dirac.EvenOdd(U, wl.L, wl.T, wl.m0, wl.csw)
    b = synth.gaussian_spinors(2, wl.volume, 21)
    lu = solve.lu_solver(eo)
    xl = lu(b)
    for i in range(2):
        x, it, res = solve.cgne(eo, b[i], tol=1e-12)
        assert res <= 1e-12
        assert np.linalg.norm(x - xl[i]) / np.linalg.norm(xl[i]) < 1e-10


def test_free_propagator_fft_closed_form():
    # free S(p) = [M - i sum gamma sin p] / [M^2 + sum sin^2 p], M = m0 + sum(1 - cos p)
    L, T, m0 = 4, 8, 0.2
    U = synth.unit_gauge(L, T)
    eo = dirac.EvenOdd(U, L, T, m0, 1.0)
    beta, col = 1, 2
    b = np.zeros((L ** 3 * T, 4, 3), dtype=np.complex128)
    b[0, beta, col] = 1.0
    x, _, res = solve.cgne(eo, b, tol=1e-13)
    # momentum grid in lexicographic (t, z, y, x) order
    kt, kz, ky, kx = np.meshgrid(np.arange(T), np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    p = [2 * np.pi * kt / T, 2 * np.pi * kx / L, 2 * np.pi * ky / L, 2 * np.pi * kz / L]
    M = m0 + sum(1 - np.cos(pm) for pm in p)
    den = M ** 2 + sum(np.sin(pm) ** 2 for pm in p)
    Sp = (M[..., None, None] * np.eye(4) - 1j * sum(np.sin(p[mu])[..., None, None] * g.GAMMA[mu] for mu in range(4))) / den[..., None, None]
    Sx = np.fft.ifftn(Sp[..., :, beta], axes=(0, 1, 2, 3)).reshape(L ** 3 * T, 4)
    want = np.zeros_like(x)
    want[:, :, col] = Sx
    assert res <= 1e-13
    assert np.abs(x - want).max() < 1e-11


@pytest.mark.parametrize("L", [4, 6])
def test_free_laplacian_spectrum(L):
    # eigenvalues of -lap are 6 - 2 sum_j cos p_j, each 3-fold in colour
    U = synth.unit_gauge(L, 1)
    Ut = lap.timeslice_links(U, L, 0)
    w = np.linalg.eigvalsh(-lap.lap_dense(Ut, L))
    k = 2 * np.pi * np.arange(L) / L
    want = np.sort(np.repeat((6 - 2 * (np.cos(k)[:, None, None] + np.cos(k)[None, :, None]
                                        + np.cos(k)[None, None, :])).ravel(), 3))
    assert np.allclose(w, want, atol=1e-12)


def test_laplacian_hermitian_nonneg_and_covariant():
    L = 4
    U = synth.gauge_field(L, 2, 0.3, 31)
    Ut = lap.timeslice_links(U, L, 1)
    A = -lap.lap_dense(Ut, L)
    assert np.abs(A - np.conj(A.T)).max() < 1e-14
    w = np.linalg.eigvalsh(A)
    assert w.min() > -1e-12 and w.max() < 12 + 1e-12
    # gauge covariance on the timeslice: U_j^G(m) = G(m) U_j(m) G(m+j)^dag
    G = synth.random_su3(L ** 3, 32)
    fwd, _ = lat.spatial_neighbours(L)
    UtG = np.stack([G @ Ut[j] @ np.conj(np.swapaxes(G[fwd[j]], -1, -2)) for j in range(3)])
    wG = np.linalg.eigvalsh(-lap.lap_dense(UtG, L))
    assert np.allclose(w, wG, atol=1e-12)
    v = (np.random.default_rng(0).standard_normal((L ** 3, 3)) + 0j)
    lhs = lap.lap_apply(UtG, L, np.einsum("mab,mb->ma", G, v))
    rhs = np.einsum("mab,mb->ma", G, lap.lap_apply(Ut, L, v))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_lanczos_matches_dense_and_projector_phase_free():
    L = 6
    U = synth.gauge_field(L, 1, 0.2, 33)
    Ut = lap.timeslice_links(U, L, 0)
    n = 12
    w_d, Vd = lap.lap_modes(Ut, L, n, dense_limit=10 ** 9)
    w_l, Vl = lap.lap_modes(Ut, L, n, dense_limit=0)
    assert np.allclose(w_d, w_l, rtol=1e-10, atol=1e-12)
    Pd = np.einsum("kmc,knd->mcnd", Vd, np.conj(Vd))
    Pl = np.einsum("kmc,knd->mcnd", Vl, np.conj(Vl))
    assert np.linalg.norm((Pd - Pl).ravel()) < 1e-8
    # residuals of the returned pairs
    for k in range(n):
        r = -lap.lap_apply(Ut, L, Vd[k]) - w_d[k] * Vd[k]
        assert np.linalg.norm(r) < 1e-11
