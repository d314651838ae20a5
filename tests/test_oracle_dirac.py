"""Pins of the oracle Wilson-clover operator and its even-odd form against
closed forms, invariants and brute force (no GPU)."""
import numpy as np
import pytest

import synth
from oracle import dirac
from oracle import gamma as g
from oracle import lattice as lat
from oracle import solve


def _free_Dp(p, m0):
    """Free-field momentum-space operator m0 + sum(1 - cos p) + i sum gamma sin p."""
    return (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(g.GAMMA[mu] * np.sin(p[mu]) for mu in range(4))


@pytest.mark.parametrize("bc_t", [0, 1])
def test_free_plane_waves(bc_t):
    L, T, m0 = 4, 6, 0.13
    U = synth.unit_gauge(L, T)
    Tc = dirac.clover_field(U, L, T, m0, 1.7)
    c = lat.coords(L, T)
    rng = np.random.Generator(np.random.PCG64(5))
    for n in [(0, 0, 0, 0), (1, 2, 3, 1), (5, 1, 0, 3), (2, 3, 3, 2)]:
        nt = n[0] + (0.5 if bc_t else 0.0)
        p = 2 * np.pi * np.array([nt / T, n[1] / L, n[2] / L, n[3] / L])
        ph = np.exp(1j * (c @ p))
        s = rng.standard_normal(4) + 1j * rng.standard_normal(4)
        col = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        psi = ph[:, None, None] * s[None, :, None] * col[None, None, :]
        want = ph[:, None, None] * (_free_Dp(p, m0) @ s)[None, :, None] * col[None, None, :]
        got = dirac.apply_dw(U, Tc, psi, L, T, bc_t)
        assert np.abs(got - want).max() < 1e-13


def test_free_dense_spectrum_brute_force():
    # eigenvalues of the free D are m0 + sum(1-cos p) +- i sqrt(sum sin^2 p), each 6-fold (2 spin x 3 colour)
    L, T, m0 = 2, 4, 0.2
    U = synth.unit_gauge(L, T)
    Tc = dirac.clover_field(U, L, T, m0, 1.0)
    D = dirac.dirac_sparse(U, Tc, L, T).toarray()
    got = np.linalg.eigvals(D)
    want = []
    for nt in range(T):
        for nx in range(L):
            for ny in range(L):
                for nz in range(L):
                    p = 2 * np.pi * np.array([nt / T, nx / L, ny / L, nz / L])
                    re = m0 + np.sum(1 - np.cos(p))
                    im = np.sqrt(np.sum(np.sin(p) ** 2))
                    want += [re + 1j * im] * 6 + [re - 1j * im] * 6
    key = lambda z: (round(z.real, 9), round(z.imag, 9))
    assert np.allclose(sorted(got, key=key), sorted(want, key=key), atol=1e-10)


def test_gamma5_hermiticity_with_clover():
    L, T = 4, 4
    U = synth.gauge_field(L, T, 0.3, 99)
    eo = dirac.EvenOdd(U, L, T, 0.05, 1.5)
    u, v = synth.gaussian_spinors(2, L ** 3 * T, 3)
    lhs = np.vdot(u.ravel(), dirac.apply_gamma5(eo.apply_full(dirac.apply_gamma5(v))).ravel())
    rhs = np.vdot(eo.apply_full(u).ravel(), v.ravel())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # same for the Schur complement on even sites
    ue, ve = u[eo.even], v[eo.even]
    lhs = np.vdot(ue.ravel(), eo.schur_dag(ve).ravel())
    rhs = np.vdot(eo.schur(ue).ravel(), ve.ravel())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_clover_hermitian_commutes_gamma5_unit():
    L, T = 4, 4
    U = synth.gauge_field(L, T, 0.3, 4)
    Tc = dirac.clover_field(U, L, T, 0.1, 1.2)
    assert np.abs(Tc - np.conj(np.swapaxes(Tc, -1, -2))).max() < 1e-14
    G5 = np.kron(g.GAMMA5, np.eye(3))
    assert np.abs(Tc @ G5 - G5 @ Tc).max() < 1e-14
    T1 = dirac.clover_field(synth.unit_gauge(L, T), L, T, 0.1, 1.2)
    assert np.abs(T1 - 4.1 * np.eye(12)).max() < 1e-15


def _flux_field(L, T, n):
    """Constant abelian flux in the (x, y) plane: every (1,2) plaquette equals
    diag(e^{i th}, e^{i th}, e^{-2i th}), th = 2 pi n / L^2."""
    th = 2 * np.pi * n / L ** 2
    c = lat.coords(L, T)

    def emb(phi):
        return np.stack([np.exp(1j * phi), np.exp(1j * phi), np.exp(-2j * phi)], -1)

    U = synth.unit_gauge(L, T)
    U[:, 1] = 0
    d = emb(-th * c[:, 2])
    for a in range(3):
        U[:, 1, a, a] = d[:, a]
    mask = c[:, 2] == L - 1
    d2 = emb(th * L * c[:, 1])
    U[mask, 2] = 0
    for a in range(3):
        U[mask, 2, a, a] = d2[mask, a]
    return U, th


@pytest.mark.parametrize("n", [1, 3])
def test_clover_constant_flux_closed_form(n):
    L, T, m0, csw = 4, 4, 0.1, 1.3
    U, th = _flux_field(L, T, n)
    Tc = dirac.clover_field(U, L, T, m0, csw)
    want = (4 + m0) * np.eye(12) - 0.5 * csw * np.kron(
        g.sigma(1, 2), np.diag([np.sin(th), np.sin(th), -np.sin(2 * th)]))
    assert np.abs(Tc - want[None]).max() < 1e-14


def test_gauge_covariance():
    L, T = 4, 4
    U = synth.gauge_field(L, T, 0.3, 8)
    G = synth.random_su3(L ** 3 * T, 9)
    fwd, _ = lat.neighbours(L, T)
    UG = np.stack([G @ U[:, mu] @ np.conj(np.swapaxes(G[fwd[mu]], -1, -2)) for mu in range(4)], axis=1)
    Tc = dirac.clover_field(U, L, T, 0.1, 1.4)
    TcG = dirac.clover_field(UG, L, T, 0.1, 1.4)
    psi = synth.gaussian_spinors(1, L ** 3 * T, 10)[0]
    Gpsi = np.einsum("xab,xsb->xsa", G, psi)
    lhs = dirac.apply_dw(UG, TcG, Gpsi, L, T, 1)
    rhs = np.einsum("xab,xsb->xsa", G, dirac.apply_dw(U, Tc, psi, L, T, 1))
    assert np.abs(lhs - rhs).max() < 1e-12


def test_sparse_matrix_equals_stencil():
    L, T = 2, 4       # L = 2: forward and backward neighbours coincide
    U = synth.gauge_field(L, T, 0.4, 12)
    Tc = dirac.clover_field(U, L, T, 0.1, 1.0)
    psi = synth.gaussian_spinors(1, L ** 3 * T, 13)[0]
    for bc in (0, 1):
        D = dirac.dirac_sparse(U, Tc, L, T, bc)
        assert np.abs(D @ psi.ravel() - dirac.apply_dw(U, Tc, psi, L, T, bc).ravel()).max() < 1e-13


def test_even_odd_schur_reproduces_full_solve():
    L, T = 4, 4
    U = synth.gauge_field(L, T, 0.2, 14)
    eo = dirac.EvenOdd(U, L, T, 0.1, 1.0)
    b = synth.gaussian_spinors(1, L ** 3 * T, 15)
    x = solve.lu_solver(eo)(b)[0]
    xe = x[eo.even]
    assert np.abs(eo.schur(xe) - eo.prepare(b[0])).max() < 1e-12
    assert np.abs(eo.reconstruct(xe, b[0]) - x).max() < 1e-12
