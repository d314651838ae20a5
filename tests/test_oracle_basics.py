"""Pins of the oracle's conventions: Dirac matrices, index tables and the
synthetic-input generator.  Nothing here compares the oracle with itself."""
import numpy as np
import pytest

import synth
from oracle import gamma as g
from oracle import lattice as lat


def test_clifford_algebra():
    for mu in range(4):
        assert np.allclose(g.GAMMA[mu], np.conj(g.GAMMA[mu].T))
        for nu in range(4):
            anti = g.GAMMA[mu] @ g.GAMMA[nu] + g.GAMMA[nu] @ g.GAMMA[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4))


def test_gamma5_chiral_diagonal():
    # chiral basis: gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3 is diag(1, 1, -1, -1)
    assert np.allclose(g.GAMMA5, np.diag([1, 1, -1, -1]))
    for mu in range(4):
        assert np.allclose(g.GAMMA5 @ g.GAMMA[mu], -g.GAMMA[mu] @ g.GAMMA5)


def test_sigma_hermitian_block_diagonal():
    for mu in range(4):
        for nu in range(4):
            s = g.sigma(mu, nu)
            assert np.allclose(s, np.conj(s.T))
            assert np.allclose(s @ g.GAMMA5, g.GAMMA5 @ s)       # chirality blocks
            assert np.allclose(s, -g.sigma(nu, mu))


@pytest.mark.parametrize("L,T", [(2, 2), (4, 8), (6, 4)])
def test_index_tables(L, T):
    V = L ** 3 * T
    c = lat.coords(L, T)
    assert np.array_equal(lat.site_index(c, L, T), np.arange(V))
    fwd, bwd = lat.neighbours(L, T)
    for mu in range(4):
        assert np.array_equal(bwd[mu][fwd[mu]], np.arange(V))
        d = (lat.coords(L, T)[fwd[mu]] - c) % np.array([T, L, L, L])
        e = np.zeros(4, dtype=int)
        e[mu] = 1
        assert np.all(d == e)
    even, odd, eo = lat.eo_tables(L, T)
    assert even.shape[0] == odd.shape[0] == V // 2
    # with even L the compressed index is s // 2 within each parity
    assert np.array_equal(eo, np.arange(V) // 2)
    p = lat.parity(L, T)
    for mu in range(4):
        assert np.all(p[fwd[mu]] != p)


def test_spatial_neighbours_match_4d_tables():
    L, T = 4, 2
    fwd4, bwd4 = lat.neighbours(L, T)
    fwd3, bwd3 = lat.spatial_neighbours(L)
    for j in range(3):
        assert np.array_equal(fwd4[j + 1][: L ** 3], fwd3[j])
        assert np.array_equal(bwd4[j + 1][: L ** 3], bwd3[j])


def test_gauge_field_is_su3_and_small_eps():
    U = synth.gauge_field(4, 4, 0.2, 7)
    Ud = np.conj(np.swapaxes(U, -1, -2))
    assert np.abs(U @ Ud - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1.0).max() < 1e-13
    # small-eps expansion U = 1 + i eps H + O(eps^2), H = sum_a w_a lambda_a / 2
    eps = 1e-5
    U2 = synth.gauge_field(2, 2, eps, 7)
    H = (U2 - np.eye(3)) / (1j * eps)
    assert np.abs(H - np.conj(np.swapaxes(H, -1, -2))).max() < 1e-4
    assert np.abs(np.trace(H, axis1=-2, axis2=-1)).max() < 1e-4
    # deterministic in the seed
    assert np.array_equal(U, synth.gauge_field(4, 4, 0.2, 7))


def test_noise_values():
    eta = synth.z2z2_noise(3, 8, 11)
    assert eta.shape == (3, 8, 4, 3)
    assert np.allclose(np.abs(eta), 1.0)
    vals = np.unique(np.round(eta * np.sqrt(2.0), 12))
    assert set(vals.tolist()) <= {1 + 1j, 1 - 1j, -1 + 1j, -1 - 1j}


def test_random_su3():
    G = synth.random_su3(50, 3)
    assert np.abs(G @ np.conj(np.swapaxes(G, -1, -2)) - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(G) - 1.0).max() < 1e-13
