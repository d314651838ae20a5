"""Pins of the oracle's diluted-wall-source estimator (Sec. 3: six colour x
even-odd diluted wall sources per noise, spin-explicit one-end insertion; no
GPU).  The solve-based contraction is checked against the trace of Eq. 3 with
the dilution outer product written out; the trace form against the exact
decomposition (full dilution is noise-free); the dilution outer product for its
structure and noise average."""
import numpy as np
import pytest

import synth
from oracle import dilution, dirac, dlma
from oracle import gamma as g
from oracle import laplacian as lap
from oracle import solve


@pytest.fixture(scope="module")
def small():
    L, T = 4, 4
    U = synth.gauge_field(L, T, 0.2, 61)
    eo = dirac.EvenOdd(U, L, T, 1.0 / (2 * 0.12) - 4.0, 1.0)
    V_all = np.stack([lap.lap_modes(lap.timeslice_links(U, L, t), L, 5)[1] for t in range(T)])
    lu = solve.lu_solver(eo)
    S = lu(dlma.point_sources(L, T, 1).reshape(-1, L ** 3 * T, 4, 3)).reshape(L ** 3, 4, 3, L ** 3 * T, 4, 3)
    return L, T, V_all, lu, S


def test_dilution_pieces_partition():
    L = 4
    eta = synth.wall_noise(2, L ** 3, 62)
    pieces = dilution.dilution_pieces(eta, L, 1)
    assert np.abs(pieces.sum(axis=1) - eta).max() == 0            # the six pieces add up to eta
    nz = np.abs(pieces) > 0
    assert np.all(nz.sum(axis=1) == 1)                               # and never overlap
    m = np.arange(L ** 3)
    par = (m % L + (m // L) % L + m // (L * L) + 1) % 2
    for c in range(3):
        for p in range(2):
            sel = nz[:, 2 * c + p]
            assert not sel[:, :, [k for k in range(3) if k != c]].any()
            assert not sel[:, par != p, :].any()


def test_outer_product_structure_and_noise_average():
    # one draw: unit diagonal, zero between different colours or parities (the
    # dilution removes those noise terms exactly); the average over draws -> 1
    L, n = 2, 3000
    eta = synth.wall_noise(n, L ** 3, 63)
    pieces = dilution.dilution_pieces(eta, L, 0)
    P1 = dilution.source_outer(pieces[0])
    assert np.abs(np.diag(P1) - 1).max() < 1e-15
    idx = np.arange(12 * L ** 3)
    m, c = idx // 12, idx % 3
    mm = np.arange(L ** 3)
    par = (mm % L + (mm // L) % L + mm // (L * L)) % 2
    diff = (c[:, None] != c[None, :]) | (par[m][:, None] != par[m][None, :])
    assert np.abs(P1[diff]).max() == 0
    Pm = sum(dilution.source_outer(pieces[r]) for r in range(n)) / n
    off = Pm - np.eye(12 * L ** 3)
    assert np.abs(off).max() < 5.0 / np.sqrt(n)


def test_full_dilution_is_exact(small):
    # with one piece per site and colour, sum_d eta_d eta_d^dag = 1 for unit-modulus
    # noise: the trace form reproduces the exact rest and mixed terms
    L, T, V_all, _, S = small
    Vs = L ** 3
    eta = synth.wall_noise(1, Vs, 64)
    pieces = np.zeros((1, 3 * Vs, Vs, 3), dtype=np.complex128)
    for m in range(Vs):
        for c in range(3):
            pieces[0, 3 * m + c, m, c] = eta[0, m, c]
    rest, mixed = dilution.diluted_trace(S, V_all, pieces, L, T, 1)
    ex = dlma.exact_parts(S, V_all, L, T, 1)
    scale = np.abs(ex["full"]).max(axis=1, keepdims=True)
    assert np.all(np.abs(rest - ex["rest"]) < 1e-12 * scale)
    assert np.all(np.abs(mixed - ex["mixed_snk"]) < 1e-12 * scale)


def test_spin_explicit_contraction_equals_trace(small):
    L, T, V_all, lu, S = small
    eta = synth.wall_noise(2, L ** 3, 65)
    r = dilution.diluted_correlators(lu, V_all, eta, L, T, 1)
    pieces = dilution.dilution_pieces(eta, L, 1)
    rest, mixed = dilution.diluted_trace(S, V_all, pieces, L, T, 1)
    scale = np.abs(r["C"]).max(axis=1, keepdims=True)
    assert np.all(np.abs(r["C_rest"] - rest) < 1e-12 * scale)
    assert np.all(np.abs(r["C_mixed"] - mixed) < 1e-12 * scale)
    # C_dist is the distillation part, unchanged by the noise treatment
    ex = dlma.exact_parts(S, V_all, L, T, 1)
    assert np.all(np.abs(r["C_dist"] - ex["dist"]) < 1e-12 * scale)


def test_planted_mistake_transposed_source_spin_matrix(small):
    # the source spin matrix B[beta, beta'] taken transposed must be caught by the
    # trace form for the vector channel (g_k g5 is not symmetric)
    L, T, V_all, lu, S = small
    eta = synth.wall_noise(1, L ** 3, 66)
    r = dilution.diluted_correlators(lu, V_all, eta, L, T, 1)
    phi, phibar = r["phi"], r["phibar"]
    ch, G = 2, g.CHANNELS[2]
    A, B = g.GAMMA5 @ G, G @ g.GAMMA5
    assert np.abs(B - B.T).max() > 0.5
    t = 2
    ph = dlma.timeslice(phi, L, t)
    pb = dlma.timeslice(phibar, L, t)
    Aph = np.einsum("st,rdbmtc->rdbmsc", A, ph - dlma.box(V_all[t], ph))
    W = np.einsum("rdqmsc,rdbmsc->rdqb", np.conj(pb), Aph)
    wrong = np.einsum("qb,rdqb->", B, W)
    pieces = dilution.dilution_pieces(eta, L, 1)
    rest, _ = dilution.diluted_trace(S, V_all, pieces, L, T, 1)
    assert abs(r["C_rest"][ch, t] - rest[ch, t]) < 1e-12 * abs(rest[ch, t])
    assert abs(wrong - rest[ch, t]) > 1e-6 * abs(rest[ch, t])
