"""Conventional low-mode averaging with Dirac low modes on the GPU (the control
of Sec. 1 and the remark after Eq. 2): the library's low modes of
Qhat = g5 Dhat against the oracle's dense eigendecomposition, and the mixed
propagator block P Dhat^-1 (1 - g5 P g5), computed with the library's own
solver and projector, vanishing to the solver tolerance -- while the same
block with the Laplacian projector of Eq. 1 does not."""
import numpy as np
import pytest

import synth
from oracle import dirac, lma

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_09729_gb300 as dl
    return dl


def test_dirac_low_modes_vs_oracle_and_vanishing_mixed_block(dl):
    L, T, N = 4, 4, 8
    m0, csw = 1.0 / (2 * 0.12) - 4.0, 1.0
    U = synth.gauge_field(L, T, 0.2, 801)
    ctx = dl.Context(L, T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(m0, csw)
    lam, u = ctx.dlma_dirac_eigs(N, 1e-10)
    eo = dirac.EvenOdd(U, L, T, m0, csw)
    wl, ul = lma.dirac_low_modes(eo, N + 1)
    assert abs(wl[N]) - abs(wl[N - 1]) > 1e-6          # the cut is not degenerate
    assert np.all(np.abs(lam - wl[:N]) <= 1e-9 * np.maximum(1.0, np.abs(wl[:N])))
    n = L ** 3 * T // 2 * 12
    Pg = u.reshape(N, n).T @ np.conj(u.reshape(N, n))
    Po = ul[:N].reshape(N, n).T @ np.conj(ul[:N].reshape(N, n))
    assert np.linalg.norm(Pg - Po) <= 1e-8
    for i in range(N):
        assert np.linalg.norm(dirac.apply_gamma5(eo.schur(u[i])) - lam[i] * u[i]) <= 1e-10 * max(1, abs(lam[i]))
    # the projector entry point
    Vh = L ** 3 * T // 2
    eta = synth.gaussian_spinors(3, Vh, 802)
    assert np.abs(ctx.dlma_dirac_project(eta) - lma.project(u, eta)).max() < 1e-12 * np.abs(eta).max()
    assert np.abs(ctx.dlma_dirac_project(eta, True) - lma.project(u, eta, True)).max() < 1e-12 * np.abs(eta).max()
    # mixed block: x = D^-1 (1 - g5 P g5) eta on the even sites (odd source 0, so x_e = Dhat^-1 y),
    # then P x_e = 0 to the solver's accuracy
    y = eta - ctx.dlma_dirac_project(eta, True)
    b = np.zeros((3, L ** 3 * T, 4, 3), dtype=np.complex128)
    b[:, eo.even] = y
    x, info = ctx.dlma_solve(b, 1e-12, dl.FP64)
    xe = np.ascontiguousarray(x[:, eo.even])
    mixed = ctx.dlma_dirac_project(xe)
    for r in range(3):
        assert np.linalg.norm(mixed[r]) <= 1e-10 * np.linalg.norm(xe[r])
    # the Laplacian projector of timeslice 0 (spin-diagonal, restricted to the even
    # sites there) leaves a mixed block of order one
    Vt = np.asarray(ctx.dlma_laplacian_eigs(0, 4, 1e-12)[1])
    sel = eo.even[eo.even < L ** 3]
    # the modes restricted to those sites, orthonormalised: a projector there, diagonal in spin
    W = np.linalg.qr(Vt[:, sel].reshape(4, -1).T)[0].T.reshape(4, len(sel), 3)

    def box(v):                              # the even sites of t = 0 come first in the compressed order
        out = np.zeros_like(v)
        c = np.einsum("kmc,rmac->rka", np.conj(W), v[:, :len(sel)])
        out[:, :len(sel)] = np.einsum("kmc,rka->rmac", W, c)
        return out
    assert np.all(eo.even[:len(sel)] == sel)
    yl = eta - box(eta)
    b[:] = 0
    b[:, eo.even] = yl
    xl, _ = ctx.dlma_solve(b, 1e-12, dl.FP64)
    ml = box(np.ascontiguousarray(xl[:, eo.even]))
    assert np.linalg.norm(ml[0]) > 1e-3 * np.linalg.norm(xl[0])
