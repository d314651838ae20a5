"""The double-float Gram matrices and rotations of the Laplacian eigensolver's
FP64 phase, against the FP64 arithmetic of the same call (DLMA_DF_EIGS=0 at
context creation) and against the oracle."""
import numpy as np
import pytest

import synth
from oracle import laplacian as lap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_09729_gb300 as dl
    return dl


def test_eigs_df_phase_against_fp64(dl, monkeypatch):
    # 8^3 x 4, N = 16 at tol 1e-10 (double-float phase B) and the same call with
    # FP64 arithmetic: eigenvalues against the dense oracle and each other,
    # residuals by the oracle's Laplacian
    L, T, N = 8, 4, 16
    U = synth.gauge_field(L, T, 0.2, 613)
    res = {}
    for flag in ("1", "tc", "0"):
        monkeypatch.setenv("DLMA_DF_EIGS", "0" if flag == "0" else "1")
        monkeypatch.setenv("DLMA_EIGS_TC", "1" if flag == "tc" else "0")
        ctx = dl.Context(L, T, 0, 0)
        ctx.dlma_set_gauge(U)
        lam, V = ctx.dlma_laplacian_eigs(-1, N, 1e-10)
        res[flag] = lam.reshape(T, N)
        V = V.reshape(T, N, L ** 3, 3)
        for t in range(T):
            Ut = lap.timeslice_links(U, L, t)
            w, _ = lap.lap_modes(Ut, L, N)
            assert np.all(np.abs(res[flag][t] - w[:N]) <= 1e-9 * np.maximum(np.abs(w[:N]), 1.0))
            for k in (0, N // 2, N - 1):
                r = -lap.lap_apply(Ut, L, V[t, k]) - res[flag][t, k] * V[t, k]
                assert np.linalg.norm(r) <= 1e-10 * max(1.0, res[flag][t, k]), (flag, t, k)
            gram = np.einsum("kmc,lmc->kl", np.conj(V[t]), V[t])
            assert np.abs(gram - np.eye(N)).max() < 1e-11
        ctx.close()
    assert np.abs(res["1"] - res["0"]).max() <= 1e-10 * np.abs(res["0"]).max()
    assert np.abs(res["tc"] - res["0"]).max() <= 1e-10 * np.abs(res["0"]).max()
