"""Failure detection through status codes, with failures made on the host:
a NaN link, a singular clover block, an unreachable tolerance, calls out of
order and bad arguments.  No test faults, traps or hangs the GPU: every wait
in the library is bounded and every failure is a returned status."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_09729_gb300 as dl
    return dl


def test_nonfinite_gauge_rejected(dl):
    L, T = 4, 4
    U = synth.gauge_field(L, T, 0.2, 501)
    U[17, 2, 1, 0] = np.nan
    ctx = dl.Context(L, T, 0, 0)
    with pytest.raises(dl.DlmaError) as e:
        ctx.dlma_set_gauge(U)
    assert e.value.status == 3                       # DLMA_ERR_NONFINITE
    with pytest.raises(dl.DlmaError) as e:           # no field: later calls report STATE
        ctx.dlma_set_params(0.1, 1.0)
    assert e.value.status == 8


def test_singular_clover_rejected(dl):
    # m0 = -4, c_sw = 0 on the unit gauge: every clover block is exactly zero
    L, T = 4, 4
    ctx = dl.Context(L, T, 0, 0)
    ctx.dlma_set_gauge(synth.unit_gauge(L, T))
    with pytest.raises(dl.DlmaError) as e:
        ctx.dlma_set_params(-4.0, 0.0)
    assert e.value.status == 4                       # DLMA_ERR_SINGULAR
    b = synth.gaussian_spinors(1, L ** 3 * T, 502)
    with pytest.raises(dl.DlmaError) as e:           # the failed parameters are not used
        ctx.dlma_solve(b, 1e-8)
    assert e.value.status == 8


def test_unreachable_tolerance_returns_best_iterate(dl):
    L, T = 4, 4
    U = synth.gauge_field(L, T, 0.2, 503)
    ctx = dl.Context(L, T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(0.1, 1.0)
    b = synth.gaussian_spinors(2, L ** 3 * T, 504)
    x, info = ctx.dlma_solve(b, 1e-30, dl.FP64, allow_not_converged=True)
    assert not any(i["converged"] for i in info)
    assert all(i["true_resid"] < 1e-12 for i in info)   # the best iterate is still returned
    with pytest.raises(dl.DlmaError) as e:
        ctx.dlma_solve(b, 1e-30, dl.FP64)
    assert e.value.status == 2                       # DLMA_ERR_NOT_CONVERGED


def test_bad_arguments(dl):
    L, T = 4, 4
    ctx = dl.Context(L, T, 0, 0)
    b = synth.gaussian_spinors(1, L ** 3 * T, 505)
    with pytest.raises(dl.DlmaError) as e:           # solve before the gauge field
        ctx.dlma_solve(b, 1e-8)
    assert e.value.status == 8
    ctx.dlma_set_gauge(synth.gauge_field(L, T, 0.2, 506))
    ctx.dlma_set_params(0.1, 1.0)
    with pytest.raises(dl.DlmaError) as e:
        ctx.dlma_solve(b, -1.0)
    assert e.value.status == 1
    with pytest.raises(dl.DlmaError) as e:           # modes not computed for this N
        ctx.dlma_correlators(0, 3, synth.z2z2_noise(1, L ** 3, 507), 1e-8)
    assert e.value.status == 8
    with pytest.raises(dl.DlmaError) as e:
        ctx.dlma_laplacian_eigs(-1, 10 ** 6, 1e-10)
    assert e.value.status == 1
