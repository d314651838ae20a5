"""The GPU sweep of the cost model (Eqs. 6-9) over the number of modes: the
measured break-even R0 exceeds the bound 2 R1 + N of Eq. 7 by the Laplacian's
share, and every quantity is consistent with its definition."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_sweep_small_lattice():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_09729_gb300 as dl
    from paper_2201_09729_gb300 import costmodel as cm
    L, T, nn = 6, 8, 2
    U = synth.gauge_field(L, T, 0.2, 505)
    ctx = dl.Context(L, T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(1 / 0.24 - 4, 1.0)
    eta = synth.z2z2_noise(nn, L ** 3, 506)
    rows = cm.sweep(ctx, 0, [4, 8], eta, 1e-10, dl.FP32)
    for row in rows:
        assert row["converged"]
        assert row["t_lap_s"] > 0 and row["t_solve_s"] > 0
        assert row["R0"] == pytest.approx(2 * row["R1"] + row["N"] + row["t_lap_s"] / row["t_solve_s"], rel=1e-12)
        assert row["R0"] > 2 * row["R1"] + row["N"]
        assert np.isfinite(row["C_dist_over_C_PS"])
        assert row["pays_off"] == (1 - row["C_dist_over_C_PS"] <= row["R1_over_R0"])
        # Table 2's split and the per-t ratios of both channels (Figs. 3 and 5)
        assert row["t_lap_matvec_s"] > 0 and row["t_lap_ortho_s"] > 0
        assert row["t_lap_matvec_s"] + row["t_lap_ortho_s"] <= 1.05 * row["t_lap_s"]
        assert len(row["C_dist_over_C_V_t"]) == T and len(row["C_dist_over_C_PS_t"]) == T
        assert row["C_dist_over_C_PS_t"][row["t"]] == pytest.approx(row["C_dist_over_C_PS"], rel=1e-12)
        assert np.all(np.isfinite(row["C_dist_over_C_V_t"]))
