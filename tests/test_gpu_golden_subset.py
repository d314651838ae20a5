"""Every correlator part of the 16^3 x 32 precision workload against the FP64
oracle, on the declared subset the oracle can solve (N_c = 2 modes, one Z2 x Z2
noise vector, t' = 0: tests/golden/oracle_correlators_precision_16c32_N2_R1.json,
written by tests/golden/make_correlator_golden.py from the oracle only).  The
library runs the same subset end to end -- its own Laplacian modes, sources,
mixed-precision solves to 1e-10, projections and contractions -- with FP32
inner solves (BiCGStab and CGNE) and FP16S inner solves; each part's error,
relative to max_t |C(t)| of its channel, is printed and must stay below 1e-8."""
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "oracle_correlators_precision_16c32_N2_R1.json")


@pytest.fixture(scope="module")
def dl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_09729_gb300 as dl
    return dl


@pytest.fixture(scope="module")
def golden():
    g = json.load(open(GOLDEN))
    parts = {k: np.array(v["re"]) + 1j * np.array(v["im"]) for k, v in g["parts"].items()}
    return g, parts


@pytest.mark.parametrize("inner,solver", [("FP32", "SOLVER_BICGSTAB"), ("FP32", "SOLVER_CGNE"),
                                          ("FP16S", "SOLVER_CGNE")])
def test_precision_workload_subset_vs_oracle(dl, golden, inner, solver):
    g, want = golden
    wl = synth.WORKLOADS["precision_16c32"]
    U, eta = synth.workload_inputs(wl, n_noise=g["n_noise"])
    ctx = dl.Context(wl.L, wl.T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(wl.m0, wl.csw)
    ctx.dlma_set_solver(getattr(dl, solver))
    lam, _ = ctx.dlma_laplacian_eigs(-1, g["n_modes"], 1e-12, want_vecs=False)
    assert np.abs(lam - np.array(g["laplacian_eigenvalues"])).max() <= 1e-9
    assert min(g["gap_above_cut"]) > 1e-4                 # the N_c = 2 projector is unique on every timeslice
    res = ctx.dlma_correlators(g["t_src"], g["n_modes"], np.ascontiguousarray(eta[0]), 1e-10, getattr(dl, inner))
    assert all(i["converged"] and i["true_resid"] <= 1e-10 for i in res["info"])
    report = {}
    for key, ref in want.items():
        scale = np.abs(want["C"]).max(axis=1)
        err = np.abs(res[key] - ref).max(axis=1) / scale
        report[key] = [float(e) for e in err]
        assert np.all(err <= 1e-8), (key, err)
    print(json.dumps({"inner": inner, "solver": solver, "rel_err_per_channel_PS_V1_V2_V3": report}))
