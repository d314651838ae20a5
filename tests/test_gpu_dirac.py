"""GPU parity of the Wilson-clover stencil and the solves against the FP64
oracle, through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import dirac, lattice, solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_09729_gb300 as dl
    return dl


def _ctx(dl, L, T, eps, m0, csw, seed, bc=0):
    U = synth.gauge_field(L, T, eps, seed)
    ctx = dl.Context(L, T, bc, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(m0, csw)
    return ctx, dirac.EvenOdd(U, L, T, m0, csw, bc)


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.mark.parametrize("L,T", [(2, 4), (4, 8), (6, 4)])
def test_index_tables_bit_exact(dl, L, T):
    ctx = dl.Context(L, T, 0, 0)
    eo, nbr = ctx.dlma_index_tables()
    even, odd, eo_o = lattice.eo_tables(L, T)
    assert np.array_equal(eo, eo_o)
    fwd, bwd = lattice.neighbours(L, T)
    for p, sites in ((0, even), (1, odd)):
        for mu in range(4):
            assert np.array_equal(nbr[p, 2 * mu], eo_o[fwd[mu][sites]])
            assert np.array_equal(nbr[p, 2 * mu + 1], eo_o[bwd[mu][sites]])


@pytest.mark.parametrize("L,T,bc", [(4, 8, 0), (6, 4, 1), (2, 4, 0)])
def test_apply_dw_fp64(dl, L, T, bc):
    ctx, eo = _ctx(dl, L, T, 0.3, 0.07, 1.4, 101, bc)
    psi = synth.gaussian_spinors(5, L ** 3 * T, 102)
    got = ctx.dlma_apply_Dw(psi, dl.FP64)
    want = eo.apply_full(psi)
    for j in range(5):
        assert _rel(got[j], want[j]) < 1e-13


def test_apply_dw_low_precision(dl):
    L, T = 4, 8
    ctx, eo = _ctx(dl, L, T, 0.2, 0.08, 1.0, 103)
    psi = synth.gaussian_spinors(3, L ** 3 * T, 104)
    want = eo.apply_full(psi)
    got32 = ctx.dlma_apply_Dw(psi, dl.FP32)
    got16 = ctx.dlma_apply_Dw(psi, dl.FP16S)
    for j in range(3):
        assert _rel(got32[j], want[j]) < 1e-6
        assert _rel(got16[j], want[j]) < 3e-3


@pytest.mark.parametrize("links", ["12", "18"])
def test_schur_fp32_link_formats(dl, links, monkeypatch):
    # the FP32 stencil reads either 12-real links (third row rebuilt) or all 18 reals
    monkeypatch.setenv("DLMA_FORCE_LINKS", links)
    L, T = 6, 4
    ctx, eo = _ctx(dl, L, T, 0.25, 0.1, 1.2, 111)
    ve = synth.gaussian_spinors(5, L ** 3 * T // 2, 112)
    for dagger in (0, 1):
        got = ctx.dlma_apply_schur(ve, dagger, dl.FP32)
        want = eo.schur_dag(ve) if dagger else eo.schur(ve)
        for j in range(5):
            assert _rel(got[j], want[j]) < 1e-6


def test_schur_block_order_chunks_bit_identical(dl, monkeypatch):
    # the chunk size of the stencil's block order only reorders the blocks: every
    # output element is computed by one thread with the same operations, so 16 and
    # 128 right-hand sides per chunk (ragged against 37 right-hand sides, two per
    # thread) give identical bits, FP32 and FP64, and match the oracle
    L, T = 6, 4
    ve = synth.gaussian_spinors(37, L ** 3 * T // 2, 113)
    out = {}
    for ch in ("16", "128"):
        monkeypatch.setenv("DLMA_FORCE_CHUNK", ch)
        monkeypatch.setenv("DLMA_FORCE_NR", "2")
        monkeypatch.setenv("DLMA_FORCE_LINKS", "12")   # the link format changes the rounding
        ctx, eo = _ctx(dl, L, T, 0.25, 0.1, 1.2, 111)
        out[ch] = (ctx.dlma_apply_schur(ve, 0, dl.FP32), ctx.dlma_apply_schur(ve, 0, dl.FP64))
        ctx.close()
    want = eo.schur(ve)
    for k in (0, 1):
        assert np.array_equal(out["16"][k], out["128"][k])
    for j in range(37):
        assert _rel(out["16"][0][j], want[j]) < 1e-6
        assert _rel(out["16"][1][j], want[j]) < 1e-13


@pytest.mark.parametrize("dagger", [0, 1])
def test_schur_fp64(dl, dagger):
    L, T = 6, 4
    ctx, eo = _ctx(dl, L, T, 0.25, 0.1, 1.2, 105)
    ve = synth.gaussian_spinors(6, L ** 3 * T // 2, 106)
    got = ctx.dlma_apply_schur(ve, dagger, dl.FP64)
    want = eo.schur_dag(ve) if dagger else eo.schur(ve)
    assert _rel(got, want) < 1e-13


def test_solve_fp64_plain_workload_vs_lu(dl):
    wl = synth.WORKLOADS["plain_4c8"]
    U, _ = synth.workload_inputs(wl)
    ctx = dl.Context(wl.L, wl.T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(wl.m0, wl.csw)
    eo = dirac.EvenOdd(U, wl.L, wl.T, wl.m0, wl.csw)
    b = synth.gaussian_spinors(3, wl.volume, 107)
    x, info = ctx.dlma_solve(b, 1e-12, dl.FP64)
    xl = solve.lu_solver(eo)(b)
    for j in range(3):
        assert info[j]["converged"] and info[j]["true_resid"] <= 1e-12
        assert _rel(x[j], xl[j]) < 1e-10


@pytest.mark.parametrize("prec,solver", [("FP32", "SOLVER_BICGSTAB"), ("FP32", "SOLVER_CGNE"), ("FP16S", "SOLVER_CGNE")])
def test_mixed_precision_solve_ragged_batch(dl, prec, solver):
    # 7 right-hand sides (ragged against the 4-rhs block), one of them zero;
    # V/2 = 432 sites: 6.75 tiles of 64; both Krylov methods of the FP32 solve
    L, T = 6, 4
    ctx, eo = _ctx(dl, L, T, 0.2, 0.0816, 1.0, 108)
    ctx.dlma_set_solver(getattr(dl, solver))
    b = synth.gaussian_spinors(7, L ** 3 * T, 109)
    b[3] = 0
    x, info = ctx.dlma_solve(b, 1e-10, getattr(dl, prec))
    lu = solve.lu_solver(eo)
    xl = lu(b)
    assert np.all(x[3] == 0) and info[3]["true_resid"] == 0
    for j in (0, 1, 2, 4, 5, 6):
        r = np.linalg.norm((b[j] - eo.apply_full(x[j])).ravel()) / np.linalg.norm(b[j].ravel())
        assert r <= 1e-10 and info[j]["true_resid"] <= 1e-10
        assert abs(r - info[j]["true_resid"]) < 1e-11
        assert _rel(x[j], xl[j]) < 1e-8


@pytest.mark.parametrize("tsl", [[3], [7, 0], [2, 3, 5]])
def test_solve_timeslice_local_sources(dl, tsl):
    # sources supported on few timeslices (one; two across the periodic boundary;
    # a run with a gap): the source preparation touches only the timeslices next
    # to the support (8^3 x 10: whole-timeslice blocks); the solutions still meet
    # the tolerance by the oracle's operator, in FP64 and mixed precision alike
    L, T = 8, 10
    ctx, eo = _ctx(dl, L, T, 0.2, 0.09, 1.0, 131)
    b = synth.gaussian_spinors(4, L ** 3 * T, 132).reshape(4, T, L ** 3, 4, 3)
    keep = np.zeros(T, bool)
    keep[tsl] = True
    b[:, ~keep] = 0
    b = b.reshape(4, L ** 3 * T, 4, 3)
    xs = []
    for prec in (dl.FP32, dl.FP64):
        x, info = ctx.dlma_solve(b, 1e-10, prec)
        for j in range(4):
            r = np.linalg.norm((b[j] - eo.apply_full(x[j])).ravel()) / np.linalg.norm(b[j].ravel())
            assert r <= 1e-10 and info[j]["converged"], (prec, j, r)
        xs.append(x)
    for j in range(4):
        assert _rel(xs[0][j], xs[1][j]) < 1e-8


def test_solve_precision_workload_residual_property(dl):
    # full 16^3 x 32 size: the oracle checks the GPU solutions by their true residual
    wl = synth.WORKLOADS["precision_16c32"]
    U, _ = synth.workload_inputs(wl)
    ctx = dl.Context(wl.L, wl.T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_set_params(wl.m0, wl.csw)
    eo = dirac.EvenOdd(U, wl.L, wl.T, wl.m0, wl.csw)
    b = synth.gaussian_spinors(2, wl.volume, 110)
    for prec, solver in ((dl.FP32, dl.SOLVER_BICGSTAB), (dl.FP32, dl.SOLVER_CGNE), (dl.FP16S, dl.SOLVER_CGNE)):
        ctx.dlma_set_solver(solver)
        x, info = ctx.dlma_solve(b, 1e-10, prec)
        for j in range(2):
            r = np.linalg.norm((b[j] - eo.apply_full(x[j])).ravel()) / np.linalg.norm(b[j].ravel())
            assert r <= 1e-10, (prec, solver, j, r, info[j])
