"""Differentiable solves and correlators on the GPU: the hand-written backward
passes (gamma_5 adjoint solves) against the oracle's LU-based adjoint and
against central finite differences (step 1e-4, FP64)."""
import numpy as np
import pytest

import synth
from oracle import dirac, dlma
from oracle import laplacian as lap
from oracle import solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_09729_gb300 as dl
    return dl


def test_solve_autograd_vs_oracle_adjoint(dl):
    import torch

    from paper_2201_09729_gb300.autograd import DLMASolve

    L, T, csw, m0 = 4, 4, 1.0, 0.15
    U = synth.gauge_field(L, T, 0.2, 601)
    ctx = dl.Context(L, T, 0, 0)
    ctx.dlma_set_gauge(U)
    b_h = synth.gaussian_spinors(2, L ** 3 * T, 602)
    c_h = synth.gaussian_spinors(2, L ** 3 * T, 603)
    b = torch.from_numpy(b_h).cuda().requires_grad_(True)
    m = torch.tensor(m0, dtype=torch.float64, requires_grad=True)
    c = torch.from_numpy(c_h).cuda()
    x = DLMASolve.apply(b, m, ctx, csw, 1e-13, dl.FP64)
    loss = torch.sum(torch.conj(c) * x).real
    loss.backward()
    eo = dirac.EvenOdd(U, L, T, m0, csw)
    y = solve.lu_solver_dag(eo)(c_h)                  # D^-dag c
    xo = solve.lu_solver(eo)(b_h)
    gb = b.grad.cpu().numpy()
    assert np.linalg.norm(gb - y) / np.linalg.norm(y) < 1e-10
    want_m0 = -np.vdot(y.ravel(), xo.ravel()).real
    assert abs(m.grad.item() - want_m0) < 1e-9 * abs(want_m0)
    # central difference in m0
    h = 1e-4
    lp = np.vdot(c_h.ravel(), solve.lu_solver(dirac.EvenOdd(U, L, T, m0 + h, csw))(b_h).ravel()).real
    lm = np.vdot(c_h.ravel(), solve.lu_solver(dirac.EvenOdd(U, L, T, m0 - h, csw))(b_h).ravel()).real
    assert abs((lp - lm) / (2 * h) - m.grad.item()) < 1e-6 * abs(want_m0)


def test_correlator_gradients_plain_workload(dl):
    import torch

    from paper_2201_09729_gb300.autograd import DLMACorrelatorPS

    wl = synth.WORKLOADS["plain_4c8"]
    U, eta = synth.workload_inputs(wl)
    w = synth.loss_weights(wl.T, synth.WEIGHT_SEED_BASE + wl.cfg)
    ctx = dl.Context(wl.L, wl.T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_laplacian_eigs(-1, wl.n_modes, 1e-13, want_vecs=False)
    e = torch.from_numpy(np.ascontiguousarray(eta[0])).cuda().requires_grad_(True)
    m = torch.tensor(wl.m0, dtype=torch.float64, requires_grad=True)
    c = DLMACorrelatorPS.apply(e, m, ctx, wl.csw, 0, wl.n_modes, 1e-13, dl.FP64)
    loss = torch.sum(torch.from_numpy(w).cuda() * c)
    loss.backward()
    # oracle adjoint (LU solves of D and D^dag, modes by dense eigh)
    eo = dirac.EvenOdd(U, wl.L, wl.T, wl.m0, wl.csw)
    V_all = np.stack([lap.lap_modes(lap.timeslice_links(U, wl.L, t), wl.L, wl.n_modes)[1] for t in range(wl.T)])
    lo, dm0, deta = dlma.ps_loss_grads(solve.lu_solver(eo), solve.lu_solver_dag(eo), V_all, eta[0], w,
                                       wl.L, wl.T, 0)
    assert abs(loss.item() - lo) < 1e-10 * abs(lo)
    assert abs(m.grad.item() - dm0) < 1e-8 * abs(dm0)
    ge = e.grad.cpu().numpy()
    assert np.linalg.norm(ge - deta) < 1e-8 * np.linalg.norm(deta)


def test_correlator_gradients_differentiation_workload_fd(dl):
    # 16^3 x 32, N = 32, 4 noise vectors, mixed-precision solves to 1e-10:
    # backward vs central differences of the GPU forward itself
    wl = synth.WORKLOADS["grad_16c32"]
    U, eta = synth.workload_inputs(wl)
    w = synth.loss_weights(wl.T, synth.WEIGHT_SEED_BASE + wl.cfg)
    ctx = dl.Context(wl.L, wl.T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_laplacian_eigs(-1, wl.n_modes, 1e-11, want_vecs=False)
    e0 = np.ascontiguousarray(eta[0])

    def loss_at(m0, e):
        ctx.dlma_set_params(m0, wl.csw)
        r = ctx.dlma_correlators(0, wl.n_modes, e, 1e-11, dl.FP32)
        return float(np.sum(w * r["C"][0].real))

    ctx.dlma_set_checkpoint(True)
    loss_at(wl.m0, e0)
    dm0, deta = ctx.dlma_correlators_backward(0, wl.n_modes, wl.n_noise, w, 1e-11, dl.FP32)
    ctx.dlma_set_checkpoint(False)
    h = 1e-4
    fd = (loss_at(wl.m0 + h, e0) - loss_at(wl.m0 - h, e0)) / (2 * h)
    assert abs(fd - dm0) < 1e-5 * abs(dm0), (fd, dm0)
    d = synth.gaussian_spinors(wl.n_noise, wl.vol_s, 604)
    fd = (loss_at(wl.m0, e0 + h * d) - loss_at(wl.m0, e0 - h * d)) / (2 * h)
    want = np.vdot(deta.ravel(), d.ravel()).real
    assert abs(fd - want) < 1e-5 * abs(want), (fd, want)


def test_two_forwards_before_one_backward(dl):
    # a loss summed over two masses and two noise draws: both forwards run before
    # either backward, so each backward must restore its own m0 and recompute its
    # replaced checkpoint; the gradients must equal those of the two losses taken
    # one at a time (each against the oracle adjoint)
    import torch

    from paper_2201_09729_gb300.autograd import DLMACorrelatorPS, DLMASolve

    wl = synth.WORKLOADS["plain_4c8"]
    U, eta = synth.workload_inputs(wl)
    w = synth.loss_weights(wl.T, synth.WEIGHT_SEED_BASE + wl.cfg)
    ctx = dl.Context(wl.L, wl.T, 0, 0)
    ctx.dlma_set_gauge(U)
    ctx.dlma_laplacian_eigs(-1, wl.n_modes, 1e-13, want_vecs=False)
    V_all = np.stack([lap.lap_modes(lap.timeslice_links(U, wl.L, t), wl.L, wl.n_modes)[1] for t in range(wl.T)])
    e_np = [np.ascontiguousarray(eta[0]), np.ascontiguousarray(synth.z2z2_noise(wl.n_noise, wl.vol_s, 611))]
    m_vals = [wl.m0, wl.m0 + 0.05]
    es = [torch.from_numpy(x).cuda().requires_grad_(True) for x in e_np]
    ms = [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in m_vals]
    wt = torch.from_numpy(w).cuda()
    cs = [DLMACorrelatorPS.apply(es[i], ms[i], ctx, wl.csw, 0, wl.n_modes, 1e-13, dl.FP64) for i in range(2)]
    (torch.sum(wt * cs[0]) + torch.sum(wt * cs[1])).backward()
    for i in range(2):
        eo = dirac.EvenOdd(U, wl.L, wl.T, m_vals[i], wl.csw)
        lo, dm0, deta = dlma.ps_loss_grads(solve.lu_solver(eo), solve.lu_solver_dag(eo), V_all, e_np[i], w,
                                           wl.L, wl.T, 0)
        assert abs(ms[i].grad.item() - dm0) < 1e-8 * abs(dm0), i
        assert np.linalg.norm(es[i].grad.cpu().numpy() - deta) < 1e-8 * np.linalg.norm(deta), i
    # the checkpoint is released after the backwards
    assert ctx.dlma_checkpoint_serial() == 0
    # a stale checkpoint is refused by the library: forward at one mass, backward at another
    ctx.dlma_set_params(wl.m0, wl.csw)
    ctx.dlma_set_checkpoint(True)
    ctx.dlma_correlators(0, wl.n_modes, e_np[0], 1e-12, dl.FP64)
    ctx.dlma_set_params(wl.m0 + 0.01, wl.csw)
    with pytest.raises(dl.DlmaError) as exc:
        ctx.dlma_correlators_backward(0, wl.n_modes, wl.n_noise, w, 1e-12, dl.FP64)
    assert exc.value.status == 8
    ctx.dlma_set_checkpoint(False)
    # the solve's backward uses the operator of its own forward
    L, T = wl.L, wl.T
    b_h = synth.gaussian_spinors(1, L ** 3 * T, 612)
    c_h = synth.gaussian_spinors(1, L ** 3 * T, 613)
    b = torch.from_numpy(b_h).cuda().requires_grad_(True)
    m = torch.tensor(0.2, dtype=torch.float64, requires_grad=True)
    x = DLMASolve.apply(b, m, ctx, wl.csw, 1e-13, dl.FP64)
    ctx.dlma_set_params(0.5, wl.csw)                       # changed between forward and backward
    torch.sum(torch.conj(torch.from_numpy(c_h).cuda()) * x).real.backward()
    y = solve.lu_solver_dag(dirac.EvenOdd(U, L, T, 0.2, wl.csw))(c_h)
    assert np.linalg.norm(b.grad.cpu().numpy() - y) / np.linalg.norm(y) < 1e-10
