"""Differentiable solves and correlators (torch.autograd.Function wrappers).

The forward and backward passes both run in libdlma.so; these classes only
move tensors across the C ABI.

DLMASolve:        x = D(m0)^-1 b.  Backward: grad_b = D^-dag grad_x, computed as
                  gamma_5 D^-1 gamma_5 grad_x (dlma_solve_adjoint), and
                  grad_m0 = -Re <grad_b, x> since dD/dm0 = 1.  Only x is kept
                  for the backward (no Krylov iterates).
DLMACorrelatorPS: C_PS(t) = Re C(t) of the pseudoscalar channel for one source
                  timeslice, C the Eq. 2 total as the library returns it,
                  differentiable in m0 and in the noise vectors eta; the forward
                  solutions are checkpointed by the library and the backward
                  runs the adjoint solves of dlma_correlators_backward.

The context is shared state: another forward, or a new m0 / c_sw, may come
between a forward and its backward (a loss summed over two masses or two noise
draws).  Each forward therefore records the (m0, c_sw) it ran with and, for
the correlator, the library's checkpoint serial; the backward restores the
parameters and, if another forward has replaced the checkpoint since, re-runs
its own forward before the adjoint solves.  The checkpoint is released once
the backward has used it.

Gradients of complex tensors follow PyTorch's convention dL/dRe + i dL/dIm.
"""
from __future__ import annotations

import torch

from . import _lib as L


def _ensure_params(ctx, params):
    if ctx.params != params:
        ctx.dlma_set_params(*params)


class DLMASolve(torch.autograd.Function):
    """x = D^-1 b for a Context whose gauge field is set; m0 is a 0-dim tensor
    (set on the context in the forward) and c_sw a float."""

    @staticmethod
    def forward(fctx, b, m0, ctx, csw, tol=1e-12, inner=L.FP64):
        params = (float(m0), float(csw))
        _ensure_params(ctx, params)
        x, _ = ctx.dlma_solve(b.detach().contiguous(), tol, inner)
        fctx.save_for_backward(x)
        fctx.dl = (ctx, tol, inner, params)
        return x

    @staticmethod
    def backward(fctx, grad_x):
        (x,) = fctx.saved_tensors
        ctx, tol, inner, params = fctx.dl
        _ensure_params(ctx, params)       # the operator of this forward, not the current one
        y = ctx.dlma_solve_adjoint(grad_x.contiguous(), tol, inner)
        grad_m0 = -ctx.dlma_real_dot(y, x)
        return y, torch.tensor(grad_m0, dtype=torch.float64), None, None, None, None


class DLMACorrelatorPS(torch.autograd.Function):
    """Real part of the pseudoscalar correlator total of Eq. 2 for source
    timeslice t_src, from the cached Laplacian modes (N per timeslice) and
    the noise eta (complex [n_noise, L^3, 4, 3], a CUDA tensor)."""

    @staticmethod
    def _forward_pass(ctx, eta, params, t_src, N, tol, inner):
        _ensure_params(ctx, params)
        ctx.dlma_set_checkpoint(True)
        res = ctx.dlma_correlators(int(t_src), int(N), eta, tol, inner)
        return res, ctx.dlma_checkpoint_serial()

    @staticmethod
    def forward(fctx, eta, m0, ctx, csw, t_src, N, tol=1e-12, inner=L.FP64):
        params = (float(m0), float(csw))
        eta_d = eta.detach().contiguous()
        res, serial = DLMACorrelatorPS._forward_pass(ctx, eta_d, params, t_src, N, tol, inner)
        fctx.save_for_backward(eta_d)
        fctx.dl = (ctx, int(t_src), int(N), int(eta.shape[0]), tol, inner, params, serial)
        return torch.as_tensor(res["C"][0].real.copy(), dtype=torch.float64, device=eta.device)

    @staticmethod
    def backward(fctx, grad_c):
        (eta_d,) = fctx.saved_tensors
        ctx, t_src, N, nn, tol, inner, params, serial = fctx.dl
        _ensure_params(ctx, params)
        if ctx.dlma_checkpoint_serial() != serial:
            # another forward replaced this one's checkpoint: recompute it
            DLMACorrelatorPS._forward_pass(ctx, eta_d, params, t_src, N, tol, inner)
        dm0, deta = ctx.dlma_correlators_backward(t_src, N, nn, grad_c.contiguous(), tol, inner)
        ctx.dlma_set_checkpoint(False)    # the checkpoint has served its backward
        return deta, torch.tensor(dm0, dtype=torch.float64), None, None, None, None, None, None
