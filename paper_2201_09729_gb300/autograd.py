"""Differentiable solves and correlators (torch.autograd.Function wrappers).

The forward and backward passes both run in libdlma.so; these classes only
move tensors across the C ABI.

DLMASolve:        x = D(m0)^-1 b.  Backward: grad_b = D^-dag grad_x, computed as
                  gamma_5 D^-1 gamma_5 grad_x (dlma_solve_adjoint), and
                  grad_m0 = -Re <grad_b, x> since dD/dm0 = 1.  Only x is kept
                  for the backward (no Krylov iterates).
DLMACorrelatorPS: C_PS(t) = Re (C_rest + 2 C_mixed + C_dist)(t) of the
                  pseudoscalar channel for one source timeslice, differentiable
                  in m0 and in the noise vectors eta; the forward solutions are
                  checkpointed by the library and the backward runs the adjoint
                  solves of dlma_correlators_backward.

Gradients of complex tensors follow PyTorch's convention dL/dRe + i dL/dIm.
"""
from __future__ import annotations

import torch

from . import _lib as L


class DLMASolve(torch.autograd.Function):
    """x = D^-1 b for a Context whose gauge field is set; m0 is a 0-dim tensor
    (set on the context in the forward) and c_sw a float."""

    @staticmethod
    def forward(fctx, b, m0, ctx, csw, tol=1e-12, inner=L.FP64):
        ctx.dlma_set_params(float(m0), float(csw))
        x, _ = ctx.dlma_solve(b.detach().contiguous(), tol, inner)
        fctx.save_for_backward(x)
        fctx.dl = (ctx, tol, inner)
        return x

    @staticmethod
    def backward(fctx, grad_x):
        (x,) = fctx.saved_tensors
        ctx, tol, inner = fctx.dl
        y = ctx.dlma_solve_adjoint(grad_x.contiguous(), tol, inner)
        grad_m0 = -ctx.dlma_real_dot(y, x)
        return y, torch.tensor(grad_m0, dtype=torch.float64), None, None, None, None


class DLMACorrelatorPS(torch.autograd.Function):
    """Real part of the pseudoscalar correlator total of Eq. 2 for source
    timeslice t_src, from the cached Laplacian modes (N per timeslice) and
    the noise eta (complex [n_noise, L^3, 4, 3], a CUDA tensor)."""

    @staticmethod
    def forward(fctx, eta, m0, ctx, csw, t_src, N, tol=1e-12, inner=L.FP64):
        ctx.dlma_set_params(float(m0), float(csw))
        ctx.dlma_set_checkpoint(True)
        res = ctx.dlma_correlators(int(t_src), int(N), eta.detach().contiguous(), tol, inner)
        fctx.dl = (ctx, int(t_src), int(N), int(eta.shape[0]), tol, inner)
        return torch.as_tensor(res["C"][0].real.copy(), dtype=torch.float64, device=eta.device)

    @staticmethod
    def backward(fctx, grad_c):
        ctx, t_src, N, nn, tol, inner = fctx.dl
        dm0, deta = ctx.dlma_correlators_backward(t_src, N, nn, grad_c.contiguous(), tol, inner)
        return deta, torch.tensor(dm0, dtype=torch.float64), None, None, None, None, None, None
