"""``torch.autograd`` face of the hand-written LBM adjoint.

``WindowMisfit.apply(f0, cs, ens, win)`` returns the per-member misfit J [k]
of an observation window (``binding.Window``) forecast from the initial state
f0 (float64 tensor [9][ny][nx][k], CUDA) with Smagorinsky coefficient cs
(0-dim float64 tensor), using the context ``ens`` (a ``binding.Ensemble`` of
the same shape; its precision decides FP64 or binary32 arithmetic). Its
backward calls ``lbm_misfit_gradient`` with the incoming gradient as member
weights (on the device), so dL/df0 and dL/dcs (summed over members on the
device) come from the CUDA adjoint sweep (with step checkpointing), not
from autograd tracing. Argument marshalling only.
"""
from __future__ import annotations

import torch

from . import binding


class WindowMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f0, cs, ens, win):
        if f0.dtype != torch.float64 or not f0.is_cuda:
            raise TypeError("f0 must be a float64 CUDA tensor [9][ny][nx][k]")
        f0 = f0.contiguous()
        ens.set_f(f0)
        ens.set_closure(float(cs))
        J = ens.misfit(win)
        ctx.save_for_backward(f0, cs)
        ctx.ens, ctx.win = ens, win
        return torch.as_tensor(J, dtype=torch.float64, device=f0.device)

    @staticmethod
    def backward(ctx, gJ):
        f0, cs = ctx.saved_tensors
        ens, win = ctx.ens, ctx.win
        ens.set_f(f0)
        ens.set_closure(float(cs))
        grad = torch.empty_like(f0)
        w = gJ.detach().to(device=f0.device, dtype=torch.float64).contiguous()
        dcs = torch.empty(1, dtype=torch.float64, device=f0.device)
        binding.lbm_misfit_gradient(ens.ctx, win, ens.members, weights=w, grad_f0=grad, dcs=dcs)
        gc = dcs.reshape(()).to(device=cs.device, dtype=cs.dtype)
        return grad, gc, None, None


def window_misfit(f0, cs, ens, win):
    """Functional form of ``WindowMisfit.apply``."""
    return WindowMisfit.apply(f0, cs, ens, win)
