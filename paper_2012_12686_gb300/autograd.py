"""``torch.autograd.Function`` over the fused loss-and-gradient call.

The loss is a scalar, so the forward pass runs the fused forward + adjoint once
(``adorym_loss_grad``) and keeps the gradients; ``backward`` only scales them by the incoming
gradient.  Gradients are computed only for the inputs that require them.  Complex probe
gradients follow PyTorch's convention for real losses (dL/dRe + i dL/dIm), which is the
library's convention too.
"""
from __future__ import annotations

import torch

from .adorym import Engine

_engines: dict = {}


def engine_for(device: torch.device) -> Engine:
    idx = device.index if device.index is not None else torch.cuda.current_device()
    key = (idx, torch.cuda.current_stream(idx).cuda_stream)
    if key not in _engines:
        _engines[key] = Engine(idx, key[1])
    return _engines[key]


class MultisliceLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, delta, beta, probe, pos, I_meas, problem):
        if not delta.is_cuda:
            raise RuntimeError("MultisliceLoss runs on the CUDA engine only (no CPU path)")
        eng = engine_for(delta.device)
        need = ctx.needs_input_grad
        want_obj = need[0] or need[1]
        gd = torch.zeros_like(delta) if want_obj else None
        gb = torch.zeros_like(beta) if want_obj else None
        gp = torch.zeros_like(probe) if need[2] else None
        gpos = torch.empty_like(pos) if need[3] else None
        loss = torch.empty((), dtype=torch.float64, device=delta.device)
        d, b = delta.detach().contiguous(), beta.detach().contiguous()
        oid = eng.register_object(d, b)
        try:
            eng.loss_grad(problem, oid, probe.detach().contiguous(), pos.detach().contiguous(),
                          I_meas.detach().contiguous(), loss, gd, gb, gp, gpos)
        finally:
            eng.unregister_object(oid)
        ctx.save_for_backward(gd, gb, gp, gpos)
        ctx.keep = (d, b)          # the registration's volumes stay alive until the call is done
        return loss

    @staticmethod
    def backward(ctx, g):
        gd, gb, gp, gpos = ctx.saved_tensors
        s32 = g.to(torch.float32)

        def sc(t):
            return None if t is None else t * (s32 if not t.is_complex() else s32.to(t.dtype))
        return sc(gd), sc(gb), sc(gp), sc(gpos), None, None


def multislice_loss(delta, beta, probe, pos, I_meas, problem):
    """Loss of Eq. lsq_loss / Eq. poisson_loss over the batch, differentiable in delta, beta, probe, pos."""
    return MultisliceLoss.apply(delta, beta, probe, pos, I_meas, problem)
