"""torch.autograd view of the forward map (velocity, wavelet) -> traces.

The backward pass is the library's own transpose: for an upstream gradient g
of the traces, the velocity gradient is mmod_gradient with g as the residual
(the zero-lag imaging condition of the adjoint wavefield, forward states
recomputed from checkpoints), and the wavelet gradient is mmod_adjoint(g).
Argument marshalling only: every step runs in libmmod.so.
"""
from __future__ import annotations

import torch

from . import CKPT_FP32, Propagator


class _ForwardMap(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vel, wavelet, prop, ckpt_count, ckpt_dtype):
        vel = vel.contiguous()
        wavelet = wavelet.contiguous()
        prop.set_model(vel)
        traces = torch.empty((prop.nt, prop.nrec), device=vel.device, dtype=torch.float32)
        prop.forward(wavelet, traces)
        ctx.prop = prop
        ctx.ckpt = (int(ckpt_count), int(ckpt_dtype))
        ctx.save_for_backward(vel, wavelet)
        return traces

    @staticmethod
    def backward(ctx, g):
        vel, wavelet = ctx.saved_tensors
        prop = ctx.prop
        g = g.contiguous().float()
        grad_vel = grad_wav = None
        if ctx.needs_input_grad[0]:
            prop.set_model(vel)   # the handle may have seen another model since
            grad_vel = torch.empty_like(vel)
            prop.gradient(wavelet, g, grad_vel, *ctx.ckpt)
        if ctx.needs_input_grad[1]:
            grad_wav = torch.empty_like(wavelet)
            prop.adjoint(g, grad_wav)
        return grad_vel, grad_wav, None, None, None


def forward_map(prop: Propagator, vel: torch.Tensor, wavelet: torch.Tensor, ckpt_count: int = 20,
                ckpt_dtype: int = CKPT_FP32) -> torch.Tensor:
    """traces [nt][nrec] = F(vel, wavelet) on prop's grid, differentiable in
    vel ([nz][ny][nx] FP32, device) and wavelet ([nsrc][nt] FP32, device).
    ckpt_count / ckpt_dtype select the checkpoints of the velocity gradient
    (the prop's MMOD_OPT_CKPT_SCHEME applies)."""
    return _ForwardMap.apply(vel, wavelet, prop, ckpt_count, ckpt_dtype)
