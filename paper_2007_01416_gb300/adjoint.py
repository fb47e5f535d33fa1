"""Gradients through n ACAT steps with respect to the initial state.

ACATRun is a torch.autograd.Function over the C ABI. The forward pass is
acat_run_record: n CFL steps on the device, the dt of each step recorded on
the device, the state kept every `every` steps (default round(sqrt(n))). The
backward pass is acat_adjoint_run: segment by segment from the last, the
states are recomputed from the checkpoint with the recorded dt (bit-identical
to the forward) and the hand-written adjoint step is applied in reverse. The
discrete choices of every step and its dt are those of the forward pass.
Only argument marshalling happens here; no step returns to the host.

FP32 contexts take and return compensated pair states [2][s][nx] (hi, lo).
Their state value is hi + lo, so the cotangent of the value is read from the
hi half of the incoming gradient, and the gradient returned for u0 carries
the cotangent of the value in both halves.
"""
from __future__ import annotations

import math

import torch


def default_every(nsteps: int) -> int:
    return max(1, int(round(math.sqrt(max(nsteps, 1)))))


class ACATRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, actx, nsteps: int, every: int = 0):
        every = every or default_every(nsteps)
        u0 = u0.detach().contiguous()
        nck = max(1, -(-nsteps // every))
        ckpt = torch.empty((nck,) + tuple(u0.shape), dtype=u0.dtype, device=u0.device)
        dts = torch.empty(max(nsteps, 1), dtype=torch.float64, device=u0.device)
        out = torch.empty_like(u0)
        if nsteps == 0:
            out.copy_(u0)
        else:
            actx.acat_run_record(u0, out, nsteps, every, ckpt, dts)
        ctx.save_for_backward(ckpt, dts)
        ctx.actx, ctx.nsteps, ctx.every = actx, nsteps, every
        return out

    @staticmethod
    def backward(ctx, gN):
        ckpt, dts = ctx.saved_tensors
        f32 = gN.dtype == torch.float32
        if f32:
            g = torch.zeros_like(gN)
            g[0] = gN[0]  # compensated cotangent (value, 0)
        else:
            g = gN.detach().contiguous().clone()
        if ctx.nsteps > 0:
            ctx.actx.acat_adjoint_run(ckpt, dts, ctx.nsteps, ctx.every, g, g)
        if f32:
            v = g[0] + g[1]
            g = torch.stack([v, v])
        return g, None, None, None


def run(u0: torch.Tensor, actx, nsteps: int, every: int = 0) -> torch.Tensor:
    """u^n as a differentiable function of u0 (1D context, FP64 or FP32)."""
    return ACATRun.apply(u0, actx, nsteps, every)


def replay(u0: torch.Tensor, actx, dts) -> torch.Tensor:
    """The forward map with a given dt sequence (for finite differences of
    the map the adjoint differentiates)."""
    u = u0.contiguous().clone()
    nxt = torch.empty_like(u)
    for d in dts:
        actx.acat_step(u, nxt, float(d))
        u, nxt = nxt, u
    return u
