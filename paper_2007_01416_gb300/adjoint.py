"""Gradients through n ACAT steps with respect to the initial state.

ACATRun is a torch.autograd.Function over the C ABI: the forward pass runs
the steps on the device (acat_step, CFL dt computed on the device and
recorded), keeping the state every `every` steps (default round(sqrt(n)));
the backward pass walks the segments from the last, recomputes each
segment's states from its checkpoint with the recorded dt (bit-identical to
the forward), and applies the hand-written adjoint step (acat_adjoint_step)
in reverse. The discrete choices of every step and its dt are those of the
forward pass. Only argument marshalling happens here.
"""
from __future__ import annotations

import math

import torch

from . import acat


class ACATRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, actx, nsteps: int, every: int = 0):
        every = every or max(1, int(round(math.sqrt(max(nsteps, 1)))))
        dts = torch.empty(max(nsteps, 1), dtype=torch.float64, device=u0.device)
        ckpts = []
        u = u0.detach().contiguous().clone()
        nxt = torch.empty_like(u)
        for n in range(nsteps):
            if n % every == 0:
                ckpts.append(u.clone())
            actx.acat_step(u, nxt, -1.0, None, dts[n:n + 1], None)
            u, nxt = nxt, u
        ctx.save_for_backward(dts, *ckpts)
        ctx.actx, ctx.nsteps, ctx.every = actx, nsteps, every
        return u.clone()

    @staticmethod
    def backward(ctx, gN):
        dts, *ckpts = ctx.saved_tensors
        actx, nsteps, every = ctx.actx, ctx.nsteps, ctx.every
        ub = gN.detach().contiguous().clone()
        ub2 = torch.empty_like(ub)
        dt = dts.cpu().tolist()
        for seg in reversed(range(len(ckpts))):
            start, end = seg * every, min(nsteps, (seg + 1) * every)
            states = [ckpts[seg]]
            for n in range(start, end - 1):
                nxt = torch.empty_like(ub)
                actx.acat_step(states[-1], nxt, dt[n])
                states.append(nxt)
            for n in reversed(range(start, end)):
                actx.acat_adjoint_step(states[n - start], dt[n], ub, ub2)
                ub, ub2 = ub2, ub
        return ub, None, None, None


def run(u0: torch.Tensor, actx, nsteps: int, every: int = 0) -> torch.Tensor:
    """u^n as a differentiable function of u0 (1D FP64 context)."""
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
