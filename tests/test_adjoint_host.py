"""Host logic of the gradient wrapper (paper_2007_01416_gb300/adjoint.py) on
the CPU: the checkpoint interval and buffer shapes it passes to the C ABI, and
the cotangent it hands back to autograd, in FP64 and in the compensated FP32
layout. A fake context stands in for libacat: its "step" is a fixed linear map
u <- A u of the state, so that the gradient of <w, u^n> is (A^T)^n w exactly.
"""
import math

import numpy as np
import pytest
import torch

from paper_2007_01416_gb300 import adjoint as AD


class FakeLinearCtx:
    """acat_run_record / acat_adjoint_run with the contracts of include/acat.h,
    on CPU tensors, for the step u <- A u (FP64 layout [s][nx], or the FP32
    pair [2][s][nx] whose value is hi + lo)."""

    def __init__(self, A, f32):
        self.A = A
        self.f32 = f32
        self.calls = []

    def _value(self, u):
        return (u[0].double() + u[1].double()) if self.f32 else u.double()

    def acat_run_record(self, u0, u_out, nsteps, every, ckpt, dts):
        self.calls.append(("record", nsteps, every, tuple(ckpt.shape), tuple(dts.shape)))
        assert ckpt.shape[0] == -(-nsteps // every)
        v = self._value(u0).reshape(-1)
        for n in range(nsteps):
            if n % every == 0:
                ckpt[n // every].copy_(u0 if n == 0 else self._store(v, u0))
            dts[n] = 0.5 + n
            v = self.A @ v
        u_out.copy_(self._store(v, u0))

    def acat_adjoint_run(self, ckpt, dts, nsteps, every, ubar_n, ubar_0):
        self.calls.append(("adjoint", nsteps, every))
        g = self._value(ubar_n).reshape(-1)
        for _ in range(nsteps):
            g = self.A.T @ g
        ubar_0.copy_(self._store(g, ubar_n))

    def _store(self, v, like):
        if self.f32:
            hi = v.to(torch.float32)
            lo = (v - hi.double()).to(torch.float32)
            return torch.stack([hi.reshape(like.shape[1:]), lo.reshape(like.shape[1:])])
        return v.reshape(like.shape).to(like.dtype)


@pytest.mark.parametrize("n,every", [(1, 1), (7, 3), (16, 4), (2000, 45)])
def test_default_every_and_checkpoint_count(n, every):
    assert AD.default_every(n) == every
    assert AD.default_every(n) == max(1, round(math.sqrt(n)))


@pytest.mark.parametrize("nsteps,every", [(5, 0), (5, 2), (9, 3), (1, 0)])
def test_gradient_fp64(nsteps, every):
    rng = np.random.default_rng(3)
    s, nx = 3, 5
    A = torch.from_numpy(rng.normal(size=(s * nx, s * nx)) / math.sqrt(s * nx))
    ctx = FakeLinearCtx(A, f32=False)
    u0 = torch.from_numpy(rng.normal(size=(s, nx))).requires_grad_(True)
    w = torch.from_numpy(rng.normal(size=(s, nx)))
    uN = AD.run(u0, ctx, nsteps, every)
    (uN * w).sum().backward()
    want = torch.linalg.matrix_power(A.T, nsteps) @ w.reshape(-1)
    assert torch.allclose(u0.grad.reshape(-1), want, rtol=1e-12, atol=1e-12)
    ev = every or AD.default_every(nsteps)
    assert ctx.calls[0] == ("record", nsteps, ev, (-(-nsteps // ev), s, nx), (nsteps,))
    assert ctx.calls[1] == ("adjoint", nsteps, ev)


def test_gradient_zero_steps_is_identity():
    ctx = FakeLinearCtx(torch.eye(4, dtype=torch.float64), f32=False)
    u0 = torch.arange(4.0, dtype=torch.float64).reshape(1, 4).requires_grad_(True)
    uN = AD.run(u0, ctx, 0)
    assert torch.equal(uN, u0.detach())
    (3.0 * uN).sum().backward()
    assert torch.equal(u0.grad, torch.full((1, 4), 3.0, dtype=torch.float64))
    assert ctx.calls == []


def test_gradient_fp32_pair_layout():
    """The FP32 state is (hi, lo) with value hi + lo: the value's cotangent
    comes from the hi half of the incoming gradient, and the returned
    gradient carries the value's cotangent in both halves (d value / d hi =
    d value / d lo = 1)."""
    rng = np.random.default_rng(4)
    s, nx, n = 3, 4, 6
    A = torch.from_numpy(rng.normal(size=(s * nx, s * nx)) / math.sqrt(s * nx))
    ctx = FakeLinearCtx(A, f32=True)
    v0 = torch.from_numpy(rng.normal(size=(s, nx)))
    hi = v0.to(torch.float32)
    lo = (v0 - hi.double()).to(torch.float32)
    u0 = torch.stack([hi, lo]).requires_grad_(True)
    w = torch.from_numpy(rng.normal(size=(s, nx))).to(torch.float32)
    uN = AD.run(u0, ctx, n, 2)
    ((uN[0] + uN[1]) * w).sum().backward()
    want = (torch.linalg.matrix_power(A.T, n) @ w.double().reshape(-1)).reshape(s, nx)
    for half in (0, 1):
        assert torch.allclose(u0.grad[half].double(), want, rtol=1e-5, atol=1e-6)
