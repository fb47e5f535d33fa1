"""Reference reverse sweep of the 1D ACAT step: plain PyTorch CPU operations
in float64, differentiated by torch.autograd.

TEST INFRASTRUCTURE. This is a second statement of the oracle's 1D step,
written for reverse-mode differentiation; it shares nothing with the CUDA
library. The step is the one of acat_oracle.c (Sec. 3.3, Eq. 2.12 with the
fluxes of Eq. 2.14 or the FL-CAT2 flux of Eq. 3.4), restated operation for
operation in the same order, vectorised over interfaces and stencil nodes:
  - the CAT2p flux by the recursion of Sec. 2.2 with the dt powers as printed;
  - the FL-CAT2 flux: the CAT2 flux (p = 1) blended with F^lo (Rusanov,
    global Lax-Friedrichs or HLL) by the superbee limiter psi^1 (Sec. 3.1;
    systems: the minimum over components and sides, Eq. 3.7);
  - the conservative update.
The discrete choices are frozen as the adjoint freezes them: the selected
orders are taken from the C oracle at the state (they are inputs here), and
every other choice (limiter piece, upwind side, argmin over components and
sides, Rusanov maximum, HLL branch) is a comparison on the values, through
which autograd passes only the selected branch. dt is a constant input.

gradient() sweeps a recorded trajectory in reverse: w_n = J(u^n)^T w_{n+1}.
"""
from __future__ import annotations

import numpy as np
import torch

from . import BURGERS, EULER1D, LINEAR, PERIODIC, Problem, flux_weights, fornberg, step_1d

_TABLES: dict = {}


def _tables(p: int):
    """gamma^{1,j}_{p,r} (g1[j][r]), gamma^{k,0}_{p,r} (gk[k][r]) and the flux
    weights gamma^{0,1/2}_{p,r} (gh[r]) of the oracle (Eqs. 2.10-2.11)."""
    if p not in _TABLES:
        n = 2 * p
        g1 = [fornberg(p, 1, float(j - p + 1)) for j in range(n)]
        gk = [fornberg(p, k, 0.0) for k in range(n)]
        _TABLES[p] = (g1, gk, flux_weights(p))
    return _TABLES[p]


def _flux(prob: Problem, u):
    """f(u) of Sec. 5 on a list of component tensors, in the oracle's order."""
    if prob.flux == LINEAR:
        return [prob.adv[0] * u[0]]
    if prob.flux == BURGERS:
        return [0.5 * u[0] * u[0]]
    rho, m, E = u
    v = m / rho
    p = (prob.gamma - 1.0) * (E - 0.5 * rho * v * v)
    return [m, m * v + p, v * (E + p)]


def _rabs(x):
    return torch.where(x < 0.0, -x, x)


def _speed(prob: Problem, u):
    if prob.flux == LINEAR:
        return torch.full_like(u[0], abs(prob.adv[0]))
    if prob.flux == BURGERS:
        return _rabs(u[0])
    rho, m, E = u
    v = m / rho
    p = (prob.gamma - 1.0) * (E - 0.5 * rho * v * v)
    return _rabs(v) + torch.sqrt(prob.gamma * p / rho)


def _eig(prob: Problem, u):
    if prob.flux == LINEAR:
        a = torch.full_like(u[0], prob.adv[0])
        return a, a
    if prob.flux == BURGERS:
        return u[0], u[0]
    rho, m, E = u
    v = m / rho
    p = (prob.gamma - 1.0) * (E - 0.5 * rho * v * v)
    c = torch.sqrt(prob.gamma * p / rho)
    return v - c, v + c


def _cat_flux(prob: Problem, p: int, us, dt: float, dx: float):
    """CAT2p flux (Eq. 2.14 by the recursion of Sec. 2.2). us[c]: tensor
    [n_if, 2p], node j = r - p + 1 in column r. Returns s tensors [n_if]."""
    g1, gk, gh = _tables(p)
    n, s = 2 * p, len(us)
    ft = _flux(prob, us)  # f~^(0)_j, [n_if, n] per component
    F = []
    for c in range(s):
        a = 0.0
        for j in range(n):
            a = a + float(gh[j]) * ft[c][:, j]
        F.append(a)
    g1t = torch.tensor(np.array(g1), dtype=torch.float64)  # [j, r]
    ut = {}
    dtk, kfact = 1.0, 1.0
    for k in range(2, n + 1):
        # (a) u~^(k-1)_j = -(sum_r g1[j][r] f~^(k-2)_r) / dx, for all j at once
        ut[k - 1] = []
        for c in range(s):
            a = 0.0
            for r in range(n):
                a = a + g1t[:, r][None, :] * ft[c][:, r:r + 1]
            ut[k - 1].append(-(a / dx))
        dtk = dtk * dt
        kfact = kfact * k
        # (b) f at the time levels, (c) the time derivative
        acc = [0.0] * s
        for rr in range(n):
            rdt = float(rr - p + 1) * dt
            st = []
            for c in range(s):
                v = us[c]
                pw, lf = 1.0, 1.0
                for ll in range(1, k):
                    pw = pw * rdt
                    lf = lf * ll
                    v = v + (pw / lf) * ut[ll][c]
                st.append(v)
            fr = _flux(prob, st)
            for c in range(s):
                acc[c] = acc[c] + float(gk[k - 1][rr]) * fr[c]
        ft = [acc[c] / dtk for c in range(s)]
        for c in range(s):
            a = 0.0
            for j in range(n):
                a = a + float(gh[j]) * ft[c][:, j]
            F[c] = F[c] + (dtk / kfact) * a
    return F


def _ratio(upw, loc):
    """r = upw / loc with the zero-jump reading (r = 1, or +-inf by sign)."""
    zero = loc == 0.0
    inf = torch.where(upw > 0.0, torch.full_like(upw, float("inf")), torch.full_like(upw, float("-inf")))
    safe = torch.where(zero, torch.ones_like(loc), loc)
    return torch.where(zero, torch.where(upw == 0.0, torch.ones_like(upw), inf), upw / safe)


def _superbee(r):
    two_r = 2.0 * r
    a = torch.where(two_r < 1.0, two_r, torch.ones_like(r))
    b = torch.where(r < 2.0, r, torch.full_like(r, 2.0))
    m = torch.where(a > b, a, b)
    return torch.where(m > 0.0, m, torch.zeros_like(m))


def _psi1(prob: Problem, line, G: int):
    """psi^1 at the interfaces of line[c] ([n_if, 2G], cell i at column G-1)."""
    ic = G - 1
    s = len(line)
    if s == 1 and prob.limiter_form == 0:
        um, u0, u1, u2 = (line[0][:, ic + d] for d in (-1, 0, 1, 2))
        r0, r1 = u0.detach(), u1.detach()
        if prob.flux == LINEAR:
            a = torch.full_like(r0, prob.adv[0])
        else:
            same = r0 == r1
            den = torch.where(same, torch.ones_like(r0), r1 - r0)
            a = torch.where(same, r0, (0.5 * r1 * r1 - 0.5 * r0 * r0) / den)
        upw = torch.where(a > 0.0, u0 - um, u2 - u1)
        return _superbee(_ratio(upw, u1 - u0))
    best = None
    for c in range(s):
        q = line[c]
        loc = q[:, ic + 1] - q[:, ic]
        pm = _superbee(_ratio(q[:, ic] - q[:, ic - 1], loc))
        pp = _superbee(_ratio(q[:, ic + 2] - q[:, ic + 1], loc))
        v = torch.where(pp < pm, pp, pm)
        best = torch.where(v < 2.0, v, torch.full_like(v, 2.0)) if best is None else torch.where(v < best, v, best)
    return best


def _flux_lo(prob: Problem, ul, ur, dt: float, dx: float):
    fl, fq = _flux(prob, ul), _flux(prob, ur)
    s = len(ul)
    if prob.lo_flux == 2:
        al, bl = _eig(prob, ul)
        ar, br = _eig(prob, ur)
        sl = torch.where(ar < al, ar, al)
        sr = torch.where(br > bl, br, bl)
        den = torch.where(sr - sl == 0.0, torch.ones_like(sl), sr - sl)
        out = []
        for c in range(s):
            mid = (sr * fl[c] - sl * fq[c] + sl * sr * (ur[c] - ul[c])) / den
            out.append(torch.where(sl >= 0.0, fl[c], torch.where(sr <= 0.0, fq[c], mid)))
        return out
    if prob.lo_flux == 1:
        alpha = dx / dt
    else:
        a_l, a_r = _speed(prob, ul), _speed(prob, ur)
        alpha = torch.where(a_r > a_l, a_r, a_l)
    return [0.5 * (fl[c] + fq[c]) - 0.5 * alpha * (ur[c] - ul[c]) for c in range(s)]


def step(prob: Problem, u: torch.Tensor, dt: float, orders) -> torch.Tensor:
    """One 1D ACAT step of u [s, nx] (torch float64) with the given order
    codes (nx + 1 values, 1 = FL-CAT2), differentiable in u."""
    N, s = prob.nx, u.shape[0]
    G = max(prob.P, 2)
    dx = (prob.x1 - prob.x0) / N
    m = np.arange(N + 1)[:, None] + np.arange(2 * G)[None, :] - G  # cells i-G+1..i+G, i = m - 1
    idx = np.mod(m, N) if prob.bc == PERIODIC else np.clip(m, 0, N - 1)
    line = [u[c][torch.from_numpy(idx)] for c in range(s)]  # [N+1, 2G]
    orders = np.asarray(orders)
    F = torch.zeros((s, N + 1), dtype=torch.float64)
    for p in sorted(set(orders.tolist())):
        sel = torch.from_numpy(np.nonzero(orders == p)[0])
        if p >= 2:
            us = [line[c][sel][:, G - p:G + p] for c in range(s)]
            Fp = _cat_flux(prob, p, us, dt, dx)
        else:
            ls = [line[c][sel] for c in range(s)]
            us = [ls[c][:, G - 1:G + 1] for c in range(s)]
            F1 = _cat_flux(prob, 1, us, dt, dx)
            ul = [ls[c][:, G - 1] for c in range(s)]
            ur = [ls[c][:, G] for c in range(s)]
            Flo = _flux_lo(prob, ul, ur, dt, dx)
            w = _psi1(prob, ls, G)
            Fp = [w * F1[c] + (1.0 - w) * Flo[c] for c in range(s)]
        for c in range(s):
            F[c, sel] = Fp[c]
    lam = dt / dx
    return torch.stack([u[c] + lam * (F[c, :-1] - F[c, 1:]) for c in range(s)])


def vjp(prob: Problem, u: np.ndarray, dt: float, w: np.ndarray) -> np.ndarray:
    """J(u)^T w of one step at fixed dt, the orders those of the C oracle at u."""
    _, _, orders = step_1d(prob, u, dt)
    ut = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float64)).requires_grad_(True)
    out = step(prob, ut, dt, orders)
    (g,) = torch.autograd.grad(out, ut, grad_outputs=torch.from_numpy(np.ascontiguousarray(w)))
    return g.numpy()


def gradient(prob: Problem, states, dts, w_last) -> np.ndarray:
    """The reverse sweep w_n = J(u^n)^T w_{n+1} over a recorded trajectory
    (states[n] = u^n, dts[n] the dt of step n); returns w_0."""
    w = np.ascontiguousarray(w_last, dtype=np.float64)
    for n in reversed(range(len(dts))):
        w = vjp(prob, states[n], float(dts[n]), w)
    return w
