"""Exact solution of the Riemann problem for the 1D Euler equations of an
ideal gas (the reference solutions of Sec. 5.3).

TEST INFRASTRUCTURE: used only by the test suite to score oracle runs on
Riemann data. Written from the classical wave analysis of gas dynamics: a
pressure function per side (shock branch from the Rankine-Hugoniot
conditions, rarefaction branch from the isentropic relation and the
Riemann invariant), Newton's method for the star pressure, then sampling of
the self-similar solution at x/t.
"""
from __future__ import annotations

import math

import numpy as np


def sound(rho: float, p: float, g: float) -> float:
    return math.sqrt(g * p / rho)


def _side(p: float, rk: float, pk: float, g: float):
    """Velocity jump f_K(p) across the wave facing side K and its derivative."""
    ck = sound(rk, pk, g)
    if p > pk:  # shock: Rankine-Hugoniot
        A = 2.0 / ((g + 1.0) * rk)
        B = (g - 1.0) / (g + 1.0) * pk
        q = math.sqrt(A / (p + B))
        f = (p - pk) * q
        df = q * (1.0 - 0.5 * (p - pk) / (p + B))
    else:  # rarefaction: isentropic + Riemann invariant
        e = (g - 1.0) / (2.0 * g)
        f = 2.0 * ck / (g - 1.0) * ((p / pk) ** e - 1.0)
        df = (1.0 / (rk * ck)) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g: float = 1.4, tol: float = 1e-14):
    """(p*, u*) between the two nonlinear waves."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = sound(rl, pl, g), sound(rr, pr, g)
    if 2.0 / (g - 1.0) * (cl + cr) <= ur - ul:
        raise ValueError("initial data generate vacuum")
    # two-rarefaction estimate as the starting guess (always positive)
    e = (g - 1.0) / (2.0 * g)
    p = ((cl + cr - 0.5 * (g - 1.0) * (ur - ul)) / (cl / pl ** e + cr / pr ** e)) ** (1.0 / e)
    p = max(p, 1e-14)
    for _ in range(200):
        fl, dl = _side(p, rl, pl, g)
        fr, dr = _side(p, rr, pr, g)
        F = fl + fr + (ur - ul)
        pn = p - F / (dl + dr)
        if pn <= 0.0:
            pn = 0.5 * p
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _side(p, rl, pl, g)
    fr, _ = _side(p, rr, pr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, xi, g: float = 1.4):
    """Primitive state (rho, u, p) at similarity coordinates xi = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, g)
    cl, cr = sound(rl, pl, g), sound(rr, pr, g)
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    out = np.zeros((3, xi.size))
    gm = (g - 1.0) / (g + 1.0)
    for n, s in enumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                SL = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
                if s <= SL:
                    st = (rl, ul, pl)
                else:
                    st = (rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps)
            else:  # left rarefaction
                rs = rl * (ps / pl) ** (1.0 / g)
                cs = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
                if s <= ul - cl:
                    st = (rl, ul, pl)
                elif s >= us - cs:
                    st = (rs, us, ps)
                else:
                    c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
                    u = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    r = rl * (c / cl) ** (2.0 / (g - 1.0))
                    st = (r, u, pl * (c / cl) ** (2.0 * g / (g - 1.0)))
        else:  # right of the contact
            if ps > pr:  # right shock
                SR = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
                if s >= SR:
                    st = (rr, ur, pr)
                else:
                    st = (rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps)
            else:  # right rarefaction
                rs = rr * (ps / pr) ** (1.0 / g)
                cs = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
                if s >= ur + cr:
                    st = (rr, ur, pr)
                elif s <= us + cs:
                    st = (rs, us, ps)
                else:
                    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
                    u = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    r = rr * (c / cr) ** (2.0 / (g - 1.0))
                    st = (r, u, pr * (c / cr) ** (2.0 * g / (g - 1.0)))
        out[:, n] = st
    return out


def cell_averages(left, right, x0: float, t: float, edges, g: float = 1.4, sub: int = 16):
    """Cell averages of the exact primitive solution (midpoint sub-sampling)."""
    edges = np.asarray(edges, dtype=np.float64)
    N = edges.size - 1
    w = (np.arange(sub) + 0.5) / sub
    xs = (edges[:-1, None] + (edges[1:] - edges[:-1])[:, None] * w[None, :]).ravel()
    prim = sample(left, right, (xs - x0) / t, g).reshape(3, N, sub)
    return prim.mean(axis=2)
