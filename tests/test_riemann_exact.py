"""Pins the exact Riemann solver (test infrastructure for Sec. 5.3) to the
physics it must satisfy, independently of the formulas inside it:
Rankine-Hugoniot conditions across shocks, constant entropy and Riemann
invariant across rarefactions, continuity of u and p at the contact, and
integral conservation of mass, momentum and energy over the wave fan."""
import math

import numpy as np
import pytest

from oracle import riemann
from paper_2007_01416_gb300 import workloads as W

G = 1.4


def cons(prim):
    rho, u, p = prim
    return np.array([rho, rho * u, p / (G - 1) + 0.5 * rho * u * u])


def flux(prim):
    rho, u, p = prim
    E = p / (G - 1) + 0.5 * rho * u * u
    return np.array([rho * u, rho * u * u + p, u * (E + p)])


CASES = list(W.RIEMANN_1D.values()) + [((0.4, 0.3, 0.8), (0.9, -0.2, 0.2)),
                                       ((0.2, -0.4, 0.15), (0.7, 0.45, 0.95))]


@pytest.mark.parametrize("left,right", CASES)
def test_wave_conditions(left, right):
    ps, us = riemann.star_state(left, right, G)
    for side, st in ((-1, left), (1, right)):
        rk, uk, pk = st
        if ps > pk:  # shock: Rankine-Hugoniot for all three conservation laws
            # star density from the sampled solution just behind the shock
            xi = np.linspace(min(uk, us) - 50, max(uk, us) + 50, 200001)
            prof = riemann.sample(left, right, xi, G)
            sel = (np.abs(prof[2] - ps) < 1e-12 * ps) & ((xi - us) * side > 0)
            rs = prof[0][sel][0 if side < 0 else -1]
            qs = (rs, us, ps)
            S = (rs * us - rk * uk) / (rs - rk)
            jump_u = cons(qs) - cons(st)
            jump_f = flux(qs) - flux(st)
            assert np.allclose(S * jump_u, jump_f, rtol=1e-9, atol=1e-9 * max(1, pk))
        else:  # rarefaction: isentropic, Riemann invariant conserved
            rs = rk * (ps / pk) ** (1 / G)
            assert abs(ps / rs ** G - pk / rk ** G) < 1e-12 * pk / rk ** G
            ck, cs = math.sqrt(G * pk / rk), math.sqrt(G * ps / rs)
            inv_k = uk - side * 2 * ck / (G - 1)
            inv_s = us - side * 2 * cs / (G - 1)
            assert abs(inv_k - inv_s) < 1e-10 * (1 + abs(inv_k))


@pytest.mark.parametrize("left,right", CASES)
def test_integral_conservation(left, right):
    # int (U(x,t) - U(x,0)) dx over [-L, L] = t (F(left) - F(right))
    t, L, n = 1.0, 200.0, 400001
    x = np.linspace(-L, L, n)
    prof = riemann.sample(left, right, x / t, G)
    U = cons(prof)
    U0 = np.where(x < 0, cons(np.array(left)[:, None] * np.ones(n)),
                  cons(np.array(right)[:, None] * np.ones(n)))
    dx = x[1] - x[0]
    lhs = ((U - U0)[:, :-1] + (U - U0)[:, 1:]).sum(axis=1) * 0.5 * dx
    rhs = t * (flux(left) - flux(right))
    scale = np.abs(flux(left)).max() + np.abs(flux(right)).max() + np.abs(cons(left)).max()
    assert np.allclose(lhs, rhs, rtol=0, atol=2e-3 * scale), (lhs, rhs)


def test_uniform_state_is_fixed():
    st = (0.6, 0.2, 0.7)
    prof = riemann.sample(st, st, np.linspace(-3, 3, 101), G)
    assert np.allclose(prof, np.array(st)[:, None], rtol=1e-12)
