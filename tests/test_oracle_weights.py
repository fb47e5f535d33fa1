"""Pins the oracle's differentiation weights (Eq. 2.10) to exact rational
solutions of the moment (Vandermonde) conditions: a formula on nodes x_r that
gives the k-th derivative at q exactly for polynomials of degree < 2p must
satisfy sum_r w_r (x_r - q)^m / m! = [m == k] for m = 0..2p-1."""
from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest


def exact_weights(p: int, k: int, q: Fraction):
    nodes = [Fraction(r) for r in range(-p + 1, p + 1)]
    n = len(nodes)
    A = [[(x - q) ** m / factorial(m) for x in nodes] for m in range(n)]
    b = [Fraction(int(m == k)) for m in range(n)]
    # Gauss-Jordan elimination in exact arithmetic
    M = [row[:] + [b[i]] for i, row in enumerate(A)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        M[col] = [v / pv for v in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [a - f * c for a, c in zip(M[r], M[col])]
    return [M[i][n] for i in range(n)]


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_fornberg_matches_exact_rationals(oracle, p):
    qs = [Fraction(j) for j in range(-p + 1, p + 1)] + [Fraction(0), Fraction(1, 2)]
    for k in range(0, 2 * p):
        for q in qs:
            w = oracle.fornberg(p, k, float(q))
            ex = exact_weights(p, k, q)
            for a, e in zip(w, ex):
                assert abs(a - float(e)) <= 4e-15 * max(1.0, abs(float(e))), (p, k, q, a, e)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_highest_derivative_is_binomial_difference(oracle, p):
    # gamma^{2p-1,1/2}_{p,.} is the (2p-1)-th undivided difference (Eq. 3.12):
    # (-1)^(2p-1-m) C(2p-1, m); the oracle must reproduce it exactly because the
    # indicator decisions are compared bit for bit.
    w = oracle.fornberg(p, 2 * p - 1, 0.5)
    ex = np.array([(-1) ** (2 * p - 1 - m) * comb(2 * p - 1, m) for m in range(2 * p)], float)
    assert np.array_equal(w, ex)
    # ... and it is the same for every evaluation point q
    for q in (-0.3, 0.0, 1.7):
        assert np.allclose(oracle.fornberg(p, 2 * p - 1, q), ex, rtol=0, atol=1e-11)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_flux_weights_satisfy_eq_2_11(oracle, p):
    # gamma^{0,1/2}: the weights with D^1_{p,i} = (A_{p,i} - A_{p,i-1}) / dx
    # (Eq. 2.11, k = 1), D^1_p the exact (2p+1)-point centred first derivative.
    cen = [Fraction(j) for j in range(-p, p + 1)]
    d = exact_weights_on(cen, 1, Fraction(0))
    w = oracle.flux_weights(p)
    ex, s = [], Fraction(0)
    for m in range(2 * p):
        s -= d[m]
        ex.append(s)
    for a, e in zip(w, ex):
        assert abs(a - float(e)) <= 1e-15 * max(1.0, abs(float(e)))
    # the shifted difference reproduces d exactly (telescoping check)
    diff = [Fraction(0)] * (2 * p + 1)
    for m, e in enumerate(ex):
        diff[m + 1] += e
        diff[m] -= e
    assert diff == d
    # symmetric, sums to one (consistency: constant flux passes unchanged)
    assert np.allclose(w, w[::-1], rtol=0, atol=1e-15)
    assert sum(ex) == 1


def exact_weights_on(nodes, k, q):
    n = len(nodes)
    A = [[(x - q) ** m / factorial(m) for x in nodes] for m in range(n)]
    M = [row[:] + [Fraction(int(m == k))] for m, row in enumerate(A)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        M[col] = [v / pv for v in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [a - f * c for a, c in zip(M[r], M[col])]
    return [M[i][n] for i in range(n)]


def test_interpolation_weights_midpoint_symmetry(oracle):
    for p in range(1, 5):
        w = oracle.fornberg(p, 0, 0.5)
        assert np.allclose(w, w[::-1], rtol=0, atol=1e-16)
        assert abs(w.sum() - 1.0) < 1e-15
