"""Pins of the oracle's rectangular 2D stencils S_{p1,p2} (the end of Sec. 4:
the x-flux of order 2 p1 and the y-flux of order 2 p2 from one block of
2 p1 x 2 p2 nodes).

Reading (the paper calls the extension straightforward and gives no more):
x-derivatives on the 2 p1 nodes of a row, y-derivatives on the 2 p2 nodes of
a column, time derivatives on the 2 max(p1, p2) time nodes, the recursion to
k = 2 max(p1, p2); F^{p1} sums to k = 2 p1, G^{p2} to k = 2 p2; a direction
on FL-CAT2 counts as p = 1.

Pins: with p1 = p2 the square block of Eqs. 4.5-4.6 operation for
operation; for linear transport the closed form below, written with
numpy's polynomial algebra (no recursion); conservation of the full step.
"""
import math
from fractions import Fraction

import numpy as np
import numpy.polynomial.polynomial as npp
import pytest

from paper_2007_01416_gb300 import workloads as W


def _tensor_interpolant(vals, xs, ys):
    """Coefficients c[i, j] of sum c_ij x^i y^j interpolating vals[b, a] at (xs[a], ys[b])."""
    V = np.array([[x ** i * y ** j for i in range(len(xs)) for j in range(len(ys))]
                  for y in ys for x in xs])
    c = np.linalg.solve(V, vals.reshape(-1))
    return c.reshape(len(xs), len(ys))


def _flux_weights(p):
    """Weights w_m of the numerical flux on the 2p nodes -p+1..p fixed by
    Eq. 2.11 at k = 1: (F_{i+1/2} - F_{i-1/2}) reproduces the centred
    (2p+1)-point first derivative, so w_m = -(d_{-p} + ... + d_{m-p})."""
    cen = [Fraction(j) for j in range(-p, p + 1)]
    d = []
    for j, xj in enumerate(cen):  # derivative at 0 of the Lagrange basis polynomial of node j
        others = [xm for m, xm in enumerate(cen) if m != j]
        den = math.prod(xj - xm for xm in others)
        d.append(sum(math.prod(-xm for xm in others if xm is not skip) for skip in others) / den)
    w, acc = [], Fraction(0)
    for m in range(2 * p):
        acc -= d[m]
        w.append(float(acc))
    return w


def _transport_flux(c, a, b, dt, m_max, pts, w, speed):
    """speed * sum_{m=0}^{m_max} dt^m/(m+1)! sum_l w_l [(-a d/dx - b d/dy)^m Pi](pts_l)."""
    total, term = 0.0, c.copy()
    for m in range(m_max + 1):
        val = sum(wl * npp.polyval2d(x, y, term) for wl, (x, y) in zip(w, pts))
        total += dt ** m / math.factorial(m + 1) * val
        dx_ = npp.polyder(term, axis=0) if term.shape[0] > 1 else np.zeros((1, term.shape[1]))
        dy_ = npp.polyder(term, axis=1) if term.shape[1] > 1 else np.zeros((term.shape[0], 1))
        nxt = np.zeros_like(term)
        nxt[:dx_.shape[0], :dx_.shape[1]] -= a * dx_
        nxt[:dy_.shape[0], :dy_.shape[1]] -= b * dy_
        term = nxt
    return speed * total


@pytest.mark.parametrize("p1,p2", [(1, 2), (2, 1), (2, 3), (3, 2), (3, 4), (4, 2), (4, 1), (2, 4), (3, 3)])
def test_rect_linear_transport_closed_form(oracle, p1, p2):
    """For f = a u, g = b u the recursion differentiates the tensor-product
    interpolant Pi of the block exactly (the node derivatives of a row or a
    column are exact on it), and the time derivatives of its Taylor
    polynomials are exact, so with the flux weights w of Eq. 2.11
    F^{p1} = a sum_{m < 2 p1} dt^m/(m+1)! sum_l w_l [(-a d_x - b d_y)^m Pi](x_l, y_0)
    over the nodes of the row j2 = 0, and likewise G^{p2} over the column
    j1 = 0."""
    a, b = 0.7, -0.45
    pr = oracle.Problem(flux=oracle.LINEAR, P=4, nx=40, ny=25, adv=(a, b), x1=1.0, y1=1.0)
    dx, dy = pr.dx, pr.dy
    rng = np.random.default_rng(10 * p1 + p2)
    blk = rng.normal(size=(1, 2 * p2, 2 * p1))
    dt = 0.3 * min(dx, dy)
    F, G = oracle.cat_flux_2d_rect(pr, p1, p2, blk, dt)
    xs = (np.arange(2 * p1) - p1 + 1) * dx
    ys = (np.arange(2 * p2) - p2 + 1) * dy
    c = _tensor_interpolant(blk[0], xs, ys)
    Fref = _transport_flux(c, a, b, dt, 2 * p1 - 1, [(x, 0.0) for x in xs], _flux_weights(p1), a)
    Gref = _transport_flux(c, a, b, dt, 2 * p2 - 1, [(0.0, y) for y in ys], _flux_weights(p2), b)
    scale = np.abs(blk).max() * max(abs(a), abs(b))
    assert abs(F[0] - Fref) < 1e-10 * scale, (F[0], Fref)
    assert abs(G[0] - Gref) < 1e-10 * scale, (G[0], Gref)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_rect_equals_square_when_orders_agree(oracle, p):
    c = W.euler2d_smooth(n=12, seed=3, P=4)
    pr = oracle.Problem(**c.problem_kwargs())
    rng = np.random.default_rng(p)
    rho = 1.0 + 0.1 * rng.random((2 * p, 2 * p))
    vx, vy, pre = 0.2 * rng.random((3, 2 * p, 2 * p))
    blk = W.prim_to_cons_2d(rho, vx, vy, 1.0 + pre)
    a = oracle.cat_flux_2d(pr, p, blk, 1e-3)
    b = oracle.cat_flux_2d_rect(pr, p, p, blk, 1e-3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_rect_step_conserves_and_differs_from_square(oracle):
    """Periodic 2D Euler data smooth in x and with a density jump in y: the
    anchors near the jump take p2 < p1, where the rectangular block changes
    the x-flux; the step still conserves every component to round-off."""
    n = 24
    x = W.centres(n, 0.0, 1.0)
    X, Y = np.meshgrid(x, x)
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * X) + 0.5 * (np.abs(Y - 0.5) < 0.25)
    u = W.prim_to_cons_2d(rho, 0.3 + 0 * rho, 0.1 + 0 * rho, 1.0 + 0 * rho)
    kw = dict(flux=oracle.EULER2D, P=3, nx=n, ny=n, bc=0, cfl=0.4)
    pr_r = oracle.Problem(**kw, rect_2d=1)
    pr_s = oracle.Problem(**kw)
    dt = oracle.dt_cfl(pr_s, u)
    ur, _, oxr, oyr = oracle.step_2d(pr_r, u, dt)
    us, _, oxs, oys = oracle.step_2d(pr_s, u, dt)
    assert np.array_equal(oxr, oxs) and np.array_equal(oyr, oys)  # orders do not depend on the stencil
    assert np.abs(ur - us).max() > 1e-8  # the x-fluxes beside the jump changed
    for c in range(4):
        assert abs(ur[c].sum() - u[c].sum()) < 1e-12 * np.abs(u[c]).sum()


@pytest.mark.parametrize("seed", [0, 2])
def test_rect_keeps_four_quadrant_data_physical_at_P4(oracle, seed):
    """With square blocks the row and column indicators do not see a jump
    that crosses the 2p x 2p block transversally, and four-quadrant Euler
    data at P = 4 goes non-physical in the first step; the rectangular block
    follows the transverse order and the run stays physical."""
    c = W.euler2d_quadrants(n=32, seed=seed, P=4)

    def physical(u):
        rho = u[0]
        p = 0.4 * (u[3] - 0.5 * (u[1] ** 2 + u[2] ** 2) / rho)
        return bool(np.all(rho > 0) and np.all(p > 0) and np.all(np.isfinite(u)))

    sq, _, _, _ = oracle.step_2d(oracle.Problem(**c.problem_kwargs()), c.u0)
    assert not physical(sq)
    pr = oracle.Problem(**dict(c.problem_kwargs(), rect_2d=1))
    u = c.u0
    for _ in range(10):
        u, _, _, _ = oracle.step_2d(pr, u)
        assert physical(u)
