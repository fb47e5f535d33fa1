"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test targets a part of the oracle with an independent statement (a closed
form, an invariant or an exact solution), so that a dropped term, a wrong sign
or index, or a transposed operand in the oracle fails at least one of them.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2007_01416_gb300 import workloads as W


def prob(oracle, **kw):
    return oracle.Problem(**kw)


# ---------------------------------------------------------------------------
# CAT2 closed forms (Eqs. 2.16-2.17 and Eqs. 4.3-4.4)
# ---------------------------------------------------------------------------
def _euler_flux(u, g=1.4):
    rho, m, E = u
    v = m / rho
    p = (g - 1.0) * (E - 0.5 * rho * v * v)
    return np.array([m, m * v + p, v * (E + p)])


@pytest.mark.parametrize("flux", ["burgers", "euler"])
def test_cat2_closed_form(oracle, flux):
    rng = np.random.default_rng(1)
    for _ in range(50):
        if flux == "burgers":
            pr = prob(oracle, flux=oracle.BURGERS, P=1, nx=10)
            st = rng.uniform(-1, 1, size=(1, 2))
            f = lambda u: 0.5 * u * u  # noqa: E731
        else:
            pr = prob(oracle, flux=oracle.EULER1D, P=1, nx=10)
            rho = rng.uniform(0.5, 1.5, 2)
            vel = rng.uniform(-0.5, 0.5, 2)
            pre = rng.uniform(0.5, 1.5, 2)
            st = W.prim_to_cons_1d(rho, vel, pre)
            f = _euler_flux
        dt = 0.3 * pr.dx
        lam = dt / pr.dx
        F = oracle.cat_flux_1d(pr, 1, st, dt)
        u0, u1 = st[:, 0], st[:, 1]
        f0, f1 = f(u0), f(u1)
        ft0 = f(u0 - lam * (f1 - f0))
        ft1 = f(u1 - lam * (f1 - f0))
        ref = 0.25 * (ft1 + ft0 + f1 + f0)
        assert np.allclose(F, ref, rtol=1e-14, atol=1e-15)


def test_cat2_2d_closed_form(oracle):
    rng = np.random.default_rng(2)
    g = 1.4
    pr = prob(oracle, flux=oracle.EULER2D, P=1, nx=10, ny=10)

    def fx(u):
        rho, mx, my, E = u
        v, w = mx / rho, my / rho
        p = (g - 1) * (E - 0.5 * rho * (v * v + w * w))
        return np.array([mx, mx * v + p, mx * w, v * (E + p)])

    def fy(u):
        rho, mx, my, E = u
        v, w = mx / rho, my / rho
        p = (g - 1) * (E - 0.5 * rho * (v * v + w * w))
        return np.array([my, my * v, my * w + p, w * (E + p)])

    for _ in range(30):
        rho = rng.uniform(0.5, 1.5, (2, 2))
        vx = rng.uniform(-0.5, 0.5, (2, 2))
        vy = rng.uniform(-0.5, 0.5, (2, 2))
        pre = rng.uniform(0.5, 1.5, (2, 2))
        blk = W.prim_to_cons_2d(rho, vx, vy, pre)  # [c, b(y), a(x)]
        dt = 0.2 * pr.dx
        F, G = oracle.cat_flux_2d(pr, 1, blk, dt)
        u = lambda a, b: blk[:, b, a]  # noqa: E731  node (j1=a, j2=b)
        dx, dy = pr.dx, pr.dy
        u1_00 = -(fx(u(1, 0)) - fx(u(0, 0))) / dx - (fy(u(0, 1)) - fy(u(0, 0))) / dy
        u1_10 = -(fx(u(1, 0)) - fx(u(0, 0))) / dx - (fy(u(1, 1)) - fy(u(1, 0))) / dy
        u1_01 = -(fx(u(1, 1)) - fx(u(0, 1))) / dx - (fy(u(0, 1)) - fy(u(0, 0))) / dy
        Fr = 0.25 * (fx(u(0, 0) + dt * u1_00) + fx(u(1, 0) + dt * u1_10) + fx(u(0, 0)) + fx(u(1, 0)))
        Gr = 0.25 * (fy(u(0, 0) + dt * u1_00) + fy(u(0, 1) + dt * u1_01) + fy(u(0, 0)) + fy(u(0, 1)))
        assert np.allclose(F, Fr, rtol=1e-13, atol=1e-14)
        assert np.allclose(G, Gr, rtol=1e-13, atol=1e-14)


# ---------------------------------------------------------------------------
# Linear flux: CAT2p is the 2p-order Lax-Wendroff scheme (Sec. 2.2)
# ---------------------------------------------------------------------------
def _lagrange_basis_at(nodes, x):
    out = []
    for j, xj in enumerate(nodes):
        v = Fraction(1)
        for m, xm in enumerate(nodes):
            if m != j:
                v *= (x - xm) / (xj - xm)
        out.append(v)
    return out


def _basis_poly(nodes, j):
    """Exact coefficients (ascending) of the j-th Lagrange basis polynomial."""
    poly, den = [Fraction(1)], Fraction(1)
    for m, xm in enumerate(nodes):
        if m == j:
            continue
        poly = [Fraction(0)] + poly
        for q in range(len(poly) - 1):
            poly[q] -= xm * poly[q + 1]
        den *= nodes[j] - xm
    return [c / den for c in poly]


def _deriv_at(poly, k, x):
    from math import factorial
    return sum(c * Fraction(factorial(d), factorial(d - k)) * x ** (d - k)
               for d, c in enumerate(poly) if d >= k)


def _linear_flux_coeffs(p, nu, a):
    """Exact flux coefficients of CAT2p for f = a u: with f = a u every local
    time derivative is exact on the interpolant Pi of u on S_p, so
    f~^{(k-1)}_j = a (-a)^{k-1} Pi^{(k-1)}(x_j) and
    F = sum_k dt^{k-1}/k! sum_j w_j f~^{(k-1)}_j, w the flux weights fixed by
    Eq. 2.11 (k = 1) from the centred first derivative (unit dx, dt = nu/a)."""
    from math import factorial
    nodes = [Fraction(r) for r in range(-p + 1, p + 1)]
    cen = [Fraction(j) for j in range(-p, p + 1)]
    d = [_deriv_at(_basis_poly(cen, j), 1, Fraction(0)) for j in range(2 * p + 1)]
    w, s = [], Fraction(0)
    for m in range(2 * p):
        s -= d[m]
        w.append(s)
    dt = nu / a
    cF = [Fraction(0)] * (2 * p)
    basis = [_basis_poly(nodes, r) for r in range(2 * p)]
    for k in range(1, 2 * p + 1):
        for jj, xj in enumerate(nodes):
            for r in range(2 * p):
                cF[r] += (dt ** (k - 1) / factorial(k) * w[jj] * a * (-a) ** (k - 1)
                          * _deriv_at(basis[r], k - 1, xj))
    return cF


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_linear_flux_closed_form(oracle, p):
    rng = np.random.default_rng(10 + p)
    a = Fraction(7, 10)
    pr = prob(oracle, flux=oracle.LINEAR, P=p, nx=16, adv=(float(a), 0.0), x0=0, x1=16)
    nu = Fraction(3, 10)
    dt = float(nu / a)  # dx = 1
    cs = _linear_flux_coeffs(p, nu, a)
    for _ in range(20):
        st = rng.normal(size=(1, 2 * p))
        F = oracle.cat_flux_1d(pr, p, st, dt)
        ref = sum(float(c) * st[0, j] for j, c in enumerate(cs))
        assert abs(F[0] - ref) <= 2e-14 * max(1.0, np.abs(st).max())


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_linear_update_is_lax_wendroff(oracle, p):
    # u_i^{n+1} = sum_{j=-p}^{p} L_j(-nu) u_{i+j}: the (2p+1)-point Lax-Wendroff
    # update (interpolation at the foot of the characteristic).
    N = 256
    a = 1.0
    pr = prob(oracle, flux=oracle.LINEAR, P=p, nx=N, adv=(a, 0.0), x0=0.0, x1=2.0, bc=0)
    x = W.centres(N, 0.0, 2.0)
    u = (0.5 * np.sin(math.pi * x) + 0.2 * np.cos(3 * math.pi * x))[None, :]
    nu = Fraction(9, 10)
    dt = float(nu) * pr.dx / a
    un, _, orders = oracle.step_1d(pr, u, dt)
    L = [float(v) for v in _lagrange_basis_at([Fraction(j) for j in range(-p, p + 1)], -nu)]
    ref = sum(L[j + p] * np.roll(u[0], -j) for j in range(-p, p + 1))
    full = (orders[:-1] == max(p, 1)) & (orders[1:] == max(p, 1)) if p >= 2 else np.ones(N, bool)
    if p == 1:
        # P = 1 is FL-CAT2: where the limiter is 1 it is CAT2 = LW2
        _, _, _, psi = oracle.step_1d(pr, u, dt, want_psi=True)
        full = (psi[:-1, 0] == 1.0) & (psi[1:, 0] == 1.0)
    assert full.sum() > (N // 2 if p >= 2 else 8)
    assert np.allclose(un[0][full], ref[full], rtol=0, atol=1e-14)


# ---------------------------------------------------------------------------
# Conservation (Eq. 2.12 / Eq. 3.19) on periodic data
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["burgers", "euler"])
def test_discrete_conservation(oracle, case):
    if case == "burgers":
        c = W.burgers_sine(nx=200, seed=3, P=3)
        pr = prob(oracle, **c.problem_kwargs())
        u = c.u0
        nsteps = 60
    else:
        c = W.acoustic_pulse(nx=256, seed=4, P=3)
        pr = prob(oracle, **c.problem_kwargs())
        u = c.u0
        nsteps = 20
    scale = np.abs(u).max()
    for _ in range(nsteps):
        un, dt, _ = oracle.step_1d(pr, u)
        for comp in range(u.shape[0]):
            s0 = math.fsum(u[comp])
            s1 = math.fsum(un[comp])
            assert abs(s1 - s0) <= 64 * u.shape[1] * 2.2e-16 * scale
        u = un


# ---------------------------------------------------------------------------
# Indicators (Sec. 3.2) and the limiter fallback (Eq. 3.4)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("P", [2, 3, 4])
def test_constant_state_selects_P_and_is_fixed(oracle, P):
    pr = prob(oracle, flux=oracle.EULER1D, P=P, nx=40, bc=1)
    # dyadic conserved values: the binomial differences of tau_p vanish exactly
    u = np.stack([np.full(40, 0.75), np.full(40, 0.25), np.full(40, 2.5)])
    un, dt, orders, psi = oracle.step_1d(pr, u, want_psi=True)
    assert np.all(orders == P)
    assert np.all(psi[:, 1:] == 1.0)  # tau = 0 exactly, I = eps/2 > 0
    assert np.array_equal(un, u)


@pytest.mark.parametrize("P", [2, 3, 4])
def test_jump_falls_back_to_first_order(oracle, P):
    N = 40
    c = W.riemann_1d("sod", N, P)
    pr = prob(oracle, **c.problem_kwargs())
    un, dt, orders, psi, F = oracle.step_1d(pr, c.u0, want_psi=True, want_flux=True)
    m = N // 2  # interface between cells m-1 and m holds the jump
    # every stencil S_p, p >= 2, containing the jump rejects it
    assert np.all(orders[m - 1:m + 2] == 1)
    # stencils that do not reach the jump see constant data: order P
    far = np.r_[0:m - P + 1, m + P:N + 1]
    assert np.all(orders[far] == P)
    # at the jump interface r = 0, psi^1 = superbee(0) = 0: F = F^lo exactly
    assert psi[m, 0] == 0.0
    ul, ur = c.u0[:, m - 1], c.u0[:, m]
    fl, fr = _euler_flux(ul), _euler_flux(ur)

    def speed(u):
        rho, mm, E = u
        v = mm / rho
        p = 0.4 * (E - 0.5 * rho * v * v)
        return abs(v) + math.sqrt(1.4 * p / rho)

    alpha = max(speed(ul), speed(ur))
    Flo = 0.5 * (fl + fr) - 0.5 * alpha * (ur - ul)
    assert np.allclose(F[m], Flo, rtol=1e-15, atol=1e-15)


def test_indicator_invariances(oracle):
    # with eps = 0, psi^p depends on the samples only up to a positive scale
    # and an additive constant (Sec. 3.2, homothetic invariance)
    rng = np.random.default_rng(5)
    N = 48
    x = W.centres(N, 0.0, 1.0)
    u = (np.sin(2 * math.pi * x) + 0.3 * np.sign(x - 0.37))[None, :] + 0.01 * rng.normal(size=(1, N))
    pr = prob(oracle, flux=oracle.LINEAR, P=4, nx=N, adv=(1.0, 0.0), eps=0.0, bc=0)
    _, _, o0, psi0 = oracle.step_1d(pr, u, 1e-3, want_psi=True)
    for alpha, shift in [(3.7, 0.0), (0.01, 0.0), (1.0, 5.0), (250.0, -2.0)]:
        _, _, o1, psi1 = oracle.step_1d(pr, alpha * u + shift, 1e-3, want_psi=True)
        assert np.allclose(psi1[:, 1:], psi0[:, 1:], rtol=1e-9, atol=1e-12)
    # the transport direction is irrelevant to psi^p
    pr2 = prob(oracle, flux=oracle.LINEAR, P=4, nx=N, adv=(-1.0, 0.0), eps=0.0, bc=0)
    _, _, _, psi2 = oracle.step_1d(pr2, u, 1e-3, want_psi=True)
    assert np.array_equal(psi2[:, 1:], psi0[:, 1:])


def test_indicator_asymptotics(oracle):
    # Prop. 3.1: smooth data, no critical point: 1 - psi^p = O(dx^{4(p-1)});
    # a jump in S_p: psi^p = O(dx^2). Measured by the log-log slope.
    def psi_at(N, data, p):
        x = W.centres(N, 0.0, 1.0)
        u = data(x)[None, :]
        pr = prob(oracle, flux=oracle.LINEAR, P=p, nx=N, adv=(1.0, 0.0), eps=0.0,
                  tau_factorial=1, bc=1)
        _, _, _, psi = oracle.step_1d(pr, u, 1e-6, want_psi=True)
        return psi

    smooth = lambda x: np.exp(x)  # noqa: E731  (no critical point)
    for p in (2, 3):
        errs = []
        for N in (64, 128):
            psi = psi_at(N, smooth, p)
            errs.append(1.0 - psi[N // 2, p - 1])
        slope = math.log2(errs[0] / errs[1])
        assert slope > 4 * (p - 1) - 0.6, (p, errs, slope)
    jump = lambda x: np.exp(x) + (x > 0.5)  # noqa: E731
    for p in (2, 3):
        vals = []
        for N in (64, 128, 256):
            psi = psi_at(N, jump, p)
            vals.append(psi[N // 2, p - 1])  # jump inside the stencil
        slope = math.log2(vals[1] / vals[2])
        assert abs(slope - 2.0) < 0.3, (p, vals, slope)


# ---------------------------------------------------------------------------
# Accuracy: order 2p on smooth solutions (Sec. 2.2, Sec. 3.3)
# ---------------------------------------------------------------------------
def _rate(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def _burgers_exact(x, t, a, b, phi):
    # u = u0(x - u t) solved by Newton (before shock formation)
    u = a + b * np.sin(math.pi * x + phi)
    for _ in range(100):
        xi = x - u * t
        g = u - (a + b * np.sin(math.pi * xi + phi))
        dg = 1.0 + b * math.pi * np.cos(math.pi * xi + phi) * t
        u = u - g / dg
    return u


@pytest.mark.parametrize("P", [2, 3])
def test_local_error_order_burgers(oracle, P):
    # one step from exact point values: where both interfaces of a cell use
    # CAT2P the local error is O(dx^{2P+1}) (order 2P, Sec. 2.2)
    rng = np.random.default_rng(0)
    a, b, phi = rng.uniform(0.2, 0.5), rng.uniform(0.5, 1.0), rng.uniform(0, 2 * math.pi)
    errs = []
    Ns = (40, 80, 160) if P == 2 else (40, 60, 90)
    for N in Ns:
        pr = prob(oracle, flux=oracle.BURGERS, P=P, nx=N, x0=-1.0, x1=1.0, cfl=0.5, bc=0)
        x = W.centres(N, -1.0, 1.0)
        u0 = (a + b * np.sin(math.pi * x + phi))[None, :]
        un, dt, orders = oracle.step_1d(pr, u0)
        full = (orders[:-1] == P) & (orders[1:] == P)
        assert full.mean() > 0.75
        errs.append(np.abs(un[0] - _burgers_exact(x, dt, a, b, phi))[full].max())
    rates = [math.log(errs[i] / errs[i + 1]) / math.log(Ns[i + 1] / Ns[i]) for i in range(2)]
    assert rates[-1] > 2 * P + 1 - 0.6, (errs, rates)


@pytest.mark.parametrize("P", [2, 3])
def test_local_error_order_euler(oracle, P):
    # entropy wave rho = 1 + 0.2 sin(2 pi x), u = 1, p = 1: exact rho(x - t)
    errs = []
    Ns = (40, 80, 160) if P == 2 else (40, 60, 90)
    for N in Ns:
        pr = prob(oracle, flux=oracle.EULER1D, P=P, nx=N, cfl=0.4, bc=0)
        x = W.centres(N, 0.0, 1.0)
        u0 = W.prim_to_cons_1d(1 + 0.2 * np.sin(2 * math.pi * x), np.ones(N), np.ones(N))
        un, dt, orders = oracle.step_1d(pr, u0)
        full = (orders[:-1] == P) & (orders[1:] == P)
        assert full.mean() > 0.75
        ex = 1 + 0.2 * np.sin(2 * math.pi * (x - dt))
        errs.append(np.abs(un[0] - ex)[full].max())
    rates = [math.log(errs[i] / errs[i + 1]) / math.log(Ns[i + 1] / Ns[i]) for i in range(2)]
    assert rates[-1] > 2 * P + 1 - 0.6, (errs, rates)


@pytest.mark.parametrize("P", [3, 4])
def test_global_order_linear_transport(oracle, P):
    # u_t + u_x = 0, u0 = sin(pi x)/2 on [0, 2], periodic (Eq. 5.2), CFL 0.9
    T = 0.5
    errs = []
    Ns = (64, 128, 256) if P == 3 else (64, 96, 128)
    for N in Ns:
        pr = prob(oracle, flux=oracle.LINEAR, P=P, nx=N, adv=(1.0, 0.0), x0=0.0, x1=2.0,
                  cfl=0.9, bc=0)
        x = W.centres(N, 0.0, 2.0)
        u0 = 0.5 * np.sin(math.pi * x)[None, :]
        u, t = oracle.run_1d(pr, u0, 10 ** 6, t_end=T)
        assert abs(t - T) < 1e-12
        errs.append(np.abs(u[0] - 0.5 * np.sin(math.pi * (x - T))).mean())
    rates = [math.log(errs[i] / errs[i + 1]) / math.log(Ns[i + 1] / Ns[i])
             for i in range(len(errs) - 1)]
    assert rates[-1] > 2 * P - 0.5, (errs, rates)


def test_global_order_burgers_before_shock(oracle):
    rng = np.random.default_rng(0)
    a, b, phi = rng.uniform(0.2, 0.5), rng.uniform(0.5, 1.0), rng.uniform(0, 2 * math.pi)
    T = 0.3 / (math.pi * b)  # shock forms at 1/(pi b)
    errs = []
    for N in (80, 160, 320):
        pr = prob(oracle, flux=oracle.BURGERS, P=3, nx=N, x0=-1.0, x1=1.0, cfl=0.5, bc=0)
        x = W.centres(N, -1.0, 1.0)
        u0 = (a + b * np.sin(math.pi * x + phi))[None, :]
        u, t = oracle.run_1d(pr, u0, 10 ** 6, t_end=T)
        errs.append(np.abs(u[0] - _burgers_exact(x, T, a, b, phi)).mean())
    rates = _rate(errs)
    assert rates[-1] > 5.5, (errs, rates)


def test_global_order_euler_entropy_wave(oracle):
    T = 0.25
    errs = []
    for N in (20, 40, 80):
        pr = prob(oracle, flux=oracle.EULER1D, P=3, nx=N, cfl=0.4, bc=0)
        x = W.centres(N, 0.0, 1.0)
        u0 = W.prim_to_cons_1d(1 + 0.2 * np.sin(2 * math.pi * x), np.ones(N), np.ones(N))
        u, t = oracle.run_1d(pr, u0, 10 ** 6, t_end=T)
        errs.append(np.abs(u[0] - (1 + 0.2 * np.sin(2 * math.pi * (x - T)))).mean())
    rates = _rate(errs)
    assert rates[-1] > 5.5, (errs, rates)


# ---------------------------------------------------------------------------
# Riemann problems against the exact solution (Sec. 5.3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,T,bound", [("sod", 0.25, 0.02), ("einfeldt123", 0.15, 0.05)])
def test_riemann_l1(oracle, name, T, bound):
    from oracle import riemann
    left, right = W.RIEMANN_1D[name]
    errs = []
    for N in (100, 200):
        c = W.riemann_1d(name, N, P=2)
        pr = prob(oracle, **c.problem_kwargs())
        u, t = oracle.run_1d(pr, c.u0, 10 ** 6, t_end=T)
        ex = riemann.cell_averages(left, right, 0.5, T, np.linspace(0, 1, N + 1))
        errs.append(np.abs(u[0] - ex[0]).mean())
    assert errs[1] < errs[0] and errs[1] < bound, errs


# ---------------------------------------------------------------------------
# Complex-step instantiation agrees with the real oracle
# ---------------------------------------------------------------------------
def test_complex_step_matches_real_and_fd(oracle):
    N = 128
    x = W.centres(N, 0.0, 1.0)
    u = W.prim_to_cons_1d(1 + 0.2 * np.sin(2 * math.pi * x), 0.3 + 0.1 * np.cos(2 * math.pi * x),
                          1 + 0.1 * np.sin(4 * math.pi * x))
    pr = prob(oracle, flux=oracle.EULER1D, P=3, nx=N, cfl=0.4, bc=0)
    dt = oracle.dt_cfl(pr, u)
    ur, _, o0 = oracle.step_1d(pr, u, dt)
    rng = np.random.default_rng(0)
    # a smooth direction, so that the +/- eps states keep every branch
    ph = rng.uniform(0, 2 * math.pi, size=(3, 1))
    d = np.sin(2 * math.pi * x[None, :] + ph) * rng.uniform(0.5, 1.0, size=(3, 1))
    h = 1e-30
    zr, zi = oracle.step_1d_complex(pr, u, h * d, dt)
    assert np.allclose(zr, ur, rtol=1e-15, atol=1e-15)
    jvp = zi / h
    eps = 1e-8
    up, _, op = oracle.step_1d(pr, u + eps * d, dt)
    um, _, om = oracle.step_1d(pr, u - eps * d, dt)
    assert np.array_equal(op, o0) and np.array_equal(om, o0)  # no branch flips
    fd = (up - um) / (2 * eps)
    assert np.allclose(jvp, fd, rtol=1e-6, atol=1e-7)


# ---------------------------------------------------------------------------
# 2D (Sec. 4)
# ---------------------------------------------------------------------------
def test_2d_reduces_to_1d_for_x_only_data(oracle):
    N, NY = 32, 6
    c1 = W.riemann_1d("sod", N, P=2)
    pr1 = prob(oracle, **c1.problem_kwargs())
    rho, vel, pre = W.cons_to_prim_1d(c1.u0)
    u2 = W.prim_to_cons_2d(*(np.repeat(a[None, :], NY, axis=0) for a in (rho, vel, 0 * vel, pre)))
    pr2 = prob(oracle, flux=oracle.EULER2D, P=2, nx=N, ny=NY, bc=1, cfl=0.8)
    dt = 0.4 * pr1.dx / 2.5
    un1, _, o1 = oracle.step_1d(pr1, c1.u0, dt)
    un2, _, ox, oy = oracle.step_2d(pr2, u2, dt)
    for row in range(NY):
        assert np.allclose(un2[0, row], un1[0], rtol=1e-13, atol=1e-13)
        assert np.allclose(un2[1, row], un1[1], rtol=1e-13, atol=1e-13)
        assert np.allclose(un2[3, row], un1[2], rtol=1e-13, atol=1e-13)
        assert np.array_equal(ox[row], o1)
    # y-momentum: only round-off from weights that sum to zero up to rounding
    assert np.abs(un2[2]).max() < 1e-13
    assert np.all(oy == 2)


def test_2d_reduces_to_1d_for_y_only_data(oracle):
    """The same Sod data laid along y (v_y the 1D velocity, v_x = 0): every
    column equals the 1D step, with the y-momentum in the place of the 1D
    momentum; the y-orders equal the 1D orders."""
    N, NX = 32, 6
    c1 = W.riemann_1d("sod", N, P=2)
    pr1 = prob(oracle, **c1.problem_kwargs())
    rho, vel, pre = W.cons_to_prim_1d(c1.u0)
    col = lambda a: np.repeat(a[:, None], NX, axis=1)  # noqa: E731
    u2 = W.prim_to_cons_2d(col(rho), col(0 * vel), col(vel), col(pre))
    pr2 = prob(oracle, flux=oracle.EULER2D, P=2, nx=NX, ny=N, bc=1, cfl=0.8, x0=0.0, x1=1.0,
               y0=c1.x0, y1=c1.x1)
    dt = 0.4 * pr1.dx / 2.5
    un1, _, o1 = oracle.step_1d(pr1, c1.u0, dt)
    un2, _, ox, oy = oracle.step_2d(pr2, u2, dt)
    for cx in range(NX):
        assert np.allclose(un2[0, :, cx], un1[0], rtol=1e-13, atol=1e-13)
        assert np.allclose(un2[2, :, cx], un1[1], rtol=1e-13, atol=1e-13)
        assert np.allclose(un2[3, :, cx], un1[2], rtol=1e-13, atol=1e-13)
        assert np.array_equal(oy[:, cx], o1)
    assert np.abs(un2[1]).max() < 1e-13
    assert np.all(ox == 2)


def test_2d_diagonal_symmetry_lax_liu(oracle):
    # configuration 8 (Table 5) is symmetric under x <-> y with u <-> v
    c = W.lax_liu(8, 24, P=2)
    pr = prob(oracle, **c.problem_kwargs())
    u = c.u0
    for _ in range(3):
        u, dt, ox, oy = oracle.step_2d(pr, u)
    ut = np.stack([u[0].T, u[2].T, u[1].T, u[3].T])
    assert np.allclose(u, ut, rtol=1e-12, atol=1e-12)
    assert np.array_equal(ox, oy.T)


def test_2d_conservation_periodic(oracle):
    N = 20
    x = W.centres(N, 0, 1)[None, :]
    y = W.centres(N, 0, 1)[:, None]
    rho = 1 + 0.2 * np.sin(2 * math.pi * x) * np.cos(2 * math.pi * y) + 0.3 * (x + 0 * y > 0.6)
    u = W.prim_to_cons_2d(rho, 0.3 + 0 * rho, -0.2 + 0 * rho, 1 + 0 * rho)
    pr = prob(oracle, flux=oracle.EULER2D, P=2, nx=N, ny=N, bc=0, cfl=0.4)
    for _ in range(3):
        un, dt, _, _ = oracle.step_2d(pr, u)
        for comp in range(4):
            assert abs(math.fsum(un[comp].ravel()) - math.fsum(u[comp].ravel())) < 1e-12 * N * N
        u = un


@pytest.mark.parametrize("P", [2, 3])
def test_2d_local_error_order_transport(oracle, P):
    # u_t + u_x + u_y = 0, smooth data without critical points; one step from
    # exact values: local error O(dx^{2P+1}) where all four interfaces use P
    errs = []
    Ns = (16, 32, 64) if P == 2 else (36, 54, 81)
    for N in Ns:
        pr = prob(oracle, flux=oracle.LINEAR, P=P, nx=N, ny=N, adv=(1.0, 1.0), bc=1, cfl=0.5)
        x = W.centres(N, 0, 1)[None, :]
        y = W.centres(N, 0, 1)[:, None]
        f = lambda x, y: np.exp(2.5 * x + 1.5 * y) + 0.3 * x * y  # noqa: E731
        u = f(x + 0 * y, y + 0 * x)[None]
        un, dt, ox, oy = oracle.step_2d(pr, u)
        ok = (ox[:, :-1] == P) & (ox[:, 1:] == P) & (oy[:-1, :] == P) & (oy[1:, :] == P)
        ok[:P + 1, :] = False  # cells fed by transmissive ghosts
        ok[:, :P + 1] = False
        ok[-P - 1:, :] = False
        ok[:, -P - 1:] = False
        assert ok.sum() >= 0.9 * (N - 2 * P - 2) ** 2
        errs.append(np.abs(un[0] - f(x - dt + 0 * y, y - dt + 0 * x))[ok].max())
    rates = [math.log(errs[i] / errs[i + 1]) / math.log(Ns[i + 1] / Ns[i]) for i in range(2)]
    assert rates[-1] > 2 * P + 1 - 0.6, (errs, rates)


# ---------------------------------------------------------------------------
# The limiter psi^1 (Eqs. 3.5-3.7): superbee values at chosen ratios
# ---------------------------------------------------------------------------
# superbee at ratios where its value is known by hand (max(0, min(2r, 1),
# min(r, 2)) read off its graph): the rising part, the plateau at 1, the
# second rise and the cap at 2, and negative ratios
SUPERBEE_AT = [(0.25, 0.5), (0.75, 1.0), (1.5, 1.5), (3.0, 2.0), (-1.0, 0.0), (0.5, 1.0),
               (2.0, 2.0), (5.0, 2.0), (1.0, 1.0), (-0.25, 0.0), (1.25, 1.25)]


def _jumps_for_ratios(ratios, upwind_left):
    """Cell jumps J_m = u_m - u_{m-1}, m = 1..K+8, such that the upwind ratio
    at interface m0 + k (between cells m0 + k - 1 and m0 + k) is ratios[k]:
    J_{m-1} / J_m for a positive speed, J_{m+1} / J_m for a negative one."""
    K, m0 = len(ratios), 4
    J = np.full(K + 9, 0.01)
    if upwind_left:
        for k, r in enumerate(ratios):
            J[m0 + k] = J[m0 + k - 1] / r
    else:
        # fill from the right: J_m = J_{m+1} / r_m
        for k in reversed(range(K)):
            J[m0 + k] = J[m0 + k + 1] / ratios[k]
    return J, m0


@pytest.mark.parametrize("positive", [True, False])
def test_limiter_superbee_values_roe_side(oracle, positive):
    """Burgers with P = 1 (FL-CAT2 everywhere): psi^1 at each interface is
    superbee of the upwind ratio, the side picked by the sign of the Roe
    speed (Eq. 3.6). Positive states take the left jump, negative states the
    right one."""
    ratios = [r for r, _ in SUPERBEE_AT]
    J, m0 = _jumps_for_ratios(ratios, upwind_left=positive)
    # u_m - u_{m-1} = J_m (positive states), or -J_m (negative states: the
    # jumps change sign together, which keeps every ratio)
    prof = np.concatenate([[0.0], np.cumsum(J[1:])])
    u = 1.0 + prof if positive else -1.0 - prof
    assert (u > 0).all() if positive else (u < 0).all()
    N = u.size
    pr = prob(oracle, flux=oracle.BURGERS, P=1, nx=N, bc=1, x0=0.0, x1=1.0, cfl=0.4)
    _, _, orders, psi = oracle.step_1d(pr, u[None, :], 1e-4, want_psi=True)
    assert (orders[1:N] == 1).all()
    for k, (_, want) in enumerate(SUPERBEE_AT):
        assert psi[m0 + k, 0] == pytest.approx(want, rel=1e-12, abs=1e-15), (k, psi[m0 + k, 0])


def test_limiter_zero_local_jump(oracle):
    """Reading of a zero local jump (Eq. 3.5 divides by it): a zero upwind jump
    gives r = 1 (psi^1 = 1), a positive upwind jump r = +inf (psi^1 = 2), a
    negative one r = -inf (psi^1 = 0)."""
    # positive states: the upwind jump is the left one
    u = np.array([1.0, 1.0, 1.0, 1.0, 1.1, 1.1, 1.1, 1.0, 1.0, 1.0, 1.0, 1.0])
    N = u.size
    pr = prob(oracle, flux=oracle.BURGERS, P=1, nx=N, bc=1, x0=0.0, x1=1.0, cfl=0.4)
    _, _, _, psi = oracle.step_1d(pr, u[None, :], 1e-4, want_psi=True)
    assert psi[2, 0] == 1.0   # cells 1, 2 equal, upwind jump u_1 - u_0 = 0
    assert psi[5, 0] == 2.0   # cells 4, 5 equal, upwind jump u_4 - u_3 = +0.1
    assert psi[8, 0] == 0.0   # cells 7, 8 equal, upwind jump u_7 - u_6 = -0.1


def test_limiter_min_form(oracle):
    """limiter_form = 1 (Eq. 3.7 for a scalar law): psi^1 = min(superbee(r-),
    superbee(r+)) with both one-sided ratios, whatever the speed's sign.
    Jumps 0.01, 0.04, 0.02, 0.06 give at the interface of the 0.04 jump the
    ratios 0.25 and 0.5, superbee 0.5 and 1, so 0.5; at the 0.02 jump the
    ratios 2 and 3, superbee 2 and 2, so 2."""
    J = np.array([0.01, 0.01, 0.01, 0.04, 0.02, 0.06, 0.06, 0.06])
    u = 1.0 + np.concatenate([[0.0], np.cumsum(J)])
    N = u.size
    pr = prob(oracle, flux=oracle.BURGERS, P=1, nx=N, bc=1, x0=0.0, x1=1.0, cfl=0.4,
              limiter_form=1)
    _, _, _, psi = oracle.step_1d(pr, u[None, :], 1e-4, want_psi=True)
    # interface m lies across the jump u_m - u_{m-1} = J[m - 1]
    assert psi[4, 0] == pytest.approx(0.5, rel=1e-12)
    assert psi[5, 0] == pytest.approx(2.0, rel=1e-12)


def test_limiter_systems_min_over_components_and_sides(oracle):
    """Euler with P = 1: psi^1 = min over components of min(superbee(r-),
    superbee(r+)) (Eq. 3.7, Sec. 3.4). Three interfaces, each with the
    minimum in a different component, the other components at ratio 1:
    rho with jumps 0.01, 0.04, 0.02 around the interface's own (ratios 0.25
    and 0.5: superbee 0.5 and 1, so 0.5); m with 0.01, 0.1, 0.01 (ratios
    0.1, 0.1: 0.2); E with 0.05, 0.1, 0.01 (ratios 0.5 and 0.1: 1 and 0.2,
    so 0.2)."""
    N = 30
    Jr = np.full(N - 1, 0.01)
    Jm = np.full(N - 1, 0.01)
    Je = np.full(N - 1, 0.02)
    # interface 8 crosses jump index 7 (u_8 - u_7): rho carries the minimum 0.5
    Jr[6], Jr[7], Jr[8] = 0.01, 0.04, 0.02
    # interface 16: m carries 0.2 (rho, E at ratio 1)
    Jm[14], Jm[15], Jm[16] = 0.01, 0.1, 0.01
    # interface 24: E carries min(superbee(0.05 / 0.1), superbee(0.01 / 0.1)) = 0.2
    Je[22], Je[23], Je[24] = 0.05, 0.1, 0.01
    rho = 1.0 + np.concatenate([[0.0], np.cumsum(Jr)])
    m = 0.2 + np.concatenate([[0.0], np.cumsum(Jm)])
    E = 3.0 + np.concatenate([[0.0], np.cumsum(Je)])
    u = np.stack([rho, m, E])
    assert ((E - 0.5 * m * m / rho) > 0).all()
    pr = prob(oracle, flux=oracle.EULER1D, P=1, nx=N, bc=1, x0=0.0, x1=1.0, cfl=0.4)
    _, _, _, psi = oracle.step_1d(pr, u, 1e-4, want_psi=True)
    assert psi[8, 0] == pytest.approx(0.5, rel=1e-12)
    assert psi[16, 0] == pytest.approx(0.2, rel=1e-12)
    assert psi[24, 0] == pytest.approx(0.2, rel=1e-12)
    # an interface away from the patterns: every ratio is 1
    assert psi[4, 0] == pytest.approx(1.0, rel=1e-12)


# ---------------------------------------------------------------------------
# CFL time step (Sec. 5: dt = CFL dx / s^max; 2D: Sec. 5.5)
# ---------------------------------------------------------------------------
def test_dt_closed_forms(oracle):
    """Hand-computed time steps: Burgers s^max = max |u|; Euler s^max =
    max(|v| + c), c = sqrt(gamma p / rho); 2D Euler CFL/2 min(dx / s_x,
    dy / s_y) with s_x from |v_x| + c and s_y from |v_y| + c."""
    N = 10
    u = np.linspace(-2.0, 1.5, N)[None, :]  # max |u| = 2
    pr = prob(oracle, flux=oracle.BURGERS, P=2, nx=N, x0=-1.0, x1=1.0, cfl=0.5)
    assert oracle.dt_cfl(pr, u) == pytest.approx(0.5 * 0.2 / 2.0, rel=1e-15)
    # Euler: rho = 1, v = 0.5, p = 1 in every cell but one with rho = 0.5,
    # v = -1, p = 2 (c = sqrt(5.6), the larger speed 1 + sqrt(5.6))
    rho = np.ones(N)
    v = np.full(N, 0.5)
    p = np.ones(N)
    rho[3], v[3], p[3] = 0.5, -1.0, 2.0
    U = np.stack([rho, rho * v, p / 0.4 + 0.5 * rho * v * v])
    pr = prob(oracle, flux=oracle.EULER1D, P=2, nx=N, x0=0.0, x1=2.0, cfl=0.4)
    assert oracle.dt_cfl(pr, U) == pytest.approx(0.4 * 0.2 / (1.0 + math.sqrt(5.6)), rel=1e-14)
    # 2D Euler on 8 x 6 cells of [0,1] x [0,0.3] (dx = 1/8, dy = 1/20): one
    # cell with (rho, vx, vy, p) = (1, 2, 0, 1.4) (c = 1.4), the rest
    # (1, 0, 0.1, 1.4); the y term is the smaller (0.05 / 1.5 < 0.125 / 3.4)
    nx, ny = 8, 6
    rho = np.ones((ny, nx))
    vx = np.zeros((ny, nx))
    vy = np.full((ny, nx), 0.1)
    p = np.full((ny, nx), 1.4)
    vx[2, 5], vy[2, 5] = 2.0, 0.0
    E = p / 0.4 + 0.5 * rho * (vx * vx + vy * vy)
    U2 = np.stack([rho, rho * vx, rho * vy, E])
    pr = prob(oracle, flux=oracle.EULER2D, P=2, nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=0.3, cfl=0.4)
    c = math.sqrt(1.4 * 1.4 / 1.0)
    sx, sy = 2.0 + c, 0.1 + c
    assert 0.05 / sy < 0.125 / sx
    want = 0.2 * min(0.125 / sx, 0.05 / sy)
    assert oracle.dt_cfl(pr, U2) == pytest.approx(want, rel=1e-14)


# ---------------------------------------------------------------------------
# Indicator values worked by hand from Eqs. 3.8-3.12 (eps = 0)
# ---------------------------------------------------------------------------
# p = 2 on (f_{i-1}, f_i, f_{i+1}, f_{i+2}) = (0, 1, 3, 4): lateral differences
# 1 (left) and 1 (right), the central one 2 left out, so I_L = I_R = 1 and
# I_2 = 1/2; the third undivided difference 4 - 3*3 + 3*1 - 0 = -2, so
# tau_2 = (3! * -2)^2 = 144 as printed, 4 without the factorial.
# p = 3 on (0, 1, 1, 2, 4, 4): left differences 1, 0 (I_L = 1), right 2, 0
# (I_R = 4), I_3 = 4/5; the fifth difference 4 - 5*4 + 10*2 - 10*1 + 5*1 - 0
# = -1, so tau_3 = (5! * -1)^2 = 14400, or 1.
PSI_BY_HAND = [(2, [0.0, 1.0, 3.0, 4.0], 1, 0.5 / 144.5), (2, [0.0, 1.0, 3.0, 4.0], 0, 0.5 / 4.5),
               (3, [0.0, 1.0, 1.0, 2.0, 4.0, 4.0], 1, 0.8 / 14400.8),
               (3, [0.0, 1.0, 1.0, 2.0, 4.0, 4.0], 0, 0.8 / 1.8)]


@pytest.mark.parametrize("p,f,fact,want", PSI_BY_HAND)
def test_indicator_values_by_hand(oracle, p, f, fact, want):
    N, m = 14, 7  # interface m between cells i = m - 1 and m
    u = np.full(N, 0.5)
    u[m - p:m + p] = f
    pr = prob(oracle, flux=oracle.LINEAR, P=p, nx=N, adv=(1.0, 0.0), eps=0.0, tau_factorial=fact, bc=1)
    _, _, _, psi = oracle.step_1d(pr, u[None, :], 1e-4, want_psi=True)
    assert psi[m, p - 1] == pytest.approx(want, rel=1e-14)


# psi~^2 (Sec. 3.2) on (0, 1, 3, 7): differences 1, 2, 4; I^1 = 1 * 20 / 21,
# I^2 = 5 * 16 / 21; the third difference 7 - 9 + 3 - 0 = 1, tau_2 = 36 (or
# 1 without the factorial); psi~^2 = max(20 / 776, 80 / 836) = 80 / 836 (or
# max(20 / 41, 80 / 101) = 80 / 101), where psi^2 (I_2 = 16 / 17) is 16 / 628.
@pytest.mark.parametrize("mod,fact,want", [(1, 1, 80.0 / 836.0), (1, 0, 80.0 / 101.0), (0, 1, 16.0 / 628.0)])
def test_modified_indicator_value_by_hand(oracle, mod, fact, want):
    N, m = 12, 6
    u = np.full(N, 0.5)
    u[m - 2:m + 2] = [0.0, 1.0, 3.0, 7.0]
    pr = prob(oracle, flux=oracle.LINEAR, P=2, nx=N, adv=(1.0, 0.0), eps=0.0, tau_factorial=fact, bc=1,
              psi2_mod=mod)
    _, _, _, psi = oracle.step_1d(pr, u[None, :], 1e-4, want_psi=True)
    assert psi[m, 1] == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("P", [2])
def test_2d_local_error_order_anisotropic(oracle, P):
    """u_t + a u_x + b u_y = 0 with a != b on cells with dy = dx / 2: one step
    from exact values has local error O(dx^{2P+1}) only if every x-quantity
    takes dx and a and every y-quantity dy and b (Eqs. 4.5-4.6, 4.9); a swap
    leaves an O(dt) error."""
    errs = []
    Ns = (16, 32, 64)
    a, b = 1.0, 0.35
    for N in Ns:
        pr = prob(oracle, flux=oracle.LINEAR, P=P, nx=N, ny=N, adv=(a, b), bc=1, cfl=0.5,
                  x0=0.0, x1=1.0, y0=0.0, y1=0.5)
        x = W.centres(N, 0.0, 1.0)[None, :]
        y = W.centres(N, 0.0, 0.5)[:, None]
        f = lambda x, y: np.exp(2.5 * x + 1.5 * y) + 0.3 * x * y  # noqa: E731
        u = f(x + 0 * y, y + 0 * x)[None]
        un, dt, ox, oy = oracle.step_2d(pr, u)
        # dt = CFL/2 min(dx / a, dy / b) with dx = 1/N, dy = 0.5/N
        assert dt == pytest.approx(0.25 * min((1.0 / N) / a, (0.5 / N) / b), rel=1e-14)
        ok = (ox[:, :-1] == P) & (ox[:, 1:] == P) & (oy[:-1, :] == P) & (oy[1:, :] == P)
        ok[:P + 1, :] = False
        ok[:, :P + 1] = False
        ok[-P - 1:, :] = False
        ok[:, -P - 1:] = False
        assert ok.sum() >= 0.9 * (N - 2 * P - 2) ** 2
        errs.append(np.abs(un[0] - f(x - a * dt + 0 * y, y - b * dt + 0 * x))[ok].max())
    rates = [math.log(errs[i] / errs[i + 1]) / math.log(Ns[i + 1] / Ns[i]) for i in range(2)]
    assert rates[-1] > 2 * P + 1 - 0.6, (errs, rates)


def test_admissibility_threshold_is_inclusive(oracle):
    """p is admissible when psi^p >= 1 - delta (Eq. 3.2 read with a threshold):
    a stencil with psi^3 = 1/2 exactly and delta = 1/2 selects p = 3. On
    (0, 1, 0, -3/2, -5/2, -3/2) the differences are 1, -1 (left), -3/2
    (central) and -1, 1 (right): I_L = I_R = 2, I_3 = 1; the fifth difference
    is 1 (tau_3 = 1 without the factorial), so psi^3 = 1/2 in exact binary
    arithmetic. psi^2 on (1, 0, -3/2, -5/2) is 1/2 / (1/2 + 1) = 1/3."""
    N, m = 14, 7
    u = np.full(N, 0.25)
    u[m - 3:m + 3] = [0.0, 1.0, 0.0, -1.5, -2.5, -1.5]
    pr = prob(oracle, flux=oracle.LINEAR, P=3, nx=N, adv=(1.0, 0.0), eps=0.0, tau_factorial=0, bc=1,
              psi_tol=0.5)
    _, _, orders, psi = oracle.step_1d(pr, u[None, :], 1e-4, want_psi=True)
    assert psi[m, 2] == 0.5 and psi[m, 1] == pytest.approx(1.0 / 3.0, rel=1e-15)
    assert orders[m] == 3


def test_transmissive_ghosts_are_copies(oracle):
    """Transmissive boundaries copy the edge cell into every ghost (reading of
    the paper's outflow / free conditions). Linear transport, P = 2, data
    starting (1, 2, ...): the stencil of interface 0 is (u_0, u_0, u_0, u_1) =
    (1, 1, 1, 2), so I_{2,L} = eps, psi^2 ~ 0 and the interface is FL-CAT2;
    there r = 0/0 reads as 1, psi^1 = 1, and the flux is the CAT2 one of the
    constant pair (u_-1, u_0) = (1, 1): F_0 = a exactly. Mirrored ghosts
    (u_-2 = u_1) would give psi^2 = 1 there instead."""
    N = 12
    u = (1.0 + np.arange(N, dtype=np.float64) ** 1.5)[None, :]
    a = 0.8
    pr = prob(oracle, flux=oracle.LINEAR, P=2, nx=N, adv=(a, 0.0), bc=1, x0=0.0, x1=1.0, cfl=0.5)
    _, _, orders, psi, F = oracle.step_1d(pr, u, 1e-3, want_psi=True, want_flux=True)
    assert orders[0] == 1 and psi[0, 1] < 1e-9 and psi[0, 0] == 1.0
    assert F[0, 0] == a * u[0, 0]
    # the right boundary likewise: interface N sees (u_{N-2}, u_{N-1}, u_{N-1}, u_{N-1})
    assert orders[N] == 1 and F[N, 0] == pytest.approx(a * u[0, N - 1], rel=1e-15)


@pytest.mark.parametrize("P", [3, 4])
def test_order_is_max_of_admissible_set(oracle, P):
    """p_s = max A (Eq. 3.3): smaller stencils need not be admissible. Data
    (x - x*)^2 + (x - x*)^3 with the critical point x* at the midpoint of cells
    m-2 and m-1, h = 0.05: the left lateral weight of S_2 is only
    (h^3/4)^2 + eps while tau_2 = (3! 6 h^3)^2, so psi^2 ~ 5e-5 rejects
    (value checked against its closed form);
    the fifth and seventh differences of a cubic vanish, so tau_3 = tau_4 = 0
    to rounding and psi^3 = psi^4 = 1 accept. The selected order is P. A rule
    taking the largest p whose smaller stencils are all admissible would give
    FL-CAT2 (code 1) here."""
    h, n, m = 0.05, 16, 8
    x = (np.arange(n) + 0.5) * h
    xs = 0.5 * (x[m - 2] + x[m - 1])
    u = ((x - xs) ** 2 + (x - xs) ** 3)[None, :]
    pr = prob(oracle, flux=oracle.LINEAR, P=P, nx=n, adv=(1.0, 0.0), bc=1)
    _, _, orders, psi = oracle.step_1d(pr, u, 1e-4, want_psi=True)
    # closed forms: d_L = h^3/4, d_R = u(x* + 5h/2) - u(x* + 3h/2) = 4h^2 + 49h^3/4,
    # third difference 6 h^3
    IL, IR = (h ** 3 / 4.0) ** 2 + 1e-12, (4.0 * h ** 2 + 12.25 * h ** 3) ** 2 + 1e-12
    I2 = IL * IR / (IL + IR)
    assert psi[m, 1] == pytest.approx(I2 / (I2 + (36.0 * h ** 3) ** 2), rel=1e-9)
    assert psi[m, 1] < 0.9
    for p in range(3, P + 1):
        assert psi[m, p - 1] > 1.0 - 1e-12
    assert orders[m] == P
