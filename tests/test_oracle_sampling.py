"""Pins of the oracle's sampling entry points against its full step.

The full-size parity tests on the GPU evaluate the oracle at sampled
interfaces and cells only (a full oracle step at the benchmark's sizes would
take too long to repeat). Those entry points restate the gather and the
update of the full step, so each is pinned here to the full step of the same
state bit for bit: fluxes and orders at sampled interfaces (Eq. 2.14 or the
FL-CAT2 flux of Eq. 3.4 as Eqs. 3.2-3.3 select), the 1D update at sampled
cells (Eq. 2.12) and the 2D update at sampled cells (Eq. 4.9), on seeded data
with jumps, both boundary conditions and every flux family.
"""
import numpy as np
import pytest

from paper_2007_01416_gb300 import workloads as W


def _case1d(kind, P, nx, bc, seed):
    if kind == "euler":
        c = W.euler1d_riemann_entropy(nx=nx, seed=seed, P=P)
    else:
        c = W.burgers_sine(nx=nx, seed=seed, P=P)
        if kind == "linear":
            c.flux = W.LINEAR
            c.adv = (-0.7, 0.0)
    c.bc = bc
    return c


CASES_1D = [("euler", 4, 777, 1, 0, {}), ("euler", 3, 500, 0, 1, {"lo_flux": 2}),
            ("euler", 2, 333, 1, 2, {"psi2_mod": 1, "lo_flux": 1}), ("burgers", 3, 400, 0, 3, {}),
            ("burgers", 1, 97, 1, 4, {}), ("linear", 4, 257, 0, 5, {})]


def _advanced(O, pr, u0, n):
    """The state after n oracle steps (sharper gradients, more FL-CAT2)."""
    u = u0.copy()
    for _ in range(n):
        u, _, _ = O.step_1d(pr, u)
    return u


@pytest.mark.parametrize("kind,P,nx,bc,seed,extra", CASES_1D)
def test_fluxes_at_and_cells_equal_the_full_step(oracle, kind, P, nx, bc, seed, extra):
    O = oracle
    c = _case1d(kind, P, nx, bc, seed)
    kw = c.problem_kwargs()
    kw.update(extra)
    pr = O.Problem(**kw)
    u = _advanced(O, pr, c.u0, 20)
    full, dt, orders, F = O.step_1d(pr, u, want_flux=True)
    if kind == "euler" and P > 1:  # both flux kinds present on Riemann data
        assert (orders == 1).any() and (orders == P).any()
    rng = np.random.default_rng(seed)
    ifaces = np.unique(np.r_[0, 1, nx - 1, nx, rng.choice(nx + 1, 96, replace=False)])
    Fs, ords = O.fluxes_1d_at(pr, u, dt, ifaces)
    assert np.array_equal(ords, orders[ifaces])
    assert np.array_equal(Fs, F[ifaces])  # bit for bit
    cells = np.unique(np.r_[0, 1, nx - 2, nx - 1, rng.choice(nx, 96, replace=False)])
    us = O.step_1d_cells(pr, u, dt, cells)
    assert np.array_equal(us, full[:, cells].T)


@pytest.mark.parametrize("P,rect,cfg", [(2, 0, None), (1, 0, None), (3, 1, None), (4, 1, None),
                                        (4, 0, "smooth"), (2, 0, 6)])
def test_step_2d_cells_equals_the_full_step(oracle, P, rect, cfg):
    O = oracle
    if cfg is None:
        c = W.euler2d_quadrants(n=23, ny=21, seed=P + 3 * rect, P=P)
    elif cfg == "smooth":  # square blocks at P >= 3 on smooth data with a contact
        c = W.euler2d_smooth(n=22, ny=19, seed=1, P=P)
    else:
        c = W.lax_liu(cfg, n=20, P=P)
    kw = c.problem_kwargs()
    kw["rect_2d"] = rect
    pr = O.Problem(**kw)
    u = c.u0.copy()
    for _ in range(3):
        u, _, _, _ = O.step_2d(pr, u)
    full, dt, ox, oy = O.step_2d(pr, u)
    assert np.isfinite(full).all()
    ny, nx = u.shape[1:]
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy = xx.ravel(), yy.ravel()  # every cell, corners and edges included
    got = O.step_2d_cells(pr, u, dt, cx, cy)
    assert np.array_equal(got, full[:, cy, cx].T)


def test_cell_flux_closed_forms(oracle):
    """The per-cell physical flux used by the FP32 free-run bar: Euler from the
    primitive variables, (rho v, rho v^2 + p, v (E + p)) with E = p/(gamma-1) +
    rho v^2/2; Burgers u^2/2; transport a u."""
    O = oracle
    rng = np.random.default_rng(7)
    rho, v, p = rng.uniform(0.1, 1.0, 50), rng.uniform(-0.5, 0.5, 50), rng.uniform(0.1, 1.0, 50)
    E = p / 0.4 + 0.5 * rho * v * v
    u = np.array([rho, rho * v, E])
    f = O.cell_flux_1d(O.Problem(flux=O.EULER1D, P=2, nx=50, gamma=1.4), u)
    assert np.allclose(f, [rho * v, rho * v * v + p, v * (E + p)], rtol=1e-14, atol=0)
    w = rng.uniform(-1, 1, (1, 50))
    assert np.array_equal(O.cell_flux_1d(O.Problem(flux=O.BURGERS, P=2, nx=50), w), 0.5 * w * w)
    assert np.array_equal(O.cell_flux_1d(O.Problem(flux=O.LINEAR, P=2, nx=50, adv=(-0.7, 0.0)), w), -0.7 * w)
