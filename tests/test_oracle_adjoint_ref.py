"""Pins of the oracle's reference reverse sweep (oracle/adjoint_ref.py): the
1D step restated in PyTorch CPU float64 for autograd.

- Its forward step equals the C oracle's step bit for bit (same operations in
  the same order; the orders are the C oracle's), on data with FL-CAT2
  interfaces, every F^lo, both limiter forms, both boundaries and P = 1..4.
- Its vector-Jacobian product equals the transpose of the C oracle's
  complex-step Jacobian (an independent derivative: complex arithmetic, with
  every discrete choice taken on real parts) to 1e-12 of max |J^T w|. The
  cases keep away from nearly constant FL-CAT2 stencils, where two correct
  evaluations of the blend's derivative differ by the conditioning of the
  limiter ratio (the adjoint tests bound that case entry by entry).
"""
import numpy as np
import pytest

from paper_2007_01416_gb300 import workloads as W


def _case(kind, nx, P, seed, extra):
    c = W.burgers_sine(nx=nx, seed=seed, P=P) if kind == "burgers" else \
        W.euler1d_riemann_entropy(nx=nx, seed=seed, P=P)
    kw = c.problem_kwargs()
    kw.update(extra)
    return c, kw


STEP_CASES = [("euler", 300, 4, 1, {}), ("euler", 300, 2, 2, {"lo_flux": 2}),
              ("euler", 257, 3, 3, {"lo_flux": 1, "bc": 0}), ("euler", 64, 1, 4, {}),
              ("burgers", 200, 3, 5, {}), ("burgers", 200, 2, 6, {"limiter_form": 1, "bc": 1}),
              ("euler", 300, 4, 7, {"limiter_form": 1, "psi2_mod": 1})]


@pytest.mark.parametrize("kind,nx,P,seed,extra", STEP_CASES)
def test_reference_step_equals_oracle(oracle, kind, nx, P, seed, extra):
    import torch
    from oracle import adjoint_ref as A
    c, kw = _case(kind, nx, P, seed, extra)
    pr = oracle.Problem(**kw)
    u = c.u0
    for _ in range(200 if kind == "burgers" else 25):  # fronts: FL-CAT2 interfaces next to high orders
        u, _, _ = oracle.step_1d(pr, u)
    ref, dt, orders = oracle.step_1d(pr, u)
    assert (orders == 1).any()
    got = A.step(pr, torch.from_numpy(u.copy()), dt, orders).numpy()
    assert np.array_equal(got, ref)


def _jacobian(O, pr, u, dt):
    h = 1e-30
    J = np.zeros((u.size, u.size))
    for k in range(u.size):
        e = np.zeros(u.size)
        e[k] = h
        _, im = O.step_1d_complex(pr, u, e.reshape(u.shape), dt)
        J[:, k] = im.ravel() / h
    return J


@pytest.mark.parametrize("kind,nx,P,extra", [("euler", 24, 2, {}), ("euler", 28, 3, {"lo_flux": 2}),
                                             ("euler", 32, 4, {"lo_flux": 1, "bc": 0}),
                                             ("burgers", 30, 2, {}), ("burgers", 30, 3, {"limiter_form": 1})])
def test_reference_vjp_is_complex_step_transpose(oracle, kind, nx, P, extra):
    from oracle import adjoint_ref as A
    c, kw = _case(kind, nx, P, 0, extra)
    pr = oracle.Problem(**kw)
    u = c.u0
    dt = oracle.dt_cfl(pr, u)
    _, _, orders = oracle.step_1d(pr, u, dt)
    assert (orders == 1).any() and (orders > 1).any()
    w = np.random.default_rng(1).normal(size=u.shape)
    ref = (_jacobian(oracle, pr, u, dt).T @ w.ravel()).reshape(u.shape)
    got = A.vjp(pr, u, dt, w)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_reference_gradient_is_the_product_of_vjps(oracle):
    """gradient() is w_0 = J_0^T ... J_{n-1}^T w_n along the given states."""
    from oracle import adjoint_ref as A
    c, kw = _case("euler", 40, 2, 9, {})
    pr = oracle.Problem(**kw)
    states, dts, u = [], [], c.u0
    for _ in range(4):
        dt = oracle.dt_cfl(pr, u)
        states.append(u)
        dts.append(dt)
        u, _, _ = oracle.step_1d(pr, u, dt)
    w = np.random.default_rng(2).normal(size=u.shape)
    want = w
    for n in reversed(range(4)):
        want = (_jacobian(oracle, pr, states[n], dts[n]).T @ want.ravel()).reshape(u.shape)
    got = A.gradient(pr, states, dts, w)
    assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()
