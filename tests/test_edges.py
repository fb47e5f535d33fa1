"""Edge cases of the CUDA path against the oracle: the smallest grids the
stencils allow (nx = ny = 2 max(P, 2), every cell a ghost of another),
zero-step runs, a batch of one instance, constant states (every order
admissible, the state a fixed point), P = 1 (FL-CAT2 only) and an order
decision exactly at the admissibility threshold."""
import numpy as np
import pytest

from paper_2007_01416_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as O
    from paper_2007_01416_gb300 import acat, build
    build.build()
    O.build()
    return torch, O, acat


def _step(torch, ctx, u, n_orders):
    ug = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    out = torch.empty_like(ug)
    dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
    orders = torch.zeros(n_orders, dtype=torch.int8, device="cuda")
    ctx.acat_step(ug, out, -1.0, None, dtv, orders)
    torch.cuda.synchronize()
    return out.cpu().numpy(), float(dtv.item()), orders.cpu().numpy()


@pytest.mark.parametrize("P", [1, 2, 3, 4])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_smallest_1d_grid(env, P, bc, prec):
    torch, O, acat = env
    nx = 2 * max(P, 2)
    c = W.euler1d_riemann_entropy(nx=nx, seed=5, P=P)
    c.bc = bc
    kw = c.problem_kwargs()
    f32 = prec == "f32"
    u = acat.to_pair(c.u0) if f32 else c.u0
    x = acat.from_pair(u) if f32 else c.u0
    with acat.Context(**kw, precision=acat.PREC_F32 if f32 else acat.PREC_F64) as ctx:
        out, dt, orders = _step(torch, ctx, u, nx + 1)
        assert ctx.acat_status() == 0
    pr = O.Problem(**kw)
    ref, _, oref = O.step_1d(pr, x, dt)
    assert np.array_equal(orders, oref)
    got = acat.from_pair(out) if f32 else out
    assert np.abs(got - ref).max() / np.abs(ref).max() < (1e-7 if f32 else 1e-12)


@pytest.mark.parametrize("P,rect", [(1, 0), (2, 0), (3, 0), (4, 0), (3, 1), (2, 1)])
def test_smallest_2d_grid(env, P, rect):
    torch, O, acat = env
    n = 2 * max(P, 2)
    c = W.euler2d_smooth(n=n, seed=2, P=P) if P >= 3 else W.euler2d_quadrants(n=n, seed=2, P=P)
    kw = dict(c.problem_kwargs(), rect_2d=rect)
    with acat.Context(**kw) as ctx:
        out, dt, o = _step(torch, ctx, c.u0, 2 * n * (n + 1))
        assert ctx.acat_status() == 0
    pr = O.Problem(**kw)
    ref, _, ox, oy = O.step_2d(pr, c.u0, dt)
    assert np.array_equal(o, np.concatenate([ox.ravel(), oy.ravel()]))
    assert np.abs(out - ref).max() / np.abs(ref).max() < 1e-12


def test_zero_steps_leave_the_state(env):
    torch, O, acat = env
    c = W.euler1d_riemann_entropy(nx=300, seed=1, P=3)
    c2 = W.euler2d_quadrants(n=20, seed=1, P=2)
    for kw, u0, extra in ((c.problem_kwargs(), c.u0, {}), (c2.problem_kwargs(), c2.u0, {}),
                          (c.problem_kwargs(), np.concatenate([c.u0, c.u0], axis=1), {"sizes": [300, 300]})):
        with acat.Context(**kw, **extra) as ctx:
            u = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
            ctx.acat_run(u, 0)
            torch.cuda.synchronize()
            assert np.array_equal(u.cpu().numpy(), u0)


def test_batch_of_one_equals_single_run(env):
    torch, O, acat = env
    c = W.euler1d_riemann_entropy(nx=777, seed=3, P=4)
    kw = c.problem_kwargs()
    with acat.Context(**kw, sizes=[777]) as b, acat.Context(**kw) as one:
        ub = torch.from_numpy(c.u0.copy()).cuda()
        us = torch.from_numpy(c.u0.copy()).cuda()
        b.acat_run(ub, 60)
        one.acat_run(us, 60)
        torch.cuda.synchronize()
        assert np.array_equal(ub.cpu().numpy(), us.cpu().numpy())


@pytest.mark.parametrize("P", [2, 4])
def test_constant_state_is_a_fixed_point(env, P):
    """A constant state admits every order (tau = 0 exactly) and no flux
    difference: orders P everywhere, the state unchanged to the last bit
    after 100 steps (FP64 and FP32)."""
    torch, O, acat = env
    nx = 500
    u0 = W.prim_to_cons_1d(np.full(nx, 0.8), np.full(nx, 0.3), np.full(nx, 0.6))
    kw = dict(flux=W.EULER1D, P=P, nx=nx, ny=1, bc=0, cfl=0.4, x0=0.0, x1=1.0)
    for prec, conv in ((acat.PREC_F64, lambda v: v), (acat.PREC_F32, acat.to_pair)):
        with acat.Context(**kw, precision=prec) as ctx:
            _, _, orders = _step(torch, ctx, conv(u0), nx + 1)
            assert np.all(orders == P)
            u = torch.from_numpy(np.ascontiguousarray(conv(u0))).cuda()
            ctx.acat_run(u, 100)
            torch.cuda.synchronize()
            assert np.array_equal(u.cpu().numpy(), conv(u0))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_order_decision_exactly_at_the_threshold(env, prec):
    """psi^3 = 1/2 exactly with delta = 1/2 (the oracle pin of the inclusive
    threshold): the filtered decision cannot certify either side, the literal
    FP64 fallback finds psi^3 >= 1 - delta, and the GPU selects p = 3 there as
    the oracle does."""
    torch, O, acat = env
    N, m = 14, 7
    i = np.arange(N, dtype=np.float64)
    u = 3.0 + 0.125 * i + 0.015625 * i * i  # no two equal neighbours, wrap included (eps = 0)
    u[m - 3:m + 3] = [0.0, 1.0, 0.0, -1.5, -2.5, -1.5]
    assert (np.diff(np.r_[u, u[0]]) != 0).all()
    u = u[None, :]
    kw = dict(flux=W.LINEAR, P=3, nx=N, ny=1, bc=0, adv=(1.0, 0.0), cfl=0.5, x0=0.0, x1=1.0,
              eps=0.0, tau_factorial=0, psi_tol=0.5)
    f32 = prec == "f32"
    with acat.Context(**kw, precision=acat.PREC_F32 if f32 else acat.PREC_F64) as ctx:
        out, dt, orders = _step(torch, ctx, acat.to_pair(u) if f32 else u, N + 1)
        assert ctx.acat_status() == 0
    pr = O.Problem(**kw)
    ref, _, oref = O.step_1d(pr, u, dt)
    assert oref[m] == 3
    assert np.array_equal(orders, oref), (orders, oref)
    got = acat.from_pair(out) if f32 else out
    assert np.abs(got - ref).max() / np.abs(ref).max() < (1e-7 if f32 else 1e-12)
