"""Parity of the switchable variants on the GPU with the oracle: the modified
indicator psi~^2 (Sec. 3.2; order codes bit-exact, decided by the same
filtered/literal scheme as psi^p) and the F^lo fluxes of FL-CAT2 (global
Lax-Friedrichs, HLL), in 1D FP64/FP32, 2D FP64/FP32, the batched step and the
adjoint (J^T against the oracle's complex-step Jacobian, 1e-10). Bars as for
the default variants: 1e-12 (FP64) and 1e-7 (FP32) of max|u| per step.
"""
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


def _case1(kind, P, nx, bc, seed=0):
    if kind in ("burgers", "linear"):
        # the seeded sine data with a jump added, so that FL-CAT2 interfaces occur
        c = W.burgers_sine(nx=nx, seed=seed, P=P)
        x = W.centres(nx, c.x0, c.x1)
        c.u0 = c.u0 + 0.5 * (x > 0.3)[None, :]
        if kind == "linear":
            c.flux = W.LINEAR
            c.adv = (-0.7, 0.0)
    else:
        c = W.euler1d_riemann_entropy(nx=nx, seed=seed, P=P)
    c.bc = bc
    return c


def _step(torch, ctx, u_np, n_orders):
    u = torch.from_numpy(np.ascontiguousarray(u_np)).cuda()
    out = torch.empty_like(u)
    dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
    orders = torch.zeros(n_orders, dtype=torch.int8, device="cuda")
    ctx.acat_step(u, out, -1.0, None, dtv, orders)
    torch.cuda.synchronize()
    return out.cpu().numpy(), float(dtv.item()), orders.cpu().numpy()


CASES_1D = [("euler", 2, 777, 1, 1, 0), ("euler", 4, 1001, 1, 0, 1), ("euler", 3, 999, 0, 0, 2),
            ("euler", 2, 640, 1, 1, 2), ("burgers", 2, 400, 0, 1, 2), ("burgers", 3, 333, 1, 1, 1),
            ("linear", 3, 257, 0, 0, 1), ("linear", 2, 130, 1, 1, 2), ("euler", 4, 12001, 1, 1, 2),
            ("euler", 1, 300, 1, 0, 2)]


@pytest.mark.parametrize("kind,P,nx,bc,mod,lo", CASES_1D)
def test_single_step_1d_variants(env, kind, P, nx, bc, mod, lo):
    torch, O, acat = env
    c = _case1(kind, P, nx, bc)
    kw = dict(c.problem_kwargs(), psi2_mod=mod, lo_flux=lo)
    with acat.Context(**kw) as ctx:
        out, dt, orders = _step(torch, ctx, c.u0, nx + 1)
        assert ctx.acat_status() == 0
    pr = O.Problem(**kw)
    assert dt == O.dt_cfl(pr, c.u0)
    ref, _, ord_ref = O.step_1d(pr, c.u0, dt)
    assert np.array_equal(orders, ord_ref), np.nonzero(orders != ord_ref)
    if lo:
        assert np.any(orders == 1)  # the variant flux is exercised
    err = np.abs(out - ref).max() / max(1.0, np.abs(ref).max())
    assert err < 1e-12, err


def test_psi2_mod_on_midpoint_critical_points(env):
    """Data with critical points of order 1 at cell-interface midpoints
    0.5 (x_{i-1} + x_i) (Sec. 3.2): psi^2 rejects S_2 there, psi~^2 accepts
    it. The GPU's order map equals the oracle's under both switches, and the
    two maps differ."""
    torch, O, acat = env
    n = 50
    x = W.centres(n, 0.0, 1.0)
    h = 1.0 / n
    # f = (x - a)^2 + (x - a)^3 near each of three minima placed at cell centres
    # shifted by h/2 (the midpoint between two cells)
    u = np.ones(n)
    for a in (x[10] + 0.5 * h, x[25] + 0.5 * h, x[40] + 0.5 * h):
        u += np.exp(-((x - a) / 0.06) ** 2) * (-(x - a) ** 2 - (x - a) ** 3)
    u = u[None, :]
    maps = []
    for mod in (0, 1):
        kw = dict(flux=W.BURGERS, P=2, nx=n, ny=1, bc=0, cfl=0.5, x0=0.0, x1=1.0, psi2_mod=mod)
        with acat.Context(**kw) as ctx:
            _, dt, orders = _step(torch, ctx, u, n + 1)
        pr = O.Problem(**kw)
        _, _, ref = O.step_1d(pr, u, dt)
        assert np.array_equal(orders, ref)
        maps.append(orders)
    assert np.sum(maps[1] == 2) > np.sum(maps[0] == 2), (maps[0], maps[1])


@pytest.mark.parametrize("kind,P,nx,bc,mod,lo", [("euler", 2, 777, 1, 1, 2), ("euler", 4, 1001, 1, 0, 1),
                                                 ("burgers", 2, 400, 0, 1, 2), ("euler", 3, 12001, 0, 1, 1)])
def test_single_step_1d_variants_f32(env, kind, P, nx, bc, mod, lo):
    torch, O, acat = env
    c = _case1(kind, P, nx, bc, seed=2)
    kw = dict(c.problem_kwargs(), psi2_mod=mod, lo_flux=lo)
    pair = acat.to_pair(c.u0)
    x = acat.from_pair(pair)
    with acat.Context(**kw, precision=acat.PREC_F32) as ctx:
        out, dt, orders = _step(torch, ctx, pair, nx + 1)
        assert ctx.acat_status() == 0
    pr = O.Problem(**kw)
    assert dt == O.dt_cfl(pr, x)
    ref, _, ord_ref = O.step_1d(pr, x, dt)
    assert np.array_equal(orders, ord_ref)
    err = np.abs(acat.from_pair(out) - ref).max() / max(1.0, np.abs(ref).max())
    assert err < 1e-7, err


@pytest.mark.parametrize("prec,mod,lo", [("f64", 1, 2), ("f64", 0, 1), ("f32", 1, 2), ("f32", 1, 1)])
def test_single_step_2d_variants(env, prec, mod, lo):
    torch, O, acat = env
    nx, ny = 47, 44
    c = W.euler2d_quadrants(n=nx, ny=ny, seed=1, P=2)
    kw = dict(c.problem_kwargs(), psi2_mod=mod, lo_flux=lo)
    f32 = prec == "f32"
    u = acat.to_pair(c.u0) if f32 else c.u0
    x = acat.from_pair(u) if f32 else c.u0
    with acat.Context(**kw, precision=acat.PREC_F32 if f32 else acat.PREC_F64) as ctx:
        out, dt, o = _step(torch, ctx, u, ny * (nx + 1) + (ny + 1) * nx)
        assert ctx.acat_status() == 0
    ox, oy = o[:ny * (nx + 1)].reshape(ny, nx + 1), o[ny * (nx + 1):].reshape(ny + 1, nx)
    pr = O.Problem(**kw)
    assert dt == O.dt_cfl(pr, x)
    ref, _, rox, roy = O.step_2d(pr, x, dt)
    assert np.array_equal(ox, rox) and np.array_equal(oy, roy)
    assert np.any(ox == 1) or np.any(oy == 1)
    got = acat.from_pair(out) if f32 else out
    err = np.abs(got - ref).max() / max(1.0, np.abs(ref).max())
    assert err < (1e-7 if f32 else 1e-12), err


def test_batched_variants_equal_single_runs(env):
    torch, O, acat = env
    sizes = [64, 333, 1001, 40]
    cases = [W.euler1d_riemann_entropy(nx=n, seed=80 + b, P=3) for b, n in enumerate(sizes)]
    kw = dict(cases[0].problem_kwargs(), psi2_mod=1, lo_flux=2)
    u = np.ascontiguousarray(np.concatenate([c.u0 for c in cases], axis=1))
    with acat.Context(**kw, sizes=sizes) as ctx:
        ug = torch.from_numpy(u).cuda()
        ctx.acat_run(ug, 37)
        torch.cuda.synchronize()
        got = ug.cpu().numpy()
    offs = np.r_[0, np.cumsum(sizes)]
    for b, c in enumerate(cases):
        with acat.Context(**{**kw, "nx": c.nx}) as one:
            v = torch.from_numpy(c.u0.copy()).cuda()
            one.acat_run(v, 37)
            torch.cuda.synchronize()
            assert np.array_equal(got[:, offs[b]:offs[b + 1]], v.cpu().numpy()), b


@pytest.mark.parametrize("mod,lo,kind", [(1, 0, "euler"), (0, 1, "euler"), (0, 2, "euler"), (1, 2, "euler"),
                                         (0, 2, "burgers"), (0, 1, "burgers")])
def test_adjoint_with_variants(env, mod, lo, kind):
    """J^T of one step with psi~^2 and the F^lo variants (global LF, HLL)
    against the complex-step Jacobian of the oracle (its discrete choices,
    the HLL branch and bounds among them, taken on real parts)."""
    torch, O, acat = env
    if kind == "euler":
        c = W.euler1d_riemann_entropy(nx=24, seed=0, P=2)
    else:
        c = _case1("burgers", 2, 24, 1)
    kw = dict(c.problem_kwargs(), psi2_mod=mod, lo_flux=lo)
    pr = O.Problem(**kw)
    u = c.u0
    dt = O.dt_cfl(pr, u)
    _, _, orders = O.step_1d(pr, u, dt)
    assert np.any(orders == 1)  # FL-CAT2 interfaces, where F^lo enters
    h = 1e-30
    J = np.zeros((u.size, u.size))
    for k in range(u.size):
        e = np.zeros(u.size)
        e[k] = h
        _, im = O.step_1d_complex(pr, u, e.reshape(u.shape), dt)
        J[:, k] = im.ravel() / h
    w = np.random.default_rng(1).normal(size=u.shape)
    ref = (J.T @ w.ravel()).reshape(u.shape)
    with acat.Context(**kw) as ctx:
        out = torch.empty(u.shape, dtype=torch.float64, device="cuda")
        ctx.acat_adjoint_step(torch.from_numpy(u.copy()).cuda(), dt, torch.from_numpy(w).cuda(), out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-10
