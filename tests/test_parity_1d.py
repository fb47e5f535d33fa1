"""Parity of the CUDA 1D step (through the C ABI) with the CPU oracle.

Bar: order codes bit-exact; FP64 states within 1e-12 relative to the state's
magnitude (max-norm) per step, and per element within 1e-12 of the magnitudes
the element is formed from, |u_i| + lam (|F_{i-1/2}| + |F_{i+1/2}|). Multi-step runs are compared step by step with
the oracle teacher-forced from the GPU state (each GPU step checked from the
same input), and free-running where the run is short.
"""
import math

import numpy as np
import pytest

from paper_2007_01416_gb300 import workloads as W

pytestmark = pytest.mark.gpu
RTOL = 1e-12
# per element, against |u_i| + lam (|F_{i-1/2}| + |F_{i+1/2}|): the recursion's
# rounding is a few units of 1e-16 of the flux terms, the update's of |u_i|
RTOL_ELEM = 1e-12


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


def _step(env, ctx, u_np, nx, dt=-1.0):
    torch, O, acat = env
    u = torch.from_numpy(np.ascontiguousarray(u_np)).cuda()
    out = torch.empty_like(u)
    dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
    orders = torch.zeros(nx + 1, dtype=torch.int8, device="cuda")
    ctx.acat_step(u, out, dt, None, dtv, orders)
    torch.cuda.synchronize()
    return out.cpu().numpy(), float(dtv.item()), orders.cpu().numpy()


def _cmp(gpu, ref):
    scale = max(1.0, np.abs(ref).max())
    return np.abs(gpu - ref).max() / scale


def _cmp_elem(gpu, ref, u_in, flux, lam):
    """Largest per-element error relative to the magnitudes the element is
    formed from: |u_i| + lam (|F_{i-1/2}| + |F_{i+1/2}|) per component (the
    terms of Eq. 2.12; flux [nx+1, s] from the oracle). A small component
    (momentum near rest) is held to its own scale, not to max |u|."""
    floor = np.abs(u_in) + lam * (np.abs(flux[:-1]) + np.abs(flux[1:])).T
    return (np.abs(gpu - ref) / np.maximum(floor, 1e-300)).max()


CASES = [
    ("burgers", 2, 400, 0), ("burgers", 3, 333, 1), ("burgers", 1, 97, 1), ("burgers", 4, 1000, 0),
    ("linear", 4, 257, 0), ("linear", 2, 130, 1),
    ("euler", 4, 16384, 1), ("euler", 3, 1001, 1), ("euler", 2, 777, 0), ("euler", 1, 64, 1),
    ("euler", 4, 16, 0), ("euler", 2, 8, 1),
    # sizes large enough for the small-CTA step with the boundary hand-off
    ("euler", 3, 12001, 0), ("burgers", 4, 15001, 1), ("linear", 2, 30001, 0), ("euler", 1, 40001, 1),
]


def _case(kind, P, nx, bc, seed=0):
    if kind == "burgers":
        c = W.burgers_sine(nx=nx, seed=seed, P=P)
    elif kind == "linear":
        c = W.burgers_sine(nx=nx, seed=seed, P=P)
        c.flux = W.LINEAR
        c.adv = (-0.7, 0.0)
    else:
        c = W.euler1d_riemann_entropy(nx=nx, seed=seed, P=P)
    c.bc = bc
    return c


@pytest.mark.parametrize("kind,P,nx,bc", CASES)
def test_single_step(env, kind, P, nx, bc):
    torch, O, acat = env
    c = _case(kind, P, nx, bc)
    kw = c.problem_kwargs()
    with acat.Context(**kw) as ctx:
        out, dt, orders = _step(env, ctx, c.u0, nx)
        assert ctx.acat_status() == 0
    pr = O.Problem(**kw)
    dt_ref = O.dt_cfl(pr, c.u0)
    assert dt == dt_ref  # same FP64 expression, correctly rounded operations
    ref, _, ord_ref, F = O.step_1d(pr, c.u0, dt, want_flux=True)
    assert np.array_equal(orders, ord_ref), np.nonzero(orders != ord_ref)
    assert _cmp(out, ref) < RTOL
    assert _cmp_elem(out, ref, c.u0, F, dt / pr.dx) < RTOL_ELEM


@pytest.mark.parametrize("kind,P,nx,bc,steps", [("burgers", 2, 400, 0, 300), ("euler", 4, 2048, 1, 200),
                                               ("euler", 3, 1500, 0, 150), ("burgers", 4, 300, 0, 200)])
def test_teacher_forced_run(env, kind, P, nx, bc, steps):
    torch, O, acat = env
    c = _case(kind, P, nx, bc, seed=3)
    kw = c.problem_kwargs()
    pr = O.Problem(**kw)
    u = c.u0.copy()
    worst = worst_e = 0.0
    with acat.Context(**kw) as ctx:
        for n in range(steps):
            out, dt, orders = _step(env, ctx, u, nx)
            ref, _, ord_ref, F = O.step_1d(pr, u, dt, want_flux=True)
            assert np.array_equal(orders, ord_ref), (n, np.nonzero(orders != ord_ref))
            worst = max(worst, _cmp(out, ref))
            worst_e = max(worst_e, _cmp_elem(out, ref, u, F, dt / pr.dx))
            u = out
        assert ctx.acat_status() == 0
    assert worst < RTOL, worst
    assert worst_e < RTOL_ELEM, worst_e


def test_free_run_burgers_config(env):
    # 1D Burgers P=2, N=400, periodic, CFL 0.5, 300 steps past shock formation
    torch, O, acat = env
    c = W.burgers_sine(nx=400, seed=0, P=2, steps=300)
    kw = c.problem_kwargs()
    pr = O.Problem(**kw)
    with acat.Context(**kw) as ctx:
        u = torch.from_numpy(c.u0.copy()).cuda()
        t = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.acat_run(u, c.steps, -1.0, None, t)
        torch.cuda.synchronize()
        assert ctx.acat_status() == 0
        ug = u.cpu().numpy()
    uo = c.u0.copy()
    tt = 0.0
    for _ in range(c.steps):
        uo, dt, _ = O.step_1d(pr, uo)
        tt += dt
    b = float(np.abs(c.u0).max())
    assert tt > 1.0 / (math.pi * 1.0)  # past the shock time for every seeded b <= 1
    assert abs(t.item() - tt) <= 1e-12 * tt
    assert _cmp(ug, uo) < 1e-10, _cmp(ug, uo)
    # discrete conservation on the periodic grid
    assert abs(math.fsum(ug[0]) - math.fsum(c.u0[0])) < 1e-11 * 400 * b


@pytest.mark.parametrize("nx", [3000, 20001])  # 8-warp fused step, small-CTA step
def test_run_equals_repeated_steps(env, nx):
    torch, O, acat = env
    c = W.euler1d_riemann_entropy(nx=nx, seed=5, P=4, steps=101)
    kw = c.problem_kwargs()
    with acat.Context(**kw) as ctx:
        u = torch.from_numpy(c.u0.copy()).cuda()
        ctx.acat_run(u, 101)
        v = torch.from_numpy(c.u0.copy()).cuda()
        w = torch.empty_like(v)
        for _ in range(101):
            ctx.acat_step(v, w)
            v, w = w, v
        torch.cuda.synchronize()
        assert torch.equal(u, v)


@pytest.mark.parametrize("prec,nx", [(0, 3000), (0, 20001), (1, 3000), (1, 16384)])
def test_steps_ordered_with_stream_kernels(env, prec, nx):
    """The 1D step kernels are launched with programmatic stream serialization:
    each waits for the previous kernel of the stream before any memory access.
    Steps and runs interleaved with PyTorch kernels that write their input and
    read and overwrite their output, with no synchronisation in between, give
    the bits of the same sequence synchronised after every operation (FP64
    fused and small-CTA grids; FP32 8- and 7-warp tiles)."""
    torch, O, acat = env
    c = W.euler1d_riemann_entropy(nx=nx, seed=11, P=4)
    u0 = torch.from_numpy(acat.to_pair(c.u0) if prec else c.u0.copy()).cuda()

    def sequence(sync):
        outs = []
        with acat.Context(**c.problem_kwargs(), precision=prec) as ctx:
            u, w = torch.empty_like(u0), torch.empty_like(u0)
            for k in range(12):
                u.copy_(u0)
                u.mul_(1.0 + 1e-3 * k)  # the step's input, written by stream kernels
                if sync:
                    torch.cuda.synchronize()
                if k % 3 == 2:
                    ctx.acat_run(u, 5)  # graph replay, in place
                    res = u
                else:
                    ctx.acat_step(u, w)
                    res = w
                if sync:
                    torch.cuda.synchronize()
                outs.append(res.clone())  # read by a stream kernel
                res.fill_(float("nan"))  # and overwritten before the next step
            torch.cuda.synchronize()
            assert ctx.acat_status() == 0
        return outs

    fast, slow = sequence(False), sequence(True)
    for x, y in zip(fast, slow):
        assert torch.equal(x, y)


@pytest.mark.parametrize("nx,t_end", [(1024, 0.01), (30001, 0.002)])
def test_t_end_clipping(env, nx, t_end):
    torch, O, acat = env
    c = W.euler1d_riemann_entropy(nx=nx, seed=6, P=2)
    kw = c.problem_kwargs()
    with acat.Context(**kw) as ctx:
        u = torch.from_numpy(c.u0.copy()).cuda()
        t = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.acat_run(u, 1000, t_end, None, t)
        torch.cuda.synchronize()
        assert t.item() == pytest.approx(t_end, rel=0, abs=1e-15)
        # every run starts at t = 0; steps past t_end do nothing
        v = torch.from_numpy(c.u0.copy()).cuda()
        ctx.acat_run(v, 1500, t_end)
        torch.cuda.synchronize()
        assert torch.equal(u, v)


def test_run_host_matches_device_run(env):
    torch, O, acat = env
    c = W.euler1d_riemann_entropy(nx=2000, seed=7, P=3)
    kw = c.problem_kwargs()
    with acat.Context(**kw) as ctx:
        u = torch.from_numpy(c.u0.copy()).cuda()
        ctx.acat_run(u, 57)
        host = torch.from_numpy(c.u0.copy()).pin_memory()
        out = torch.empty_like(host).pin_memory()
        ctx.acat_run_host(host, out, 57)
        torch.cuda.synchronize()
        assert torch.equal(out, u.cpu())


@pytest.mark.parametrize("step", [0, 1500, 3999])
def test_full_size_euler_sampled(env, step):
    """1D Euler P=4, N=16384, transmissive, CFL 0.4, in the launch
    configuration of the benchmark: the GPU state after `step` steps is
    advanced one more step by the GPU and by the oracle at 512 sampled cells
    (plus the fixed ends) from the same input and dt."""
    torch, O, acat = env
    c = W.euler1d_riemann_entropy(nx=16384, seed=0, P=4, steps=4000)
    kw = c.problem_kwargs()
    pr = O.Problem(**kw)
    with acat.Context(**kw) as ctx:
        u = torch.from_numpy(c.u0.copy()).cuda()
        if step:
            ctx.acat_run(u, step)
        torch.cuda.synchronize()
        un = u.cpu().numpy()
        out, dt, orders = _step(env, ctx, un, c.nx)
        assert ctx.acat_status() == 0
    rng = np.random.default_rng(step)
    cells = np.unique(np.r_[0, 1, 2, c.nx - 3, c.nx - 2, c.nx - 1,
                            rng.choice(c.nx, 512, replace=False)])
    ifaces = np.unique(np.r_[cells, cells + 1])
    F, ord_ref = O.fluxes_1d_at(pr, un, dt, ifaces)
    assert np.array_equal(orders[ifaces], ord_ref)
    ref = O.step_1d_cells(pr, un, dt, cells).T
    assert np.abs(out[:, cells] - ref).max() <= RTOL * max(1.0, np.abs(un).max())
    pos = np.searchsorted(ifaces, cells)
    lam = dt / pr.dx
    floor = np.abs(un[:, cells]) + lam * (np.abs(F[pos]) + np.abs(F[pos + 1])).T
    assert (np.abs(out[:, cells] - ref) <= RTOL_ELEM * floor).all()


def test_nonphysical_state_sets_status(env):
    torch, O, acat = env
    c = W.euler1d_riemann_entropy(nx=256, seed=1, P=2)
    u0 = c.u0.copy()
    u0[0, 100] = -1.0  # negative density
    with acat.Context(**c.problem_kwargs()) as ctx:
        _step(env, ctx, u0, c.nx)
        assert ctx.acat_status() & acat.STATUS_NONPHYSICAL
        ctx.acat_clear_status()
        assert ctx.acat_status() == 0
