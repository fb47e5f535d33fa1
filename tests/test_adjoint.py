"""The hand-written adjoint step and the checkpointed gradient.

Single step: the GPU adjoint J^T w equals the transpose of the Jacobian that
the oracle's complex-step instantiation computes column by column (branches
on real parts, dt fixed), element by element to 1e-10 relative plus the
conditioning bound of the FL-CAT2 blend (below).
Many steps: <ubar_0, d> equals <ubar_N, J_N ... J_1 d> with the products
J d propagated by complex-step oracle steps along the GPU's own trajectory
(real parts and dt taken from the GPU forward), and,
on the 1D Euler acoustic-pulse configuration (N = 8192, P = 2, 2000 steps,
periodic), the gradient of the L2 misfit matches central finite differences
of the replayed map on 32 random directions.
"""
import math

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
    from paper_2007_01416_gb300 import acat, adjoint, build
    build.build()
    O.build()
    return torch, O, acat, adjoint


def _jacobian(O, pr, u, dt):
    h = 1e-30
    n = u.size
    J = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        _, im = O.step_1d_complex(pr, u, e.reshape(u.shape), dt)
        J[:, k] = im.ravel() / h
    return J


def _blend_conditioning(pr, u, dt, orders, flux, w):
    """Entry-wise bound on how far two correct evaluations of J^T w may differ.

    At an FL-CAT2 interface (Eq. 3.4) the flux is F_lo + psi^1 (F_1 - F_lo),
    so the Jacobian holds d psi^1/du (F_1 - F_lo). Where the state is nearly
    constant the limiter ratio r = (upwind jump)/(local jump) has a tiny
    denominator: |d psi/du| reaches 2 (1 + |r|)/|local jump| while F_1 - F_lo
    carries a rounding error of a few ulps of |F|. Two evaluations that round
    differently (FMA contraction, operation order) then differ in that entry
    by about |d psi/du| * eps * |F| * dt/dx, which the tolerance admits."""
    N, s = pr.nx, pr.nvars
    q = u.reshape(s, N)
    wv = w.reshape(s, N)
    err = np.zeros((s, N))
    fscale = np.abs(flux).max()
    per_flux = 64 * np.finfo(float).eps * fscale * dt / pr.dx

    def cell(j):
        return j % N if pr.bc == 0 else min(max(j, 0), N - 1)

    for m in np.nonzero(orders == 1)[0]:
        i = m - 1
        wsum = sum(abs(wv[c2, cell(i)]) + abs(wv[c2, cell(i + 1)]) for c2 in range(s))
        for c in range(s):
            qq = [q[c, cell(j)] for j in range(i - 1, i + 3)]
            loc = qq[2] - qq[1]
            if loc == 0.0:
                continue
            for upw, cells in ((qq[1] - qq[0], (i - 1, i, i + 1)), (qq[3] - qq[2], (i, i + 1, i + 2))):
                r = upw / loc
                slope = 2.0 if 0.0 < r < 0.5 else (1.0 if 1.0 < r < 2.0 else 0.0)
                if slope == 0.0:
                    continue
                d = slope * (1.0 + abs(r)) / abs(loc) * per_flux * wsum
                for j in cells:
                    err[c, cell(j)] += d
    return err


def _state(kind, N, P, bc, seed=0):
    if kind == "riemann":
        c = W.euler1d_riemann_entropy(nx=N, seed=seed, P=P)
    elif kind == "pulse":
        c = W.acoustic_pulse(nx=N, seed=seed, P=P)
        c.u0[1] += 0.3 * c.u0[0]  # moving, so every component varies
    elif kind == "burgers":
        c = W.burgers_sine(nx=N, seed=seed, P=P)
    else:
        c = W.burgers_sine(nx=N, seed=seed, P=P)
        c.flux = W.LINEAR
        c.adv = (0.8, 0.0)
    c.bc = bc
    return c


@pytest.mark.parametrize("kind,P,N,bc", [("riemann", 2, 24, 1), ("riemann", 3, 28, 1), ("riemann", 4, 32, 0),
                                         ("pulse", 2, 24, 0), ("burgers", 2, 30, 0), ("burgers", 3, 30, 1),
                                         ("linear", 3, 26, 0), ("riemann", 1, 20, 1)])
def test_adjoint_step_is_jacobian_transpose(env, kind, P, N, bc):
    torch, O, acat, adjoint = env
    c = _state(kind, N, P, bc)
    kw = c.problem_kwargs()
    pr = O.Problem(**kw)
    u = c.u0
    dt = O.dt_cfl(pr, u)
    J = _jacobian(O, pr, u, dt)
    rng = np.random.default_rng(1)
    w = rng.normal(size=u.shape)
    ref = (J.T @ w.ravel()).reshape(u.shape)
    _, _, orders, flux = O.step_1d(pr, u, dt, want_flux=True)
    with acat.Context(**kw) as ctx:
        ug = torch.from_numpy(u.copy()).cuda()
        wb = torch.from_numpy(w).cuda()
        out = torch.empty_like(wb)
        ctx.acat_adjoint_step(ug, dt, wb, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    tol = 1e-10 * np.abs(ref).max() + _blend_conditioning(pr, u, dt, orders, flux, w)
    excess = np.abs(got - ref) - tol
    assert excess.max() <= 0.0, (np.unravel_index(excess.argmax(), excess.shape),
                                 np.abs(got - ref).max() / np.abs(ref).max(), np.bincount(orders))


def _smooth_euler(N):
    """Periodic Euler state with every component varying everywhere."""
    x = W.centres(N, 0.0, 1.0)
    rho = 1.0 + 0.2 * np.sin(2 * math.pi * x) + 0.1 * np.sin(6 * math.pi * x + 1.0)
    vel = 0.3 + 0.1 * np.cos(2 * math.pi * x)
    p = 1.0 + 0.2 * np.sin(4 * math.pi * x + 0.5)
    c = W.euler1d_riemann_entropy(nx=N, seed=0, P=3)
    c.u0 = W.prim_to_cons_1d(rho, vel, p)
    c.bc = 0
    return c


@pytest.mark.parametrize("kind", ["riemann", "smooth"])
def test_adjoint_many_steps_dot_complex_step(env, kind):
    """<ubar_0, d> = <w_N, J_N ... J_1 d> over 60 steps.

    Each J_n is the complex-step Jacobian at the GPU's state u^n and dt^n.
    The two sides may differ by the blend conditioning of every step,
    sum_n sum_k E_n[k] |v_n[k]|, with v_n the tangent entering step n and E_n
    the entry-wise bound of the single-step test for the adjoint w_{n+1}."""
    torch, O, acat, adjoint = env
    c = _state("riemann", 512, 3, 1, seed=2) if kind == "riemann" else _smooth_euler(512)
    kw = c.problem_kwargs()
    pr = O.Problem(**kw)
    nsteps = 60
    rng = np.random.default_rng(3)
    wN = rng.normal(size=c.u0.shape)
    with acat.Context(**kw) as ctx:
        u0 = torch.from_numpy(c.u0.copy()).cuda().requires_grad_(True)
        uN = adjoint.run(u0, ctx, nsteps, every=7)
        (uN * torch.from_numpy(wN).cuda()).sum().backward()
        g0 = u0.grad.cpu().numpy()
        # the GPU forward trajectory: states u^n and the dt of each step
        dts, states = [], []
        u = torch.from_numpy(c.u0.copy()).cuda()
        nxt = torch.empty_like(u)
        dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(nsteps):
            states.append(u.cpu().numpy())
            ctx.acat_step(u, nxt, -1.0, None, dtv, None)
            dts.append(float(dtv.item()))
            u, nxt = nxt, u
        # adjoints w_{n+1} entering each reverse step, for the bound
        ws = [None] * (nsteps + 1)
        ws[nsteps] = wN
        wb = torch.from_numpy(wN.copy()).cuda()
        out = torch.empty_like(wb)
        for n in reversed(range(nsteps)):
            ctx.acat_adjoint_step(torch.from_numpy(states[n]).cuda(), dts[n], wb, out)
            wb, out = out, wb
            ws[n] = wb.cpu().numpy()
    assert np.allclose(ws[0], g0, rtol=0, atol=1e-12 * np.abs(g0).max())
    x = np.linspace(0, 1, c.nx)
    d = np.stack([np.sin(2 * math.pi * x + k) for k in range(3)])
    h = 1e-30
    im = h * d
    bound = 0.0
    for n in range(nsteps):
        _, _, orders, flux = O.step_1d(pr, states[n], dts[n], want_flux=True)
        E = _blend_conditioning(pr, states[n], dts[n], orders, flux, ws[n + 1])
        bound += float((E * np.abs(im / h)).sum())
        # J(u^n) applied to the tangent, with the branches the GPU took
        _, im = O.step_1d_complex(pr, states[n], im, dts[n])
    lhs = float((g0 * d).sum())
    rhs = float((wN * im / h).sum())
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs) + bound, (lhs, rhs, bound)


def test_gradient_acoustic_pulse_finite_differences(env):
    """1D Euler P = 2, N = 8192 periodic, 2000 steps, isentropic pulse;
    L = dx/2 sum |u^N - u_target|^2 with the target from a second seed."""
    torch, O, acat, adjoint = env
    c = W.acoustic_pulse(nx=8192, seed=0, P=2, steps=2000)
    tgt_case = W.acoustic_pulse(nx=8192, seed=1, P=2, steps=2000)
    kw = c.problem_kwargs()
    dx = (c.x1 - c.x0) / c.nx
    with acat.Context(**kw) as ctx:
        target = torch.from_numpy(tgt_case.u0.copy()).cuda()
        ctx.acat_run(target, c.steps)
        u0 = torch.from_numpy(c.u0.copy()).cuda().requires_grad_(True)
        uN = adjoint.run(u0, ctx, c.steps)
        loss = 0.5 * dx * ((uN - target) ** 2).sum()
        loss.backward()
        g = u0.grad.detach()
        # the dt sequence of the forward pass, for the replayed map
        dts, u = [], torch.from_numpy(c.u0.copy()).cuda()
        nxt = torch.empty_like(u)
        dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(c.steps):
            ctx.acat_step(u, nxt, -1.0, None, dtv, None)
            dts.append(float(dtv.item()))
            u, nxt = nxt, u

        def L(v):
            w = adjoint.replay(v, ctx, dts)
            return float((0.5 * dx * ((w - target) ** 2).sum()).item())

        rng = np.random.default_rng(7)
        x = torch.linspace(0, 1, c.nx, dtype=torch.float64, device="cuda")
        worst = 0.0
        for k in range(32):
            # smooth random direction, unit max-norm
            a, ph = rng.uniform(-1, 1, size=(3, 3)), rng.uniform(0, 2 * math.pi, size=(3, 3))
            d = torch.stack([sum(a[cc, m] * torch.sin(2 * math.pi * (m + 1) * x + ph[cc, m])
                                 for m in range(3)) for cc in range(3)])
            d = d / d.abs().max()
            eps = 1e-6
            fd = (L(u0.detach() + eps * d) - L(u0.detach() - eps * d)) / (2 * eps)
            ad = float((g * d).sum().item())
            worst = max(worst, abs(fd - ad) / max(abs(ad), 1e-12))
        assert worst < 1e-5, worst


def test_record_and_reverse_run_checkpoint_intervals(env):
    """The recorded forward equals acat_run, its checkpoints are the states
    it passed, and the reverse run gives the same cotangent for every
    checkpoint interval (the recompute is bit-identical to the forward)."""
    torch, O, acat, adjoint = env
    c = _state("riemann", 256, 3, 1, seed=4)
    n = 23
    with acat.Context(**c.problem_kwargs()) as ctx:
        u0 = torch.from_numpy(c.u0.copy()).cuda()
        ref = u0.clone()
        ctx.acat_run(ref, n)
        wN = torch.from_numpy(np.random.default_rng(5).normal(size=c.u0.shape)).cuda()
        outs = []
        for every in (1, 4, 7, 23, 40):
            nck = -(-n // every)
            ckpt = torch.empty((nck,) + tuple(u0.shape), dtype=torch.float64, device="cuda")
            dts = torch.empty(n, dtype=torch.float64, device="cuda")
            uN = torch.empty_like(u0)
            ctx.acat_run_record(u0, uN, n, every, ckpt, dts)
            assert torch.equal(uN, ref)
            assert torch.equal(ckpt[0], u0)
            if nck > 1:
                v = u0.clone()
                ctx.acat_run(v, every)
                assert torch.equal(ckpt[1], v)
            g = torch.empty_like(u0)
            ctx.acat_adjoint_run(ckpt, dts, n, every, wN, g)
            g2 = wN.clone()
            ctx.acat_adjoint_run(ckpt, dts, n, every, g2, g2)  # in place
            assert torch.equal(g, g2)
            outs.append(g.cpu().numpy())
        assert ctx.acat_status() == 0
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


# ---------------------------------------------------------------------------
# FP32 adjoint (compensated state and cotangent)
# ---------------------------------------------------------------------------
F32_STEP_TOL = 2e-6


@pytest.mark.parametrize("kind,P,N,bc", [("riemann", 2, 64, 1), ("riemann", 3, 96, 1), ("riemann", 4, 128, 0),
                                         ("pulse", 2, 64, 0), ("burgers", 3, 60, 1)])
def test_adjoint_step_f32_matches_f64(env, kind, P, N, bc):
    """The FP32 adjoint step against the FP64 adjoint step at the same state
    value hi + lo (same order decisions): float rounding of the reverse sweep
    only. Bound: a node cotangent is a sum of about 30 products of O(1)
    Jacobian entries and weights with the interface cotangent, each rounded
    within eps32 = 6e-8 of its size: 30 x 6e-8 < 2e-6 of max|J^T w| (observed
    2e-7)."""
    torch, O, acat, adjoint = env
    c = _state(kind, N, P, bc)
    kw = c.problem_kwargs()
    pair = acat.to_pair(c.u0)
    x = acat.from_pair(pair)
    pr = O.Problem(**kw)
    dt = O.dt_cfl(pr, x)
    w = np.random.default_rng(11).normal(size=c.u0.shape)
    with acat.Context(**kw) as c64, acat.Context(**kw, precision=acat.PREC_F32) as c32:
        out64 = torch.empty(c.u0.shape, dtype=torch.float64, device="cuda")
        c64.acat_adjoint_step(torch.from_numpy(x).cuda(), dt, torch.from_numpy(w).cuda(), out64)
        wp = torch.from_numpy(acat.to_pair(w)).cuda()
        out32 = torch.empty_like(wp)
        c32.acat_adjoint_step(torch.from_numpy(pair).cuda(), dt, wp, out32)
        torch.cuda.synchronize()
        ref = out64.cpu().numpy()
        got = acat.from_pair(out32.cpu().numpy())
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"f32 adjoint {kind} P={P}: rel err {err:.2e}")
    assert err < F32_STEP_TOL, err


def test_adjoint_run_f32_along_its_trajectory(env):
    """60 steps: the FP32 gradient (recorded FP32 forward, FP32 reverse run)
    against FP64 adjoint steps applied along the same FP32 trajectory (states
    hi + lo, recorded dt); per-step float rounding accumulates at most
    linearly: 60 x 2e-6 (observed 2e-6)."""
    torch, O, acat, adjoint = env
    c = _state("riemann", 512, 3, 1, seed=2)
    kw = c.problem_kwargs()
    n = 60
    wN = np.random.default_rng(3).normal(size=c.u0.shape)
    with acat.Context(**kw, precision=acat.PREC_F32) as c32, acat.Context(**kw) as c64:
        u0 = torch.from_numpy(acat.to_pair(c.u0)).cuda().requires_grad_(True)
        uN = adjoint.run(u0, c32, n, every=7)
        (uN * torch.from_numpy(np.stack([wN, wN])).cuda().float()).sum().backward()
        g32 = u0.grad[0].double().cpu().numpy()
        assert np.array_equal(u0.grad[0].cpu().numpy(), u0.grad[1].cpu().numpy())
        # the FP32 trajectory and its dt: the recorded run with every state kept
        p0 = torch.from_numpy(acat.to_pair(c.u0)).cuda()
        ckpt = torch.empty((n,) + tuple(p0.shape), dtype=torch.float32, device="cuda")
        dtt = torch.empty(n, dtype=torch.float64, device="cuda")
        c32.acat_run_record(p0, torch.empty_like(p0), n, 1, ckpt, dtt)
        torch.cuda.synchronize()
        states = [acat.from_pair(ckpt[k].cpu().numpy()) for k in range(n)]
        dts = dtt.cpu().tolist()
        wb = torch.from_numpy(wN.copy()).cuda()
        out = torch.empty_like(wb)
        for k in reversed(range(n)):
            c64.acat_adjoint_step(torch.from_numpy(states[k]).cuda(), dts[k], wb, out)
            wb, out = out, wb
        g64 = wb.cpu().numpy()
    err = np.abs(g32 - g64).max() / np.abs(g64).max()
    print(f"f32 gradient 60 steps: rel err {err:.2e}")
    assert err < n * F32_STEP_TOL, err


def test_gradient_acoustic_pulse_against_reference_sweep(env):
    """C5 in FP64 (1D Euler P = 2, N = 8192 periodic, 2000 steps, isentropic
    pulse, L = dx/2 sum |u^N - u_target|^2): the GPU's dL/du^0 element by
    element against the oracle's reverse sweep (oracle/adjoint_ref.py, the
    step restated in PyTorch CPU float64 and differentiated by autograd, with
    the orders the C oracle selects at each state). Both sweep the trajectory
    the GPU recorded (every state and dt), so the two take the same discrete
    choices. Bar: 1e-10 of the entry plus 1e-12 of max |dL/du^0| (the floor
    takes the entries near zero)."""
    torch, O, acat, adjoint = env
    from oracle import adjoint_ref as A
    c = W.acoustic_pulse(nx=8192, seed=0, P=2, steps=2000)
    tgt_case = W.acoustic_pulse(nx=8192, seed=1, P=2, steps=2000)
    kw = c.problem_kwargs()
    dx = (c.x1 - c.x0) / c.nx
    n = c.steps
    with acat.Context(**kw) as ctx:
        target = torch.from_numpy(tgt_case.u0.copy()).cuda()
        ctx.acat_run(target, n)
        u0 = torch.from_numpy(c.u0.copy()).cuda()
        ckpt = torch.empty((n,) + tuple(u0.shape), dtype=torch.float64, device="cuda")
        dts = torch.empty(n, dtype=torch.float64, device="cuda")
        uN = torch.empty_like(u0)
        ctx.acat_run_record(u0, uN, n, 1, ckpt, dts)  # every state of the run
        wN = dx * (uN - target)
        g = torch.empty_like(u0)
        ctx.acat_adjoint_run(ckpt, dts, n, 1, wN, g)
        torch.cuda.synchronize()
        assert ctx.acat_status() == 0
        states, dt_seq = ckpt.cpu().numpy(), dts.cpu().numpy()
        got, w_last = g.cpu().numpy(), wN.cpu().numpy()
    del ckpt
    pr = O.Problem(**kw)
    ref = A.gradient(pr, states, dt_seq, w_last)
    bar = 1e-10 * np.abs(ref) + 1e-12 * np.abs(ref).max()
    err = np.abs(got - ref)
    print(f"C5 gradient against the reference sweep: max |err| / max |ref| {err.max() / np.abs(ref).max():.2e}, "
          f"max |err| / (|ref| + 1e-2 max|ref|) {(err / (np.abs(ref) + 1e-2 * np.abs(ref).max())).max():.2e}")
    assert (err <= bar).all(), (np.unravel_index((err - bar).argmax(), err.shape), err.max() / np.abs(ref).max())
