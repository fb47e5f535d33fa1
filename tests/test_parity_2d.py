"""Parity of the CUDA 2D step (Sec. 4) with the CPU oracle.

FP64: order codes of both directions bit-exact, states within 1e-12 of
max|u| per step (teacher-forced over several steps). FP32 (delta form on the
compensated state): same order codes from the same state value, states within
1e-7 of max|u| per step.
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


def _step2(env, ctx, u_np, nx, ny, dt=-1.0):
    torch, O, acat = env
    u = torch.from_numpy(np.ascontiguousarray(u_np)).cuda()
    out = torch.empty_like(u)
    dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
    orders = torch.zeros(ny * (nx + 1) + (ny + 1) * nx, dtype=torch.int8, device="cuda")
    ctx.acat_step(u, out, dt, None, dtv, orders)
    torch.cuda.synchronize()
    o = orders.cpu().numpy()
    ox = o[:ny * (nx + 1)].reshape(ny, nx + 1)
    oy = o[ny * (nx + 1):].reshape(ny + 1, nx)
    return out.cpu().numpy(), float(dtv.item()), ox, oy


def _transport(nx, ny, P, bc):
    x = W.centres(nx, 0, 1)[None, :]
    y = W.centres(ny, 0, 1)[:, None]
    u = (np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0.5 * (x + 0 * y > 0.55))[None]
    c = W.Case("transport2d", W.LINEAR, P, nx, ny, bc, 0.5, 0, 1, 0, 1, u, 1, adv=(0.7, -0.4))
    return c


CASES = [
    ("lax_liu_4", 2, 33, 30, 1), ("lax_liu_6", 2, 40, 16, 1), ("lax_liu_8", 1, 31, 31, 1),
    ("quadrants", 2, 47, 44, 1), ("quadrants", 2, 32, 32, 0), ("quadrants", 1, 20, 23, 0),
    ("transport", 2, 45, 38, 0), ("transport", 1, 30, 17, 1), ("quadrants", 2, 8, 9, 1),
    # P = 3, 4: the shared-memory block kernel (square blocks S_p1, S_p2). Four-
    # quadrant Euler data is left out at these orders: with square blocks the
    # row/column indicators do not see a transverse jump inside the 2p x 2p
    # block, and one step already produces negative pressures (the oracle's
    # too); the cases below are smooth Euler data with a contact and transport
    ("smooth2d", 3, 97, 90, 1), ("smooth2d", 4, 96, 96, 0), ("smooth2d", 3, 50, 61, 0),
    ("transport", 3, 30, 28, 0), ("transport", 4, 26, 25, 1),
]


def _smooth2d(nx, ny, P, bc):
    """Smooth 2D Euler data with a contact at x = 0.6 (u, v, p continuous)."""
    x = W.centres(nx, 0, 1)[None, :]
    y = W.centres(ny, 0, 1)[:, None]
    rho = 1 + 0.2 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) + 0.3 * (x + 0 * y > 0.6)
    u = 0.3 + 0.1 * np.cos(2 * np.pi * y) + 0 * x
    v = -0.2 + 0.1 * np.sin(2 * np.pi * x) + 0 * y
    p = 1 + 0.1 * np.cos(2 * np.pi * (x + y))
    return W.Case("smooth2d", W.EULER2D, P, nx, ny, bc, 0.4, 0, 1, 0, 1, W.prim_to_cons_2d(rho, u, v, p), 1)


def _case(kind, P, nx, ny, bc, seed=0):
    if kind.startswith("lax_liu"):
        c = W.lax_liu(int(kind.split("_")[-1]), nx, P)
        if ny != nx:
            c = W._quadrants(c.name, W.LAX_LIU[int(kind.split("_")[-1])], nx, ny, P, 1, c.cfl)
    elif kind == "quadrants":
        c = W.euler2d_quadrants(n=nx, ny=ny, seed=seed, P=P)
    elif kind == "smooth2d":
        c = _smooth2d(nx, ny, P, bc)
    else:
        c = _transport(nx, ny, P, bc)
    c.bc = bc
    return c


@pytest.mark.parametrize("kind,P,nx,ny,bc", CASES)
def test_single_step_2d(env, kind, P, nx, ny, bc):
    torch, O, acat = env
    c = _case(kind, P, nx, ny, bc)
    kw = c.problem_kwargs()
    with acat.Context(**kw) as ctx:
        out, dt, ox, oy = _step2(env, ctx, c.u0, nx, ny)
        assert ctx.acat_status() == 0
    pr = O.Problem(**kw)
    assert dt == O.dt_cfl(pr, c.u0)
    ref, _, rox, roy = O.step_2d(pr, c.u0, dt)
    assert np.array_equal(ox, rox), np.argwhere(ox != rox)[:5]
    assert np.array_equal(oy, roy), np.argwhere(oy != roy)[:5]
    err = np.abs(out - ref).max() / max(1.0, np.abs(ref).max())
    assert err < 1e-12, err


@pytest.mark.parametrize("P", [2, 3])
def test_teacher_forced_2d(env, P):
    torch, O, acat = env
    c = W.euler2d_quadrants(n=40, ny=36, seed=3, P=P) if P == 2 else _smooth2d(61, 58, P, 1)
    kw = c.problem_kwargs()
    pr = O.Problem(**kw)
    u = c.u0.copy()
    worst = 0.0
    with acat.Context(**kw) as ctx:
        for n in range(25):
            out, dt, ox, oy = _step2(env, ctx, u, c.nx, c.ny)
            ref, _, rox, roy = O.step_2d(pr, u, dt)
            assert np.array_equal(ox, rox) and np.array_equal(oy, roy), n
            worst = max(worst, np.abs(out - ref).max() / np.abs(ref).max())
            u = out
    assert worst < 1e-12, worst


@pytest.mark.parametrize("P", [2, 4])
def test_run_2d_matches_steps_and_conserves(env, P):
    torch, O, acat = env
    c = _transport(64, 48, P, 0)
    kw = c.problem_kwargs()
    with acat.Context(**kw) as ctx:
        u = torch.from_numpy(c.u0.copy()).cuda()
        ctx.acat_run(u, 53)
        v = torch.from_numpy(c.u0.copy()).cuda()
        w = torch.empty_like(v)
        for _ in range(53):
            ctx.acat_step(v, w)
            v, w = w, v
        torch.cuda.synchronize()
        assert torch.equal(u, v)
        s0, s1 = float(c.u0.sum()), float(u.sum().item())
        assert abs(s1 - s0) < 1e-11 * np.abs(c.u0).sum()


@pytest.mark.parametrize("kind,P,nx,ny,bc", [("quadrants", 2, 47, 44, 1), ("lax_liu_8", 2, 40, 40, 1),
                                             ("transport", 2, 45, 38, 0), ("quadrants", 1, 20, 23, 0)])
def test_single_step_2d_f32(env, kind, P, nx, ny, bc):
    torch, O, acat = env
    c = _case(kind, P, nx, ny, bc, seed=5)
    kw = c.problem_kwargs()
    pair = acat.to_pair(c.u0)
    xval = acat.from_pair(pair)
    with acat.Context(**kw, precision=acat.PREC_F32) as ctx:
        out, dt, ox, oy = _step2(env, ctx, pair, nx, ny)
        assert ctx.acat_status() == 0
    pr = O.Problem(**kw)
    assert dt == O.dt_cfl(pr, xval)
    ref, _, rox, roy = O.step_2d(pr, xval, dt)
    assert np.array_equal(ox, rox) and np.array_equal(oy, roy)
    err = np.abs(acat.from_pair(out) - ref).max() / max(1.0, np.abs(ref).max())
    assert err < 1e-7, err


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_full_size_2d_sampled(env, prec):
    """2D Euler P=2, 4096 x 4096, transmissive, CFL 0.4, in the launch
    configuration of the benchmark: after 3 GPU steps, one more GPU step is
    compared with the oracle's update of 256 sampled cells (and the four
    corners) from the same state and dt."""
    torch, O, acat = env
    c = W.euler2d_quadrants(n=4096, seed=0, P=2)
    kw = c.problem_kwargs()
    pr = O.Problem(**kw)
    f32 = prec == "f32"
    with acat.Context(**kw, precision=acat.PREC_F32 if f32 else acat.PREC_F64) as ctx:
        host = acat.to_pair(c.u0) if f32 else c.u0
        u = torch.from_numpy(host).cuda()
        ctx.acat_run(u, 3)
        out = torch.empty_like(u)
        dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.acat_step(u, out, -1.0, None, dtv, None)
        torch.cuda.synchronize()
        assert ctx.acat_status() == 0
        un = u.cpu().numpy()
        got = out.cpu().numpy()
    if f32:
        un, got = acat.from_pair(un), acat.from_pair(got)
    dt = float(dtv.item())
    assert dt == O.dt_cfl(pr, un)
    rng = np.random.default_rng(1)
    cx = np.r_[0, 4095, 0, 4095, 2047, 2048, rng.integers(0, 4096, 250)]
    cy = np.r_[0, 0, 4095, 4095, 2047, 2048, rng.integers(0, 4096, 250)]
    ref = O.step_2d_cells(pr, un, dt, cx, cy)
    gpu = got[:, cy, cx].T
    err = np.abs(gpu - ref).max() / np.abs(un).max()
    assert err < (1e-7 if f32 else 1e-12), err


# ---------------------------------------------------------------------------
# Rectangular stencils S_{p1,p2} (rect_2d = 1): one block of 2 p1 x 2 p2
# nodes per anchor, in the shared-memory block kernel (FP64, P = 2..4)
# ---------------------------------------------------------------------------
RECT_CASES = [("quadrants", 2, 40, 37, 1), ("quadrants", 3, 45, 40, 1), ("quadrants", 4, 40, 44, 0),
              ("quadrants", 4, 27, 13, 1), ("smooth2d", 3, 50, 61, 0), ("smooth2d", 4, 37, 33, 1),
              ("transport", 4, 26, 25, 1), ("transport", 3, 30, 28, 0), ("lax_liu_6", 3, 40, 16, 1)]


@pytest.mark.parametrize("kind,P,nx,ny,bc", RECT_CASES)
def test_single_step_2d_rect(env, kind, P, nx, ny, bc):
    torch, O, acat = env
    c = _case(kind, P, nx, ny, bc, seed=1)
    kw = dict(c.problem_kwargs(), rect_2d=1)
    with acat.Context(**kw) as ctx:
        out, dt, ox, oy = _step2(env, ctx, c.u0, nx, ny)
        assert ctx.acat_status() == 0
    pr = O.Problem(**kw)
    assert dt == O.dt_cfl(pr, c.u0)
    ref, _, rox, roy = O.step_2d(pr, c.u0, dt)
    assert np.array_equal(ox, rox), np.argwhere(ox != rox)[:5]
    assert np.array_equal(oy, roy), np.argwhere(oy != roy)[:5]
    err = np.abs(out - ref).max() / max(1.0, np.abs(ref).max())
    assert err < 1e-12, err
    if kind == "quadrants":
        # anchors with p1 != p2 and a block exist (at P = 2 the pairs (2, 1) and
        # (1, 2)), and there the rectangular block changes the flux
        px, py = ox[:, :-1], oy[:-1, :]
        assert np.any(((px >= 2) | (py >= 2)) & (px != py))
        with acat.Context(**c.problem_kwargs()) as sq:
            out_sq, _, _, _ = _step2(env, sq, c.u0, nx, ny, dt)
        assert np.abs(out_sq - out).max() > 1e-10


def test_teacher_forced_2d_rect_quadrants(env):
    """Four-quadrant Euler data at P = 4 with rectangular stencils: 8 steps
    against the oracle from the GPU state, every state physical (with square
    blocks the first step already produces negative pressures here)."""
    torch, O, acat = env
    c = _case("quadrants", 4, 36, 36, 1, seed=2)
    kw = dict(c.problem_kwargs(), rect_2d=1)
    pr = O.Problem(**kw)
    u = c.u0
    with acat.Context(**kw) as ctx:
        for n in range(8):
            out, dt, ox, oy = _step2(env, ctx, u, c.nx, c.ny)
            assert ctx.acat_status() == 0, n
            ref, _, rox, roy = O.step_2d(pr, u, dt)
            assert np.array_equal(ox, rox) and np.array_equal(oy, roy), n
            assert np.abs(out - ref).max() / np.abs(ref).max() < 1e-12, n
            u = out


# FP32 with P >= 3 and the FP32 rectangular stencils: the block kernel in the
# delta formulation on the compensated state (orders bit-exact, 1e-7 per step)
F32_HI_CASES = [("smooth2d", 3, 50, 61, 0, 0), ("smooth2d", 4, 37, 33, 1, 0), ("transport", 3, 30, 28, 0, 0),
                ("transport", 4, 26, 25, 1, 0), ("quadrants", 3, 45, 40, 1, 1), ("quadrants", 4, 40, 44, 0, 1),
                ("quadrants", 2, 40, 37, 1, 1), ("smooth2d", 3, 25, 27, 1, 1)]


@pytest.mark.parametrize("kind,P,nx,ny,bc,rect", F32_HI_CASES)
def test_single_step_2d_f32_high_order(env, kind, P, nx, ny, bc, rect):
    torch, O, acat = env
    c = _case(kind, P, nx, ny, bc, seed=1)
    kw = dict(c.problem_kwargs(), rect_2d=rect)
    pair = acat.to_pair(c.u0)
    x = acat.from_pair(pair)
    with acat.Context(**kw, precision=acat.PREC_F32) as ctx:
        out, dt, ox, oy = _step2(env, ctx, pair, nx, ny)
        assert ctx.acat_status() == 0
    pr = O.Problem(**kw)
    assert dt == O.dt_cfl(pr, x)
    ref, _, rox, roy = O.step_2d(pr, x, dt)
    assert np.array_equal(ox, rox), np.argwhere(ox != rox)[:5]
    assert np.array_equal(oy, roy), np.argwhere(oy != roy)[:5]
    err = np.abs(acat.from_pair(out) - ref).max() / max(1.0, np.abs(ref).max())
    assert err < 1e-7, err


def test_teacher_forced_2d_f32_rect_quadrants(env):
    """FP32 with rectangular stencils on four-quadrant data at P = 4: 6 steps
    against the oracle from the GPU state (value hi + lo)."""
    torch, O, acat = env
    c = _case("quadrants", 4, 32, 30, 1, seed=3)
    kw = dict(c.problem_kwargs(), rect_2d=1)
    pr = O.Problem(**kw)
    pair = acat.to_pair(c.u0)
    with acat.Context(**kw, precision=acat.PREC_F32) as ctx:
        for n in range(6):
            x = acat.from_pair(pair)
            out, dt, ox, oy = _step2(env, ctx, pair, c.nx, c.ny)
            assert ctx.acat_status() == 0, n
            ref, _, rox, roy = O.step_2d(pr, x, dt)
            assert np.array_equal(ox, rox) and np.array_equal(oy, roy), n
            assert np.abs(acat.from_pair(out) - ref).max() / np.abs(ref).max() < 1e-7, n
            pair = out
