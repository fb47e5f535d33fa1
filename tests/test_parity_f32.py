"""FP32 path (ACAT_PREC_F32): float recursion on a compensated (hi, lo) state;
order decisions and limiter as FP64 takes them on hi + lo; the first step's
dt from an FP64 wave-speed reduction (later steps of a run reduce in float).

Bars (from the arithmetic of the float path): the order codes of one step
match the FP64 oracle bit for bit from the same state value hi + lo (the
decisions are taken in FP64 on that exact value); one step agrees with the
oracle within 1e-7 of max|u| (float rounding of flux increments, at most
O(1) across a discontinuity: eps32 * lambda * |jump of f| * 4 < 1e-7).
Free runs: the scheme is a discontinuous map of the state (order thresholds),
so trajectories that differ by rounding split locally where a decision is near
its threshold. FP64 GPU runs from initial states perturbed at FP32 rounding
size show the same against the oracle, so the FP32 run's L1 and Linf distances
to the oracle are bounded by SPLIT_K times theirs plus the accumulated FP32
rounding bound, and its order histogram must track the FP64 run's (see
test_free_run_f32_against_oracle).
"""
import numpy as np
import pytest

from paper_2007_01416_gb300 import workloads as W

pytestmark = pytest.mark.gpu
STEP_TOL = 1e-7
EPS32 = 2.0 ** -24
ROUND_C = 8.0     # float roundings an increment of the FP32 update carries, at most
SPLIT_K = 4.0     # free runs: FP32 may deviate from the oracle 4x as much as the yardstick runs
HIST_TOL = 0.005  # free runs: order histograms within 0.5 % of the interfaces per order
NPERT = 3         # free runs: FP64 runs from eps32-perturbed initial states (the yardstick)


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


def _step32(env, ctx, pair, nx):
    torch, O, acat = env
    u = torch.from_numpy(np.ascontiguousarray(pair)).cuda()
    out = torch.empty_like(u)
    dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
    orders = torch.zeros(nx + 1, dtype=torch.int8, device="cuda")
    ctx.acat_step(u, out, -1.0, None, dtv, orders)
    torch.cuda.synchronize()
    return out.cpu().numpy(), float(dtv.item()), orders.cpu().numpy()


@pytest.mark.parametrize("kind,P,nx,bc,lpn,nw", [
    ("euler", 4, 16384, 1, 1, 8), ("euler", 3, 1001, 0, 1, 8), ("euler", 2, 777, 1, 1, 8),
    ("burgers", 2, 400, 0, 1, 8), ("burgers", 4, 513, 1, 1, 8), ("euler", 1, 64, 1, 1, 8),
    ("euler", 4, 16384, 1, 2, 8), ("euler", 4, 1001, 0, 2, 8), ("euler", 2, 777, 1, 2, 8),
    ("burgers", 2, 400, 0, 2, 8), ("burgers", 4, 513, 1, 2, 8), ("linear", 4, 300, 0, 2, 8),
    # the small-CTA step with the boundary hand-off; the last CTA holds 1, 2 and 10 interfaces
    ("euler", 4, 16384, 1, 1, 2), ("euler", 3, 1001, 0, 1, 2), ("euler", 2, 777, 1, 1, 2),
    ("burgers", 4, 513, 1, 1, 2), ("euler", 1, 64, 1, 1, 2), ("linear", 4, 300, 0, 1, 2),
    # the fused step in 7-warp tiles
    ("euler", 4, 16384, 1, 1, 7), ("euler", 3, 1001, 0, 1, 7), ("euler", 2, 777, 1, 1, 7),
    ("burgers", 2, 400, 0, 1, 7), ("euler", 1, 64, 1, 1, 7)])
def test_single_step_f32(env, kind, P, nx, bc, lpn, nw):
    """lpn = 2: two lanes per stencil node (the node's sums split in two);
    nw = 2: the small-CTA step; nw = 7: the fused step in 7-warp tiles."""
    torch, O, acat = env
    if kind == "linear":
        c = W.burgers_sine(nx=nx, seed=2, P=P)
        c.u0 = c.u0 + 0.5 * (W.centres(nx, c.x0, c.x1) > 0.3)[None, :]
        c.flux, c.adv = W.LINEAR, (0.8, 0.0)
    else:
        c = W.burgers_sine(nx=nx, seed=2, P=P) if kind == "burgers" else \
            W.euler1d_riemann_entropy(nx=nx, seed=2, P=P)
    c.bc = bc
    kw = c.problem_kwargs()
    pair = acat.to_pair(c.u0)
    x = acat.from_pair(pair)  # the exact value the GPU sees
    with acat.Context(**kw, precision=acat.PREC_F32) as ctx:
        ctx.acat_set_launch_shape(nw, lpn, 0)
        assert ctx.acat_launch_shape() == (nw, lpn, 0)
        out, dt, orders = _step32(env, ctx, pair, nx)
        assert ctx.acat_status() == 0
    pr = O.Problem(**kw)
    assert dt == O.dt_cfl(pr, x)
    ref, _, ord_ref = O.step_1d(pr, x, dt)
    assert np.array_equal(orders, ord_ref)
    err = np.abs(acat.from_pair(out) - ref).max() / max(1.0, np.abs(ref).max())
    print(f"single step f32 {kind} P={P} nx={nx} lpn={lpn} nw={nw}: rel err {err:.2e}")
    assert err < STEP_TOL, err


@pytest.mark.parametrize("lpn,nw", [(1, 8), (2, 8), (1, 2)])
def test_teacher_forced_f32(env, lpn, nw):
    torch, O, acat = env
    c = W.euler1d_riemann_entropy(nx=2048, seed=4, P=4)
    kw = c.problem_kwargs()
    pr = O.Problem(**kw)
    pair = acat.to_pair(c.u0)
    worst = 0.0
    with acat.Context(**kw, precision=acat.PREC_F32) as ctx:
        ctx.acat_set_launch_shape(nw, lpn, 0)
        for n in range(100):
            x = acat.from_pair(pair)
            out, dt, orders = _step32(env, ctx, pair, c.nx)
            ref, _, ord_ref = O.step_1d(pr, x, dt)
            assert np.array_equal(orders, ord_ref), n
            worst = max(worst, np.abs(acat.from_pair(out) - ref).max() / np.abs(ref).max())
            pair = out
    print(f"teacher-forced f32 worst step err {worst:.2e}")
    assert worst < STEP_TOL, worst


def _cell_left(a, bc):
    """a[:, i-1] with the boundary's ghost at i = 0 (periodic wrap or copy)."""
    g = a[:, -1:] if bc == 0 else a[:, :1]
    return np.concatenate([g, a[:, :-1]], axis=1)


def _rounding_bound(O, pr, u, dt):
    """Per-cell bound of the FP32 path's rounding in one step from u: the
    update adds lam (B + G_l - G_r), B = f(u_{i-1}) - f(u_i), G_l =
    F_{i-1/2} - f(u_{i-1}), G_r = F_{i+1/2} - f(u_i), each a float increment
    carrying at most ROUND_C float roundings relative to itself; the
    compensated pair itself rounds at eps32^2 |u_i|. Returns (u_next, bound)."""
    new, _, orders, F = O.step_1d(pr, u, dt, want_flux=True)
    f = O.cell_flux_1d(pr, u)
    fl = _cell_left(f, pr.bc)
    lam = dt / pr.dx
    b = ROUND_C * EPS32 * lam * (np.abs(fl - f) + np.abs(F[:-1].T - fl) + np.abs(F[1:].T - f)) + \
        EPS32 ** 2 * np.abs(u)
    return new, b


def _run64(env, kw, u0, steps, nx):
    """A free FP64 GPU run; returns the final state and its last step's orders."""
    torch, O, acat = env
    with acat.Context(**kw) as ctx:
        u = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
        ctx.acat_run(u, steps)
        torch.cuda.synchronize()
        assert ctx.acat_status() == 0
        _, _, orders = _step32(env, ctx, u.cpu().numpy(), nx)
        return u.cpu().numpy(), orders


@pytest.mark.parametrize("P,nx,steps,lpn,nw", [(4, 4096, 1000, 1, 8), (2, 4096, 1000, 1, 2),
                                               (3, 4096, 1000, 1, 8), (4, 4096, 1000, 2, 8),
                                               (4, 16384, 4000, 1, 2)])
def test_free_run_f32_against_oracle(env, P, nx, steps, lpn, nw):
    """Free-running FP32 and FP64 GPU runs of the 1D Euler workload (the last
    case at the benchmark's size and step count) against the oracle run.

    The scheme is a discontinuous map of the state (the order thresholds of
    Eq. 3.2, the limiter's pieces): two evaluations that differ only in
    rounding split where a decision is near its threshold, and the split
    persists. The yardstick is what rounding of FP32 size does to the scheme
    evaluated in FP64: NPERT FP64 GPU runs (pinned to 1e-12 per step) from the
    initial state perturbed by eps32 relative noise (seeded), and the
    unperturbed FP64 run. Per component:
      L1, Linf of FP32 - oracle <= SPLIT_K x the largest of those runs'
                                   + the accumulated FP32 rounding bound;
      the order histograms of the FP32 and FP64 runs' last step within
      HIST_TOL of the interfaces per order; the interfaces where the FP32 and
      FP64 trajectories' orders differ at most SPLIT_K x the most that a
      perturbed run's differ from the unperturbed one's (or HIST_TOL)."""
    torch, O, acat = env
    c = W.euler1d_riemann_entropy(nx=nx, seed=0, P=P, steps=steps)
    kw = c.problem_kwargs()
    pr = O.Problem(**kw)
    ref = c.u0.copy()
    b1, binf = np.zeros(3), np.zeros(3)
    for _ in range(steps):
        ref, b = _rounding_bound(O, pr, ref, O.dt_cfl(pr, ref))
        b1 += b.sum(1)
        binf += b.max(1)
    with acat.Context(**kw, precision=acat.PREC_F32) as ctx:
        ctx.acat_set_launch_shape(nw, lpn, 0)
        u = torch.from_numpy(acat.to_pair(c.u0)).cuda()
        ctx.acat_run(u, steps)
        torch.cuda.synchronize()
        assert ctx.acat_status() == 0
        _, _, ord32 = _step32(env, ctx, u.cpu().numpy(), nx)
        got32 = acat.from_pair(u.cpu().numpy())
    got64, ord64 = _run64(env, kw, c.u0, steps, nx)
    s1 = np.abs(ref).sum(1)
    l1_yard, li_yard, mis_yard = np.abs(got64 - ref).sum(1) / s1, np.abs(got64 - ref).max(1), 0
    rng = np.random.default_rng(100 + P)
    for _ in range(NPERT):
        up = c.u0 * (1.0 + EPS32 * rng.uniform(-1.0, 1.0, c.u0.shape))
        gp, op = _run64(env, kw, up, steps, nx)
        l1_yard = np.maximum(l1_yard, np.abs(gp - ref).sum(1) / s1)
        li_yard = np.maximum(li_yard, np.abs(gp - ref).max(1))
        mis_yard = max(mis_yard, int((op != ord64).sum()))
    l1_32, li_32 = np.abs(got32 - ref).sum(1) / s1, np.abs(got32 - ref).max(1)
    h32, h64 = np.bincount(ord32, minlength=5), np.bincount(ord64, minlength=5)
    mis32 = int((ord32 != ord64).sum())
    print(f"P={P} nx={nx} steps={steps} lpn={lpn} nw={nw}: L1 FP32 {l1_32} yardstick {l1_yard} bound {b1 / s1}; "
          f"Linf FP32 {li_32} yardstick {li_yard} bound {binf}; orders FP32 {h32} FP64 {h64}; "
          f"mismatch FP32-FP64 {mis32}, perturbed FP64-FP64 up to {mis_yard}")
    assert (l1_32 <= SPLIT_K * l1_yard + b1 / s1).all()
    assert (li_32 <= SPLIT_K * li_yard + binf).all()
    assert (np.abs(h32 - h64) <= HIST_TOL * (nx + 1)).all()
    assert mis32 <= max(SPLIT_K * mis_yard, HIST_TOL * (nx + 1))


@pytest.mark.parametrize("P,nx", [(4, 16384), (2, 777), (3, 1001)])
def test_small_cta_equals_fused(env, P, nx):
    """The small-CTA step (boundary cells handed off between CTAs) and the
    fused step in 8- and 7-warp tiles compute every interface and cell from
    the same values with the same operations: 200-step runs agree bit for
    bit."""
    torch, O, acat = env
    c = W.euler1d_riemann_entropy(nx=nx, seed=8, P=P)
    runs = []
    for nw in (2, 8, 7):
        with acat.Context(**c.problem_kwargs(), precision=acat.PREC_F32) as ctx:
            ctx.acat_set_launch_shape(nw, 1, 0)
            u = torch.from_numpy(acat.to_pair(c.u0)).cuda()
            t = torch.zeros(1, dtype=torch.float64, device="cuda")
            ctx.acat_run(u, 200, -1.0, None, t)
            torch.cuda.synchronize()
            assert ctx.acat_status() == 0
            runs.append((u.cpu(), t.item()))
    for r in runs[1:]:
        assert torch.equal(runs[0][0], r[0]) and runs[0][1] == r[1]


def test_run_host_f32(env):
    torch, O, acat = env
    c = W.euler1d_riemann_entropy(nx=3000, seed=9, P=3)
    with acat.Context(**c.problem_kwargs(), precision=acat.PREC_F32) as ctx:
        pair = torch.from_numpy(acat.to_pair(c.u0))
        u = pair.clone().cuda()
        ctx.acat_run(u, 41)
        out = torch.empty_like(pair).pin_memory()
        ctx.acat_run_host(pair.pin_memory(), out, 41)
        torch.cuda.synchronize()
        assert torch.equal(out, u.cpu())


def _default_nw_f32(torch, nx, P):
    """Warps per CTA a single FP32 context starts with: 8 or 7, whichever
    leaves the busiest SM the fewer warps of work (ties keep 8)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    load = {}
    for nw in (8, 7):
        T = nw * (32 // (2 * P)) - 1
        load[nw] = -(-(-(-nx // T)) // sms) * nw
    return 7 if load[7] < load[8] else 8


@pytest.mark.parametrize("nx,P", [(4096, 4), (16384, 4), (16384, 3), (16384, 2), (777, 1)])
def test_default_shape_f32(env, nx, P):
    """The default warps per CTA of a single FP32 context follow the load
    rule (at N = 16384 on 152 SMs: 7 at P = 2 and 4, 8 at P = 3)."""
    torch, O, acat = env
    kw = W.euler1d_riemann_entropy(nx=nx, seed=1, P=P).problem_kwargs()
    with acat.Context(**kw, precision=acat.PREC_F32) as ctx:
        assert ctx.acat_launch_shape() == (_default_nw_f32(torch, nx, P), 1, 0)
    if torch.cuda.get_device_properties(0).multi_processor_count == 152 and nx == 16384:
        assert _default_nw_f32(torch, nx, P) == {2: 7, 3: 8, 4: 7}[P]


def test_single_instance_shape_and_autotune(env):
    """Single-instance shapes: FP32 may switch lanes per node (P = 2, 4); the
    tile width and grid are fixed; FP64 and lpn = 2 at P = 3 are refused.
    acat_autotune on a single FP32 instance keeps the state it reads."""
    torch, O, acat = env
    c = W.euler1d_riemann_entropy(nx=4096, seed=1, P=4)
    kw = c.problem_kwargs()
    with acat.Context(**kw, precision=acat.PREC_F32) as ctx:
        assert ctx.acat_launch_shape() == (_default_nw_f32(torch, 4096, 4), 1, 0)
        with pytest.raises(acat.AcatError) as ei:
            ctx.acat_set_launch_shape(4, 1, 0)
        assert ei.value.code == -5
        with pytest.raises(acat.AcatError) as ei:
            ctx.acat_set_launch_shape(8, 3, 0)
        assert ei.value.code == -1
        ctx.acat_set_launch_shape(2, 1, 0)  # the small-CTA step (one lane per node only)
        assert ctx.acat_launch_shape() == (2, 1, 0)
        with pytest.raises(acat.AcatError) as ei:
            ctx.acat_set_launch_shape(2, 2, 0)
        assert ei.value.code == -1
        ctx.acat_set_launch_shape(7, 1, 0)  # the fused step in 7-warp tiles (one lane per node only)
        assert ctx.acat_launch_shape() == (7, 1, 0)
        with pytest.raises(acat.AcatError) as ei:
            ctx.acat_set_launch_shape(7, 2, 0)
        assert ei.value.code == -1
        u = torch.from_numpy(acat.to_pair(c.u0)).cuda()
        keep = u.clone()
        nw, lpn, cps = ctx.acat_autotune(u, steps=50)
        assert torch.equal(u, keep) and (nw, lpn) in ((8, 1), (8, 2), (7, 1), (2, 1)) and cps == 0
        assert ctx.acat_launch_shape() == (nw, lpn, 0)
    with acat.Context(**{**kw, "P": 3}, precision=acat.PREC_F32) as ctx:
        with pytest.raises(acat.AcatError) as ei:
            ctx.acat_set_launch_shape(8, 2, 0)
        assert ei.value.code == -1
    with acat.Context(**kw) as ctx:
        nw = ctx.acat_launch_shape()[0]
        with pytest.raises(acat.AcatError) as ei:
            ctx.acat_set_launch_shape(nw, 2, 0)
        assert ei.value.code == -5
        with pytest.raises(acat.AcatError) as ei:
            ctx.acat_autotune(torch.from_numpy(c.u0).cuda())
        assert ei.value.code == -5


@pytest.mark.parametrize("amp", [1e-9, 1e-12])
def test_orders_with_eps_zero_on_nearly_constant_data(env, amp):
    """eps = 0 and differences far below the float rounding of the state: the
    differences carry relative errors too large for the float filter, which
    must leave the decisions to the literal FP64 evaluation; the order codes
    equal the oracle's."""
    torch, O, acat = env
    nx = 1000
    x = W.centres(nx, 0.0, 1.0)
    rho = 1.0 + amp * np.sin(2 * np.pi * x) + 1e-3 * (x > 0.5)
    u0 = W.prim_to_cons_1d(rho, np.full(nx, 0.25), np.full(nx, 0.7) + amp * np.cos(6 * np.pi * x))
    kw = dict(flux=W.EULER1D, P=4, nx=nx, ny=1, bc=1, cfl=0.4, x0=0.0, x1=1.0, eps=0.0)
    pair = acat.to_pair(u0)
    xval = acat.from_pair(pair)
    with acat.Context(**kw, precision=acat.PREC_F32) as ctx:
        out, dt, orders = _step32(env, ctx, pair, nx)
    pr = O.Problem(**kw)
    ref, _, oref = O.step_1d(pr, xval, dt)
    assert np.array_equal(orders, oref), np.nonzero(orders != oref)
    err = np.abs(acat.from_pair(out) - ref).max() / np.abs(ref).max()
    assert err < STEP_TOL, err
