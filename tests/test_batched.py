"""Batches of independent ragged 1D instances in one persistent launch per
step (acat_create_batched), each with its own CFL dt.

Per instance the batched step does exactly the arithmetic of a single-instance
step (same tiles from the instance's first cell), so a batch must reproduce
single-instance runs bit for bit; against the oracle the bars are those of the
1D tests (orders bit-exact, FP64 1e-12 per step)."""
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


def _concat(states):
    return np.ascontiguousarray(np.concatenate(states, axis=1))


def _split(u, sizes):
    offs = np.r_[0, np.cumsum(sizes)]
    return [u[..., offs[b]:offs[b + 1]] for b in range(len(sizes))]


@pytest.mark.parametrize("P", [2, 3, 4])
def test_batched_step_vs_oracle(env, P):
    torch, O, acat = env
    sizes = [17, 64, 97, 300, 31, 8 if P <= 4 else 16, 1001]
    sizes = [max(s, 2 * max(P, 2)) for s in sizes]
    cases = [W.euler1d_riemann_entropy(nx=n, seed=40 + b, P=P) for b, n in enumerate(sizes)]
    kw = cases[0].problem_kwargs()
    u = _concat([c.u0 for c in cases])
    with acat.Context(**kw, sizes=sizes) as ctx:
        ug = torch.from_numpy(u).cuda()
        out = torch.empty_like(ug)
        dts = torch.zeros(len(sizes), dtype=torch.float64, device="cuda")
        orders = torch.zeros(sum(sizes) + len(sizes), dtype=torch.int8, device="cuda")
        ctx.acat_step(ug, out, -1.0, None, dts, orders)
        torch.cuda.synchronize()
        assert ctx.acat_status() == 0
        out, dts, orders = out.cpu().numpy(), dts.cpu().numpy(), orders.cpu().numpy()
    ordsplit = np.split(orders, np.cumsum([n + 1 for n in sizes])[:-1])
    for b, (c, got) in enumerate(zip(cases, _split(out, sizes))):
        pr = O.Problem(**{**kw, "nx": c.nx})
        assert dts[b] == O.dt_cfl(pr, c.u0)
        ref, _, ord_ref = O.step_1d(pr, c.u0, dts[b])
        assert np.array_equal(ordsplit[b], ord_ref), b
        assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max()), b


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batched_run_equals_single_runs(env, prec):
    torch, O, acat = env
    sizes = list(W.batched_sizes(24, seed=3, lo=40, hi=3000))
    cases = [W.euler1d_riemann_entropy(nx=int(n), seed=70 + b, P=3) for b, n in enumerate(sizes)]
    kw = cases[0].problem_kwargs()
    pr = acat.PREC_F32 if prec == "f32" else acat.PREC_F64
    conv = acat.to_pair if prec == "f32" else (lambda x: x)
    u = _concat([c.u0 for c in cases])
    with acat.Context(**kw, precision=pr, sizes=sizes) as ctx:
        ug = torch.from_numpy(conv(u)).cuda()
        tb = torch.zeros(len(sizes), dtype=torch.float64, device="cuda")
        ctx.acat_run(ug, 151, 0.05, None, tb)
        torch.cuda.synchronize()
        assert ctx.acat_status() == 0
        got = ug.cpu().numpy()
        times = tb.cpu().numpy()
    offs = np.r_[0, np.cumsum(sizes)]
    for b, c in enumerate(cases):
        with acat.Context(**{**kw, "nx": c.nx}, precision=pr) as one:
            v = torch.from_numpy(conv(c.u0)).cuda()
            t = torch.zeros(1, dtype=torch.float64, device="cuda")
            one.acat_run(v, 151, 0.05, None, t)
            torch.cuda.synchronize()
            ref = v.cpu().numpy()
        assert np.array_equal(got[..., offs[b]:offs[b + 1]], ref), b
        assert times[b] == t.item()


def test_full_size_batch_sampled(env):
    """4096 instances, N uniform in [256, 16384], P = 3, FP32, in the launch
    configuration of the benchmark: 20 batched steps; three instances are
    re-run alone and must match bit for bit."""
    torch, O, acat = env
    sizes, states = W.euler1d_batched(n_inst=4096, seed=0)
    kw = W.euler1d_riemann_entropy(nx=256, seed=0, P=3).problem_kwargs()
    u = acat.to_pair(_concat(states))
    with acat.Context(**kw, precision=acat.PREC_F32, sizes=sizes) as ctx:
        ug = torch.from_numpy(u).cuda()
        ctx.acat_run(ug, 20)
        torch.cuda.synchronize()
        assert ctx.acat_status() == 0
        got = ug.cpu().numpy()
    offs = np.r_[0, np.cumsum(sizes)]
    for b in (0, 2047, 4095):
        with acat.Context(**{**kw, "nx": int(sizes[b])}, precision=acat.PREC_F32) as one:
            v = torch.from_numpy(acat.to_pair(states[b])).cuda()
            one.acat_run(v, 20)
            torch.cuda.synchronize()
            assert np.array_equal(got[..., offs[b]:offs[b + 1]], v.cpu().numpy()), b


def test_every_launch_shape_gives_identical_states(env):
    """Tile width (warps per CTA) and grid (CTAs per SM) only move work
    between CTAs: at a fixed number of lanes per node every shape gives the
    same states bit for bit, over a run long enough to replay the captured
    step graph. Two lanes per node (FP32) regroup the recursion's sums; its
    shapes agree among themselves bit for bit and with one lane per node to
    the FP32 bar."""
    torch, O, acat = env
    sizes = list(W.batched_sizes(37, seed=5, lo=12, hi=2500))
    cases = [W.euler1d_riemann_entropy(nx=int(n), seed=90 + b, P=4) for b, n in enumerate(sizes)]
    kw = cases[0].problem_kwargs()
    for prec, conv in ((acat.PREC_F64, lambda x: x), (acat.PREC_F32, acat.to_pair)):
        u = torch.from_numpy(conv(_concat([c.u0 for c in cases]))).cuda()
        with acat.Context(**kw, precision=prec, sizes=sizes) as ctx:
            assert ctx.acat_launch_shape()[:2] == (8, 1)
            ref = {}
            for lpn in ((1, 2) if prec == acat.PREC_F32 else (1,)):
                for nw in (8, 4, 16):
                    for cps in (0, 1):
                        ctx.acat_set_launch_shape(nw, lpn, cps)
                        got_nw, got_lpn, got_cps = ctx.acat_launch_shape()
                        assert (got_nw, got_lpn) == (nw, lpn) and (cps == 0 or got_cps == cps)
                        v = u.clone()
                        ctx.acat_run(v, 61)
                        torch.cuda.synchronize()
                        assert ctx.acat_status() == 0
                        if lpn not in ref:
                            ref[lpn] = v.cpu().numpy()
                        else:
                            assert np.array_equal(v.cpu().numpy(), ref[lpn]), (prec, nw, lpn, cps)
            if 2 in ref:
                a, b = acat.from_pair(ref[1]), acat.from_pair(ref[2])
                assert np.abs(a - b).mean() / np.abs(a).mean() < 61 * 1e-7
            with pytest.raises(acat.AcatError) as ei:
                ctx.acat_set_launch_shape(5, 1, 0)
            assert ei.value.code == -1
            with pytest.raises(acat.AcatError):
                ctx.acat_set_launch_shape(8, 1, 10 ** 6)
            assert ctx.acat_launch_shape()[0] == 16


def test_batched_two_lanes_per_node_vs_oracle(env):
    """One FP32 batched step with two lanes per stencil node against the
    oracle per instance: orders bit-exact, 1e-7 of max|u|."""
    torch, O, acat = env
    sizes = [17, 64, 97, 300, 31, 1001]
    cases = [W.euler1d_riemann_entropy(nx=n, seed=60 + b, P=4) for b, n in enumerate(sizes)]
    kw = cases[0].problem_kwargs()
    u = acat.to_pair(_concat([c.u0 for c in cases]))
    with acat.Context(**kw, precision=acat.PREC_F32, sizes=sizes) as ctx:
        ctx.acat_set_launch_shape(4, 2, 0)
        ug = torch.from_numpy(u).cuda()
        out = torch.empty_like(ug)
        dts = torch.zeros(len(sizes), dtype=torch.float64, device="cuda")
        orders = torch.zeros(sum(sizes) + len(sizes), dtype=torch.int8, device="cuda")
        ctx.acat_step(ug, out, -1.0, None, dts, orders)
        torch.cuda.synchronize()
        assert ctx.acat_status() == 0
        out, dts, orders = acat.from_pair(out.cpu().numpy()), dts.cpu().numpy(), orders.cpu().numpy()
    x = acat.from_pair(u)
    ordsplit = np.split(orders, np.cumsum([n + 1 for n in sizes])[:-1])
    for b, (c, got, xb) in enumerate(zip(cases, _split(out, sizes), _split(x, sizes))):
        pr = O.Problem(**{**kw, "nx": c.nx})
        ref, _, ord_ref = O.step_1d(pr, xb, dts[b])
        assert np.array_equal(ordsplit[b], ord_ref), b
        assert np.abs(got - ref).max() < 1e-7 * max(1.0, np.abs(ref).max()), b


def test_autotune_keeps_results(env, tmp_path):
    """acat_autotune picks a shape from timed runs on a copy of the state (the
    state itself is not modified); a run after it equals a run with the
    chosen shape set by hand, bit for bit. The cached form applies a stored
    shape without timing."""
    torch, O, acat = env
    sizes = list(W.batched_sizes(64, seed=8, lo=40, hi=4000))
    cases = [W.euler1d_riemann_entropy(nx=int(n), seed=120 + b, P=4) for b, n in enumerate(sizes)]
    kw = cases[0].problem_kwargs()
    u = torch.from_numpy(acat.to_pair(_concat([c.u0 for c in cases]))).cuda()
    u_keep = u.clone()
    with acat.Context(**kw, precision=acat.PREC_F32, sizes=sizes) as ctx:
        nw, lpn, cps = ctx.acat_autotune(u, steps=3)
        assert torch.equal(u, u_keep)
        assert nw in (4, 8, 16) and lpn in (1, 2) and cps >= 1
        assert ctx.acat_launch_shape() == (nw, lpn, cps)
        v = u.clone()
        ctx.acat_run(v, 50)
        torch.cuda.synchronize()
        assert ctx.acat_status() == 0
        tuned = v.cpu().numpy()
    with acat.Context(**kw, precision=acat.PREC_F32, sizes=sizes) as ctx:
        ctx.acat_set_launch_shape(8, lpn, 0)
        v = u.clone()
        ctx.acat_run(v, 50)
        torch.cuda.synchronize()
        assert np.array_equal(v.cpu().numpy(), tuned)
        cache = str(tmp_path / "tune.json")
        name = torch.cuda.get_device_name()
        first = acat.autotune_cached(ctx, u, cache, name)
        n0 = ctx.launch_count()
        assert acat.autotune_cached(ctx, u, cache, name) == first
        assert ctx.launch_count() == n0  # applied from the file, not timed
    with acat.Context(**W.euler2d_quadrants(n=16, ny=16, seed=0, P=2).problem_kwargs()) as two_d:
        with pytest.raises(acat.AcatError) as ei:
            two_d.acat_launch_shape()
        assert ei.value.code == -5
