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
