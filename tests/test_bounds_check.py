"""The bounds-checked build of the library (ACAT_BOUNDS_CHECK): every checked
tile, shared-memory and global index that would fall outside its buffer sets
ACAT_STATUS_BOUNDS and skips the access instead of faulting the GPU. The small
cases below run every kernel family (1D fused and small-CTA steps in FP64 and
FP32, one and two lanes per node, the batched step, the 2D steps at P <= 2 and
P >= 3 with square and rectangular blocks, the adjoint step) once with the
product library and once, in a child process, with the checked build: no
status bit may be set, and the states must agree bit for bit (the checks only
skip accesses that fail them)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2007_01416_gb300 import workloads as W

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _cases():
    """(name, problem kwargs, precision, launch shape or None, steps, case)."""
    e1 = W.euler1d_riemann_entropy
    q2 = W.euler2d_quadrants
    cases = [("f64_fused", e1(nx=777, seed=1, P=3), 0, None, 4),
             ("f64_small_cta", e1(nx=20001, seed=2, P=4), 0, None, 3),
             ("f32_fused", e1(nx=1001, seed=3, P=4), 1, (8, 1, 0), 3),
             ("f32_two_lanes", e1(nx=777, seed=4, P=2), 1, (8, 2, 0), 3),
             ("f32_small_cta", e1(nx=777, seed=5, P=2), 1, (2, 1, 0), 3),
             ("burgers_f64", W.burgers_sine(nx=400, seed=6, P=4), 0, None, 5),
             ("2d_p2_f32", q2(n=47, ny=44, seed=7, P=2), 1, None, 2),
             ("2d_p2_f64", q2(n=47, ny=44, seed=8, P=2), 0, None, 2),
             ("2d_p3_f64", W.euler2d_smooth(n=40, ny=36, seed=9, P=3), 0, None, 2),
             ("2d_p4_rect_f32", q2(n=32, ny=30, seed=10, P=4), 1, None, 2)]
    out = []
    for name, c, prec, shape, steps in cases:
        kw = c.problem_kwargs()
        if name.endswith("rect_f32"):
            kw["rect_2d"] = 1
        out.append((name, kw, prec, shape, steps, c))
    return out


def _run_all(torch, acat):
    """States after a few steps and the status word of every case, batched
    and adjoint cases included."""
    out = {}
    for name, kw, prec, shape, steps, c in _cases():
        with acat.Context(**kw, precision=prec) as ctx:
            if shape:
                ctx.acat_set_launch_shape(*shape)
            u = torch.from_numpy(acat.to_pair(c.u0) if prec == 1 else c.u0.copy()).cuda()
            ctx.acat_run(u, steps)
            torch.cuda.synchronize()
            out[name] = u.cpu().numpy()
            out[name + "_status"] = np.array(ctx.acat_status())
    sizes = list(W.batched_sizes(12, seed=3, lo=40, hi=3000))
    states = [W.euler1d_riemann_entropy(nx=int(n), seed=40 + b, P=3).u0 for b, n in enumerate(sizes)]
    kw = W.euler1d_riemann_entropy(nx=256, seed=0, P=3).problem_kwargs()
    for prec in (0, 1):
        u0 = np.ascontiguousarray(np.concatenate(states, axis=1))
        with acat.Context(**kw, precision=prec, sizes=sizes) as ctx:
            u = torch.from_numpy(acat.to_pair(u0) if prec else u0).cuda()
            ctx.acat_run(u, 5)
            torch.cuda.synchronize()
            out[f"batched_{prec}"] = u.cpu().numpy()
            out[f"batched_{prec}_status"] = np.array(ctx.acat_status())
    c = W.acoustic_pulse(nx=64, seed=1, P=2)
    with acat.Context(**c.problem_kwargs()) as ctx:
        u = torch.from_numpy(c.u0.copy()).cuda()
        w = torch.from_numpy(np.cos(np.arange(c.u0.size)).reshape(c.u0.shape)).cuda()
        bar = torch.empty_like(w)
        ctx.acat_adjoint_step(u, 1e-4, w, bar)
        torch.cuda.synchronize()
        out["adjoint"] = bar.cpu().numpy()
        out["adjoint_status"] = np.array(ctx.acat_status())
    return out


def _child(path):
    """Entry point of the child process (ACAT_LIBRARY set to the checked build)."""
    import torch

    from paper_2007_01416_gb300 import acat
    assert acat.LIB_PATH.endswith("libacat_bounds.so"), acat.LIB_PATH
    np.savez(path, **_run_all(torch, acat))


def test_bounds_checked_build_matches(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_01416_gb300 import acat, build
    build.build()
    checked = build.build(variant="bounds")
    ref = _run_all(torch, acat)
    path = str(tmp_path / "checked.npz")
    env = dict(os.environ, ACAT_LIBRARY=checked)
    root = os.path.dirname(HERE)
    code = (f"import sys; sys.path[:0] = [{HERE!r}, {root!r}]; import test_bounds_check as T; "
            f"T._child({path!r})")
    res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-3000:]
    got = np.load(path)
    for name in ref:
        if name.endswith("_status"):
            assert int(ref[name]) == 0 and int(got[name]) == 0, (name, int(got[name]))
        else:
            assert np.array_equal(ref[name], got[name]), name
