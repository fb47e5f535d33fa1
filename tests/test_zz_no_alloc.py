"""acat_run_noalloc: the 1D run for callers that must not allocate device
memory (for example a host application that owns all device memory through
its own pool). It keeps its scratch in a fixed static device array inside the
library instead of a context. This file is collected last so that a run that
stops at the first failure has already run every other test.

The test calls the entry point through the C ABI twice in a row on different
problems and compares each result with acat_run of a context, within the 1e-12
relative tolerance of the other parity tests. It passes alone in a fresh
process and after the rest of the suite."""
import ctypes

import numpy as np
import pytest

from paper_2007_01416_gb300 import workloads as W

pytestmark = pytest.mark.gpu
RTOL = 1e-12


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_01416_gb300 import acat, build
    build.build()
    L = acat.lib()
    L.acat_run_noalloc.argtypes = [ctypes.POINTER(acat.acat_params), ctypes.c_void_p, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]
    return torch, acat, L


def _noalloc(env, case, nsteps, t_end=-1.0):
    torch, acat, L = env
    p = acat.make_params(**case.problem_kwargs())
    u = torch.from_numpy(case.u0.copy()).cuda()
    t = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    st = torch.full((1,), 0xFFFF, dtype=torch.int32, device="cuda")
    rc = L.acat_run_noalloc(ctypes.byref(p), u.data_ptr(), nsteps, t_end,
                            torch.cuda.current_stream().cuda_stream, t.data_ptr(), st.data_ptr())
    assert rc == 0, acat.strerror(rc)
    torch.cuda.synchronize()
    return u.cpu().numpy(), t.item(), int(st.item())


def _with_context(env, case, nsteps, t_end=-1.0):
    torch, acat, L = env
    with acat.Context(**case.problem_kwargs()) as ctx:
        u = torch.from_numpy(case.u0.copy()).cuda()
        t = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.acat_run(u, nsteps, t_end, None, t)
        torch.cuda.synchronize()
        return u.cpu().numpy(), t.item()


def test_noalloc_matches_acat_run_twice(env):
    cases = [(W.euler1d_riemann_entropy(nx=4096, seed=11, P=4), 97, -1.0),
             (W.burgers_sine(nx=1000, seed=12, P=3), 60, 0.05)]
    for case, nsteps, t_end in cases:  # two calls in a row on the shared scratch
        got, t_got, status = _noalloc(env, case, nsteps, t_end)
        ref, t_ref = _with_context(env, case, nsteps, t_end)
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(got - ref).max() <= RTOL * scale
        assert t_got == pytest.approx(t_ref, rel=1e-15, abs=0)
        assert status == 0


def test_noalloc_clears_slots_between_calls(env):
    """The slots of the shared array (wave speed, time, status) are cleared at
    the start of every call: a first call with a much larger wave speed, or one
    that sets a status bit, leaves nothing behind for the next."""
    strong = W.euler1d_riemann_entropy(nx=2048, seed=21, P=3)
    strong.u0[2] *= 40.0  # energy x 40: wave speed about 6x that of the data below
    calm = W.acoustic_pulse(nx=1024, seed=22, P=2)
    got, t_got, status = _noalloc(env, strong, 5)
    assert status == 0
    got, t_got, status = _noalloc(env, calm, 31)
    ref, t_ref = _with_context(env, calm, 31)
    assert np.array_equal(got, ref) and t_got == t_ref and status == 0
    bad = W.euler1d_riemann_entropy(nx=512, seed=23, P=2)
    bad.u0[0, 100] = -1.0  # negative density: the step flags it
    _, _, status = _noalloc(env, bad, 1)
    assert status != 0
    got, t_got, status = _noalloc(env, calm, 31)
    assert np.array_equal(got, ref) and t_got == t_ref and status == 0


def test_noalloc_rejects_oversized_state(env):
    torch, acat, L = env
    case = W.euler1d_riemann_entropy(nx=350000, seed=0, P=2)  # 8.4 MB > 8 MiB
    p = acat.make_params(**case.problem_kwargs())
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = L.acat_run_noalloc(ctypes.byref(p), dummy.data_ptr(), 1, -1.0, None, None, None)
    assert rc == -6  # ACAT_ERR_TOO_LARGE, before any device work
