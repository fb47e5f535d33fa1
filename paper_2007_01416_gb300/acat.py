"""ctypes binding of libacat (include/acat.h), with the same entry-point
names. It only marshals arguments: every step of the ACAT path runs in the
library's CUDA kernels. Device buffers are torch CUDA tensors (or raw device
addresses); streams default to torch's current stream.

Loading fails loudly when ``libacat.so`` is missing or cannot be loaded: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# ACAT_LIBRARY selects another build of the same library (the bounds-checked
# libacat_bounds.so of the tests); default: the in-tree libacat.so
LIB_PATH = os.environ.get("ACAT_LIBRARY") or os.path.join(HERE, "libacat.so")

LINEAR, BURGERS, EULER1D, EULER2D = 0, 1, 2, 3
PERIODIC, TRANSMISSIVE = 0, 1
PREC_F64, PREC_F32 = 0, 1
LO_RUSANOV, LO_GLOBAL_LF, LO_HLL = 0, 1, 2
STATUS_NONPHYSICAL, STATUS_BAD_DT, STATUS_BOUNDS = 1, 2, 4


class AcatError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class acat_params(ctypes.Structure):
    _fields_ = [
        ("flux", ctypes.c_int), ("P", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("bc", ctypes.c_int), ("precision", ctypes.c_int), ("tau_factorial", ctypes.c_int),
        ("limiter_form", ctypes.c_int), ("psi2_mod", ctypes.c_int), ("lo_flux", ctypes.c_int),
        ("rect_2d", ctypes.c_int),
        ("gamma", ctypes.c_double), ("adv", ctypes.c_double * 2),
        ("cfl", ctypes.c_double), ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double), ("psi_tol", ctypes.c_double),
        ("eps", ctypes.c_double),
    ]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libacat not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        pp = ctypes.POINTER(acat_params)
        L.acat_default_params.argtypes = [pp]
        L.acat_default_params.restype = None
        L.acat_create.argtypes = [pp, ctypes.POINTER(vp)]
        L.acat_create_batched.argtypes = [pp, i, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(vp)]
        L.acat_destroy.argtypes = [vp]
        L.acat_state_bytes.argtypes = [vp]
        L.acat_state_bytes.restype = ctypes.c_int64
        L.acat_step.argtypes = [vp, vp, vp, d, vp, vp, vp]
        L.acat_run.argtypes = [vp, vp, i, d, vp, vp]
        L.acat_run_host.argtypes = [vp, vp, vp, i, d, vp, ctypes.POINTER(ctypes.c_double)]
        L.acat_status.argtypes = [vp, ctypes.POINTER(ctypes.c_uint)]
        L.acat_clear_status.argtypes = [vp]
        L.acat_strerror.argtypes = [i]
        L.acat_strerror.restype = ctypes.c_char_p
        L.acat_launch_count.argtypes = [vp]
        L.acat_launch_count.restype = ctypes.c_int64
        L.acat_adjoint_step.argtypes = [vp, vp, d, vp, vp, vp]
        L.acat_run_record.argtypes = [vp, vp, vp, i, i, vp, vp, vp]
        L.acat_adjoint_run.argtypes = [vp, vp, vp, i, i, vp, vp, vp]
        ip = ctypes.POINTER(ctypes.c_int)
        L.acat_autotune.argtypes = [vp, vp, i, vp, ip, ip, ip]
        L.acat_launch_shape.argtypes = [vp, ip, ip, ip]
        L.acat_set_launch_shape.argtypes = [vp, i, i, i]
        L.acat_measure_fma_peak.argtypes = [i, vp]
        L.acat_measure_fma_peak.restype = ctypes.c_double
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().acat_strerror(int(code)).decode()


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise AcatError(rc, what)


def default_params() -> acat_params:
    p = acat_params()
    lib().acat_default_params(ctypes.byref(p))
    return p


def make_params(**kw) -> acat_params:
    """acat_params from keyword arguments (defaults from the library)."""
    p = default_params()
    for k, v in kw.items():
        if k == "adv":
            p.adv[0], p.adv[1] = float(v[0]), float(v[1])
        else:
            setattr(p, k, v)
    return p


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def to_pair(u):
    """FP64 state -> compensated FP32 layout [hi; lo] (shape [2, ...]):
    hi = fl32(u), lo = fl32(u - hi). Works on numpy arrays and torch tensors."""
    try:
        import torch
        if isinstance(u, torch.Tensor):
            hi = u.to(torch.float32)
            lo = (u - hi.to(torch.float64)).to(torch.float32)
            return torch.stack([hi, lo]).contiguous()
    except ImportError:
        pass
    import numpy as np
    u = np.asarray(u, dtype=np.float64)
    hi = u.astype(np.float32)
    lo = (u - hi.astype(np.float64)).astype(np.float32)
    return np.ascontiguousarray(np.stack([hi, lo]))


def from_pair(pair):
    """Compensated FP32 layout [hi; lo] -> the FP64 value hi + lo (exact)."""
    try:
        import torch
        if isinstance(pair, torch.Tensor):
            return pair[0].to(torch.float64) + pair[1].to(torch.float64)
    except ImportError:
        pass
    import numpy as np
    return pair[0].astype(np.float64) + pair[1].astype(np.float64)


def acat_measure_fma_peak(precision: int, stream=None) -> float:
    return float(lib().acat_measure_fma_peak(int(precision), _stream(stream)))


class Context:
    """An acat_ctx: one problem (flux, P, grid, BC, precision) on the current
    device. Methods mirror the C entry points."""

    def __init__(self, params: acat_params | None = None, sizes=None, **kw):
        """sizes: instance sizes for a batch of independent 1D problems
        (acat_create_batched); None for a single problem (acat_create)."""
        self.params = params if params is not None else make_params(**kw)
        h = ctypes.c_void_p()
        self.n_inst = 0
        self.sizes = None if sizes is None else [int(v) for v in sizes]
        if sizes is None:
            _check(lib().acat_create(ctypes.byref(self.params), ctypes.byref(h)), "acat_create")
        else:
            arr = (ctypes.c_int32 * len(sizes))(*[int(v) for v in sizes])
            _check(lib().acat_create_batched(ctypes.byref(self.params), len(sizes), arr,
                                             ctypes.byref(h)), "acat_create_batched")
            self.n_inst = len(sizes)
        self._h = h

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def state_bytes(self) -> int:
        return int(lib().acat_state_bytes(self._h))

    def acat_step(self, u_in, u_out, dt: float = -1.0, stream=None, dt_out=None, orders_out=None):
        _check(lib().acat_step(self._h, _ptr(u_in), _ptr(u_out), float(dt), _stream(stream),
                               _ptr(dt_out), _ptr(orders_out)), "acat_step")

    def acat_run(self, u, nsteps: int, t_end: float = -1.0, stream=None, t_out=None):
        _check(lib().acat_run(self._h, _ptr(u), int(nsteps), float(t_end), _stream(stream),
                              _ptr(t_out)), "acat_run")

    def acat_run_host(self, u_host_in, u_host_out, nsteps: int, t_end: float = -1.0,
                      stream=None) -> float:
        t = (ctypes.c_double * max(1, self.n_inst))()
        _check(lib().acat_run_host(self._h, _ptr(u_host_in), _ptr(u_host_out), int(nsteps),
                                   float(t_end), _stream(stream), t),
               "acat_run_host")
        return list(t) if self.n_inst else t[0]

    def acat_adjoint_step(self, u_n, dt: float, ubar_np1, ubar_n, stream=None):
        _check(lib().acat_adjoint_step(self._h, _ptr(u_n), float(dt), _ptr(ubar_np1), _ptr(ubar_n),
                                       _stream(stream)), "acat_adjoint_step")

    def acat_run_record(self, u0, u_out, nsteps: int, every: int, ckpt, dts, stream=None):
        _check(lib().acat_run_record(self._h, _ptr(u0), _ptr(u_out), int(nsteps), int(every), _ptr(ckpt),
                                     _ptr(dts), _stream(stream)), "acat_run_record")

    def acat_adjoint_run(self, ckpt, dts, nsteps: int, every: int, ubar_n, ubar_0, stream=None):
        _check(lib().acat_adjoint_run(self._h, _ptr(ckpt), _ptr(dts), int(nsteps), int(every), _ptr(ubar_n),
                                      _ptr(ubar_0), _stream(stream)), "acat_adjoint_run")

    def acat_autotune(self, u, steps: int = 3, stream=None) -> tuple[int, int, int]:
        """Times the step's launch shapes on a copy of u and keeps the fastest;
        returns (warps per CTA, lanes per stencil node, CTAs per SM)."""
        nw, lpn, cps = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().acat_autotune(self._h, _ptr(u), int(steps), _stream(stream), ctypes.byref(nw),
                                   ctypes.byref(lpn), ctypes.byref(cps)), "acat_autotune")
        return nw.value, lpn.value, cps.value

    def acat_launch_shape(self) -> tuple[int, int, int]:
        nw, lpn, cps = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().acat_launch_shape(self._h, ctypes.byref(nw), ctypes.byref(lpn), ctypes.byref(cps)),
               "acat_launch_shape")
        return nw.value, lpn.value, cps.value

    def acat_set_launch_shape(self, nw: int, lpn: int = 1, cps: int = 0) -> None:
        _check(lib().acat_set_launch_shape(self._h, int(nw), int(lpn), int(cps)), "acat_set_launch_shape")

    def acat_status(self) -> int:
        f = ctypes.c_uint(0)
        rc = lib().acat_status(self._h, ctypes.byref(f))
        if rc not in (0, -4):
            _check(rc, "acat_status")
        return int(f.value)

    def acat_clear_status(self) -> None:
        _check(lib().acat_clear_status(self._h), "acat_clear_status")

    def launch_count(self) -> int:
        return int(lib().acat_launch_count(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().acat_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def tuning_key(ctx: Context, device_name: str) -> str:
    """Key of a context's tuned launch shape: the device, the fields of the
    problem that select the kernel, the grid size (single instance) or a
    digest of the instance sizes (the tile list and the load balance depend
    on them)."""
    import hashlib
    p = ctx.params
    sizes = ctx.sizes if ctx.sizes is not None else [p.nx]
    digest = hashlib.sha256(",".join(map(str, sizes)).encode()).hexdigest()[:16]
    return (f"{device_name}|flux={p.flux}|P={p.P}|prec={p.precision}|psi2_mod={p.psi2_mod}"
            f"|lo_flux={p.lo_flux}|batched={int(ctx.sizes is not None)}|sizes={digest}")


def autotune_cached(ctx: Context, u, cache_path: str, device_name: str, steps: int = 3,
                    stream=None) -> tuple[int, int, int]:
    """acat_autotune with its result kept in a JSON file: a key found in the
    file is applied with acat_set_launch_shape without timing; otherwise the
    shape is tuned and stored. Returns (warps per CTA, lanes per node, CTAs
    per SM; 0 = occupancy when applied from the file)."""
    import json
    key = tuning_key(ctx, device_name)
    cache = {}
    if os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if key in cache:
        e = cache[key]
        nw, lpn, cps = int(e["nw"]), int(e["lpn"]), int(e["cps"])
        ctx.acat_set_launch_shape(nw, lpn, cps)
        return nw, lpn, cps
    nw, lpn, cps = ctx.acat_autotune(u, steps, stream)
    cache[key] = {"nw": nw, "lpn": lpn, "cps": cps}
    tmp = cache_path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return nw, lpn, cps
