"""CPU oracle of the ACAT method (Carrillo, Macca, Pares, Russo, Zorio,
arXiv 2007.01416): ctypes wrapper around ``acat_oracle.c``.

TEST INFRASTRUCTURE. The oracle is a plain, slow FP64 restatement of the
paper used to check the CUDA library. It shares no code with that library and
the library never loads it; only the test suite, the package smoke check and
the benchmark's CPU-baseline leg import this module.

Functions take and return numpy float64 arrays in SoA layout:
1D ``u[s, nx]``, 2D ``u[s, ny, nx]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "acat_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

LINEAR, BURGERS, EULER1D, EULER2D = 0, 1, 2, 3
PERIODIC, TRANSMISSIVE = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available). Returns the path."""
    srcs = [_SRC, os.path.join(_HERE, "acat_oracle_impl.h"), os.path.join(_HERE, "acat_oracle.h")]
    if not force and os.path.exists(_LIB):
        if os.path.getmtime(_LIB) >= max(os.path.getmtime(s) for s in srcs):
            return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-lm"]
    tmp = _LIB + f".tmp{os.getpid()}"
    try:
        subprocess.run(base[:6] + ["-fopenmp"] + base[6:] + ["-o", tmp], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp], check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("flux", ctypes.c_int), ("P", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("bc", ctypes.c_int), ("tau_factorial", ctypes.c_int), ("limiter_form", ctypes.c_int),
        ("psi2_mod", ctypes.c_int), ("lo_flux", ctypes.c_int), ("rect_2d", ctypes.c_int),
        ("gamma", ctypes.c_double), ("adv", ctypes.c_double * 2), ("cfl", ctypes.c_double),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double),
        ("y1", ctypes.c_double), ("psi_tol", ctypes.c_double), ("eps", ctypes.c_double),
    ]


@dataclass
class Problem:
    """Problem description in the paper's terms (flux family, P, CFL, grid, BC)."""
    flux: int
    P: int
    nx: int
    ny: int = 1
    bc: int = PERIODIC
    gamma: float = 1.4
    adv: tuple = (1.0, 1.0)
    cfl: float = 0.5
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    psi_tol: float = 0.1
    eps: float = 1e-12
    tau_factorial: int = 1
    limiter_form: int = 0
    psi2_mod: int = 0   # 1: modified indicator psi~^2 (Sec. 3.2)
    lo_flux: int = 0    # F^lo: 0 Rusanov, 1 global Lax-Friedrichs, 2 HLL
    rect_2d: int = 0    # 2D: 1 = one rectangular block S_{p1,p2} per anchor (Sec. 4, end)
    extra: dict = field(default_factory=dict)

    @property
    def nvars(self) -> int:
        return {EULER1D: 3, EULER2D: 4}.get(self.flux, 1)

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self) -> float:
        return (self.y1 - self.y0) / self.ny

    def _c(self) -> _Params:
        p = _Params()
        p.flux, p.P, p.nx, p.ny, p.bc = self.flux, self.P, self.nx, self.ny, self.bc
        p.tau_factorial, p.limiter_form = self.tau_factorial, self.limiter_form
        p.psi2_mod, p.lo_flux, p.rect_2d = self.psi2_mod, self.lo_flux, self.rect_2d
        p.gamma = self.gamma
        p.adv[0], p.adv[1] = self.adv
        p.cfl, p.x0, p.x1, p.y0, p.y1 = self.cfl, self.x0, self.x1, self.y0, self.y1
        p.psi_tol, p.eps = self.psi_tol, self.eps
        return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i = ctypes.POINTER(ctypes.c_double), ctypes.c_int
        pp = ctypes.POINTER(_Params)
        i8 = ctypes.POINTER(ctypes.c_int8)
        i32 = ctypes.POINTER(ctypes.c_int32)
        _lib.or_fornberg.argtypes = [i, i, ctypes.c_double, d]
        _lib.or_flux_weights.argtypes = [i, d]
        _lib.or_flux_x.argtypes = [pp, d, d]
        _lib.or_flux_y.argtypes = [pp, d, d]
        _lib.or_cell_flux_1d.argtypes = [pp, d, d]
        _lib.or_dt_1d.argtypes = [pp, d]
        _lib.or_dt_1d.restype = ctypes.c_double
        _lib.or_dt_2d.argtypes = [pp, d]
        _lib.or_dt_2d.restype = ctypes.c_double
        _lib.or_cat_flux_1d.argtypes = [pp, i, d, ctypes.c_double, ctypes.c_double, d]
        _lib.or_cat_flux_2d.argtypes = [pp, i, d, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, d, d]
        _lib.or_cat_flux_2d_rect.argtypes = [pp, i, i, d, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, d, d]
        _lib.or_step_1d.argtypes = [pp, d, d, d, i8, d, d]
        _lib.or_fluxes_1d_at.argtypes = [pp, d, ctypes.c_double, i, i32, d, i8]
        _lib.or_step_1d_cells.argtypes = [pp, d, ctypes.c_double, i, i32, d]
        _lib.or_step_1d_z.argtypes = [pp, d, d, ctypes.c_double, d, d]
        _lib.or_step_2d.argtypes = [pp, d, d, d, i8, i8]
        _lib.or_step_2d_cells.argtypes = [pp, d, ctypes.c_double, i, i32, i32, d]
        _lib.or_set_threads.argtypes = [i]
        _lib.or_get_threads.restype = i
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


def fornberg(p: int, k: int, q: float) -> np.ndarray:
    """gamma^{k,q}_{p,r}, r = -p+1..p (Eq. 2.10), by Fornberg's algorithm."""
    w = np.zeros(2 * p)
    if lib().or_fornberg(p, k, float(q), _dp(w)) != 0:
        raise ValueError("bad weight request")
    return w


def flux_weights(p: int) -> np.ndarray:
    """gamma^{0,1/2}_{p,r}: the flux weights of Eq. 2.14 (Eq. 2.11 at k = 1)."""
    w = np.zeros(2 * p)
    if lib().or_flux_weights(p, _dp(w)) != 0:
        raise ValueError("bad p")
    return w


def flux_x(prob: Problem, u) -> np.ndarray:
    u = _f64(u)
    f = np.zeros(prob.nvars)
    pr = prob._c()
    lib().or_flux_x(ctypes.byref(pr), _dp(u), _dp(f))
    return f


def flux_y(prob: Problem, u) -> np.ndarray:
    u = _f64(u)
    f = np.zeros(prob.nvars)
    pr = prob._c()
    lib().or_flux_y(ctypes.byref(pr), _dp(u), _dp(f))
    return f


def cell_flux_1d(prob: Problem, u) -> np.ndarray:
    """The physical flux f(u_i) of every cell of a 1D state u[s, nx]."""
    u = _f64(u)
    f = np.empty_like(u)
    pr = prob._c()
    lib().or_cell_flux_1d(ctypes.byref(pr), _dp(u), _dp(f))
    return f


def dt_cfl(prob: Problem, u) -> float:
    u = _f64(u)
    pr = prob._c()
    if prob.ny > 1 or u.ndim == 3:
        return float(lib().or_dt_2d(ctypes.byref(pr), _dp(u)))
    return float(lib().or_dt_1d(ctypes.byref(pr), _dp(u)))


def cat_flux_1d(prob: Problem, p: int, stencil, dt: float) -> np.ndarray:
    """CAT2p flux (Eq. 2.14) from stencil[s, 2p] = u_{i-p+1..i+p}."""
    st = _f64(stencil)
    F = np.zeros(prob.nvars)
    pr = prob._c()
    rc = lib().or_cat_flux_1d(ctypes.byref(pr), p, _dp(st), dt, prob.dx, _dp(F))
    if rc:
        raise ValueError(rc)
    return F


def cat_flux_2d(prob: Problem, p: int, block, dt: float):
    """2D CAT2p fluxes (Eqs. 4.5-4.6) from block[s, 2p(y), 2p(x)] anchored at i."""
    b = _f64(block)
    F = np.zeros(prob.nvars)
    G = np.zeros(prob.nvars)
    pr = prob._c()
    rc = lib().or_cat_flux_2d(ctypes.byref(pr), p, _dp(b), dt, prob.dx, prob.dy, _dp(F), _dp(G))
    if rc:
        raise ValueError(rc)
    return F, G


def cat_flux_2d_rect(prob: Problem, p1: int, p2: int, block, dt: float):
    """2D CAT fluxes of the rectangular block S_{p1,p2} from block[s, 2p2(y), 2p1(x)]
    anchored at i: F^{p1} along the row j2 = 0, G^{p2} along the column j1 = 0."""
    b = _f64(block)
    F = np.zeros(prob.nvars)
    G = np.zeros(prob.nvars)
    pr = prob._c()
    rc = lib().or_cat_flux_2d_rect(ctypes.byref(pr), p1, p2, _dp(b), dt, prob.dx, prob.dy, _dp(F), _dp(G))
    if rc:
        raise ValueError(rc)
    return F, G


def step_1d(prob: Problem, u, dt: float | None = None, want_psi: bool = False,
            want_flux: bool = False):
    """One ACAT2P step (Eq. 3.19). Returns (u_new, dt, orders[, psi][, flux])."""
    u = _f64(u)
    out = np.empty_like(u)
    dtv = ctypes.c_double(dt if dt is not None else -1.0)
    orders = np.zeros(prob.nx + 1, dtype=np.int8)
    psi = np.zeros((prob.nx + 1, prob.P)) if want_psi else None
    flux = np.zeros((prob.nx + 1, prob.nvars)) if want_flux else None
    pr = prob._c()
    rc = lib().or_step_1d(ctypes.byref(pr), _dp(u), _dp(out), ctypes.byref(dtv),
                          orders.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                          _dp(psi) if psi is not None else None,
                          _dp(flux) if flux is not None else None)
    if rc:
        raise RuntimeError(f"oracle step failed ({rc})")
    res = [out, dtv.value, orders]
    if want_psi:
        res.append(psi)
    if want_flux:
        res.append(flux)
    return tuple(res)


def fluxes_1d_at(prob: Problem, u, dt: float, ifaces):
    """Numerical fluxes at the given interfaces (m between cells m-1 and m)."""
    u = _f64(u)
    idx = np.ascontiguousarray(ifaces, dtype=np.int32)
    F = np.zeros((len(idx), prob.nvars))
    orders = np.zeros(len(idx), dtype=np.int8)
    pr = prob._c()
    rc = lib().or_fluxes_1d_at(ctypes.byref(pr), _dp(u), float(dt), len(idx),
                               idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(F),
                               orders.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)))
    if rc:
        raise RuntimeError(rc)
    return F, orders


def step_1d_cells(prob: Problem, u, dt: float, cells) -> np.ndarray:
    """u^{n+1} at selected cells only (Eq. 2.12); returns [len(cells), s]."""
    u = _f64(u)
    idx = np.ascontiguousarray(cells, dtype=np.int32)
    out = np.zeros((len(idx), prob.nvars))
    pr = prob._c()
    rc = lib().or_step_1d_cells(ctypes.byref(pr), _dp(u), float(dt), len(idx),
                                idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(out))
    if rc:
        raise RuntimeError(rc)
    return out


def step_1d_complex(prob: Problem, u_re, u_im, dt: float):
    """One 1D step on a complex state at fixed dt, branches on real parts."""
    a, b = _f64(u_re), _f64(u_im)
    ore, oim = np.empty_like(a), np.empty_like(a)
    pr = prob._c()
    rc = lib().or_step_1d_z(ctypes.byref(pr), _dp(a), _dp(b), float(dt), _dp(ore), _dp(oim))
    if rc:
        raise RuntimeError(rc)
    return ore, oim


def step_2d(prob: Problem, u, dt: float | None = None):
    """One 2D ACAT2P step (Eq. 4.9). Returns (u_new, dt, orders_x, orders_y)."""
    u = _f64(u)
    out = np.empty_like(u)
    dtv = ctypes.c_double(dt if dt is not None else -1.0)
    ox = np.zeros((prob.ny, prob.nx + 1), dtype=np.int8)
    oy = np.zeros((prob.ny + 1, prob.nx), dtype=np.int8)
    pr = prob._c()
    rc = lib().or_step_2d(ctypes.byref(pr), _dp(u), _dp(out), ctypes.byref(dtv),
                          ox.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                          oy.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)))
    if rc:
        raise RuntimeError(f"oracle 2D step failed ({rc})")
    return out, dtv.value, ox, oy


def step_2d_cells(prob: Problem, u, dt: float, cx, cy) -> np.ndarray:
    """u^{n+1} at selected cells only; returns [len(cx), s]."""
    u = _f64(u)
    cx = np.ascontiguousarray(cx, dtype=np.int32)
    cy = np.ascontiguousarray(cy, dtype=np.int32)
    out = np.zeros((len(cx), prob.nvars))
    pr = prob._c()
    rc = lib().or_step_2d_cells(ctypes.byref(pr), _dp(u), float(dt), len(cx),
                                cx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                cy.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(out))
    if rc:
        raise RuntimeError(rc)
    return out


def run_1d(prob: Problem, u, nsteps: int, t_end: float | None = None):
    """nsteps oracle steps (dt from the CFL rule, clipped at t_end)."""
    u = _f64(u).copy()
    t = 0.0
    for _ in range(nsteps):
        dt = dt_cfl(prob, u)
        if t_end is not None:
            if t >= t_end:
                break
            dt = min(dt, t_end - t)
        u, dt, _ = step_1d(prob, u, dt)
        t += dt
    return u, t
