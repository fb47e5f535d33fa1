"""Seeded synthetic inputs shaped like the paper's test problems.

This module holds input generation only (initial data, grid sizes, named
initial states printed in the paper) and none of the ACAT arithmetic. Both the
CUDA path and the CPU oracle are fed from here. All generators use
``numpy.random.default_rng(seed)``; states are returned as float64 SoA arrays
of conserved variables: 1D ``[s, nx]``, 2D ``[s, ny, nx]``. Cell centres are
``x_i = x0 + (i + 1/2) dx``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

LINEAR, BURGERS, EULER1D, EULER2D = 0, 1, 2, 3
PERIODIC, TRANSMISSIVE = 0, 1
GAMMA = 1.4


@dataclass
class Case:
    """A problem in the terms the paper states it (flux, P, CFL, grid, BC)
    plus its initial state and step count."""
    name: str
    flux: int
    P: int
    nx: int
    ny: int
    bc: int
    cfl: float
    x0: float
    x1: float
    y0: float
    y1: float
    u0: np.ndarray
    steps: int
    gamma: float = GAMMA
    adv: tuple = (1.0, 1.0)
    t_end: float = -1.0

    def problem_kwargs(self) -> dict:
        return dict(flux=self.flux, P=self.P, nx=self.nx, ny=self.ny, bc=self.bc,
                    gamma=self.gamma, adv=tuple(self.adv), cfl=self.cfl, x0=self.x0,
                    x1=self.x1, y0=self.y0, y1=self.y1)


def centres(n: int, a: float, b: float) -> np.ndarray:
    return a + (np.arange(n) + 0.5) * (b - a) / n


def prim_to_cons_1d(rho, u, p, gamma=GAMMA) -> np.ndarray:
    """(rho, u, p) -> (rho, rho u, E) with E = p/(gamma-1) + rho u^2 / 2."""
    rho, u, p = (np.asarray(a, dtype=np.float64) for a in (rho, u, p))
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])


def cons_to_prim_1d(U, gamma=GAMMA) -> np.ndarray:
    rho, m, E = U
    u = m / rho
    return np.stack([rho, u, (gamma - 1.0) * (E - 0.5 * rho * u * u)])


def prim_to_cons_2d(rho, u, v, p, gamma=GAMMA) -> np.ndarray:
    rho, u, v, p = (np.asarray(a, dtype=np.float64) for a in (rho, u, v, p))
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


# --------------------------------------------------------------------------
# Configurations of the benchmark and of the parity tests
# --------------------------------------------------------------------------
def burgers_sine(nx: int = 400, seed: int = 0, P: int = 2, steps: int = 300,
                 cfl: float = 0.5) -> Case:
    """Inviscid Burgers, u0 = a + b sin(pi x + phi) on [-1, 1], periodic
    (the Burgers test of Sec. 5.2 with seeded amplitude, offset and phase)."""
    rng = np.random.default_rng(seed)
    a, b, phi = rng.uniform(0.2, 0.5), rng.uniform(0.5, 1.0), rng.uniform(0.0, 2.0 * math.pi)
    x = centres(nx, -1.0, 1.0)
    u0 = (a + b * np.sin(math.pi * x + phi))[None, :]
    return Case("burgers_sine", BURGERS, P, nx, 1, PERIODIC, cfl, -1.0, 1.0, 0.0, 1.0, u0, steps)


def euler1d_riemann_entropy(nx: int = 16384, seed: int = 0, P: int = 4, steps: int = 4000,
                            cfl: float = 0.4) -> Case:
    """1D Euler Riemann problem on [0, 1], jump at 1/2 (Sec. 5.3) with seeded
    left/right states (rho, u, p) in [0.1,1] x [-0.5,0.5] x [0.1,1], and an
    entropy wave rho <- rho (1 + 0.2 sin(k x)), k in [4, 8]; transmissive."""
    rng = np.random.default_rng(seed)
    rl, ul, pl = rng.uniform(0.1, 1.0), rng.uniform(-0.5, 0.5), rng.uniform(0.1, 1.0)
    rr, ur, pr = rng.uniform(0.1, 1.0), rng.uniform(-0.5, 0.5), rng.uniform(0.1, 1.0)
    k = rng.uniform(4.0, 8.0)
    x = centres(nx, 0.0, 1.0)
    left = x < 0.5
    rho = np.where(left, rl, rr) * (1.0 + 0.2 * np.sin(k * x))
    u = np.where(left, ul, ur)
    p = np.where(left, pl, pr)
    return Case("euler1d_riemann_entropy", EULER1D, P, nx, 1, TRANSMISSIVE, cfl, 0.0, 1.0, 0.0,
                1.0, prim_to_cons_1d(rho, u, p), steps)


def euler2d_quadrants(n: int = 4096, seed: int = 0, P: int = 2, steps: int = 500,
                      cfl: float = 0.4, ny: int | None = None) -> Case:
    """2D Euler four-quadrant Riemann data on [0,1]^2 (the Lax-Liu setting of
    Sec. 5.5) with seeded constant states: rho, p in [0.1, 1.5], u, v in
    [-0.8, 0.8]; quadrants numbered 1 (x>1/2, y>1/2), 2 (x<1/2, y>1/2),
    3 (x<1/2, y<1/2), 4 (x>1/2, y<1/2); transmissive boundaries."""
    rng = np.random.default_rng(seed)
    ny = n if ny is None else ny
    st = [(rng.uniform(0.1, 1.5), rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8),
           rng.uniform(0.1, 1.5)) for _ in range(4)]
    return _quadrants(f"euler2d_quadrants", st, n, ny, P, steps, cfl)


def euler2d_smooth(n: int = 1024, seed: int = 0, P: int = 3, steps: int = 10, cfl: float = 0.4,
                   ny: int | None = None) -> Case:
    """Smooth 2D Euler data with a contact, periodic on [0,1]^2, for the
    high-order (P >= 3) 2D step: rho = 1 + a sin(2 pi x) sin(2 pi y) +
    0.3 [x > x_c], u = 0.3 + 0.1 cos(2 pi y), v = -0.2 + 0.1 sin(2 pi x),
    p = 1 + 0.1 cos(2 pi (x + y) + phi); a in [0.1, 0.3], x_c in [0.4, 0.7],
    phi in [0, 2 pi) seeded."""
    rng = np.random.default_rng(seed)
    a, xc, phi = rng.uniform(0.1, 0.3), rng.uniform(0.4, 0.7), rng.uniform(0.0, 2.0 * math.pi)
    ny = n if ny is None else ny
    x = centres(n, 0.0, 1.0)[None, :]
    y = centres(ny, 0.0, 1.0)[:, None]
    rho = 1.0 + a * np.sin(2 * math.pi * x) * np.sin(2 * math.pi * y) + 0.3 * (x + 0 * y > xc)
    u = 0.3 + 0.1 * np.cos(2 * math.pi * y) + 0 * x
    v = -0.2 + 0.1 * np.sin(2 * math.pi * x) + 0 * y
    p = 1.0 + 0.1 * np.cos(2 * math.pi * (x + y) + phi)
    return Case("euler2d_smooth", EULER2D, P, n, ny, PERIODIC, cfl, 0.0, 1.0, 0.0, 1.0,
                prim_to_cons_2d(rho, u, v, p), steps)


def _quadrants(name, st, nx, ny, P, steps, cfl) -> Case:
    x = centres(nx, 0.0, 1.0)[None, :]
    y = centres(ny, 0.0, 1.0)[:, None]
    q = np.where(x > 0.5, np.where(y > 0.5, 0, 3), np.where(y > 0.5, 1, 2))
    prim = np.zeros((4, ny, nx))
    for k in range(4):
        for c in range(4):
            prim[c][q == k] = st[k][c]
    rho, u, v, p = prim
    return Case(name, EULER2D, P, nx, ny, TRANSMISSIVE, cfl, 0.0, 1.0, 0.0, 1.0,
                prim_to_cons_2d(rho, u, v, p), steps)


def batched_sizes(n_inst: int = 4096, seed: int = 0, lo: int = 256, hi: int = 16384) -> np.ndarray:
    """Seeded instance sizes N_b uniform on {lo..hi}."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=n_inst).astype(np.int32)


def euler1d_batched(n_inst: int = 4096, seed: int = 0, lo: int = 256, hi: int = 16384):
    """Ragged batch of independent 1D Euler Riemann + entropy-wave instances;
    returns (sizes, list of [3, N_b] states)."""
    sizes = batched_sizes(n_inst, seed, lo, hi)
    states = [euler1d_riemann_entropy(int(n), seed=seed * 100003 + b + 1).u0
              for b, n in enumerate(sizes)]
    return sizes, states


def acoustic_pulse(nx: int = 8192, seed: int = 0, P: int = 2, steps: int = 2000,
                   cfl: float = 0.4) -> Case:
    """Isentropic acoustic pulse on [0,1], periodic:
    rho = 1 + 0.01 exp(-(x - x0)^2 / w^2), u = 0, p = rho^gamma / gamma,
    x0 in [0.3, 0.7], w in [0.02, 0.08]."""
    rng = np.random.default_rng(seed)
    xc, w = rng.uniform(0.3, 0.7), rng.uniform(0.02, 0.08)
    x = centres(nx, 0.0, 1.0)
    rho = 1.0 + 0.01 * np.exp(-((x - xc) ** 2) / (w * w))
    p = rho ** GAMMA / GAMMA
    return Case("acoustic_pulse", EULER1D, P, nx, 1, PERIODIC, cfl, 0.0, 1.0, 0.0, 1.0,
                prim_to_cons_1d(rho, np.zeros_like(x), p), steps)


# --------------------------------------------------------------------------
# Initial states printed in the paper
# --------------------------------------------------------------------------
RIEMANN_1D = {
    # (rho, u, p) left, right; jump at x = 1/2 on [0, 1] (Sec. 5.3)
    "sod": ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),            # Eq. 5.10
    "einfeldt123": ((1.0, -2.0, 0.4), (1.0, 2.0, 0.4)),     # Eq. 5.11
    "blast_right": ((1.0, 0.0, 1000.0), (1.0, 0.0, 0.01)),  # Eq. 5.12
}


def riemann_1d(name: str, nx: int, P: int, cfl: float = 0.8, steps: int = 10 ** 9) -> Case:
    left, right = RIEMANN_1D[name]
    x = centres(nx, 0.0, 1.0)
    prim = [np.where(x < 0.5, left[c], right[c]) for c in range(3)]
    return Case(name, EULER1D, P, nx, 1, TRANSMISSIVE, cfl, 0.0, 1.0, 0.0, 1.0,
                prim_to_cons_1d(*prim), steps)


LAX_LIU = {
    # quadrant states (rho, u, v, p), quadrants 1..4 (Tables 3-5 of Sec. 5.5)
    4: [(1.1, 0.0, 0.0, 1.1), (0.5065, 0.8939, 0.0, 0.35), (1.1, 0.8939, 0.8939, 1.1),
        (0.5065, 0.0, 0.8939, 0.35)],
    6: [(1.0, 0.75, -0.5, 1.0), (2.0, 0.75, 0.5, 1.0), (1.0, -0.75, 0.5, 1.0),
        (3.0, -0.75, -0.5, 1.0)],
    8: [(0.5197, 0.1, 0.1, 0.4), (1.0, -0.6259, 0.1, 1.0), (0.8, 0.1, 0.1, 1.0),
        (1.0, 0.1, -0.6259, 1.0)],
}


def lax_liu(config: int, n: int, P: int, cfl: float = 0.475, steps: int = 10 ** 9) -> Case:
    return _quadrants(f"lax_liu_{config}", LAX_LIU[config], n, n, P, steps, cfl)
