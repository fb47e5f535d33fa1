"""Algorithmic operation counts of the ACAT step (roofline numerators): the
reference count of the method's work (a Horner pass per time level, the
*_ref functions), and the leaner count of the formulation the CUDA kernels
use (running Taylor sums, the other functions).

Counting convention: an FMA is 2 flops; add, multiply, divide and square root
are 1 each. Counts are per interface for the flux work and per cell for the
update, so a launch's work follows from the histogram of selected orders.

CAT2p flux of one interface (n = 2p nodes, S components, PHI flops per flux
evaluation), in the dt-scaled recursion with running Taylor sums:
  f(u_j) at the n nodes                                   n PHI
  for each of the n-1 orders k = 2..2p:
    U^(k-1)_j = -lambda sum_r g1[j][r] F_r               2 n^2 S + n S
    acc_j = g[k-1][0] f(u_j)                              n S
    at the n-1 levels r != 0: Taylor update, f, acc      n (n-1) (2S + PHI + 2S)
    F_sum += acc / k!                                     2 n S
  sum_j gamma^{0,1/2}_j F_sum_j                           2 n S
"""
from __future__ import annotations

# flops of one flux evaluation f(u)
PHI = {0: 1, 1: 2, 2: 10, 3: 19}  # linear, Burgers, Euler 1D (1 divide), Euler 2D f+g pair
NVARS = {0: 1, 1: 1, 2: 3, 3: 4}


def cat_flux_flops(p: int, flux: int) -> int:
    n, S, phi = 2 * p, NVARS[flux], PHI[flux]
    per_k = 2 * n * n * S + n * S + n * S + n * (n - 1) * (4 * S + phi) + 2 * n * S
    return n * phi + (n - 1) * per_k + 2 * n * S


def indicator_flops(P: int, flux: int) -> int:
    S = NVARS[flux]
    tot = 0
    for p in range(2, P + 1):
        tot += S * (6 * (p - 1) + 2 + 3 + 4 * p + 2 + 2)
    return tot


def flcat2_flops(flux: int) -> int:
    S, phi = NVARS[flux], PHI[flux]
    return 4 * phi + 28 * S + 16


def update_flops(flux: int) -> int:
    return 3 * NVARS[flux] + 8


# The reference count of the method's work (one Horner pass per time level):
# per interface at the selected order p (n = 2p nodes, S components),
#   FMA(p) = S [(n-1) 2 n^2 + n(n-1) n(n-1)/2 + n^2]   (2 flops each)
#   n (n-1)^2 flux evaluations of PHI_REF flops (f(u_j) at r = 0 reused);
# FL-CAT2 interfaces 100 S; the indicators 10 P S per interface; the update
# 20 S per cell. At p = 4 for 1D Euler: 2 x 7584 + 392 x 8 = 18304 flops.
PHI_REF = {0: 1, 1: 2, 2: 8}


def cat_flux_flops_ref(p: int, flux: int) -> int:
    n, S = 2 * p, NVARS[flux]
    fma = S * ((n - 1) * 2 * n * n + n * (n - 1) * n * (n - 1) // 2 + n * n)
    return 2 * fma + n * (n - 1) ** 2 * PHI_REF[flux]


def step_flops_1d_ref(order_hist: dict, P: int, flux: int, cells: int) -> float:
    """step_flops_1d in the reference count (above)."""
    S = NVARS[flux]
    f = 0.0
    for code, cnt in order_hist.items():
        f += cnt * (100 * S if code == 1 else cat_flux_flops_ref(code, flux))
    f += sum(order_hist.values()) * 10 * P * S + cells * 20 * S
    return f


def step_flops_1d(order_hist: dict, P: int, flux: int, cells: int) -> float:
    """Flops of one 1D step: order_hist maps order code (1 = FL-CAT2) to the
    number of interfaces that selected it."""
    f = 0.0
    for code, cnt in order_hist.items():
        f += cnt * (flcat2_flops(flux) if code == 1 else cat_flux_flops(code, flux))
    nif = sum(order_hist.values())
    f += nif * indicator_flops(P, flux) + cells * update_flops(flux)
    return f


def cat2d_flops(p: int, flux: int) -> int:
    """2D block recursion on the 2p x 2p block (Eqs. 4.5-4.6), F and G
    together: per node the x- and y-derivative sums (n terms each), the
    Taylor update, the f/g pair at the n-1 levels r != 0 and both time sums."""
    n, S, phi = 2 * p, NVARS[flux], PHI[3] if flux == 3 else 2 * PHI[0]
    nodes = n * n
    per_k = nodes * (2 * 2 * n * S + 2 * S) + nodes * 2 * S \
        + nodes * (n - 1) * (2 * S + phi + 4 * S) + nodes * 4 * S
    return nodes * phi + (n - 1) * per_k + 2 * 2 * n * S


def cat2d_rect_flops(p1: int, p2: int, flux: int) -> int:
    """2D block recursion on the rectangular block S_{p1,p2} (2 p1 x 2 p2
    nodes, 2 max(p1, p2) time levels): per node the x-derivative sum over a
    row (2 p1 terms), the y-derivative sum over a column (2 p2 terms), the
    Taylor update, the f/g pair at the levels r != 0 and both time sums."""
    n1, n2, S = 2 * p1, 2 * p2, NVARS[flux]
    n = 2 * max(p1, p2)
    phi = PHI[3] if flux == 3 else 2 * PHI[0]
    nodes = n1 * n2
    per_k = nodes * (2 * n1 * S + 2 * n2 * S + 2 * S) + nodes * 2 * S \
        + nodes * (n - 1) * (2 * S + phi + 4 * S) + nodes * 4 * S
    return nodes * phi + (n - 1) * per_k + 2 * (n1 + n2) * S


def flcat2_2d_flops(flux: int) -> int:
    S, phi = NVARS[flux], PHI[3] if flux == 3 else 2 * PHI[0]
    return 6 * phi + 40 * S + 30


def step_flops_2d(blocks: int, flcat: int, anchors: int, P: int, flux: int, cells: int) -> float:
    """blocks: block recursions run (one per anchor whose directions select
    p = 2; two only when both select different p >= 2), flcat: directions
    on FL-CAT2, anchors: both indicator lines per anchor."""
    S = NVARS[flux]
    ind = 2 * sum(S * (6 * (p - 1) + 2 + 3 + 4 * p + 2 + 2) for p in range(2, P + 1))
    return blocks * cat2d_flops(P, flux) + flcat * flcat2_2d_flops(flux) + anchors * ind \
        + cells * (5 * S + 14)


def state_bytes_1d(cells: int, flux: int, prec: int = 0) -> int:
    """Compulsory HBM traffic of one step: read and write the state once
    (FP64, or the FP32 hi/lo pair: 8 bytes per value either way)."""
    return 2 * cells * NVARS[flux] * 8


def step_flops_2d_tasks(blocks_by_p: dict, flcat: int, anchors: int, P: int, flux: int, cells: int) -> float:
    """As step_flops_2d with the block recursions counted per order p
    (blocks_by_p maps p to the number of 2p x 2p block recursions run)."""
    S = NVARS[flux]
    ind = 2 * sum(S * (6 * (p - 1) + 2 + 3 + 4 * p + 2 + 2) for p in range(2, P + 1))
    return sum(cnt * cat2d_flops(p, flux) for p, cnt in blocks_by_p.items()) \
        + flcat * flcat2_2d_flops(flux) + anchors * ind + cells * (5 * S + 14)
