"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only samples level-set functions on grids and describes the
workloads; it holds none of the solver's arithmetic.  Both the CUDA library's
callers and the CPU oracle's callers take their inputs from here.

Geometries (all analytic, so no dataset is needed):
  * disk          phi = |x - x0| - R                     (Sec. 4.1, Eq. test13)
  * star          phi = r - r0 - A sin(k theta)           (five-lobed star)
  * rounded box   phi = |max(|x| - b, 0)|_2 - rho         (3-D)
  * random star   phi = r - 0.5 - sum_k a_k sin(k theta + p_k), k = 2..6
  * square + disks (Sec. 4.1, Eq. test24)
"""
from __future__ import annotations

import math

import numpy as np

# Model constants of Sec. 4 (Eq. dataeq) and the initial/boundary data of the
# multigrid-efficiency tests (Eq. BCnumtests): a, d, m_s, m_c, alpha, beta,
# s_ext, s0, c0.
PAPER_MODEL = (1.0e4, 0.1, 64.06, 100.09, 0.01, 0.1, 1.0, 0.0, 10.0)


def node_coords(dim: int, lo: float, hi: float, N: int):
    """Node coordinates x_i = lo + i h, i = 0..N, as dim arrays of shape
    (N+1,)*dim in (z, y, x) index order so that x varies fastest in memory."""
    h = (hi - lo) / N
    x = lo + h * np.arange(N + 1, dtype=np.float64)
    if dim == 2:
        Y, X = np.meshgrid(x, x, indexing="ij")
        return (X, Y)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return (X, Y, Z)


def disk(N: int, R: float = 0.8, center=(0.0, 0.0), lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    X, Y = node_coords(2, lo, hi, N)
    return np.ascontiguousarray(np.sqrt((X - center[0]) ** 2 + (Y - center[1]) ** 2) - R)


def star(N: int, r0: float = 0.6, amp: float = 0.2, k: int = 5, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    X, Y = node_coords(2, lo, hi, N)
    r = np.sqrt(X * X + Y * Y)
    th = np.arctan2(Y, X)
    return np.ascontiguousarray(r - r0 - amp * np.sin(k * th))


def rounded_box(N: int, b: float = 0.6, rho: float = 0.2, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    X, Y, Z = node_coords(3, lo, hi, N)
    q = [np.maximum(np.abs(A) - b, 0.0) for A in (X, Y, Z)]
    return np.ascontiguousarray(np.sqrt(q[0] ** 2 + q[1] ** 2 + q[2] ** 2) - rho)


def random_star_params(rng: np.random.Generator):
    a = rng.uniform(0.0, 0.05, size=5)
    p = rng.uniform(0.0, 2.0 * math.pi, size=5)
    s_ext = float(rng.uniform(0.5, 1.0))
    return a, p, s_ext


def random_star(N: int, a, p, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    X, Y = node_coords(2, lo, hi, N)
    r = np.sqrt(X * X + Y * Y)
    th = np.arctan2(Y, X)
    phi = r - 0.5
    for j, k in enumerate(range(2, 7)):
        phi = phi - a[j] * np.sin(k * th + p[j])
    return np.ascontiguousarray(phi)


def random_rounded_box(N: int, rng: np.random.Generator, lo: float = -1.0, hi: float = 1.0):
    while True:
        b = float(rng.uniform(0.4, 0.65))
        rho = float(rng.uniform(0.1, 0.2))
        if b + rho <= 0.85:
            break
    return rounded_box(N, b, rho, lo, hi), b, rho


def paper_test1(N: int, lo: float = -2.0, hi: float = 2.0) -> np.ndarray:
    """Disk of Sec. 4.1 (Eq. test13): centre (sqrt2/30, sqrt3/40), R = 1.486."""
    return disk(N, 1.486, (math.sqrt(2.0) / 30.0, math.sqrt(3.0) / 40.0), lo, hi)


def paper_test2(N: int, lo: float = -2.0, hi: float = 2.0) -> np.ndarray:
    """Square with four disks on its vertices (Sec. 4.1, Eq. test24)."""
    X, Y = node_coords(2, lo, hi, N)
    Lh, D = 0.9567, 0.3
    p1 = np.maximum(np.abs(X), np.abs(Y)) - Lh
    p2 = np.sqrt((np.abs(X) - Lh) ** 2 + (np.abs(Y) - Lh) ** 2) - D
    return np.ascontiguousarray(np.minimum(p1, p2))


# The workloads the library is measured on.  N counts intervals per axis, so
# "1025^2 nodes" is N = 1024.  dt = dt_factor * h on [-1, 1], h = 2 / N.
# coarsest is the N of the coarsest multigrid level: 4 in 3-D keeps the dense
# direct solve there at 2 x 81 unknowns (a 9^3 coarsest box of the rounded box
# has ~600 active nodes, whose dense FP64 factorisation per Newton iteration
# costs more than the cycles).  The 65^2 disk has no discrete solution at its
# second step with dt = h (the ghost c-equation loses its real roots), so it
# runs with dt = h/4.  oracle_step_s_estimate: seconds one CN step of the CPU
# oracle takes (one core of the build host); oracle_cycles_per_step: multigrid
# cycles the oracle counted on the workload's first CN step (used to scale a
# sampled oracle cycle to a step where a step is too long to time).
WORKLOADS = {
    "disk65": dict(dim=2, N=64, coarsest=8, geometry="disk", steps=10, precision="fp64", dt_factor=0.25,
                   oracle_step_s_estimate=0.05),
    "star1025": dict(dim=2, N=1024, coarsest=8, geometry="star", steps=200, precision="fp64", dt_factor=1.0,
                     oracle_step_s_estimate=2.4),
    "rbox257": dict(dim=3, N=256, coarsest=4, geometry="rounded_box", steps=50, precision="fp64", dt_factor=1.0,
                    oracle_step_s_estimate=225.0, oracle_cycles_per_step=55),
    # the same box at half the resolution: parity tests and small profiles
    "rbox129": dict(dim=3, N=128, coarsest=4, geometry="rounded_box", steps=50, precision="fp64", dt_factor=1.0,
                    oracle_step_s_estimate=38.0, oracle_cycles_per_step=59),
}


def workload_levelset(name: str) -> np.ndarray:
    w = WORKLOADS[name]
    if w["geometry"] == "disk":
        return disk(w["N"])
    if w["geometry"] == "star":
        return star(w["N"])
    return rounded_box(w["N"])
