"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle's tests.

This module holds no arithmetic of the finite-element method: only counter-based random
numbers, index conventions and workload-mix draws.  Both sides receive the arrays it makes.

Random values: SplitMix64 (Steele, Lea, Flood 2014; the mixing step as published by Vigna) applied
to the counter ``seed * 2**32 + index``; the top 53 bits give a uniform in [0, 1), mapped to
[-1, 1).  A primal (continuous) field is drawn per *unique* node, in lexicographic global order
``(gz*Ny + gy)*Nx + gx`` with ``Nx = mx*p + 1``; a dual (cell-wise) field is drawn per cell-wise
entry in canonical order ``((cz*my + cy)*mx + cx)*n^3 + (k*n + j)*n + i``.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """One SplitMix64 output for each 64-bit counter value (vectorised, wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = counter.astype(np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` values uniform in [-1, 1) for counters seed*2^32 + offset + [0, count)."""
    idx = np.arange(count, dtype=np.uint64) + np.uint64(offset)
    ctr = (np.uint64(seed) << np.uint64(32)) + idx
    u = (splitmix64(ctr) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


def global_shape(m, p: int):
    mx, my, mz = (m, m, m) if np.isscalar(m) else tuple(m)
    return (mz * p + 1, my * p + 1, mx * p + 1)


def boundary_nodes(m, p: int) -> np.ndarray:
    """Boolean mask of unique nodes on the boundary of the unit cube (lexicographic order)."""
    Nz, Ny, Nx = global_shape(m, p)
    gz, gy, gx = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    b = (gx == 0) | (gx == Nx - 1) | (gy == 0) | (gy == Ny - 1) | (gz == 0) | (gz == Nz - 1)
    return b.reshape(-1)


def primal_unique(m, p: int, seed: int = 0, dirichlet: bool = False) -> np.ndarray:
    """Continuous input drawn per unique node; Dirichlet nodes set to zero when requested."""
    Nz, Ny, Nx = global_shape(m, p)
    x = uniform_pm1(seed, Nz * Ny * Nx)
    if dirichlet:
        x[boundary_nodes(m, p)] = 0.0
    return x


def dual_cellwise(m, p: int, seed: int = 0) -> np.ndarray:
    """Unassembled (dual) vector drawn independently per cell-wise entry."""
    mx, my, mz = (m, m, m) if np.isscalar(m) else tuple(m)
    n = p + 1
    return uniform_pm1(seed, mx * my * mz * n ** 3)


def batched_problems(count: int = 256, seed: int = 0, degrees=(2, 3, 5, 7), mmin: int = 4,
                     mmax: int = 32, amp_max: float = 0.15):
    """Mix of independent problems: m ~ U{mmin..mmax}, p ~ U(degrees), amp ~ U[0, amp_max]."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(mmin, mmax + 1, size=count)
    ps = rng.choice(np.asarray(degrees), size=count)
    amps = rng.uniform(0.0, amp_max, size=count)
    return [dict(m=int(a), p=int(b), amp=float(c), seed=seed * 100003 + i)
            for i, (a, b, c) in enumerate(zip(ms, ps, amps))]


def poisson_arrivals(rate: float, count: int, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative sums of exponential gaps."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def serving_requests(count: int, seed: int = 0, degrees=(2, 3, 7), median_m: int = 16,
                     max_m: int = 64, sigma: float = 0.5, min_m: int = 4):
    """Request mix: m = clip(round(median * exp(sigma z)), min, max), p ~ U(degrees)."""
    rng = np.random.default_rng(seed + 7)
    z = rng.standard_normal(count)
    ms = np.clip(np.rint(median_m * np.exp(sigma * z)), min_m, max_m).astype(int)
    ps = rng.choice(np.asarray(degrees), size=count)
    return [dict(m=int(a), p=int(b), seed=seed * 1000003 + i) for i, (a, b) in enumerate(zip(ms, ps))]
