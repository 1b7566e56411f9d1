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


# ---------------------------------------------------------------- block-structured test meshes
# Macro-meshes given as vertex coordinates and, per block, the macro-vertices of its eight local
# corners c = i + 2j + 4k.  Each block's local frame is turned by a random proper rotation (a
# signed permutation of the axes with determinant +1), so that neighbouring blocks meet with
# every kind of relative face orientation.  Data only: no finite-element arithmetic.

def _rotations():
    """The 24 signed permutation matrices with determinant +1."""
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), dtype=np.int64)
            for r in range(3):
                R[r, perm[r]] = signs[r]
            if round(np.linalg.det(R)) == 1:
                out.append(R)
    return out


def _rotate_block(corners, R):
    """Corner list of the same hexahedron seen through the local frame turned by R."""
    new = [0] * 8
    for c in range(8):
        u = np.array([2 * (c & 1) - 1, 2 * ((c >> 1) & 1) - 1, 2 * ((c >> 2) & 1) - 1])
        v = R @ u
        c2 = int((v[0] + 1) // 2) + 2 * int((v[1] + 1) // 2) + 4 * int((v[2] + 1) // 2)
        new[c2] = corners[c]
    return new


def _right_handed(vxyz, corners):
    """Swap the local x and y axes if the block's corner frame is left-handed."""
    X = np.asarray(vxyz)
    e = [X[corners[1]] - X[corners[0]], X[corners[2]] - X[corners[0]], X[corners[4]] - X[corners[0]]]
    if np.linalg.det(np.array(e)) > 0:
        return list(corners)
    return [corners[c ^ 3 if (c & 3) in (1, 2) else c] for c in range(8)]


def mb_cube_in_cube(m: int, a: float = 0.5, seed: int = 0, rotate: bool = True):
    """Seven blocks: the cube [-a,a]^3 and the six blocks between its faces and those of
    [-1,1]^3 (edges of valence 3, corners of valence 4).  Returns (vxyz, block_verts, dims)."""
    rng = np.random.default_rng(seed)
    vxyz = [[(2 * (c & 1) - 1) * a, (2 * ((c >> 1) & 1) - 1) * a, (2 * ((c >> 2) & 1) - 1) * a]
            for c in range(8)]
    vxyz += [[2 * (c & 1) - 1.0, 2 * ((c >> 1) & 1) - 1.0, 2 * ((c >> 2) & 1) - 1.0]
             for c in range(8)]
    blocks = [list(range(8))]
    for axis in range(3):
        for side in (0, 1):
            # the inner face (axis at side) and the outer face; local z runs outwards
            t1, t2 = [d for d in range(3) if d != axis]
            corners = []
            for k in range(2):
                for j in range(2):
                    for i in range(2):
                        c = (side << axis) | (i << t1) | (j << t2)
                        corners.append(c if k == 0 else 8 + c)
            blocks.append(corners)
    rots = _rotations()
    out = []
    for b in blocks:
        b = _right_handed(vxyz, b)
        if rotate:
            b = _rotate_block(b, rots[int(rng.integers(len(rots)))])
        out.append(b)
    return np.array(vxyz), np.array(out, dtype=np.int32), np.full((7, 3), m, dtype=np.int32)


def mb_star(nsect: int, m: int, mz: int = 1, seed: int = 0, rotate: bool = True):
    """nsect quadrilateral sectors around the z-axis, extruded over z in [0, 1]: the vertical
    macro-edge through the centre has valence nsect.  Returns (vxyz, block_verts, dims)."""
    rng = np.random.default_rng(seed)
    pts = [(0.0, 0.0)]
    for k in range(nsect):
        th = 2 * np.pi * k / nsect
        pts.append((np.cos(th), np.sin(th)))
    for k in range(nsect):
        th = 2 * np.pi * (k + 0.5) / nsect
        pts.append((1.1 * np.cos(th), 1.1 * np.sin(th)))
    npt = len(pts)
    vxyz = [[x, y, 0.0] for x, y in pts] + [[x, y, 1.0] for x, y in pts]
    rots = _rotations()
    blocks = []
    for k in range(nsect):
        quad = [0, 1 + k, 1 + (k + 1) % nsect, 1 + nsect + k]  # (0,0), (1,0), (0,1), (1,1)
        b = quad + [q + npt for q in quad]
        b = _right_handed(vxyz, b)
        if rotate:
            b = _rotate_block(b, rots[int(rng.integers(len(rots)))])
        blocks.append(b)
    dims = []
    for b in blocks:
        d = [m, m, m]
        # the extruded direction keeps mz cells: find the local axis joining z = 0 and z = 1
        X = np.asarray(vxyz)
        for ax, bit in enumerate((1, 2, 4)):
            if abs(X[b[bit]][2] - X[b[0]][2]) > 0.5:
                d[ax] = mz
        dims.append(d)
    return np.array(vxyz), np.array(blocks, dtype=np.int32), np.array(dims, dtype=np.int32)
