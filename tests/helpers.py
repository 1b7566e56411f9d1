"""Shared helpers of the test-suite: mesh pairs (oracle + CUDA), error norms, sampling."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2607_02335_gb300 import synth as S


def rel_max_err(y, yref) -> float:
    y = np.asarray(y, dtype=np.float64)
    yref = np.asarray(yref, dtype=np.float64)
    den = np.abs(yref).max()
    return float(np.abs(y - yref).max() / (den if den > 0 else 1.0))


def as_tuple(m):
    return (m, m, m) if np.isscalar(m) else tuple(m)


def oracle_mesh(m, p, amp=0.0, dirichlet=False):
    return O.Mesh(as_tuple(m), p, amp=amp, dirichlet=dirichlet)


def cell_local_to_global(m, p, cell, loc):
    mx, my, mz = as_tuple(m)
    n = p + 1
    cx, cy, cz = cell % mx, (cell // mx) % my, cell // (mx * my)
    i, j, k = loc % n, (loc // n) % n, loc // (n * n)
    Nx, Ny = mx * p + 1, my * p + 1
    return ((cz * p + k) * Ny + (cy * p + j)) * Nx + (cx * p + i)


def cells_of_global(m, p, g):
    """All (cell, local) copies of global node g."""
    mx, my, mz = as_tuple(m)
    n = p + 1
    Nx, Ny = mx * p + 1, my * p + 1
    gx, gy, gz = g % Nx, (g // Nx) % Ny, g // (Nx * Ny)
    out = []

    def axis(gv, mm):
        c = [gv // p] if gv % p else [gv // p - 1, gv // p]
        return [(cc, gv - cc * p) for cc in c if 0 <= cc < mm]

    for cz, k in axis(gz, mz):
        for cy, j in axis(gy, my):
            for cx, i in axis(gx, mx):
                out.append(((cz * my + cy) * mx + cx, (k * n + j) * n + i))
    return out


def sampled_assembled(mesh: O.Mesh, op: int, x_glob: np.ndarray, samples):
    """Oracle value of (A_D x_glob) at the global node of each sampled (cell, local) entry,
    computed from element rows of every cell sharing the node."""
    m = (mesh.mx, mesh.my, mesh.mz)
    p, n3 = mesh.p, mesh.n ** 3
    bnd = None
    out = []
    for cell, loc in samples:
        g = cell_local_to_global(m, p, cell, loc)
        if mesh.dirichlet:
            if bnd is None:
                bnd = S.boundary_nodes(m, p)
            if bnd[g]:
                out.append(0.0)
                continue
        acc = 0.0
        for c2, l2 in cells_of_global(m, p, g):
            row = O.element_row(mesh, op, c2, l2)
            xl = np.array([x_glob[cell_local_to_global(m, p, c2, j)] for j in range(n3)])
            if mesh.dirichlet:
                xl = xl * ~bnd[[cell_local_to_global(m, p, c2, j) for j in range(n3)]]
            acc += float(row @ xl)
        out.append(acc)
    return np.array(out)
