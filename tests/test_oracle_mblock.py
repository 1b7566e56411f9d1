"""Pins of the block-structured oracle (Sec. 4.2): its global numbering comes from node
coordinates, its element matrices from the trilinear block maps; both are checked against closed
forms and against the structured oracle on the same physical meshes."""
import numpy as np
import pytest

import oracle as O
from paper_2607_02335_gb300 import synth as S


def unique_cube_in_cube(m, p):
    """Seven blocks of m^3 cells: 7 block interiors, 24 faces, 32 edges, 16 vertices."""
    k = m * p - 1
    return 7 * k ** 3 + 24 * k ** 2 + 32 * k + 16


def unique_star(ns, m, mz, p):
    """ns extruded sectors of m x m x mz cells: 2D count times the layers along z."""
    k = m * p - 1
    return (ns * k * k + 3 * ns * k + 2 * ns + 1) * (mz * p + 1)


def star_area(ns):
    """Shoelace area of the star's ns quadrilaterals (centre, P_k, M_k, P_k+1)."""
    a = 0.0
    for k in range(ns):
        t0, t1, tm = 2 * np.pi * k / ns, 2 * np.pi * (k + 1) / ns, 2 * np.pi * (k + 0.5) / ns
        q = [(0, 0), (np.cos(t0), np.sin(t0)), (1.1 * np.cos(tm), 1.1 * np.sin(tm)),
             (np.cos(t1), np.sin(t1))]
        a += 0.5 * sum(q[i][0] * q[(i + 1) % 4][1] - q[(i + 1) % 4][0] * q[i][1] for i in range(4))
    return a


@pytest.mark.parametrize("p,m", [(1, 1), (1, 2), (2, 2), (3, 1), (3, 2)])
def test_cube_in_cube_counts_volume_constants(p, m):
    mb = O.MBMesh(*S.mb_cube_in_cube(m, seed=p), p)
    assert mb.n_unique == unique_cube_in_cube(m, p)
    assert mb.n_cellwise == 7 * m ** 3 * (p + 1) ** 3
    # every node's copies carry 1/mult each: the sum over cell-wise entries counts the nodes
    assert (1.0 / mb.multiplicity()).sum() == pytest.approx(mb.n_unique, rel=1e-12)
    one = np.ones(mb.n_unique)
    # trilinear blocks: detJ has degree <= 2 per direction, exact with n >= 2 Gauss points
    assert abs(mb.apply_assembled(O.MASS, one).sum() - 8.0) <= 1e-12
    assert np.abs(mb.apply_assembled(O.LAPLACE, one)).max() <= 1e-13


@pytest.mark.parametrize("ns,p", [(3, 1), (3, 2), (5, 1), (5, 2)])
def test_star_counts_and_area(ns, p):
    m, mz = 2, 1
    mb = O.MBMesh(*S.mb_star(ns, m, mz, seed=ns), p)
    assert mb.n_unique == unique_star(ns, m, mz, p)
    assert abs(mb.apply_assembled(O.MASS, np.ones(mb.n_unique)).sum() - star_area(ns)) <= 1e-12


def _sorted_by_coords(xyz, vals):
    key = np.round(xyz, 9)
    order = np.lexsort((key[:, 2], key[:, 1], key[:, 0]))
    return key[order], vals[order]


def _gll(p):
    x = np.zeros(p + 1)
    O._L().or_gll(p, x.ctypes.data_as(O._D))
    return x


def test_rotated_blocks_reproduce_the_structured_operator():
    """The unit cube split into two blocks along x (each m^3 cells, the second with a turned
    local frame) is the structured (2m, m, m) mesh: A_CG applied to the same smooth nodal field
    must agree node by node, for both operators."""
    m, p = 2, 3
    vxyz = np.array([[x, y, z] for z in (0, 1) for y in (0, 1) for x in (0, 0.5, 1)], float)
    vid = lambda i, j, k: k * 6 + j * 3 + i  # noqa: E731
    b0 = [vid(i, j, k) for k in (0, 1) for j in (0, 1) for i in (0, 1)]
    b1 = [vid(1 + i, j, k) for k in (0, 1) for j in (0, 1) for i in (0, 1)]
    rots = S._rotations()
    b1 = S._rotate_block(b1, rots[7])
    mb = O.MBMesh(vxyz, [b0, b1], [[m, m, m], [m, m, m]], p)
    om = O.Mesh((2 * m, m, m), p)
    assert mb.n_unique == (2 * m * p + 1) * (m * p + 1) ** 2
    f = lambda X: np.sin(2 * X[:, 0]) * np.cos(3 * X[:, 1]) + X[:, 2] ** 2  # noqa: E731
    xyz_mb = mb.node_coords()
    # structured node coordinates, lexicographic global order
    t = (1 + _gll(p)) / 2
    axes = [np.concatenate([[0.0]] + [(c + t[1:]) / mm for c in range(mm)])
            for mm in (2 * m, m, m)]
    gz, gy, gx = np.meshgrid(*(np.arange(len(a)) for a in axes[::-1]), indexing="ij")
    xyz_s = np.stack([axes[0][gx.ravel()], axes[1][gy.ravel()], axes[2][gz.ravel()]], axis=1)
    for op in (O.LAPLACE, O.MASS):
        y_mb = mb.apply_assembled(op, f(xyz_mb))
        y_s = np.zeros(len(xyz_s))
        O._L().or_apply_assembled(om._c, op, np.ascontiguousarray(f(xyz_s)).ctypes.data_as(O._D),
                                  y_s.ctypes.data_as(O._D), 0)
        k1, v1 = _sorted_by_coords(xyz_mb, y_mb)
        k2, v2 = _sorted_by_coords(xyz_s, y_s)
        assert np.array_equal(k1, k2)
        assert np.abs(v1 - v2).max() <= 1e-12 * np.abs(v2).max()


def test_assembled_operator_symmetric():
    mb = O.MBMesh(*S.mb_star(5, 2, 1, seed=3), 2)
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(mb.n_unique), rng.standard_normal(mb.n_unique)
    for op in (O.LAPLACE, O.MASS):
        a, b = mb.apply_assembled(op, x) @ y, mb.apply_assembled(op, y) @ x
        assert abs(a - b) <= 1e-12 * abs(a)
