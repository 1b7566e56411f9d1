"""Pins for the FP64 CPU oracle: values fixed by the paper, closed forms, invariants, library
routines and brute force on tiny inputs (no GPU).  Each pin is chosen so that a plausible slip in
the oracle (a dropped term, a sign, a transposed Jacobian, a wrong index) fails at least one."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2607_02335_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- 1D rules
@pytest.mark.parametrize("n", range(1, 11))
def test_gauss_matches_library(n):
    x, w = O.gauss(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, xr, atol=1e-15, rtol=0)
    assert np.allclose(w, wr, atol=1e-15, rtol=0)


@pytest.mark.parametrize("n", range(1, 9))
def test_gauss_exact_to_degree_2n_minus_1(n):
    x, w = O.gauss(n)
    for k in range(2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, x ** k) - exact) < 1e-14
    assert abs(w.sum() - 2.0) < 1e-15


def test_gll_closed_forms():
    assert np.allclose(O.gll(1), [-1, 1], atol=0)
    assert np.allclose(O.gll(2), [-1, 0, 1], atol=1e-16)
    assert np.allclose(O.gll(3), [-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1], atol=1e-15)
    assert np.allclose(O.gll(4), [-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1], atol=1e-15)
    a = math.sqrt(1 / 3 - 2 * math.sqrt(7) / 21)
    b = math.sqrt(1 / 3 + 2 * math.sqrt(7) / 21)
    assert np.allclose(O.gll(5), [-1, -b, -a, a, b, 1], atol=1e-15)


@pytest.mark.parametrize("p", range(2, 8))
def test_gll_interior_are_roots_of_legendre_derivative(p):
    dP = np.polynomial.legendre.Legendre.basis(p).deriv()
    roots = np.sort(dP.roots().real)
    assert np.allclose(O.gll(p)[1:-1], roots, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3, 5, 7])
def test_lagrange_cardinal_and_partition_of_unity(p):
    t = 0.5 * (1 + O.gll(p))
    n = p + 1
    for i in range(n):
        for j in range(n):
            assert abs(O.lagrange(t, i, t[j]) - (1.0 if i == j else 0.0)) < 1e-14
    for s in np.linspace(-0.2, 1.2, 13):
        assert abs(sum(O.lagrange(t, i, s) for i in range(n)) - 1.0) < 1e-12
        assert abs(sum(O.lagrange(t, i, s, deriv=True) for i in range(n))) < 1e-10


def test_lagrange_derivative_vs_polynomial_fit():
    p = 4
    t = 0.5 * (1 + O.gll(p))
    for i in range(p + 1):
        y = np.zeros(p + 1)
        y[i] = 1.0
        poly = np.polynomial.Polynomial.fit(t, y, p, domain=[0, 1], window=[0, 1])
        for s in [0.1, 0.37, 0.8]:
            assert abs(O.lagrange(t, i, s, deriv=True) - poly.deriv()(s)) < 1e-10


# ---------------------------------------------------------------- counts (Table tab:memory_overhead)
def test_memory_overhead_table():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "memory_overhead.txt"))
            if l.strip() and not l.startswith("#")]
    for name, edge, stored, unique, sratio, tratio in rows:
        edge = int(edge)
        # one storage unit with `edge` nodes per edge is a single Q_{edge-1} cell
        mesh1 = O.Mesh(1, edge - 1)
        assert mesh1.n_cellwise == int(stored)
        big = O.Mesh(4000, edge - 1)  # unique nodes per unit, asymptotically
        unique_per_cell = big.n_unique / big.n_cells
        assert abs(unique_per_cell - int(unique)) / int(unique) < 2e-3
        assert round(int(stored) / int(unique), 2) == float(sratio)
        # cell-wise: one read + one write of the stored values; assembled: read x, read-add-write
        # y.  The printed transfer ratios are 2/3 of the printed (rounded) storage ratios, e.g.
        # Q7: 2/3 * 1.49 = 0.99 while 2*512/(3*343) = 0.995.
        assert round(2.0 / 3.0 * float(sratio), 2) == float(tratio)
        assert abs(2 * int(stored) / (3 * int(unique)) - float(tratio)) < 0.006


def test_unique_count_closed_form():
    for m, p in [(1, 1), (3, 2), (5, 3), (2, 7)]:
        assert O.Mesh(m, p).n_unique == (m * p + 1) ** 3
        assert O.Mesh(m, p).n_cellwise == m ** 3 * (p + 1) ** 3
    assert O.Mesh((2, 3, 4), 2).n_unique == 5 * 7 * 9


# ---------------------------------------------------------------- geometry
def test_affine_jacobian_is_diagonal_cell_size():
    mesh = O.Mesh((2, 3, 4), 3)
    xn = O.cell_nodes(mesh, 1, 2, 3)
    J = O.jacobian(mesh, xn, [0.3, 0.6, 0.1])
    assert np.allclose(J, np.diag([1 / 2, 1 / 3, 1 / 4]), atol=1e-14)


def test_isoparametric_jacobian_approximates_map_derivative():
    # J_ab = d x_a / d xi_b.  The map adds amp*s(X)*(1,1,1), so the exact derivative is
    # (I + amp (1,1,1) grad s^T) / m -- not symmetric, which catches a transposed J.
    m, amp = 3, 0.1
    mesh = O.Mesh(m, 7, amp=amp)
    xn = O.cell_nodes(mesh, 1, 0, 2)
    xi = np.array([0.3, 0.7, 0.45])
    X = (np.array([1, 0, 2]) + xi) / m
    pi = math.pi
    gs = pi * np.array([math.cos(pi * X[0]) * math.sin(pi * X[1]) * math.sin(pi * X[2]),
                        math.sin(pi * X[0]) * math.cos(pi * X[1]) * math.sin(pi * X[2]),
                        math.sin(pi * X[0]) * math.sin(pi * X[1]) * math.cos(pi * X[2])])
    Jex = (np.eye(3) + amp * np.outer(np.ones(3), gs)) / m
    J = O.jacobian(mesh, xn, xi)
    assert np.abs(J - Jex).max() < 1e-6
    assert np.abs(J - J.T).max() > 1e-3


def test_map_fixes_boundary():
    for X in ([0, 0.3, 0.7], [1, 0.5, 0.5], [0.2, 0.0, 0.9], [0.4, 0.6, 1.0]):
        assert np.allclose(O.map_point(0.15, X), X, atol=1e-16)


# ---------------------------------------------------------------- element matrices (closed forms)
def _q1_pattern(h, diag, one, two, three):
    A = np.zeros((8, 8))
    for a in range(8):
        for b in range(8):
            d = bin(a ^ b).count("1")
            A[a, b] = [diag, one, two, three][d]
    return A


def test_q1_affine_stiffness_closed_form():
    m = 3
    h = 1.0 / m
    mesh = O.Mesh(m, 1)
    K = O.element_matrix(mesh, O.LAPLACE, 13)
    ref = h * _q1_pattern(h, 1 / 3, 0.0, -1 / 12, -1 / 12)
    assert np.abs(K - ref).max() < 1e-15


def test_q1_affine_mass_closed_form():
    m = 2
    h = 1.0 / m
    mesh = O.Mesh(m, 1)
    M = O.element_matrix(mesh, O.MASS, 5)
    ref = h ** 3 * _q1_pattern(h, 1 / 27, 1 / 54, 1 / 108, 1 / 216)
    assert np.abs(M - ref).max() < 1e-16


def test_q2_affine_matches_textbook_kronecker_form():
    # textbook 1D quadratic element on [0,1] with nodes 0, 1/2, 1
    S1 = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / 3.0
    M1 = np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) / 30.0
    hx, hy, hz = 1 / 2, 1 / 3, 1 / 4
    mesh = O.Mesh((2, 3, 4), 2)
    Sx, Sy, Sz = S1 / hx, S1 / hy, S1 / hz
    Mx, My, Mz = M1 * hx, M1 * hy, M1 * hz
    # local index (k*n + j)*n + i  <->  kron(z, y, x)
    Kref = np.kron(np.kron(Mz, My), Sx) + np.kron(np.kron(Mz, Sy), Mx) + np.kron(np.kron(Sz, My), Mx)
    Mref = np.kron(np.kron(Mz, My), Mx)
    K = O.element_matrix(mesh, O.LAPLACE, 7)
    M = O.element_matrix(mesh, O.MASS, 7)
    assert np.abs(K - Kref).max() < 1e-13 * np.abs(Kref).max()
    assert np.abs(M - Mref).max() < 1e-15


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_element_matrices_symmetric_and_rows_consistent(p):
    mesh = O.Mesh(2, p, amp=0.1)
    for op in (O.LAPLACE, O.MASS):
        A = O.element_matrix(mesh, op, 5)
        assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
        r = O.element_row(mesh, op, 5, 3)
        assert np.abs(r - A[3]).max() <= 1e-15 * np.abs(A).max()
        w = np.linalg.eigvalsh(A)
        assert w.min() > -1e-12 * w.max()


def test_q7_single_cell_laplace_annihilates_constants():
    mesh = O.Mesh(1, 7, amp=0.1)
    K = O.element_matrix(mesh, O.LAPLACE, 0)
    assert np.abs(K.sum(axis=1)).max() < 1e-12 * np.abs(K).max()


# ---------------------------------------------------------------- global invariants
@pytest.mark.parametrize("p,amp", [(1, 0.1), (2, 0.1), (3, 0.1), (4, 0.05)])
def test_laplace_annihilates_constants(p, amp):
    mesh = O.Mesh(2, p, amp=amp)
    y = O.apply_assembled(mesh, O.LAPLACE, np.ones(mesh.n_unique))
    K = O.element_matrix(mesh, O.LAPLACE, 0)
    assert np.abs(y).max() < 1e-13 * np.abs(K).max() * 8


@pytest.mark.parametrize("p,amp,tol", [(1, 0.0, 1e-14), (3, 0.0, 1e-14), (5, 0.0, 1e-13),
                                       (1, 0.1, 1e-14), (2, 0.1, 1e-14), (3, 0.1, 1e-5)])
def test_mass_of_ones_is_volume(p, amp, tol):
    mesh = O.Mesh(2, p, amp=amp)
    one = np.ones(mesh.n_unique)
    y = O.apply_assembled(mesh, O.MASS, one)
    assert abs(one @ y - 1.0) < tol


def test_symmetry_of_assembled_operator():
    mesh = O.Mesh((2, 3, 2), 3, amp=0.1, dirichlet=True)
    x = S.primal_unique((2, 3, 2), 3, seed=1)
    y = S.primal_unique((2, 3, 2), 3, seed=2)
    for op in (O.LAPLACE, O.MASS):
        ax, ay = O.apply_assembled(mesh, op, x), O.apply_assembled(mesh, op, y)
        assert abs(ax @ y - ay @ x) < 1e-13 * np.abs(ax).max() * len(x) ** 0.5


def test_csr_equals_elementwise_and_dense_brute_force():
    mesh = O.Mesh((2, 1, 2), 2, amp=0.1, dirichlet=True)
    csr = O.assemble_csr(mesh, O.LAPLACE)
    nu = mesh.n_unique
    dense = np.zeros((nu, nu))
    for c in range(nu):  # column by column through the element-wise apply
        e = np.zeros(nu)
        e[c] = 1.0
        dense[:, c] = O.apply_assembled(mesh, O.LAPLACE, e)
    x = S.primal_unique((2, 1, 2), 2, seed=3)
    y_csr = O.apply_dirichlet_csr(mesh, csr, x)
    assert np.abs(y_csr - dense @ x).max() < 1e-13 * np.abs(y_csr).max()
    free = ~O.boundary_global(mesh)
    Af = dense[np.ix_(free, free)]
    assert np.abs(Af - Af.T).max() < 1e-14 * np.abs(Af).max()
    assert np.linalg.eigvalsh(Af).min() > 0
    d = O.diag_global(mesh, O.LAPLACE)
    assert np.allclose(d[free], np.diag(dense)[free], rtol=1e-14, atol=0)
    assert np.all(d[~free] == 1.0)


def test_csr_without_dirichlet_matches_elementwise():
    mesh = O.Mesh((3, 2, 2), 3, amp=0.1)
    csr = O.assemble_csr(mesh, O.MASS)
    x = S.primal_unique((3, 2, 2), 3, seed=5)
    assert np.abs(O.csr_spmv(csr, x) - O.apply_assembled(mesh, O.MASS, x)).max() < 1e-15


# ---------------------------------------------------------------- gather / scatter / DSS
def test_pairing_lemma_gather_scatter_adjoint():
    mesh = O.Mesh((2, 3, 2), 2)
    f = S.dual_cellwise((2, 3, 2), 2, seed=4)
    u = S.primal_unique((2, 3, 2), 2, seed=6)
    lhs = f @ O.gather(mesh, u)
    rhs = O.scatter(mesh, f) @ u
    assert abs(lhs - rhs) < 1e-12 * np.abs(f).sum()


def _closed_form_multiplicity(mesh):
    n, p = mesh.n, mesh.p
    out = np.zeros(mesh.n_cellwise)
    e = 0
    for cz in range(mesh.mz):
        for cy in range(mesh.my):
            for cx in range(mesh.mx):
                for k in range(n):
                    for j in range(n):
                        for i in range(n):
                            mult = 1
                            for c, l, mm in ((cx, i, mesh.mx), (cy, j, mesh.my), (cz, k, mesh.mz)):
                                g = c * p + l
                                if g % p == 0 and 0 < g < mm * p:
                                    mult *= 2
                            out[e] = mult
                            e += 1
    return out


@pytest.mark.parametrize("m,p", [((2, 2, 2), 1), ((3, 2, 2), 2), ((2, 3, 1), 4)])
def test_dss_of_ones_is_multiplicity(m, p):
    mesh = O.Mesh(m, p)
    s1 = O.dss(mesh, np.ones(mesh.n_cellwise))
    assert np.array_equal(s1, _closed_form_multiplicity(mesh))
    assert np.array_equal(O.multiplicity(mesh), s1)


def test_dss_worked_example_four_copies():
    lines = [l.split() for l in open(os.path.join(GOLDEN, "dss_four_copies.txt"))
             if l.strip() and not l.startswith("#")]
    examples = [list(map(float, l)) for l in lines if len(l) == 5]
    # 2 x 2 x 1 mesh of Q1 cells: the central vertical edge carries nodes shared by four cells
    mesh = O.Mesh((2, 2, 1), 1)
    n3 = 8
    for a, b, c, d, expect in examples:
        y = np.zeros(mesh.n_cellwise)
        # node (x=1/2, y=1/2, z=0): local (1,1,0) in cell 0, (0,1,0) in 1, (1,0,0) in 2, (0,0,0) in 3
        slots = [0 * n3 + 3, 1 * n3 + 2, 2 * n3 + 1, 3 * n3 + 0]
        for s, v in zip(slots, (a, b, c, d)):
            y[s] = v
        z = O.dss(mesh, y)
        assert all(z[s] == expect for s in slots)
        others = np.ones(mesh.n_cellwise, bool)
        others[slots] = False
        assert np.all(z[others] == 0.0)
    rep = [l for l in lines if len(l) == 3][0]
    copies, init, assembled = int(rep[0]), float(rep[1]), float(rep[2])
    s1 = O.dss(mesh, init * np.ones(mesh.n_cellwise))
    assert s1[3] == assembled and copies == 4


def test_dss_is_idempotent_up_to_multiplicity():
    mesh = O.Mesh((2, 2, 3), 2)
    y = S.dual_cellwise((2, 2, 3), 2, seed=9)
    z = O.dss(mesh, y)
    mult = O.multiplicity(mesh)
    assert np.abs(O.dss(mesh, z / mult) - z).max() < 1e-14


# ---------------------------------------------------------------- rhs, solves, convergence
def test_rhs_integrates_f():
    # sum of the unassembled load = integral of f (partition of unity); 24/pi for the sine case
    mesh = O.Mesh(4, 3, amp=0.1)
    b = O.rhs(mesh, O.RHS_SINE)
    assert abs(b.sum() - 24.0 / math.pi) < 2e-4


@pytest.mark.parametrize("p", [2, 3])
def test_quadratic_manufactured_solution_is_exact(p):
    m = 3
    mesh = O.Mesh(m, p, dirichlet=True)
    bg = O.scatter(mesh, O.rhs(mesh, O.RHS_QUADRATIC))
    res = O.cg(mesh, O.LAPLACE, bg, rtol=1e-14, maxit=2000)
    assert res["status"] == 0
    u = O.exact_nodal(mesh, O.RHS_QUADRATIC)
    assert np.abs(res["x"] - u).max() < 1e-12


def test_sine_l2_convergence_rate():
    for p in (1, 2):
        errs = []
        for m in (3, 6):
            mesh = O.Mesh(m, p, amp=0.05, dirichlet=True)
            bg = O.scatter(mesh, O.rhs(mesh, O.RHS_SINE))
            res = O.cg(mesh, O.LAPLACE, bg, rtol=1e-13, maxit=5000)
            errs.append(O.l2_error(mesh, O.gather(mesh, res["x"]), O.RHS_SINE))
        rate = math.log2(errs[0] / errs[1])
        assert rate > p + 1 - 0.35, (p, errs, rate)


def test_cg_matches_direct_solve_and_fcg():
    scipy_sparse = pytest.importorskip("scipy.sparse")
    spla = pytest.importorskip("scipy.sparse.linalg")
    mesh = O.Mesh((3, 2, 3), 3, amp=0.1, dirichlet=True)
    b = O.scatter(mesh, S.dual_cellwise((3, 2, 3), 3, seed=11))
    free = ~O.boundary_global(mesh)
    rowptr, col, val = O.assemble_csr(mesh, O.LAPLACE)
    A = scipy_sparse.csr_matrix((val, col, rowptr), shape=(mesh.n_unique,) * 2)
    Af = A[free][:, free]
    xd = np.zeros(mesh.n_unique)
    xd[free] = spla.spsolve(Af.tocsc(), b[free])
    r1 = O.cg(mesh, O.LAPLACE, b, rtol=1e-13, maxit=3000)
    r2 = O.cg(mesh, O.LAPLACE, b, rtol=1e-13, maxit=3000, flexible=True)
    assert r1["status"] == 0 and r2["status"] == 0
    assert np.abs(r1["x"] - xd).max() < 1e-10 * np.abs(xd).max()
    assert np.abs(r2["x"] - xd).max() < 1e-10 * np.abs(xd).max()
    # with a fixed preconditioner the two beta formulas agree in exact arithmetic
    k = 8
    assert np.allclose(r1["alpha"][:k], r2["alpha"][:k], rtol=1e-8)
    assert np.allclose(r1["beta"][:k], r2["beta"][:k], rtol=1e-6)
    assert np.all(np.diff(r1["relres"][:3]) < 1)


# ---------------------------------------------------------------- element-matrix apply, L2 norm
@pytest.mark.parametrize("p,dirichlet", [(2, True), (3, True), (4, False)])
def test_apply_local_mats_equals_apply_local(p, dirichlet):
    """The CPU baseline's apply (precomputed element matrices, a range of cells) is A_K x_K of
    Sec. 3.1: bitwise the on-the-fly element apply on the same cells, and within rounding of a
    numpy product with the masks applied by hand (Dirichlet rows and columns zeroed)."""
    m = (3, 4, 2)
    mesh = O.Mesh(m, p, amp=0.1, dirichlet=dirichlet)
    n3 = (p + 1) ** 3
    xc = S.dual_cellwise(m, p, seed=21)
    yref = O.apply_local(mesh, O.LAPLACE, xc)
    cell0, ncell = 5, 11
    mats = O.element_matrices(mesh, O.LAPLACE, cell0, ncell)
    sl = slice(cell0 * n3, (cell0 + ncell) * n3)
    y = O.apply_local_mats(mesh, cell0, mats, xc[sl])
    assert np.array_equal(y, yref[sl])
    keep = np.ones(mesh.n_cellwise)
    if dirichlet:
        bnd = O.boundary_global(mesh)
        gidx = O.gather(mesh, np.arange(mesh.n_unique, dtype=np.float64)).astype(np.int64)
        keep = (~bnd[gidx]).astype(np.float64)
    kx = (xc * keep)[sl].reshape(ncell, n3)
    yn = np.einsum("cab,cb->ca", mats, kx).reshape(-1) * keep[sl]
    assert np.abs(y - yn).max() <= 1e-14 * np.abs(yn).max()
    if dirichlet:
        assert np.all(y[keep[sl] == 0] == 0.0)


def test_l2_error_closed_forms():
    """||u_h - u||_{L2(unit cube)} against closed forms: u_h = 0 gives ||u|| = (1/30)^{3/2} for
    u = prod x(1-x) and (1/8)^{1/2} for the sine; u_h = I u (p >= 2, affine) gives 0; u_h = 2 I u
    gives ||u|| (a sign slip gives 3 ||u||); u_h = c gives sqrt(c^2 - 2c/216 + 1/27000) on a
    deformed mesh (det J weighting, exact in physical space up to quadrature)."""
    quad = (1.0 / 30.0) ** 1.5
    for p in (2, 3):
        mesh = O.Mesh(3, p)
        zero = np.zeros(mesh.n_cellwise)
        assert abs(O.l2_error(mesh, zero, O.RHS_QUADRATIC) - quad) <= 1e-14
        uq = O.gather(mesh, O.exact_nodal(mesh, O.RHS_QUADRATIC))
        assert O.l2_error(mesh, uq, O.RHS_QUADRATIC) <= 1e-14
        assert abs(O.l2_error(mesh, 2.0 * uq, O.RHS_QUADRATIC) - quad) <= 1e-14
    mesh = O.Mesh(4, 3)
    assert abs(O.l2_error(mesh, np.zeros(mesh.n_cellwise), O.RHS_SINE) - math.sqrt(0.125)) <= 1e-9
    c = 0.3
    for amp in (0.0, 0.1):
        mesh = O.Mesh(4, 3, amp=amp)
        e = O.l2_error(mesh, np.full(mesh.n_cellwise, c), O.RHS_QUADRATIC)
        assert abs(e - math.sqrt(c * c - 2 * c / 216 + 1 / 27000)) <= 1e-7, amp
