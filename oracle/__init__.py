"""FP64 CPU oracle for the cell-wise matrix-free finite-element path (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
this package.  It wraps ``liboracle.so`` (plain C, ``oracle.c``), which is written from the
paper's definitions and shares nothing with the CUDA library:

* element operators, Eq. (mass_operator) / Eq. (laplace_operator), formed entry by entry with
  general per-quadrature-point geometry (Sec. 2.3);
* gather ``G`` / scatter ``G^T`` (Sec. 2.1), the constrained system and ``A_CG = G^T A G``
  (Sec. 3.1, Eq. (constrained_system));
* DSS ``S = G I_Riesz G^T`` (Sec. 3.3, Eq. (dss_operator)) and the Jacobi diagonal;
* assembled Jacobi-PCG/FCG (Algorithm "Communication-Free (Flexible) PCG" on global vectors).

Conventions: canonical cell-wise order ``((cz*my+cy)*mx+cx)*n^3 + (k*n+j)*n+i`` and lexicographic
global order ``(gz*Ny+gy)*Nx+gx``, ``Nx = mx*p+1``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

LAPLACE, MASS = 0, 1
RHS_SINE, RHS_QUADRATIC = 0, 1


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (FP contraction off, OpenMP on)."""
    hdr = os.path.join(_HERE, "oracle.h")
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(hdr))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class _Mesh(ctypes.Structure):
    _fields_ = [("mx", ctypes.c_int), ("my", ctypes.c_int), ("mz", ctypes.c_int),
                ("p", ctypes.c_int), ("amp", ctypes.c_double), ("dirichlet", ctypes.c_int)]


class _MB(ctypes.Structure):
    _fields_ = [("nblocks", ctypes.c_int), ("p", ctypes.c_int),
                ("dims", ctypes.POINTER(ctypes.c_int)),
                ("block_verts", ctypes.POINTER(ctypes.c_int)),
                ("vxyz", ctypes.POINTER(ctypes.c_double))]


class _CGOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("maxit", ctypes.c_int), ("flexible", ctypes.c_int)]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        M = ctypes.POINTER(_Mesh)
        ll, i32 = ctypes.c_longlong, ctypes.c_int
        sig = {
            "or_gauss": (i32, [i32, _D, _D]),
            "or_gll": (i32, [i32, _D]),
            "or_lagrange": (ctypes.c_double, [_D, i32, i32, ctypes.c_double]),
            "or_lagrange_deriv": (ctypes.c_double, [_D, i32, i32, ctypes.c_double]),
            "or_n_cells": (ll, [M]), "or_n_cellwise": (ll, [M]), "or_n_unique": (ll, [M]),
            "or_map": (None, [ctypes.c_double, _D, _D]),
            "or_cell_nodes": (None, [M, i32, i32, i32, _D]),
            "or_jacobian": (None, [M, _D, _D, _D]),
            "or_element_matrix": (i32, [M, i32, ll, _D]),
            "or_element_row": (i32, [M, i32, ll, i32, _D]),
            "or_gather": (None, [M, _D, _D]),
            "or_scatter": (None, [M, _D, _D]),
            "or_boundary_global": (None, [M, ctypes.POINTER(ctypes.c_ubyte)]),
            "or_multiplicity": (None, [M, _D]),
            "or_apply_local": (i32, [M, i32, _D, _D, i32]),
            "or_apply_assembled": (i32, [M, i32, _D, _D, i32]),
            "or_dss": (i32, [M, _D, _D]),
            "or_diag_global": (i32, [M, i32, _D, i32]),
            "or_element_matrices": (i32, [M, i32, ll, ll, _D, i32]),
            "or_apply_local_mats": (i32, [M, ll, ll, _D, _D, _D, i32]),
            "or_csr_nnz": (ll, [M]),
            "or_assemble_csr": (i32, [M, i32, ctypes.POINTER(ll), ctypes.POINTER(i32), _D, i32]),
            "or_csr_spmv": (None, [ll, ctypes.POINTER(ll), ctypes.POINTER(i32), _D, _D, _D]),
            "or_rhs": (i32, [M, i32, _D]),
            "or_exact_nodal": (None, [M, i32, _D]),
            "or_l2_error": (i32, [M, i32, _D, _D]),
            "or_cg": (i32, [M, i32, _D, _D, ctypes.POINTER(_CGOpts), ctypes.POINTER(i32),
                            _D, _D, _D, i32]),
            "or_mb_n_cellwise": (ll, [ctypes.POINTER(_MB)]),
            "or_mb_cell_offset": (ll, [ctypes.POINTER(_MB), i32]),
            "or_mb_cell_nodes": (None, [ctypes.POINTER(_MB), i32, i32, i32, i32, _D]),
            "or_mb_element_matrix": (i32, [ctypes.POINTER(_MB), i32, ll, _D]),
            "or_mb_apply_local": (i32, [ctypes.POINTER(_MB), i32, _D, _D, i32]),
            "or_mb_numbering": (ll, [ctypes.POINTER(_MB), ctypes.c_double, ctypes.POINTER(ll)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


class Mesh:
    """Structured hexahedral mesh of the unit cube, deformed by
    ``Phi(X) = X + amp sin(pi X) sin(pi Y) sin(pi Z) (1,1,1)`` and interpolated isoparametrically."""

    def __init__(self, m, p: int, amp: float = 0.0, dirichlet: bool = False):
        mx, my, mz = (m, m, m) if np.isscalar(m) else tuple(m)
        self.mx, self.my, self.mz, self.p = int(mx), int(my), int(mz), int(p)
        self.n = self.p + 1
        self.amp, self.dirichlet = float(amp), bool(dirichlet)
        self._c = _Mesh(self.mx, self.my, self.mz, self.p, self.amp, int(self.dirichlet))

    @property
    def ref(self):
        return ctypes.byref(self._c)

    @property
    def n_cells(self) -> int:
        return _L().or_n_cells(self.ref)

    @property
    def n_cellwise(self) -> int:
        return _L().or_n_cellwise(self.ref)

    @property
    def n_unique(self) -> int:
        return _L().or_n_unique(self.ref)

    @property
    def global_shape(self):
        p = self.p
        return (self.mz * p + 1, self.my * p + 1, self.mx * p + 1)


# ---- 1D rules -------------------------------------------------------------------------------
def gauss(n: int):
    x, w = np.zeros(n), np.zeros(n)
    assert _L().or_gauss(n, _dp(x), _dp(w)) == 0
    return x, w


def gll(p: int):
    x = np.zeros(p + 1)
    assert _L().or_gll(p, _dp(x)) == 0
    return x


def lagrange(t: np.ndarray, i: int, s: float, deriv: bool = False) -> float:
    t = np.ascontiguousarray(t, dtype=np.float64)
    f = _L().or_lagrange_deriv if deriv else _L().or_lagrange
    return f(_dp(t), len(t), i, float(s))


# ---- geometry --------------------------------------------------------------------------------
def map_point(amp: float, X) -> np.ndarray:
    Xa = np.ascontiguousarray(X, dtype=np.float64)
    x = np.zeros(3)
    _L().or_map(float(amp), _dp(Xa), _dp(x))
    return x


def cell_nodes(mesh: Mesh, cx: int, cy: int, cz: int) -> np.ndarray:
    xn = np.zeros((mesh.n ** 3, 3))
    _L().or_cell_nodes(mesh.ref, cx, cy, cz, _dp(xn))
    return xn


def jacobian(mesh: Mesh, xn: np.ndarray, xi) -> np.ndarray:
    J = np.zeros(9)
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    _L().or_jacobian(mesh.ref, _dp(np.ascontiguousarray(xn)), _dp(xi), _dp(J))
    return J.reshape(3, 3)


# ---- element level ---------------------------------------------------------------------------
def element_matrix(mesh: Mesh, op: int, cell: int) -> np.ndarray:
    nn = mesh.n ** 3
    A = np.zeros((nn, nn))
    st = _L().or_element_matrix(mesh.ref, op, cell, _dp(A))
    if st:
        raise RuntimeError(f"or_element_matrix status {st}")
    return A


def element_row(mesh: Mesh, op: int, cell: int, row: int) -> np.ndarray:
    out = np.zeros(mesh.n ** 3)
    st = _L().or_element_row(mesh.ref, op, cell, row, _dp(out))
    if st:
        raise RuntimeError(f"or_element_row status {st}")
    return out


def element_matrices(mesh: Mesh, op: int, cell0: int, ncell: int, nthreads: int = 0):
    nn = mesh.n ** 3
    mats = np.zeros((ncell, nn, nn))
    st = _L().or_element_matrices(mesh.ref, op, cell0, ncell, _dp(mats), nthreads)
    if st:
        raise RuntimeError(f"or_element_matrices status {st}")
    return mats


def apply_local_mats(mesh: Mesh, cell0: int, mats: np.ndarray, xc: np.ndarray,
                     nthreads: int = 0) -> np.ndarray:
    ncell = mats.shape[0]
    yc = np.zeros(ncell * mesh.n ** 3)
    _L().or_apply_local_mats(mesh.ref, cell0, ncell, _dp(mats), _dp(np.ascontiguousarray(xc)),
                             _dp(yc), nthreads)
    return yc


# ---- gather / scatter ------------------------------------------------------------------------
def gather(mesh: Mesh, xg: np.ndarray) -> np.ndarray:
    xc = np.zeros(mesh.n_cellwise)
    _L().or_gather(mesh.ref, _dp(np.ascontiguousarray(xg, dtype=np.float64)), _dp(xc))
    return xc


def scatter(mesh: Mesh, yc: np.ndarray) -> np.ndarray:
    yg = np.zeros(mesh.n_unique)
    _L().or_scatter(mesh.ref, _dp(np.ascontiguousarray(yc, dtype=np.float64)), _dp(yg))
    return yg


def boundary_global(mesh: Mesh) -> np.ndarray:
    b = np.zeros(mesh.n_unique, dtype=np.uint8)
    _L().or_boundary_global(mesh.ref, b.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    return b.astype(bool)


def multiplicity(mesh: Mesh) -> np.ndarray:
    m = np.zeros(mesh.n_cellwise)
    _L().or_multiplicity(mesh.ref, _dp(m))
    return m


# ---- operators -------------------------------------------------------------------------------
def apply_local(mesh: Mesh, op: int, xc: np.ndarray, nthreads: int = 0) -> np.ndarray:
    yc = np.zeros(mesh.n_cellwise)
    st = _L().or_apply_local(mesh.ref, op, _dp(np.ascontiguousarray(xc, dtype=np.float64)),
                             _dp(yc), nthreads)
    if st:
        raise RuntimeError(f"or_apply_local status {st}")
    return yc


def apply_assembled(mesh: Mesh, op: int, xg: np.ndarray, nthreads: int = 0) -> np.ndarray:
    yg = np.zeros(mesh.n_unique)
    st = _L().or_apply_assembled(mesh.ref, op, _dp(np.ascontiguousarray(xg, dtype=np.float64)),
                                 _dp(yg), nthreads)
    if st:
        raise RuntimeError(f"or_apply_assembled status {st}")
    return yg


def dss(mesh: Mesh, yc: np.ndarray) -> np.ndarray:
    zc = np.zeros(mesh.n_cellwise)
    assert _L().or_dss(mesh.ref, _dp(np.ascontiguousarray(yc, dtype=np.float64)), _dp(zc)) == 0
    return zc


def diag_global(mesh: Mesh, op: int, nthreads: int = 0) -> np.ndarray:
    d = np.zeros(mesh.n_unique)
    st = _L().or_diag_global(mesh.ref, op, _dp(d), nthreads)
    if st:
        raise RuntimeError(f"or_diag_global status {st}")
    return d


def assemble_csr(mesh: Mesh, op: int, nthreads: int = 0):
    """Return (rowptr, colidx, vals) of the unconstrained A_CG."""
    nnz = _L().or_csr_nnz(mesh.ref)
    nu = mesh.n_unique
    rowptr = np.zeros(nu + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz)
    st = _L().or_assemble_csr(mesh.ref, op,
                              rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                              col.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(val), nthreads)
    if st:
        raise RuntimeError(f"or_assemble_csr status {st}")
    return rowptr, col, val


def csr_spmv(csr, x: np.ndarray) -> np.ndarray:
    rowptr, col, val = csr
    y = np.zeros(len(rowptr) - 1)
    _L().or_csr_spmv(len(rowptr) - 1, rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                     col.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(val),
                     _dp(np.ascontiguousarray(x, dtype=np.float64)), _dp(y))
    return y


def apply_dirichlet_csr(mesh: Mesh, csr, xg: np.ndarray) -> np.ndarray:
    """A_D x = R A_CG R x with R zeroing Dirichlet nodes (identity without Dirichlet)."""
    x = np.array(xg, dtype=np.float64)
    if mesh.dirichlet:
        b = boundary_global(mesh)
        x[b] = 0.0
        y = csr_spmv(csr, x)
        y[b] = 0.0
        return y
    return csr_spmv(csr, x)


# ---- rhs, exact solution, error --------------------------------------------------------------
def rhs(mesh: Mesh, kind: int = RHS_SINE) -> np.ndarray:
    b = np.zeros(mesh.n_cellwise)
    st = _L().or_rhs(mesh.ref, kind, _dp(b))
    if st:
        raise RuntimeError(f"or_rhs status {st}")
    return b


def exact_nodal(mesh: Mesh, kind: int = RHS_SINE) -> np.ndarray:
    u = np.zeros(mesh.n_unique)
    _L().or_exact_nodal(mesh.ref, kind, _dp(u))
    return u


def l2_error(mesh: Mesh, uc: np.ndarray, kind: int = RHS_SINE) -> float:
    e = ctypes.c_double(0.0)
    _L().or_l2_error(mesh.ref, kind, _dp(np.ascontiguousarray(uc, dtype=np.float64)),
                     ctypes.byref(e))
    return e.value


# ---- assembled CG ----------------------------------------------------------------------------
def cg(mesh: Mesh, op: int, bg: np.ndarray, x0=None, rtol: float = 1e-10, maxit: int = 1000,
       flexible: bool = False, nthreads: int = 0):
    """Jacobi-PCG (or FCG) on the assembled global system.  Returns dict with x, status, iters,
    alpha, beta, relres."""
    nu = mesh.n_unique
    x = np.zeros(nu) if x0 is None else np.array(x0, dtype=np.float64)
    alpha, beta, relres = np.zeros(maxit + 1), np.zeros(maxit + 1), np.zeros(maxit + 2)
    it = ctypes.c_int(0)
    o = _CGOpts(rtol, maxit, int(flexible))
    st = _L().or_cg(mesh.ref, op, _dp(np.ascontiguousarray(bg, dtype=np.float64)), _dp(x),
                    ctypes.byref(o), ctypes.byref(it), _dp(alpha), _dp(beta), _dp(relres), nthreads)
    k = it.value
    return {"x": x, "status": st, "iters": k, "alpha": alpha[:k], "beta": beta[:max(k - 1, 0)],
            "relres": relres[:k + 1]}


class MBMesh:
    """Block-structured mesh (Sec. 4.2): macro-blocks given by eight corner vertices each
    (local corner c = i + 2j + 4k), a structured grid of dims[b] cells per block, trilinear
    geometry.  Cell-wise layout: blocks one after the other, each block's cells lexicographic,
    the canonical node order inside a cell.  The global numbering comes from the nodes'
    coordinates (``or_mb_numbering``); gather, scatter and DSS are then the plain definitions
    G, G^T and S = G G^T of Sec. 2.1 and Eq. (dss_operator)."""

    def __init__(self, vxyz, block_verts, dims, p: int, tol: float = 1e-9):
        self.vxyz = np.ascontiguousarray(np.asarray(vxyz, dtype=np.float64).reshape(-1, 3))
        self.block_verts = np.ascontiguousarray(np.asarray(block_verts, dtype=np.int32).reshape(-1, 8))
        self.dims = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(-1, 3))
        self.p, self.n = int(p), int(p) + 1
        self.nblocks = len(self.block_verts)
        self._c = _MB(self.nblocks, self.p, self.dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      self.block_verts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      self.vxyz.ctypes.data_as(_D))
        self.n_cellwise = int(_L().or_mb_n_cellwise(ctypes.byref(self._c)))
        self.gid = np.zeros(self.n_cellwise, dtype=np.int64)
        nu = _L().or_mb_numbering(ctypes.byref(self._c), tol,
                                  self.gid.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
        if nu < 0:
            raise MemoryError("or_mb_numbering")
        self.n_unique = int(nu)

    def cell_offset(self, block: int) -> int:
        return int(_L().or_mb_cell_offset(ctypes.byref(self._c), block))

    def cell_nodes(self, block, cx, cy, cz):
        xn = np.zeros(3 * self.n ** 3)
        _L().or_mb_cell_nodes(ctypes.byref(self._c), block, cx, cy, cz, _dp(xn))
        return xn.reshape(-1, 3)

    def node_coords(self):
        """Physical coordinates of every global node (from its first copy)."""
        xyz = np.zeros((self.n_unique, 3))
        n3 = self.n ** 3
        e = 0
        for b in range(self.nblocks):
            mx, my, mz = (int(v) for v in self.dims[b])
            for cz in range(mz):
                for cy in range(my):
                    for cx in range(mx):
                        xyz[self.gid[e:e + n3]] = self.cell_nodes(b, cx, cy, cz)
                        e += n3
        return xyz

    def gather(self, xg):
        return np.asarray(xg, dtype=np.float64)[self.gid]

    def scatter(self, yc):
        yg = np.zeros(self.n_unique)
        np.add.at(yg, self.gid, np.asarray(yc, dtype=np.float64))
        return yg

    def dss(self, yc):
        return self.gather(self.scatter(yc))

    def multiplicity(self):
        return self.gather(np.bincount(self.gid, minlength=self.n_unique).astype(np.float64))

    def element_matrix(self, op: int, cell: int):
        nn = self.n ** 3
        A = np.zeros(nn * nn)
        st = _L().or_mb_element_matrix(ctypes.byref(self._c), op, cell, _dp(A))
        if st:
            raise RuntimeError(f"or_mb_element_matrix: status {st}")
        return A.reshape(nn, nn)

    def apply_local(self, op: int, xc, nthreads: int = 0):
        xc = np.ascontiguousarray(xc, dtype=np.float64)
        yc = np.zeros(self.n_cellwise)
        st = _L().or_mb_apply_local(ctypes.byref(self._c), op, _dp(xc), _dp(yc), nthreads)
        if st:
            raise RuntimeError(f"or_mb_apply_local: status {st}")
        return yc

    def apply_assembled(self, op: int, xg, nthreads: int = 0):
        """A_CG x_glob = G^T (blockdiag A_K) G x_glob (Sec. 3.1)."""
        return self.scatter(self.apply_local(op, self.gather(xg), nthreads))


class Packed:
    """2^3 packing of a structured mesh (Sec. 2.2, the optional storage unit of Table
    "tab:memory_overhead"): each unit stores the (2p+1)^3 distinct nodes of a 2x2x2 cluster of
    cells, unit (ux, uy, uz) lexicographic over (mx/2, my/2, mz/2), local node (i, j, k) at
    (k N + j) N + i with N = 2p+1.  Built on the structured oracle: P maps a unit vector to the
    cell-wise copies of its eight cells, so the unit-level operators are the definitions
    P^T A_K P (local), G_u = P^{-1}-free gather from global nodes, and S_u = G_u G_u^T."""

    def __init__(self, mesh: Mesh):
        if mesh.mx % 2 or mesh.my % 2 or mesh.mz % 2:
            raise ValueError("packing needs even cell counts")
        self.mesh = mesh
        p, n = mesh.p, mesh.n
        self.N = N = 2 * p + 1
        self.ux, self.uy, self.uz = mesh.mx // 2, mesh.my // 2, mesh.mz // 2
        self.n_units = self.ux * self.uy * self.uz
        self.length = self.n_units * N ** 3
        Nx, Ny = mesh.mx * p + 1, mesh.my * p + 1
        # global node of every unit-storage entry
        u = np.arange(self.n_units)
        ux, uy, uz = u % self.ux, (u // self.ux) % self.uy, u // (self.ux * self.uy)
        loc = np.arange(N ** 3)
        i, j, k = loc % N, (loc // N) % N, loc // (N * N)
        gx = (2 * p * ux)[:, None] + i[None, :]
        gy = (2 * p * uy)[:, None] + j[None, :]
        gz = (2 * p * uz)[:, None] + k[None, :]
        self.gid = ((gz * Ny + gy) * Nx + gx).ravel()
        # P: for every cell-wise entry, the unit-storage entry holding the same node
        c = np.arange(mesh.mx * mesh.my * mesh.mz)
        cx, cy, cz = c % mesh.mx, (c // mesh.mx) % mesh.my, c // (mesh.mx * mesh.my)
        cl = np.arange(n ** 3)
        ci, cj, ck = cl % n, (cl // n) % n, cl // (n * n)
        unit = ((cz // 2) * self.uy + cy // 2) * self.ux + cx // 2
        li = (p * (cx % 2))[:, None] + ci[None, :]
        lj = (p * (cy % 2))[:, None] + cj[None, :]
        lk = (p * (cz % 2))[:, None] + ck[None, :]
        self.P = (unit[:, None] * N ** 3 + (lk * N + lj) * N + li).ravel()

    def gather(self, xg):
        return np.asarray(xg, dtype=np.float64)[self.gid]

    def scatter(self, yu):
        yg = np.zeros(or_n_unique(self.mesh))
        np.add.at(yg, self.gid, np.asarray(yu, dtype=np.float64))
        return yg

    def dss(self, yu):
        return self.gather(self.scatter(yu))

    def multiplicity(self):
        return self.gather(np.bincount(self.gid, minlength=or_n_unique(self.mesh)).astype(float))

    def to_cellwise(self, xu):
        return np.asarray(xu, dtype=np.float64)[self.P]

    def from_cellwise(self, yc):
        yu = np.zeros(self.length)
        np.add.at(yu, self.P, np.asarray(yc, dtype=np.float64))
        return yu

    def apply_local(self, op: int, xu, nthreads: int = 0):
        """sum over the unit's cells K of P_K^T A_K P_K x_unit (Dirichlet rows/columns as in the
        structured oracle)."""
        return self.from_cellwise(apply_local(self.mesh, op, self.to_cellwise(xu), nthreads))


def or_n_unique(mesh: Mesh) -> int:
    return int(_L().or_n_unique(mesh.ref))


class Adaptive:
    """Two-level Cartesian refinement of the unit cube (Appendix "Extension of DSS algorithms onto
    Non-Conforming Interfaces"): a coarse grid of mc^3 cells, the cells of the box
    [lo, hi) (coarse cell coordinates, strictly inside the domain) each refined into 2x2x2 fine
    cells.  Storage: the full coarse grid (the cells inside the box are dormant and stay zero),
    then the fine grid of the box, both in layout 0.  The conforming space constrains every fine
    node on the box boundary to the trace of the coarse polynomial of its parent cell, so the
    gather G_c maps global DoFs (nodes of the active coarse cells, fine nodes off the box boundary)
    to copies, with interpolation weights P(i, J) = prod_d l_J_d(xi_d(i)) on the constrained fine
    copies.  DSS is S = G_c G_c^T on the active copies, zero on the dormant ones."""

    def __init__(self, mc: int, lo, hi, p: int):
        self.mc, self.lo, self.hi, self.p = mc, tuple(lo), tuple(hi), p
        n = self.n = p + 1
        assert all(1 <= lo[d] < hi[d] <= mc - 1 for d in range(3)), "box strictly inside"
        self.fd = tuple(2 * (hi[d] - lo[d]) for d in range(3))  # fine cells per direction
        nc_coarse = mc ** 3
        nc_fine = self.fd[0] * self.fd[1] * self.fd[2]
        n3 = n ** 3
        self.length = (nc_coarse + nc_fine) * n3
        t = (1.0 + gll(p)) / 2.0
        self.t = t
        rows, cols, vals = [], [], []
        key_id = {}

        def node_key(x):  # coinciding nodes agree to rounding; distinct ones differ by >= 1e-4
            return tuple(int(round(v * 2 ** 30)) for v in x)

        def dof(x):
            k = node_key(x)
            if k not in key_id:
                key_id[k] = len(key_id)
            return key_id[k]

        self.active = np.zeros(nc_coarse + nc_fine, dtype=bool)
        # coarse active cells
        for cz in range(mc):
            for cy in range(mc):
                for cx in range(mc):
                    c = (cz * mc + cy) * mc + cx
                    if all(lo[d] <= (cx, cy, cz)[d] < hi[d] for d in range(3)):
                        continue
                    self.active[c] = True
                    for a in range(n3):
                        i, j, k = a % n, (a // n) % n, a // (n * n)
                        x = ((cx + t[i]) / mc, (cy + t[j]) / mc, (cz + t[k]) / mc)
                        rows.append(c * n3 + a)
                        cols.append(dof(x))
                        vals.append(1.0)
        # fine cells: free nodes, or constrained to the parent's coarse nodes on the box boundary
        H = 2 * mc
        fine_cols, fine_rows, fine_vals = [], [], []
        for fz in range(self.fd[2]):
            for fy in range(self.fd[1]):
                for fx in range(self.fd[0]):
                    c = nc_coarse + (fz * self.fd[1] + fy) * self.fd[0] + fx
                    self.active[c] = True
                    g = (2 * lo[0] + fx, 2 * lo[1] + fy, 2 * lo[2] + fz)  # fine cell, global
                    par = tuple(gg // 2 for gg in g)
                    half = tuple(gg % 2 for gg in g)
                    for a in range(n3):
                        ijk = (a % n, (a // n) % n, a // (n * n))
                        x = tuple((g[d] + t[ijk[d]]) / H for d in range(3))
                        fidx = [g[d] * p + ijk[d] for d in range(3)]  # fine node lattice index
                        on_bnd = any(fidx[d] in (2 * lo[d] * p, 2 * hi[d] * p) for d in range(3))
                        if not on_bnd:
                            fine_rows.append(c * n3 + a)
                            fine_cols.append(x)
                            fine_vals.append(None)
                            continue
                        xi = [(half[d] + t[ijk[d]]) / 2.0 for d in range(3)]  # in the parent
                        for b in range(n3):
                            J = (b % n, (b // n) % n, b // (n * n))
                            w = 1.0
                            for d in range(3):
                                w *= lagrange(t, J[d], xi[d])
                            if w == 0.0:
                                continue
                            xJ = tuple((par[d] + t[J[d]]) / mc for d in range(3))
                            fine_rows.append(c * n3 + a)
                            fine_cols.append(xJ)
                            fine_vals.append(w)
        ncoarse_dofs = len(key_id)
        for r, x, w in zip(fine_rows, fine_cols, fine_vals):
            if w is None:
                rows.append(r)
                cols.append(dof(x))
                vals.append(1.0)
            else:
                k = node_key(x)
                assert k in key_id and key_id[k] < ncoarse_dofs, "constraint to a non-coarse node"
                rows.append(r)
                cols.append(key_id[k])
                vals.append(w)
        self.n_unique = len(key_id)
        import scipy.sparse as sp
        self.G = sp.csr_matrix((vals, (rows, cols)), shape=(self.length, self.n_unique))
        self.active_entries = np.repeat(self.active, n3)

    def gather(self, xg):
        return self.G @ np.asarray(xg, dtype=np.float64)

    def scatter(self, yc):
        return self.G.T @ np.asarray(yc, dtype=np.float64)

    def dss(self, yc):
        return self.G @ (self.G.T @ np.asarray(yc, dtype=np.float64))

    def cell_corners(self, c):
        """(8, 3) corner coordinates of storage cell c (coarse or fine)."""
        mc, n = self.mc, self.n
        if c < mc ** 3:
            g, h = ((c % mc), (c // mc) % mc, c // (mc * mc)), 1.0 / mc
        else:
            f = c - mc ** 3
            fx, fy = f % self.fd[0], (f // self.fd[0]) % self.fd[1]
            fz = f // (self.fd[0] * self.fd[1])
            g = (2 * self.lo[0] + fx, 2 * self.lo[1] + fy, 2 * self.lo[2] + fz)
            h = 1.0 / (2 * mc)
        return np.array([[(g[0] + (k & 1)) * h, (g[1] + ((k >> 1) & 1)) * h,
                          (g[2] + ((k >> 2) & 1)) * h] for k in range(8)])

    def apply_local(self, op: int, xc):
        """Per active cell A_K x_K (element matrices of the oracle's trilinear cells)."""
        n3 = self.n ** 3
        ncell = len(self.active)
        vx = np.concatenate([self.cell_corners(c) for c in range(ncell)])
        mb = MBMesh(vx, np.arange(8 * ncell).reshape(ncell, 8), np.ones((ncell, 3)), self.p,
                    tol=-1.0)
        yc = np.zeros(self.length)
        xc = np.asarray(xc, dtype=np.float64)
        for c in np.nonzero(self.active)[0]:
            A = mb.element_matrix(op, int(c))
            yc[c * n3:(c + 1) * n3] = A @ xc[c * n3:(c + 1) * n3]
        return yc
