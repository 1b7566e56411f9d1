"""Thin ctypes binding of ``libfe.so`` (C ABI in ``include/fe.h``).

The functions below carry the C names and only marshal arguments: device vectors are passed as
raw pointers (``torch.Tensor.data_ptr()``), streams as ``cudaStream_t`` handles.  Every step of
the computation runs in the library's CUDA kernels; there is no fallback.  Importing this module
raises ``ImportError`` when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libfe.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libfe.so not built ({_LIB_PATH}); run `python -m paper_2607_02335_gb300.build`")
_lib = ctypes.CDLL(_LIB_PATH)

# ---- enums (mirrors of include/fe.h) ----------------------------------------------------------
FE_OK, FE_ERR_INVALID, FE_ERR_OOM, FE_ERR_CUDA = 0, 1, 2, 3
FE_ERR_NOT_CONVERGED, FE_ERR_BREAKDOWN, FE_ERR_TIMEOUT, FE_ERR_BUSY, FE_ERR_COMM = 4, 5, 6, 7, 8
FE_LAPLACE, FE_MASS = 0, 1
FE_F64, FE_F32, FE_BF16_F32ACC, FE_F16_F32ACC = 0, 1, 2, 3
FE_GEOM_STORED, FE_GEOM_RECOMPUTE, FE_GEOM_AFFINE = 0, 1, 2
FE_LAYOUT_CELLS, FE_LAYOUT_PACKED2 = 0, 1
FE_ASSEMBLE, FE_NATIVE_F64 = 1, 2
FE_RHS_SINE, FE_RHS_QUADRATIC = 0, 1

STATUS_NAMES = {0: "FE_OK", 1: "FE_ERR_INVALID", 2: "FE_ERR_OOM", 3: "FE_ERR_CUDA",
                4: "FE_ERR_NOT_CONVERGED", 5: "FE_ERR_BREAKDOWN", 6: "FE_ERR_TIMEOUT",
                7: "FE_ERR_BUSY", 8: "FE_ERR_COMM"}


class fe_mesh_desc(ctypes.Structure):
    _fields_ = [("mx", ctypes.c_int), ("my", ctypes.c_int), ("mz", ctypes.c_int),
                ("degree", ctypes.c_int), ("deform_amp", ctypes.c_double),
                ("geom_mode", ctypes.c_int), ("dirichlet", ctypes.c_int), ("device", ctypes.c_int),
                ("layout", ctypes.c_int)]


class fe_layout(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_longlong), ("nodes_per_cell", ctypes.c_longlong),
                ("cellwise_len", ctypes.c_longlong), ("unique_dofs", ctypes.c_longlong),
                ("layout_id", ctypes.c_int)]


class fe_cg_opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("maxit", ctypes.c_int), ("mixed", ctypes.c_int),
                ("flexible", ctypes.c_int), ("inner_rtol", ctypes.c_double),
                ("history", ctypes.c_void_p)]


class fe_cg_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("status", ctypes.c_int)]


class fe_mb_desc(ctypes.Structure):
    _fields_ = [("nblocks", ctypes.c_int), ("nverts", ctypes.c_int), ("degree", ctypes.c_int),
                ("dims", ctypes.POINTER(ctypes.c_int)), ("block_verts", ctypes.POINTER(ctypes.c_int)),
                ("vxyz", ctypes.POINTER(ctypes.c_double)), ("device", ctypes.c_int)]


class fe_amr_desc(ctypes.Structure):
    _fields_ = [("mc", ctypes.c_int), ("lo", ctypes.c_int * 3), ("hi", ctypes.c_int * 3),
                ("degree", ctypes.c_int), ("device", ctypes.c_int)]


class fe_slab_desc(ctypes.Structure):
    _fields_ = [("global_", fe_mesh_desc), ("z0", ctypes.c_int), ("z1", ctypes.c_int)]


# int exchange(void* ctx, int sides, int elem_bytes, long long count, void* stream)
FE_EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_longlong, ctypes.c_void_p)
# int allgather(void* ctx, int n, void* stream)
FE_ALLGATHER_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p)


class fe_comm(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int), ("size", ctypes.c_int), ("send", ctypes.c_void_p * 2),
                ("recv", ctypes.c_void_p * 2), ("red_send", ctypes.c_void_p),
                ("red_all", ctypes.c_void_p), ("exchange", FE_EXCHANGE_FN),
                ("allgather", FE_ALLGATHER_FN), ("ctx", ctypes.c_void_p)]


_vp, _i, _u, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_double
_MESH = ctypes.c_void_p
_SIGS = {
    "fe_mesh_create": [ctypes.POINTER(fe_mesh_desc), _vp, ctypes.POINTER(_MESH)],
    "fe_mesh_destroy": [_MESH],
    "fe_mesh_layout": [_MESH, ctypes.POINTER(fe_layout)],
    "fe_gather": [_MESH, _vp, _vp, _vp],
    "fe_apply": [_MESH, _i, _i, _vp, _vp, _u, _vp],
    "fe_apply_host": [_MESH, _i, ctypes.POINTER(_i), _vp, ctypes.POINTER(_vp), _u, _vp],
    "fe_dss": [_MESH, _i, _vp, _vp, _vp],
    "fe_diag": [_MESH, _i, _vp, _vp],
    "fe_pairing": [_MESH, _i, _vp, _vp, _vp, _vp],
    "fe_pairing_noalloc": [_MESH, _i, _vp, _vp, _vp, _vp],
    "fe_cg_solve": [_MESH, _vp, _vp, ctypes.POINTER(fe_cg_opts), ctypes.POINTER(fe_cg_result), _vp],
    "fe_rhs": [_MESH, _i, _vp, _vp],
    "fe_serve_create": [ctypes.c_size_t, _i, _i, ctypes.POINTER(_vp)],
    "fe_serve_submit": [_vp, ctypes.POINTER(fe_mesh_desc), _vp, ctypes.POINTER(fe_cg_opts),
                        ctypes.POINTER(ctypes.c_longlong)],
    "fe_serve_poll": [_vp, ctypes.c_longlong, ctypes.POINTER(fe_cg_result), _vp],
    "fe_serve_stats": [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                       ctypes.POINTER(ctypes.c_double)],
    "fe_serve_destroy": [_vp],
    "fe_cg_solve_batched": [_i, ctypes.POINTER(_MESH), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                            ctypes.POINTER(fe_cg_opts), ctypes.POINTER(fe_cg_result), _vp],
    "fe_l2_error": [_MESH, _i, _vp, ctypes.POINTER(ctypes.c_double), _vp],
    "fe_mb_create": [ctypes.POINTER(fe_mb_desc), _vp, ctypes.POINTER(_vp)],
    "fe_mb_destroy": [_vp],
    "fe_mb_layout": [_vp, ctypes.POINTER(fe_layout)],
    "fe_mb_info": [_vp, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_i),
                   ctypes.POINTER(_i)],
    "fe_mb_apply": [_vp, _i, _i, _vp, _vp, _u, _vp],
    "fe_mb_dss": [_vp, _i, _vp, _vp, _vp],
    "fe_amr_create": [ctypes.POINTER(fe_amr_desc), _vp, ctypes.POINTER(_vp)],
    "fe_amr_destroy": [_vp],
    "fe_amr_layout": [_vp, ctypes.POINTER(fe_layout)],
    "fe_amr_apply": [_vp, _i, _i, _vp, _vp, _u, _vp],
    "fe_amr_dss": [_vp, _i, _vp, _vp, _vp],
    "fe_slab_create": [ctypes.POINTER(fe_slab_desc), _vp, ctypes.POINTER(_MESH)],
    "fe_slab_plane_len": [_MESH, ctypes.POINTER(ctypes.c_longlong)],
    "fe_slab_face_pack": [_MESH, _i, _vp, _i, _vp, _vp],
    "fe_slab_face_add": [_MESH, _i, _vp, _i, _vp, _vp],
    "fe_slab_dss": [_MESH, _i, _vp, _vp, ctypes.POINTER(fe_comm), _vp],
    "fe_slab_apply": [_MESH, _i, _i, _vp, _vp, _u, ctypes.POINTER(fe_comm), _vp],
    "fe_slab_cg_solve": [_MESH, _vp, _vp, ctypes.POINTER(fe_cg_opts), ctypes.POINTER(fe_comm),
                         ctypes.POINTER(fe_cg_result), _vp],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.fe_last_error.argtypes = []
_lib.fe_last_error.restype = ctypes.c_char_p

EXPORTED = tuple(_SIGS) + ("fe_last_error",)


class FeError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {fe_last_error()}")


def fe_last_error() -> str:
    return _lib.fe_last_error().decode()


def _check(status: int, where: str) -> int:
    if status != FE_OK:
        raise FeError(status, where)
    return status


def _ptr(t) -> int:
    if t is None:
        return None
    return t if isinstance(t, int) else t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


# ---- calls with the C names ---------------------------------------------------------------------
def fe_mesh_create(desc: fe_mesh_desc, stream=None) -> int:
    h = _MESH()
    _check(_lib.fe_mesh_create(ctypes.byref(desc), _stream(stream), ctypes.byref(h)), "fe_mesh_create")
    return h.value


def fe_mesh_destroy(mesh: int) -> None:
    _check(_lib.fe_mesh_destroy(mesh), "fe_mesh_destroy")


def fe_mesh_layout(mesh: int) -> fe_layout:
    out = fe_layout()
    _check(_lib.fe_mesh_layout(mesh, ctypes.byref(out)), "fe_mesh_layout")
    return out


def fe_gather(mesh: int, x_unique_host, x_cell_dev, stream=None) -> None:
    import numpy as np
    xu = np.ascontiguousarray(x_unique_host, dtype=np.float64)
    _check(_lib.fe_gather(mesh, xu.ctypes.data, _ptr(x_cell_dev), _stream(stream)), "fe_gather")


def fe_apply(mesh: int, op: int, prec: int, x, y, flags: int = 0, stream=None) -> None:
    _check(_lib.fe_apply(mesh, op, prec, _ptr(x), _ptr(y), flags, _stream(stream)), "fe_apply")


def fe_apply_host(mesh: int, ops, x_unique_host, y_unique_host, flags: int = 0, stream=None) -> None:
    """ops: sequence of 1 or 2 operators; x_unique_host / y_unique_host: host buffers (numpy arrays,
    pinned torch CPU tensors or raw addresses) of unique_dofs doubles; stream-ordered (see
    include/fe.h)."""
    def addr(b):
        if isinstance(b, int):
            return b
        if hasattr(b, "data_ptr"):
            return b.data_ptr()
        return b.ctypes.data
    n = len(ops)
    o = (_i * max(n, 1))(*ops)
    ys = (_vp * max(len(y_unique_host), 1))(*[addr(y) for y in y_unique_host])
    _check(_lib.fe_apply_host(mesh, n, o, addr(x_unique_host), ys, flags, _stream(stream)),
           "fe_apply_host")


def fe_dss(mesh: int, prec: int, r, z, stream=None) -> None:
    _check(_lib.fe_dss(mesh, prec, _ptr(r), _ptr(z), _stream(stream)), "fe_dss")


def fe_diag(mesh: int, op: int, d, stream=None) -> None:
    _check(_lib.fe_diag(mesh, op, _ptr(d), _stream(stream)), "fe_diag")


def fe_pairing(mesh: int, prec: int, a, b, result_dev, stream=None) -> None:
    _check(_lib.fe_pairing(mesh, prec, _ptr(a), _ptr(b), _ptr(result_dev), _stream(stream)),
           "fe_pairing")


def fe_pairing_noalloc(mesh: int, prec: int, a, b, result_dev, stream=None) -> None:
    """fe_pairing without any device allocation (static scratch; see include/fe.h)."""
    _check(_lib.fe_pairing_noalloc(mesh, prec, _ptr(a), _ptr(b), _ptr(result_dev), _stream(stream)),
           "fe_pairing_noalloc")


def fe_rhs(mesh: int, kind: int, b, stream=None) -> None:
    _check(_lib.fe_rhs(mesh, kind, _ptr(b), _stream(stream)), "fe_rhs")


def fe_l2_error(mesh: int, kind: int, u, stream=None) -> float:
    err = ctypes.c_double(0.0)
    _check(_lib.fe_l2_error(mesh, kind, _ptr(u), ctypes.byref(err), _stream(stream)), "fe_l2_error")
    return err.value


def fe_cg_solve(mesh: int, b, x, opts: fe_cg_opts, stream=None) -> fe_cg_result:
    """Returns the fe_cg_result; FE_ERR_NOT_CONVERGED / FE_ERR_BREAKDOWN are reported in
    ``result.status`` instead of raising."""
    res = fe_cg_result()
    st = _lib.fe_cg_solve(mesh, _ptr(b), _ptr(x), ctypes.byref(opts), ctypes.byref(res),
                          _stream(stream))
    if st not in (FE_OK, FE_ERR_NOT_CONVERGED, FE_ERR_BREAKDOWN):
        raise FeError(st, "fe_cg_solve")
    res.status = st
    return res


def fe_cg_solve_batched(meshes, b, x, opts: fe_cg_opts, stream=None):
    """meshes: list of mesh handles; b, x: lists of device tensors (or pointers).  Returns the list
    of fe_cg_result; non-convergence is reported per problem in result.status."""
    n = len(meshes)
    hs = (_MESH * n)(*meshes)
    bs = (_vp * n)(*[_ptr(v) for v in b])
    xs = (_vp * n)(*[_ptr(v) for v in x])
    res = (fe_cg_result * n)()
    st = _lib.fe_cg_solve_batched(n, hs, bs, xs, ctypes.byref(opts), res, _stream(stream))
    if st not in (FE_OK, FE_ERR_NOT_CONVERGED, FE_ERR_BREAKDOWN):
        raise FeError(st, "fe_cg_solve_batched")
    return list(res)


def fe_serve_create(mem_budget: int, max_slots: int, device: int = 0) -> int:
    h = _vp()
    _check(_lib.fe_serve_create(int(mem_budget), max_slots, device, ctypes.byref(h)), "fe_serve_create")
    return h.value


def fe_serve_submit(server: int, desc: fe_mesh_desc, b_host, opts: fe_cg_opts) -> int:
    import numpy as np
    t = ctypes.c_longlong(0)
    ptr = None
    if b_host is not None:
        b_host = np.ascontiguousarray(b_host, dtype=np.float64)
        ptr = b_host.ctypes.data
    _check(_lib.fe_serve_submit(server, ctypes.byref(desc), ptr, ctypes.byref(opts), ctypes.byref(t)),
           "fe_serve_submit")
    return t.value


def fe_serve_poll(server: int, ticket: int, x_host=None):
    """Returns None while the request is pending, else the fe_cg_result (x copied into the numpy
    array x_host when given)."""
    res = fe_cg_result()
    ptr = None if x_host is None else x_host.ctypes.data
    st = _lib.fe_serve_poll(server, ticket, ctypes.byref(res), ptr)
    if st == FE_ERR_BUSY:
        return None
    _check(st, "fe_serve_poll")
    return res


def fe_serve_stats(server: int):
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.fe_serve_stats(server, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "fe_serve_stats")
    return a.value, b.value, c.value


def fe_serve_destroy(server: int) -> None:
    _check(_lib.fe_serve_destroy(server), "fe_serve_destroy")


# ---- convenience object ---------------------------------------------------------------------------
class Mesh:
    """Owns an ``fe_mesh``; vectors are torch CUDA tensors of ``cellwise_len`` elements."""

    def __init__(self, m, degree: int, deform_amp: float = 0.0, geom_mode: int = FE_GEOM_STORED,
                 dirichlet: bool = False, device: int = 0, stream=None, layout: int = 0):
        mx, my, mz = (m, m, m) if isinstance(m, int) else tuple(m)
        self.desc = fe_mesh_desc(mx, my, mz, degree, deform_amp, geom_mode, int(dirichlet), device,
                                 layout)
        self.handle = fe_mesh_create(self.desc, stream)
        lay = fe_mesh_layout(self.handle)
        self.n_cells, self.nodes_per_cell = lay.n_cells, lay.nodes_per_cell
        self.cellwise_len, self.unique_dofs = lay.cellwise_len, lay.unique_dofs
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            fe_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self, prec: int = FE_F64):
        import torch
        dt = torch.float64 if prec == FE_F64 else torch.float32
        return torch.empty(self.cellwise_len, dtype=dt, device=f"cuda:{self.device}")

    def gather(self, x_unique_host):
        import torch
        out = torch.empty(self.cellwise_len, dtype=torch.float64, device=f"cuda:{self.device}")
        fe_gather(self.handle, x_unique_host, out)
        return out

    def apply(self, x, op=FE_LAPLACE, prec=FE_F64, flags=0, y=None, stream=None):
        y = self.empty(prec) if y is None else y
        fe_apply(self.handle, op, prec, x, y, flags, stream)
        return y

    def dss(self, r, prec=FE_F64, z=None, stream=None):
        z = self.empty(prec) if z is None else z
        fe_dss(self.handle, prec, r, z, stream)
        return z

    def diag(self, op=FE_LAPLACE, stream=None):
        d = self.empty(FE_F64)
        fe_diag(self.handle, op, d, stream)
        return d

    def pairing(self, a, b, prec=FE_F64, stream=None) -> float:
        import torch
        out = torch.empty(1, dtype=torch.float64, device=f"cuda:{self.device}")
        fe_pairing(self.handle, prec, a, b, out, stream)
        return float(out.item())

    def rhs(self, kind=FE_RHS_SINE, stream=None):
        b = self.empty(FE_F64)
        fe_rhs(self.handle, kind, b, stream)
        return b

    def l2_error(self, u, kind=FE_RHS_SINE, stream=None) -> float:
        return fe_l2_error(self.handle, kind, u, stream)

    def cg_solve(self, b, x, rtol=1e-10, maxit=1000, mixed=0, flexible=False, inner_rtol=1e-2,
                 history=False, stream=None):
        """Returns the fe_cg_result, or (result, history[iters, 3]) with history=True."""
        import numpy as np
        hist = np.zeros(3 * maxit) if history else None
        o = fe_cg_opts(rtol, maxit, mixed, int(flexible), inner_rtol,
                       hist.ctypes.data if history else None)
        res = fe_cg_solve(self.handle, b, x, o, stream)
        if history:
            return res, hist.reshape(maxit, 3)[: res.iters]
        return res


# ---- block-structured meshes (Sec. 4.2) ---------------------------------------------------------
def fe_mb_create(desc: fe_mb_desc, stream=None) -> int:
    h = _vp()
    _check(_lib.fe_mb_create(ctypes.byref(desc), _stream(stream), ctypes.byref(h)), "fe_mb_create")
    return h.value


def fe_mb_destroy(mesh: int) -> None:
    _check(_lib.fe_mb_destroy(mesh), "fe_mb_destroy")


def fe_mb_layout(mesh: int) -> fe_layout:
    out = fe_layout()
    _check(_lib.fe_mb_layout(mesh, ctypes.byref(out)), "fe_mb_layout")
    return out


def fe_mb_info(mesh: int):
    f, v, mv = _i(), _i(), _i()
    e = ctypes.c_longlong()
    _check(_lib.fe_mb_info(mesh, ctypes.byref(f), ctypes.byref(e), ctypes.byref(v), ctypes.byref(mv)),
           "fe_mb_info")
    return {"face_pairs": f.value, "edge_entities": e.value, "vertex_entities": v.value,
            "max_valence": mv.value}


def fe_mb_apply(mesh: int, op: int, prec: int, x, y, flags: int = 0, stream=None) -> None:
    _check(_lib.fe_mb_apply(mesh, op, prec, _ptr(x), _ptr(y), flags, _stream(stream)), "fe_mb_apply")


def fe_mb_dss(mesh: int, prec: int, r, z, stream=None) -> None:
    _check(_lib.fe_mb_dss(mesh, prec, _ptr(r), _ptr(z), _stream(stream)), "fe_mb_dss")


class MBMesh:
    """Block-structured mesh handle: vertex coordinates, eight corner vertices per block (local
    corner c = i + 2j + 4k) and the cells per block direction."""

    def __init__(self, vxyz, block_verts, dims, degree: int, device: int = 0, stream=None):
        import numpy as np
        self._v = np.ascontiguousarray(np.asarray(vxyz, dtype=np.float64).reshape(-1, 3))
        self._b = np.ascontiguousarray(np.asarray(block_verts, dtype=np.int32).reshape(-1, 8))
        self._d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(-1, 3))
        desc = fe_mb_desc(len(self._b), len(self._v), degree,
                          self._d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                          self._b.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                          self._v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), device)
        self.handle = fe_mb_create(desc, stream)
        lay = fe_mb_layout(self.handle)
        self.n_cells, self.cellwise_len, self.unique_dofs = lay.n_cells, lay.cellwise_len, lay.unique_dofs
        self.device = device

    def info(self):
        return fe_mb_info(self.handle)

    def empty(self, prec=FE_F64):
        import torch
        dt = torch.float64 if prec == FE_F64 else torch.float32
        return torch.empty(self.cellwise_len, dtype=dt, device=f"cuda:{self.device}")

    def apply(self, x, op=FE_LAPLACE, prec=FE_F64, flags=0, y=None, stream=None):
        y = self.empty(prec) if y is None else y
        fe_mb_apply(self.handle, op, prec, x, y, flags, stream)
        return y

    def dss(self, r, prec=FE_F64, z=None, stream=None):
        z = self.empty(prec) if z is None else z
        fe_mb_dss(self.handle, prec, r, z, stream)
        return z

    def close(self):
        if self.handle:
            fe_mb_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- hanging nodes on a two-level Cartesian refinement (Appendix) ---------------------------------
def fe_amr_create(desc: fe_amr_desc, stream=None) -> int:
    h = _vp()
    _check(_lib.fe_amr_create(ctypes.byref(desc), _stream(stream), ctypes.byref(h)), "fe_amr_create")
    return h.value


def fe_amr_destroy(mesh: int) -> None:
    _check(_lib.fe_amr_destroy(mesh), "fe_amr_destroy")


def fe_amr_layout(mesh: int) -> fe_layout:
    out = fe_layout()
    _check(_lib.fe_amr_layout(mesh, ctypes.byref(out)), "fe_amr_layout")
    return out


def fe_amr_apply(mesh: int, op: int, prec: int, x, y, flags: int = 0, stream=None) -> None:
    _check(_lib.fe_amr_apply(mesh, op, prec, _ptr(x), _ptr(y), flags, _stream(stream)),
           "fe_amr_apply")


def fe_amr_dss(mesh: int, prec: int, r, z, stream=None) -> None:
    _check(_lib.fe_amr_dss(mesh, prec, _ptr(r), _ptr(z), _stream(stream)), "fe_amr_dss")


class AMRMesh:
    """Two-level Cartesian refinement: coarse grid mc^3, cells of the box [lo, hi) refined."""

    def __init__(self, mc: int, lo, hi, degree: int, device: int = 0, stream=None):
        desc = fe_amr_desc(mc, (ctypes.c_int * 3)(*lo), (ctypes.c_int * 3)(*hi), degree, device)
        self.handle = fe_amr_create(desc, stream)
        lay = fe_amr_layout(self.handle)
        self.cellwise_len, self.unique_dofs = lay.cellwise_len, lay.unique_dofs
        self.device = device

    def empty(self, prec=FE_F64):
        import torch
        dt = torch.float64 if prec == FE_F64 else torch.float32
        return torch.empty(self.cellwise_len, dtype=dt, device=f"cuda:{self.device}")

    def apply(self, x, op=FE_LAPLACE, prec=FE_F64, flags=0, y=None, stream=None):
        y = self.empty(prec) if y is None else y
        fe_amr_apply(self.handle, op, prec, x, y, flags, stream)
        return y

    def dss(self, r, prec=FE_F64, z=None, stream=None):
        z = self.empty(prec) if z is None else z
        fe_amr_dss(self.handle, prec, r, z, stream)
        return z

    def close(self):
        if self.handle:
            fe_amr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- slab decomposition (one structured mesh over several slabs) ---------------------------------
def fe_slab_create(desc: fe_slab_desc, stream=None) -> int:
    h = _MESH()
    _check(_lib.fe_slab_create(ctypes.byref(desc), _stream(stream), ctypes.byref(h)), "fe_slab_create")
    return h.value


def fe_slab_plane_len(mesh: int) -> int:
    c = ctypes.c_longlong(0)
    _check(_lib.fe_slab_plane_len(mesh, ctypes.byref(c)), "fe_slab_plane_len")
    return c.value


def fe_slab_face_pack(mesh: int, prec: int, v, side: int, plane, stream=None) -> None:
    _check(_lib.fe_slab_face_pack(mesh, prec, _ptr(v), side, _ptr(plane), _stream(stream)),
           "fe_slab_face_pack")


def fe_slab_face_add(mesh: int, prec: int, v, side: int, plane, stream=None) -> None:
    _check(_lib.fe_slab_face_add(mesh, prec, _ptr(v), side, _ptr(plane), _stream(stream)),
           "fe_slab_face_add")


def fe_slab_dss(mesh: int, prec: int, r, z, comm: fe_comm, stream=None) -> None:
    _check(_lib.fe_slab_dss(mesh, prec, _ptr(r), _ptr(z), ctypes.byref(comm), _stream(stream)),
           "fe_slab_dss")


def fe_slab_apply(mesh: int, op: int, prec: int, x, y, flags: int, comm, stream=None) -> None:
    c = None if comm is None else ctypes.byref(comm)
    _check(_lib.fe_slab_apply(mesh, op, prec, _ptr(x), _ptr(y), flags, c, _stream(stream)),
           "fe_slab_apply")


def fe_slab_cg_solve(mesh: int, b, x, opts: fe_cg_opts, comm: fe_comm, stream=None) -> fe_cg_result:
    """As fe_cg_solve: FE_ERR_NOT_CONVERGED / FE_ERR_BREAKDOWN are reported in result.status."""
    res = fe_cg_result()
    st = _lib.fe_slab_cg_solve(mesh, _ptr(b), _ptr(x), ctypes.byref(opts), ctypes.byref(comm),
                               ctypes.byref(res), _stream(stream))
    if st not in (FE_OK, FE_ERR_NOT_CONVERGED, FE_ERR_BREAKDOWN):
        raise FeError(st, "fe_slab_cg_solve")
    res.status = st
    return res
