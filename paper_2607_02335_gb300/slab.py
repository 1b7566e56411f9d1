"""Slab decomposition of one structured mesh (``fe_slab_*`` in include/fe.h).

The cells of an ``mx x my x mz`` mesh split into slabs of whole z-layers.  Each slab is an
``fe_mesh`` whose kernels do every step of the computation; between slabs the library asks the
caller's communicator, through two callbacks, to move the interface planes (one exchange per DSS)
and the scalars of the solver (one allgather of three values per CG iteration).  This module holds
that plumbing:

* :func:`slab_ranges` -- the z-layers of each slab;
* :class:`DistSlabComm` -- one slab per process over ``torch.distributed`` (NCCL on device buffers,
  ordered on the library's stream; gloo through host staging);
* :class:`ThreadSlabGroup` -- several slabs driven by threads of one process, on one device or
  several, exchanging by device copies between host barriers;
* :class:`Slab` -- a slab handle with the calls of :class:`fe.Mesh` plus the exchanged ones.
"""
from __future__ import annotations

import ctypes
import threading

from . import fe


def slab_ranges(mz: int, nslabs: int):
    """Contiguous z-layer ranges ``[(z0, z1), ...]`` of ``nslabs`` slabs, sizes differing by at most
    one layer (the lower slabs take the extra layers)."""
    if not 1 <= nslabs <= mz:
        raise ValueError(f"cannot split {mz} layers into {nslabs} slabs")
    base, extra = divmod(mz, nslabs)
    out, z = [], 0
    for r in range(nslabs):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


class SlabComm:
    """Buffers and callbacks of one slab's ``fe_comm``.  Subclasses implement
    ``exchange(sides, elem_bytes, count, stream)`` and ``allgather(n, stream)`` with the semantics of
    include/fe.h: ``send[s]`` goes to the neighbour on side ``s`` (0 below, 1 above) and its plane
    arrives in ``recv[s]``; ``red_send[:n]`` of every slab lands in ``red_all[r*n : (r+1)*n]``."""

    def __init__(self, rank: int, size: int, plane_len: int, device):
        import torch
        if not 0 <= rank < size:
            raise ValueError(f"rank {rank} outside [0, {size})")
        self.rank, self.size, self.plane_len = rank, size, int(plane_len)
        self.device = torch.device(device)
        self.has = (rank > 0, rank < size - 1)
        f64 = dict(dtype=torch.float64, device=self.device)
        self.send = [torch.zeros(self.plane_len, **f64) if h else None for h in self.has]
        self.recv = [torch.zeros(self.plane_len, **f64) if h else None for h in self.has]
        self.red_send = torch.zeros(4, **f64)
        self.red_all = torch.zeros(4 * size, **f64)
        self.error = None
        # the callbacks must outlive every library call that holds the struct
        self._xfn = fe.FE_EXCHANGE_FN(self._exchange_cb)
        self._gfn = fe.FE_ALLGATHER_FN(self._allgather_cb)
        c = fe.fe_comm()
        c.rank, c.size = rank, size
        for s in (0, 1):
            c.send[s] = self.send[s].data_ptr() if self.has[s] else None
            c.recv[s] = self.recv[s].data_ptr() if self.has[s] else None
        c.red_send = self.red_send.data_ptr()
        c.red_all = self.red_all.data_ptr()
        c.exchange = self._xfn
        c.allgather = self._gfn
        c.ctx = None
        self.c = c

    @staticmethod
    def _dtype(elem_bytes: int):
        import torch
        if elem_bytes not in (4, 8):
            raise ValueError(f"plane element of {elem_bytes} bytes")
        return torch.float64 if elem_bytes == 8 else torch.float32

    def view(self, buf, elem_bytes: int, count: int):
        """The first ``count`` elements of a plane buffer in the call's element type."""
        return buf.view(self._dtype(elem_bytes))[:count]

    def _stream(self, stream):
        """The library's stream as a torch stream (None / 0: the device's default stream)."""
        import torch
        if stream:
            return torch.cuda.ExternalStream(stream, device=self.device)
        return torch.cuda.default_stream(self.device)

    def _sync(self, stream):
        if self.device.type == "cuda":
            self._stream(stream).synchronize()

    def _exchange_cb(self, ctx, sides, elem_bytes, count, stream):
        try:
            self.exchange(sides, elem_bytes, count, stream)
            return 0
        except BaseException as e:  # noqa: BLE001 -- reported through FE_ERR_COMM
            self.error = e
            return 1

    def _allgather_cb(self, ctx, n, stream):
        try:
            self.allgather(n, stream)
            return 0
        except BaseException as e:  # noqa: BLE001
            self.error = e
            return 1

    def exchange(self, sides, elem_bytes, count, stream):
        raise NotImplementedError

    def allgather(self, n, stream):
        raise NotImplementedError


class DistSlabComm(SlabComm):
    """One slab per process of a ``torch.distributed`` group; slab ``r`` is the group's rank ``r``.
    With the NCCL backend and device buffers the transfers are issued on the library's stream; any
    other backend stages the buffers through host memory after synchronizing that stream."""

    def __init__(self, plane_len: int, device, group=None):
        import torch.distributed as dist
        self.group = group
        super().__init__(dist.get_rank(group), dist.get_world_size(group), plane_len, device)
        self.nccl = dist.get_backend(group) == "nccl" and self.device.type == "cuda"

    def _peer(self, side: int) -> int:
        import torch.distributed as dist
        r = self.rank - 1 if side == 0 else self.rank + 1
        return r if self.group is None else dist.get_global_rank(self.group, r)

    def exchange(self, sides, elem_bytes, count, stream):
        import torch
        import torch.distributed as dist
        todo = [s for s in (0, 1) if (sides >> s) & 1]
        if self.nccl:
            with torch.cuda.stream(self._stream(stream)):
                ops = []
                for s in todo:
                    ops.append(dist.P2POp(dist.isend, self.view(self.send[s], elem_bytes, count),
                                          self._peer(s), self.group))
                    ops.append(dist.P2POp(dist.irecv, self.view(self.recv[s], elem_bytes, count),
                                          self._peer(s), self.group))
                for req in dist.batch_isend_irecv(ops):
                    req.wait()
            return
        self._sync(stream)
        out = {s: self.view(self.send[s], elem_bytes, count).cpu() for s in todo}
        inc = {s: torch.empty(count, dtype=self._dtype(elem_bytes)) for s in todo}
        reqs = []
        for s in todo:
            reqs.append(dist.isend(out[s], self._peer(s), self.group))
            reqs.append(dist.irecv(inc[s], self._peer(s), self.group))
        for req in reqs:
            req.wait()
        for s in todo:
            self.view(self.recv[s], elem_bytes, count).copy_(inc[s])

    def allgather(self, n, stream):
        import torch
        import torch.distributed as dist
        if self.nccl:
            with torch.cuda.stream(self._stream(stream)):
                dist.all_gather_into_tensor(self.red_all[: self.size * n], self.red_send[:n],
                                            group=self.group)
            return
        self._sync(stream)
        mine = self.red_send[:n].cpu()
        parts = [torch.empty(n, dtype=torch.float64) for _ in range(self.size)]
        dist.all_gather(parts, mine, group=self.group)
        self.red_all[: self.size * n].copy_(torch.cat(parts))


class ThreadSlabGroup:
    """Slabs driven by threads of one process.  Every callback waits (at most ``timeout`` seconds)
    at a barrier until all slabs have enqueued and finished their packing, copies the neighbours'
    planes with device copies, and waits again before any slab may refill its send buffers.  Only
    the host waits: no kernel waits for another slab."""

    def __init__(self, size: int, timeout: float = 120.0):
        self.size = size
        self.barrier = threading.Barrier(size, timeout=timeout)
        self.comms = [None] * size

    def comm(self, rank: int, plane_len: int, device) -> "ThreadSlabComm":
        c = ThreadSlabComm(self, rank, plane_len, device)
        self.comms[rank] = c
        return c


class ThreadSlabComm(SlabComm):
    def __init__(self, group: ThreadSlabGroup, rank: int, plane_len: int, device):
        self.group = group
        super().__init__(rank, group.size, plane_len, device)

    def _copy_done(self):
        import torch
        if self.device.type == "cuda":
            torch.cuda.current_stream(self.device).synchronize()

    def exchange(self, sides, elem_bytes, count, stream):
        self._sync(stream)
        self.group.barrier.wait()
        try:
            for s in (0, 1):
                if (sides >> s) & 1:
                    peer = self.group.comms[self.rank - 1 if s == 0 else self.rank + 1]
                    self.view(self.recv[s], elem_bytes, count).copy_(
                        self.view(peer.send[1 - s], elem_bytes, count))
            self._copy_done()
        finally:
            self.group.barrier.wait()

    def allgather(self, n, stream):
        self._sync(stream)
        self.group.barrier.wait()
        try:
            for r, peer in enumerate(self.group.comms):
                self.red_all[r * n:(r + 1) * n].copy_(peer.red_send[:n])
            self._copy_done()
        finally:
            self.group.barrier.wait()


class Slab(fe.Mesh):
    """Slab ``[z0, z1)`` of the ``mx x my x mz`` mesh; vectors are torch CUDA tensors of
    ``cellwise_len`` elements, the slab's contiguous part of the whole mesh's vectors."""

    def __init__(self, m, degree: int, z0: int, z1: int, deform_amp: float = 0.0,
                 geom_mode: int = fe.FE_GEOM_STORED, dirichlet: bool = False, device: int = 0,
                 stream=None):
        mx, my, mz = (m, m, m) if isinstance(m, int) else tuple(m)
        whole = fe.fe_mesh_desc(mx, my, mz, degree, deform_amp, geom_mode, int(dirichlet), device, 0)
        self.desc = fe.fe_slab_desc(whole, z0, z1)
        self.handle = fe.fe_slab_create(self.desc, stream)
        lay = fe.fe_mesh_layout(self.handle)
        self.n_cells, self.nodes_per_cell = lay.n_cells, lay.nodes_per_cell
        self.cellwise_len, self.unique_dofs = lay.cellwise_len, lay.unique_dofs
        self.device = device
        self.z0, self.z1 = z0, z1
        self.plane_len = fe.fe_slab_plane_len(self.handle)

    def apply(self, x, op=fe.FE_LAPLACE, prec=fe.FE_F64, flags=0, y=None, stream=None, comm=None):
        y = self.empty(prec) if y is None else y
        fe.fe_slab_apply(self.handle, op, prec, x, y, flags, None if comm is None else comm.c, stream)
        return y

    def dss(self, r, prec=fe.FE_F64, z=None, stream=None, comm=None):
        if comm is None:
            raise ValueError("Slab.dss needs the slab's communicator")
        z = self.empty(prec) if z is None else z
        fe.fe_slab_dss(self.handle, prec, r, z, comm.c, stream)
        return z

    def face_pack(self, v, side: int, plane, prec=fe.FE_F64, stream=None):
        fe.fe_slab_face_pack(self.handle, prec, v, side, plane, stream)

    def face_add(self, v, side: int, plane, prec=fe.FE_F64, stream=None):
        fe.fe_slab_face_add(self.handle, prec, v, side, plane, stream)

    def cg_solve(self, b, x, comm=None, rtol=1e-10, maxit=1000, history=False, stream=None, **kw):
        """Jacobi PCG over all slabs (every slab calls it with its own comm).  Returns the
        fe_cg_result, or (result, history[iters, 3]) with history=True."""
        import numpy as np
        if comm is None:
            raise ValueError("Slab.cg_solve needs the slab's communicator")
        if kw.get("mixed", 0) or kw.get("flexible", False):
            raise ValueError("slab solves are FP64 PCG only")
        hist = np.zeros(3 * maxit) if history else None
        o = fe.fe_cg_opts(rtol, maxit, 0, 0, 0.0, hist.ctypes.data if history else None)
        res = fe.fe_slab_cg_solve(self.handle, b, x, o, comm.c, stream)
        if comm.error is not None:
            raise RuntimeError(f"slab communicator failed: {comm.error!r}")
        if history:
            return res, hist.reshape(maxit, 3)[: res.iters]
        return res
