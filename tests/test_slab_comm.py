"""Host logic of the slab decomposition on CPU ranks (gloo processes): the layer split, the
interface-plane exchange and the scalar allgather of ``DistSlabComm``.  Each rank plays its slab
with the oracle standing in for the device kernels: the structured DSS inside the slab, then the
planes packed in the order include/fe.h specifies, exchanged, and added.  The result must be the
whole mesh's DSS restricted to the slab."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

import oracle  # noqa: E402

MX, MY, P = 3, 2, 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _layer_view(v, mzl, n):
    # cell-wise vector -> [cz][cy][cx][k][j][i]
    return v.reshape(mzl, MY, MX, n, n, n)


def _pack(v, mzl, n, side):
    """Plane of `side` in the documented order: entry ((cy mx + cx) n + j) n + i."""
    layer, k = (0, 0) if side == 0 else (mzl - 1, n - 1)
    return np.ascontiguousarray(_layer_view(v, mzl, n)[layer, :, :, k, :, :]).reshape(-1)


def _add(v, mzl, n, side, plane):
    layer, k = (0, 0) if side == 0 else (mzl - 1, n - 1)
    _layer_view(v, mzl, n)[layer, :, :, k, :, :] += plane.reshape(MY, MX, n, n)


def _worker(rank, world, port, mz, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2607_02335_gb300.slab import DistSlabComm, slab_ranges
        n = P + 1
        n3 = n ** 3
        z0, z1 = slab_ranges(mz, world)[rank]
        mzl = z1 - z0
        whole = oracle.Mesh((MX, MY, mz), P)
        rng = np.random.default_rng(7)  # the same dual vector on every rank
        y = rng.standard_normal(whole.n_cellwise)
        expect = oracle.dss(whole, y)[z0 * MX * MY * n3:z1 * MX * MY * n3]
        mine = y[z0 * MX * MY * n3:z1 * MX * MY * n3].copy()
        local = oracle.dss(oracle.Mesh((MX, MY, mzl), P), mine)

        plane_len = MX * MY * n * n
        comm = DistSlabComm(plane_len, "cpu")
        sides = (1 if rank > 0 else 0) | (2 if rank < world - 1 else 0)
        # FP64 planes
        for s in (0, 1):
            if (sides >> s) & 1:
                comm.send[s].copy_(torch.from_numpy(_pack(local, mzl, n, s)))
        comm.exchange(sides, 8, plane_len, None)
        got = local.copy()
        for s in (0, 1):
            if (sides >> s) & 1:
                _add(got, mzl, n, s, comm.recv[s].numpy())
        err64 = float(np.max(np.abs(got - expect)) / np.max(np.abs(expect)))
        # FP32 planes in the same buffers
        local32 = local.astype(np.float32)
        for s in (0, 1):
            if (sides >> s) & 1:
                comm.view(comm.send[s], 4, plane_len).copy_(
                    torch.from_numpy(_pack(local32, mzl, n, s)))
        comm.exchange(sides, 4, plane_len, None)
        got32 = local32.copy()
        for s in (0, 1):
            if (sides >> s) & 1:
                _add(got32, mzl, n, s, comm.view(comm.recv[s], 4, plane_len).numpy())
        err32 = float(np.max(np.abs(got32 - expect)) / np.max(np.abs(expect)))
        # allgather of three scalars, in rank order
        comm.red_send[:3] = torch.tensor([rank + 0.5, -rank, 10.0 * rank], dtype=torch.float64)
        comm.allgather(3, None)
        gathered = comm.red_all[:3 * world].tolist()
        out[rank] = (err64, err32, gathered, sides)
    finally:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


@pytest.mark.parametrize("world,mz", [(2, 3), (3, 5), (4, 4)])
def test_plane_exchange_completes_the_whole_mesh_dss(world, mz):
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, mz, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        res = dict(out)
    want = [v for r in range(world) for v in (r + 0.5, -r, 10.0 * r)]
    for r in range(world):
        err64, err32, gathered, sides = res[r]
        assert err64 <= 1e-14, (r, err64)
        assert err32 <= 1e-6, (r, err32)
        assert gathered == want
        assert sides == (1 if r > 0 else 0) | (2 if r < world - 1 else 0)


def test_slab_ranges():
    from paper_2607_02335_gb300.slab import slab_ranges
    assert slab_ranges(7, 3) == [(0, 3), (3, 5), (5, 7)]
    assert slab_ranges(4, 4) == [(0, 1), (1, 2), (2, 3), (3, 4)]
    assert slab_ranges(5, 1) == [(0, 5)]
    for mz in range(1, 12):
        for k in range(1, mz + 1):
            r = slab_ranges(mz, k)
            assert r[0][0] == 0 and r[-1][1] == mz
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [z1 - z0 for z0, z1 in r]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slab_ranges(3, 4)
    with pytest.raises(ValueError):
        slab_ranges(3, 0)


def test_invalid_slab_descriptors_rejected_on_host():
    import ctypes
    from paper_2607_02335_gb300 import fe
    whole = fe.fe_mesh_desc(2, 2, 4, 2, 0.0, 0, 0, 0, 0)
    for z0, z1 in ((-1, 2), (2, 2), (3, 2), (0, 5), (0, 0)):
        h = ctypes.c_void_p()
        st = fe._lib.fe_slab_create(ctypes.byref(fe.fe_slab_desc(whole, z0, z1)), None,
                                    ctypes.byref(h))
        assert st == fe.FE_ERR_INVALID and h.value is None, (z0, z1)
        assert fe.fe_last_error()
    packed = fe.fe_mesh_desc(2, 2, 4, 2, 0.0, 0, 0, 0, fe.FE_LAYOUT_PACKED2)
    h = ctypes.c_void_p()
    assert fe._lib.fe_slab_create(ctypes.byref(fe.fe_slab_desc(packed, 0, 2)), None,
                                  ctypes.byref(h)) == fe.FE_ERR_INVALID
    assert fe._lib.fe_slab_create(None, None, None) == fe.FE_ERR_INVALID
    assert fe._lib.fe_slab_dss(None, 0, None, None, None, None) == fe.FE_ERR_INVALID
    assert fe._lib.fe_slab_cg_solve(None, None, None, None, None, None, None) == fe.FE_ERR_INVALID
    assert fe._lib.fe_slab_plane_len(None, None) == fe.FE_ERR_INVALID


def test_single_reduction_recurrence_equals_the_two_reduction_pcg():
    """The slab solver's recurrence (z = P r, s = A z; gamma = <r,z>, delta = <s,z>; beta =
    gamma/gamma_old, alpha = gamma/(delta - beta gamma/alpha_old); p = z + beta p, q = s + beta q)
    written out on the oracle's assembled Jacobi-PCG system: its alpha_k and beta_k are the
    oracle's two-reduction PCG's (equal in exact arithmetic)."""
    import scipy.sparse as sp
    m, p = (4, 3, 5), 3
    om = oracle.Mesh(m, p, amp=0.1, dirichlet=True)
    rowptr, col, val = oracle.assemble_csr(om, oracle.LAPLACE)
    A = sp.csr_matrix((val, col, rowptr))
    free = ~oracle.boundary_global(om)
    R = sp.diags(free.astype(float))
    A = R @ A @ R
    d = np.where(free, oracle.diag_global(om, oracle.LAPLACE), 1.0)
    rng = np.random.default_rng(11)
    b = rng.standard_normal(A.shape[0]) * free
    ref = oracle.cg(om, oracle.LAPLACE, b, rtol=1e-12, maxit=400)
    x = np.zeros_like(b)
    r = b.copy()
    pv = np.zeros_like(b)
    q = np.zeros_like(b)
    alphas, betas = [], []
    z = r * free / d
    s = A @ z
    gamma, delta = r @ z, s @ z
    alpha, beta = gamma / delta, 0.0
    for k in range(30):
        pv = z + beta * pv
        q = s + beta * q
        x += alpha * pv
        r -= alpha * q
        alphas.append(alpha)
        z = r * free / d
        s = A @ z
        g_new, delta = r @ z, s @ z
        beta = g_new / gamma
        betas.append(beta)
        alpha = g_new / (delta - beta * g_new / alpha)
        gamma = g_new
    k = 25
    assert np.allclose(alphas[:k], ref["alpha"][:k], rtol=1e-9, atol=0)
    assert np.allclose(betas[:k - 1], ref["beta"][:k - 1], rtol=1e-8, atol=0)
