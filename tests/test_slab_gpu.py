"""Slab decomposition on one GPU.  The slabs of one mesh run as threads of this process (each on
its own stream; only the host waits at the exchange barriers, no kernel waits for another slab) or
are exchanged by hand with the plane entry points.  Checks: a slab's unassembled apply, geometry
and manufactured data are bitwise those of the whole mesh; the DSS completed by one plane exchange
is the whole mesh's DSS; the slab PCG follows the oracle's assembled Jacobi-PCG (the iterates of the
single-reduction recurrence equal those of the two-reduction one in exact arithmetic) with one
plane exchange and one allgather per iteration."""
import threading

import numpy as np
import pytest

import oracle as O
from paper_2607_02335_gb300 import synth as S
from tests.helpers import oracle_mesh, rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    from paper_2607_02335_gb300 import fe as F
    return F


@pytest.fixture(scope="module")
def sl():
    from paper_2607_02335_gb300 import slab as M
    return M


def cells(m, p, z0, z1):
    mx, my, _ = m
    n3 = (p + 1) ** 3
    return slice(z0 * mx * my * n3, z1 * mx * my * n3)


def continuous(fe_mesh, m, p, seed, dirichlet=False):
    return fe_mesh.gather(S.primal_unique(m, p, seed=seed, dirichlet=dirichlet))


def run_slabs(n, fn, timeout=300):
    """fn(rank) in one thread per slab, each on its own CUDA stream; returns the results."""
    out, errs = [None] * n, [None] * n

    def body(r):
        try:
            torch.cuda.set_device(0)
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                out[r] = fn(r)
            st.synchronize()
        except BaseException as e:  # noqa: BLE001
            errs[r] = e

    th = [threading.Thread(target=body, args=(r,)) for r in range(n)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout)
        assert not t.is_alive()
    for e in errs:
        if e is not None:
            raise e
    torch.cuda.synchronize()
    return out


class CountingGroup:
    """ThreadSlabGroup whose communicators count their callbacks."""

    def __init__(self, sl, n):
        self.g = sl.ThreadSlabGroup(n)
        self.calls = [[0, 0] for _ in range(n)]
        base = sl.ThreadSlabComm
        calls = self.calls

        class Comm(base):
            def exchange(self, *a):
                calls[self.rank][0] += 1
                return super().exchange(*a)

            def allgather(self, *a):
                calls[self.rank][1] += 1
                return super().allgather(*a)

        self.Comm = Comm

    def comm(self, rank, plane_len):
        c = self.Comm(self.g, rank, plane_len, "cuda:0")
        self.g.comms[rank] = c
        return c


@pytest.mark.parametrize("geom,op,p", [(0, 0, 3), (0, 1, 2), (1, 0, 3), (2, 0, 4), (0, 0, 7)])
def test_unassembled_apply_and_data_bitwise(fe, sl, geom, op, p):
    m = (5, 3, 7)
    amp = 0.0 if geom == fe.FE_GEOM_AFFINE else 0.1
    whole = fe.Mesh(m, p, deform_amp=amp, geom_mode=geom, dirichlet=True)
    x = continuous(whole, m, p, seed=3)
    y = whole.apply(x, op=op)
    b = whole.rhs() if geom != fe.FE_GEOM_AFFINE else None
    for z0, z1 in sl.slab_ranges(m[2], 3):
        s = sl.Slab(m, p, z0, z1, deform_amp=amp, geom_mode=geom, dirichlet=True)
        assert s.cellwise_len == cells(m, p, z0, z1).stop - cells(m, p, z0, z1).start
        assert s.unique_dofs == (m[0] * p + 1) * (m[1] * p + 1) * ((z1 - z0) * p + 1)
        assert s.plane_len == m[0] * m[1] * (p + 1) ** 2
        ys = s.apply(x[cells(m, p, z0, z1)].clone(), op=op)
        torch.cuda.synchronize()
        assert torch.equal(ys, y[cells(m, p, z0, z1)])
        if b is not None:
            assert torch.equal(s.rhs(), b[cells(m, p, z0, z1)])


@pytest.mark.parametrize("prec", [0, 1])
def test_dss_completed_by_plane_exchange(fe, sl, prec):
    m, p, nslabs = (4, 3, 7), 3, 3
    dt = torch.float64 if prec == fe.FE_F64 else torch.float32
    whole = fe.Mesh(m, p)
    r = torch.from_numpy(S.dual_cellwise(m, p, seed=5)).cuda().to(dt)
    z = whole.dss(r, prec=prec)
    slabs = [sl.Slab(m, p, z0, z1) for z0, z1 in sl.slab_ranges(m[2], nslabs)]
    loc, planes = [], []
    for s in slabs:
        zs = torch.empty(s.cellwise_len, dtype=dt, device="cuda")
        fe.fe_dss(s.handle, prec, r[cells(m, p, s.z0, s.z1)].clone(), zs)
        pl = [torch.empty(s.plane_len, dtype=dt, device="cuda") for _ in range(2)]
        for side in (0, 1):
            s.face_pack(zs, side, pl[side], prec=prec)
        loc.append(zs)
        planes.append(pl)
    for i in range(nslabs - 1):  # interface between slab i (its top) and slab i+1 (its bottom)
        slabs[i].face_add(loc[i], 1, planes[i + 1][0], prec=prec)
        slabs[i + 1].face_add(loc[i + 1], 0, planes[i][1], prec=prec)
    torch.cuda.synchronize()
    got = torch.cat(loc)
    # the planes are added after all passes here: the same pairs, summed in another order
    tol = 1e-15 if prec == fe.FE_F64 else 1e-6
    assert rel_max_err(got.double().cpu().numpy(), z.double().cpu().numpy()) <= tol
    if prec == fe.FE_F64:
        om = oracle_mesh(m, p)
        assert rel_max_err(got.cpu().numpy(), O.dss(om, r.cpu().numpy())) <= 1e-14


@pytest.mark.parametrize("prec,nslabs", [(0, 2), (0, 4), (1, 3)])
def test_slab_dss_is_bitwise_the_whole_mesh_dss(fe, sl, prec, nslabs):
    m, p = (5, 3, 8), 3
    dt = torch.float64 if prec == fe.FE_F64 else torch.float32
    whole = fe.Mesh(m, p)
    r = torch.from_numpy(S.dual_cellwise(m, p, seed=6)).cuda().to(dt)
    z = whole.dss(r, prec=prec)
    ranges = sl.slab_ranges(m[2], nslabs)
    slabs = [sl.Slab(m, p, z0, z1) for z0, z1 in ranges]
    grp = CountingGroup(sl, nslabs)
    comms = [grp.comm(k, slabs[k].plane_len) for k in range(nslabs)]
    rs = [r[cells(m, p, z0, z1)].clone() for z0, z1 in ranges]
    torch.cuda.synchronize()
    zs = run_slabs(nslabs, lambda k: slabs[k].dss(rs[k], prec=prec, comm=comms[k]))
    assert torch.equal(torch.cat(zs), z)  # per node the same pair sums in the same order
    assert all(c == [1, 0] for c in grp.calls)


@pytest.mark.parametrize("p,prec", [(2, 0), (3, 1), (5, 0)])
def test_assembled_apply_over_thread_slabs(fe, sl, p, prec):
    m, nslabs = (5, 4, 6), 3
    dt = torch.float64 if prec == fe.FE_F64 else torch.float32
    whole = fe.Mesh(m, p, deform_amp=0.1, dirichlet=True)
    x = continuous(whole, m, p, seed=9, dirichlet=True).to(dt)
    y = whole.apply(x, prec=prec, flags=fe.FE_ASSEMBLE)
    ranges = sl.slab_ranges(m[2], nslabs)
    slabs = [sl.Slab(m, p, z0, z1, deform_amp=0.1, dirichlet=True) for z0, z1 in ranges]
    grp = CountingGroup(sl, nslabs)
    comms = [grp.comm(r, slabs[r].plane_len) for r in range(nslabs)]
    xs = [x[cells(m, p, z0, z1)].clone() for z0, z1 in ranges]
    torch.cuda.synchronize()
    ys = run_slabs(nslabs, lambda r: slabs[r].apply(xs[r], prec=prec, flags=fe.FE_ASSEMBLE,
                                                     comm=comms[r]))
    got = torch.cat(ys)
    assert torch.equal(got, y)  # brick-fused (p <= 3) and unfused alike
    assert all(c == [1, 0] for c in grp.calls)
    if prec == fe.FE_F64:
        om = oracle_mesh(m, p, amp=0.1, dirichlet=True)
        xg = S.primal_unique(m, p, seed=9, dirichlet=True)
        ref = O.gather(om, O.apply_assembled(om, O.LAPLACE, xg))
        assert rel_max_err(got.cpu().numpy(), ref) <= 1e-12


def _unique_from_cellwise(om, xc):
    gidx = O.gather(om, np.arange(om.n_unique, dtype=np.float64)).astype(np.int64)
    xg = np.zeros(om.n_unique)
    xg[gidx] = xc
    return xg, gidx


@pytest.mark.parametrize("nslabs", [1, 2, 3])
def test_slab_pcg_follows_the_assembled_pcg(fe, sl, nslabs):
    m, p = (4, 3, 6), 3
    om = oracle_mesh(m, p, amp=0.1, dirichlet=True)
    bc = S.dual_cellwise(m, p, seed=21)
    ref = O.cg(om, O.LAPLACE, O.scatter(om, bc), rtol=1e-12, maxit=500)
    assert ref["status"] == 0
    ranges = sl.slab_ranges(m[2], nslabs)
    slabs = [sl.Slab(m, p, z0, z1, deform_amp=0.1, dirichlet=True) for z0, z1 in ranges]
    grp = CountingGroup(sl, nslabs)
    comms = [grp.comm(r, slabs[r].plane_len) for r in range(nslabs)]
    bs = [torch.from_numpy(bc[cells(m, p, z0, z1)].copy()).cuda() for z0, z1 in ranges]
    xs = [torch.zeros(s.cellwise_len, dtype=torch.float64, device="cuda") for s in slabs]
    torch.cuda.synchronize()
    out = run_slabs(nslabs, lambda r: slabs[r].cg_solve(bs[r], xs[r], comm=comms[r], rtol=1e-12,
                                                         maxit=500, history=True))
    res = [o[0] for o in out]
    hist = out[0][1]
    assert all(r_.status == fe.FE_OK for r_ in res)
    assert len({r_.iters for r_ in res}) == 1 and len({r_.rel_res for r_ in res}) == 1
    for o in out[1:]:
        assert np.array_equal(o[1], hist)  # every slab took the same scalars
    assert abs(res[0].iters - ref["iters"]) <= 1
    k = 25
    assert np.allclose(hist[:k, 0], ref["alpha"][:k], rtol=1e-8, atol=0)
    assert np.allclose(hist[:k - 1, 1], ref["beta"][:k - 1], rtol=1e-7, atol=0)
    assert np.allclose(hist[:k, 2], ref["relres"][1:k + 1], rtol=1e-8, atol=0)
    # the solution is continuous across the slab interfaces and solves the assembled system
    xc = torch.cat(xs).cpu().numpy()
    xg, gidx = _unique_from_cellwise(om, xc)
    assert np.array_equal(xc, xg[gidx])
    assert rel_max_err(xg, ref["x"]) <= 1e-9
    # one plane exchange and one allgather per iteration (plus the set-up ones: the diagonal's
    # exchange, and the allgather of the largest |b| that scales the system)
    for r, (nx, ng) in enumerate(grp.calls):
        if nslabs == 1:
            assert (nx, ng) == (0, 0)
        else:
            assert nx == ng
            assert 0 <= ng - 3 - res[r].iters <= 3  # flag read every 4 iterations


def test_slab_pcg_manufactured_solution(fe, sl):
    m, p, nslabs = (6, 6, 8), 4, 4
    whole = fe.Mesh(m, p, deform_amp=0.1, dirichlet=True)
    xw = torch.zeros(whole.cellwise_len, dtype=torch.float64, device="cuda")
    rw = whole.cg_solve(whole.rhs(), xw, rtol=1e-10, maxit=2000)
    assert rw.status == fe.FE_OK
    ranges = sl.slab_ranges(m[2], nslabs)
    slabs = [sl.Slab(m, p, z0, z1, deform_amp=0.1, dirichlet=True) for z0, z1 in ranges]
    g = sl.ThreadSlabGroup(nslabs)
    comms = [g.comm(r, slabs[r].plane_len, "cuda:0") for r in range(nslabs)]
    xs = [torch.zeros(s.cellwise_len, dtype=torch.float64, device="cuda") for s in slabs]
    res = run_slabs(nslabs, lambda r: slabs[r].cg_solve(slabs[r].rhs(), xs[r], comm=comms[r],
                                                        rtol=1e-10, maxit=2000))
    assert all(r_.status == fe.FE_OK for r_ in res)
    assert abs(res[0].iters - rw.iters) <= 2
    xc = torch.cat(xs)
    assert rel_max_err(xc.cpu().numpy(), xw.cpu().numpy()) <= 1e-8
    e2 = sum(s.l2_error(x) ** 2 for s, x in zip(slabs, xs)) ** 0.5
    assert e2 == pytest.approx(whole.l2_error(xw), rel=1e-6)


@pytest.mark.parametrize("scale", [1e-300, 1e30])
def test_slab_pcg_badly_scaled_rhs(fe, sl, scale):
    """Right-hand sides far from unit size solve like the unscaled one: the system is scaled by an
    exact power of two taken from the largest |b| over all slabs."""
    m, p, nslabs = (4, 4, 6), 2, 2
    ranges = sl.slab_ranges(m[2], nslabs)
    slabs = [sl.Slab(m, p, z0, z1, deform_amp=0.1, dirichlet=True) for z0, z1 in ranges]
    g = sl.ThreadSlabGroup(nslabs)
    comms = [g.comm(r, slabs[r].plane_len, "cuda:0") for r in range(nslabs)]
    sols = {}
    for sc in (1.0, scale):
        xs = [torch.zeros(s.cellwise_len, dtype=torch.float64, device="cuda") for s in slabs]
        res = run_slabs(nslabs, lambda r: slabs[r].cg_solve(slabs[r].rhs() * sc, xs[r],
                                                            comm=comms[r], rtol=1e-10, maxit=500))
        assert all(r_.status == fe.FE_OK and r_.iters > 0 for r_ in res), (sc, res[0].iters)
        sols[sc] = torch.cat(xs).cpu().numpy() / sc
    assert rel_max_err(sols[scale], sols[1.0]) <= 1e-8


def test_slab_errors(fe, sl):
    m, p = (3, 3, 4), 2
    s0, s1 = sl.Slab(m, p, 0, 2), sl.Slab(m, p, 2, 4)
    x = torch.zeros(s0.cellwise_len, dtype=torch.float64, device="cuda")
    # the whole-mesh solvers refuse slabs
    with pytest.raises(fe.FeError) as e:
        fe.Mesh.cg_solve(s0, x, x.clone())
    assert e.value.status == fe.FE_ERR_INVALID
    g = sl.ThreadSlabGroup(2)
    c0, c1 = g.comm(0, s0.plane_len, "cuda:0"), g.comm(1, s1.plane_len, "cuda:0")
    # a communicator whose rank does not match the slab
    with pytest.raises(fe.FeError) as e:
        s0.apply(x, flags=fe.FE_ASSEMBLE, comm=c1)
    assert e.value.status == fe.FE_ERR_INVALID

    class Failing(sl.ThreadSlabComm):
        def exchange(self, *a):
            raise RuntimeError("link down")

    f0 = Failing(g, 0, s0.plane_len, "cuda:0")
    with pytest.raises(fe.FeError) as e:
        s0.apply(x, flags=fe.FE_ASSEMBLE, comm=f0)
    assert e.value.status == fe.FE_ERR_COMM
    assert isinstance(f0.error, RuntimeError)
    assert c0.error is None
