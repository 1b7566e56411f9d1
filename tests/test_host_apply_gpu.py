"""fe_apply_host: the assembled operator on host vectors in unique-node form, y = G^T A_D G x.
Against the oracle's assembled apply (which works on unique-node vectors directly), against the
device path (fe_apply with FE_ASSEMBLE, one copy per node picked on the host) bit for bit, and a
closed form on a large affine mesh."""
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


def owner_copies(m, p):
    """Cell-wise index of one copy of every unique node (lexicographic node order)."""
    mx, my, mz = m
    n = p + 1
    Nx, Ny, Nz = mx * p + 1, my * p + 1, mz * p + 1
    g = np.arange(Nx * Ny * Nz)
    gx, gy, gz = g % Nx, (g // Nx) % Ny, g // (Nx * Ny)
    cx, cy, cz = np.minimum(gx // p, mx - 1), np.minimum(gy // p, my - 1), np.minimum(gz // p, mz - 1)
    i, j, k = gx - cx * p, gy - cy * p, gz - cz * p
    return ((cz * my + cy) * mx + cx) * n ** 3 + (k * n + j) * n + i


@pytest.mark.parametrize("m,p,dirichlet,geom", [((5, 4, 3), 1, False, 0), ((4, 3, 5), 3, True, 0),
                                                ((3, 2, 2), 7, False, 0), ((6, 5, 4), 2, True, 0),
                                                ((4, 3, 5), 3, True, 1), ((3, 3, 3), 5, False, 1)])
def test_host_apply_matches_oracle_and_device_path(fe, m, p, dirichlet, geom):
    gm = fe.Mesh(m, p, deform_amp=0.1, dirichlet=dirichlet, geom_mode=geom)
    om = oracle_mesh(m, p, amp=0.1, dirichlet=dirichlet)
    xu = S.primal_unique(m, p, seed=4)
    ys = [np.empty(gm.unique_dofs), np.empty(gm.unique_dofs)]
    fe.fe_apply_host(gm.handle, [fe.FE_LAPLACE, fe.FE_MASS], xu, ys)
    torch.cuda.synchronize()
    own = owner_copies(m, p)
    xc = gm.gather(xu)
    for op, y in zip((fe.FE_LAPLACE, fe.FE_MASS), ys):
        ref = O.apply_assembled(om, op, xu)
        assert rel_max_err(y, ref) <= 1e-12
        dev = gm.apply(xc, op=op, flags=fe.FE_ASSEMBLE).cpu().numpy()
        assert np.array_equal(y, dev[own])
    # one operator per call gives the same bits as two
    y1 = np.empty(gm.unique_dofs)
    fe.fe_apply_host(gm.handle, [fe.FE_MASS], xu, [y1])
    torch.cuda.synchronize()
    assert np.array_equal(y1, ys[1])


@pytest.mark.parametrize("chunks", [2, 3, 7])
@pytest.mark.parametrize("m,p,dirichlet", [((5, 3, 7), 2, True), ((4, 4, 9), 3, False),
                                           ((3, 3, 7), 7, True), ((5, 5, 8), 1, False)])
def test_chunked_host_apply_is_bitwise_the_device_path(fe, monkeypatch, chunks, m, p, dirichlet):
    """z-chunks forced through FE_HOST_CHUNKS: per chunk the apply, its z-pass and the one across the
    chunk's lower interface, then the y/x passes of the layers whose z-sums are complete, and the
    read-back of the node layers that are final (cell offsets of odd length included)."""
    monkeypatch.setenv("FE_HOST_CHUNKS", str(chunks))
    gm = fe.Mesh(m, p, deform_amp=0.1, dirichlet=dirichlet)
    xu = S.primal_unique(m, p, seed=6)
    ys = [np.full(gm.unique_dofs, np.nan), np.full(gm.unique_dofs, np.nan)]
    fe.fe_apply_host(gm.handle, [fe.FE_LAPLACE, fe.FE_MASS], xu, ys)
    torch.cuda.synchronize()
    own = owner_copies(m, p)
    xc = gm.gather(xu)
    for op, y in zip((fe.FE_LAPLACE, fe.FE_MASS), ys):
        dev = gm.apply(xc, op=op, flags=fe.FE_ASSEMBLE).cpu().numpy()
        assert np.array_equal(y, dev[own])


def test_host_apply_pinned_buffers_on_streams(fe):
    """Stream-ordered calls with page-locked buffers, two meshes on two streams, repeated."""
    cases = [((8, 8, 8), 3), ((4, 4, 4), 7)]
    meshes = [fe.Mesh(m, p, deform_amp=0.1) for m, p in cases]
    streams = [torch.cuda.Stream() for _ in meshes]
    xs, ys, want = [], [], []
    for (m, p), gm in zip(cases, meshes):
        xu = S.primal_unique(m, p, seed=8)
        xs.append(torch.from_numpy(xu).pin_memory())
        ys.append([torch.empty(gm.unique_dofs, dtype=torch.float64).pin_memory() for _ in range(2)])
        own = owner_copies(m, p)
        xc = gm.gather(xu)
        want.append([gm.apply(xc, op=op, flags=fe.FE_ASSEMBLE).cpu().numpy()[own]
                     for op in (fe.FE_LAPLACE, fe.FE_MASS)])
    torch.cuda.synchronize()
    for _ in range(3):
        for gm, st, x, y in zip(meshes, streams, xs, ys):
            fe.fe_apply_host(gm.handle, [fe.FE_LAPLACE, fe.FE_MASS], x, y, 0, st)
        for st in streams:
            st.synchronize()
        for y, w in zip(ys, want):
            assert np.array_equal(y[0].numpy(), w[0]) and np.array_equal(y[1].numpy(), w[1])
        for y in ys:
            y[0].zero_()
            y[1].zero_()


def test_host_apply_on_a_slab(fe):
    from paper_2607_02335_gb300.slab import Slab
    m, p = (4, 3, 6), 2
    s = Slab(m, p, 2, 5, deform_amp=0.1)
    xu = S.primal_unique((4, 3, 3), p, seed=2)  # the slab's own node numbering
    y = np.empty(s.unique_dofs)
    fe.fe_apply_host(s.handle, [fe.FE_LAPLACE], xu, [y])
    torch.cuda.synchronize()
    yc = s.empty()
    fe.fe_apply(s.handle, fe.FE_LAPLACE, fe.FE_F64, s.gather(xu), yc, fe.FE_ASSEMBLE)  # inside the slab
    torch.cuda.synchronize()
    assert np.array_equal(y, yc.cpu().numpy()[owner_copies((4, 3, 3), p)])


def test_host_apply_rejects_bad_arguments(fe):
    gm = fe.Mesh(2, 2)
    x, y = np.zeros(gm.unique_dofs), np.zeros(gm.unique_dofs)
    for ops, flags in (([], 0), ([0, 1, 0], 0), ([5], 0), ([0], fe.FE_ASSEMBLE)):
        with pytest.raises(fe.FeError) as e:
            fe.fe_apply_host(gm.handle, ops, x, [y] * max(len(ops), 1), flags)
        assert e.value.status == fe.FE_ERR_INVALID
    pk = fe.Mesh(2, 2, layout=fe.FE_LAYOUT_PACKED2)
    with pytest.raises(fe.FeError) as e:
        fe.fe_apply_host(pk.handle, [0], np.zeros(pk.unique_dofs), [np.zeros(pk.unique_dofs)])
    assert e.value.status == fe.FE_ERR_INVALID


def test_host_apply_closed_form_beyond_two_billion_copies(fe):
    """Q1 mass on an affine 1290 x 1290 x 162 mesh (2.16e9 cell-wise entries, 64-bit offsets):
    for x = gx + 2 gy + 3 gz the assembled Q1 mass (2-point Gauss is exact) is the tensor product of
    1D masses h/6 [1 4 1] (ends h/6 [2 1]), so y has a closed form at every node."""
    mx, my, mz = 1290, 1290, 162
    gm = fe.Mesh((mx, my, mz), 1, geom_mode=fe.FE_GEOM_AFFINE)
    assert gm.cellwise_len > 2 ** 31
    Nx, Ny, Nz = mx + 1, my + 1, mz + 1
    ax = [np.arange(N, dtype=np.float64) for N in (Nx, Ny, Nz)]
    x = (ax[0][None, None, :] + 2 * ax[1][None, :, None] + 3 * ax[2][:, None, None]).reshape(-1)
    y = np.empty_like(x)
    fe.fe_apply_host(gm.handle, [fe.FE_MASS], x, [y])
    torch.cuda.synchronize()
    del x

    def one_d(N, h, scale):
        u = scale * np.arange(N, dtype=np.float64)
        mu = h * u  # interior rows: h/6 (u_{i-1} + 4 u_i + u_{i+1}) = h u_i for linear u
        mu[0] = h * (2 * u[0] + u[1]) / 6
        mu[-1] = h * (u[-2] + 2 * u[-1]) / 6
        m1 = np.full(N, h)
        m1[0] = m1[-1] = h / 2
        return mu, m1

    (ux, ox), (uy, oy), (uz, oz) = one_d(Nx, 1 / mx, 1), one_d(Ny, 1 / my, 2), one_d(Nz, 1 / mz, 3)
    want = (ux[None, None, :] * oy[None, :, None] * oz[:, None, None]
            + ox[None, None, :] * uy[None, :, None] * oz[:, None, None]
            + ox[None, None, :] * oy[None, :, None] * uz[:, None, None]).reshape(-1)
    assert rel_max_err(y, want) <= 1e-12
