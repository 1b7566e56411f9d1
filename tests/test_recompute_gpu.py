"""Recomputed geometry (metric formed on the fly from cell-wise nodal coordinates, Sec. 2.3 and
Sec. 6.2) against the FP64 CPU oracle and against the stored-metric mode of the same mesh.

The two modes describe the same operator, so they must agree to the FP64 bar (1e-12 relative
max-norm).  Meshes of the chunked sizes make the apply walk several L2-sized chunks of cells with
a ragged last chunk."""
import numpy as np
import pytest

import oracle as O
from paper_2607_02335_gb300 import synth as S
from tests.helpers import oracle_mesh, rel_max_err, sampled_assembled

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5

SHAPES = {1: (5, 5, 5), 2: (5, 4, 3), 3: (5, 4, 3), 4: (7, 3, 3), 5: (5, 4, 3), 6: (7, 3, 3),
          7: (3, 3, 2)}


@pytest.fixture(scope="module")
def fe():
    from paper_2607_02335_gb300 import fe as F
    return F


def to_host(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_recompute_vs_oracle_and_stored(fe, p):
    m = SHAPES[p]
    om = oracle_mesh(m, p, amp=0.1)
    gr = fe.Mesh(m, p, deform_amp=0.1, geom_mode=fe.FE_GEOM_RECOMPUTE)
    gs = fe.Mesh(m, p, deform_amp=0.1, geom_mode=fe.FE_GEOM_STORED)
    xc = O.gather(om, S.primal_unique(m, p, seed=1))
    x = torch.from_numpy(xc).cuda()
    for op in (fe.FE_LAPLACE, fe.FE_MASS):
        yref = O.apply_local(om, op, xc)
        yr = to_host(gr.apply(x, op=op))
        assert rel_max_err(yr, yref) <= TOL64, (p, op)
        assert rel_max_err(yr, to_host(gs.apply(x, op=op))) <= TOL64, (p, op, "stored")
        yn = to_host(gr.apply(x, op=op, flags=fe.FE_NATIVE_F64))
        assert rel_max_err(yn, yref) <= TOL64, (p, op, "native")
        y32 = to_host(gr.apply(x.float(), op=op, prec=fe.FE_F32))
        assert rel_max_err(y32, yref) <= TOL32, (p, op, "fp32")


@pytest.mark.parametrize("p,m", [(2, (4, 3, 5)), (5, (2, 3, 2))])
def test_recompute_assembled_dirichlet_and_diag(fe, p, m):
    om = oracle_mesh(m, p, amp=0.1, dirichlet=True)
    gm = fe.Mesh(m, p, deform_amp=0.1, geom_mode=fe.FE_GEOM_RECOMPUTE, dirichlet=True)
    xg = S.primal_unique(m, p, seed=3, dirichlet=True)
    x = gm.gather(xg)
    for op in (O.LAPLACE, O.MASS):
        yref = O.gather(om, O.apply_dirichlet_csr(om, O.assemble_csr(om, op), xg))
        y = to_host(gm.apply(x, op=op, flags=fe.FE_ASSEMBLE))
        assert rel_max_err(y, yref) <= TOL64, op
        dref = O.gather(om, O.diag_global(om, op))
        assert rel_max_err(to_host(gm.diag(op)), dref) <= TOL64, op


@pytest.mark.parametrize("p,m", [(3, 32), (7, (14, 14, 15)), (1, 64)])
def test_recompute_several_chunks(fe, p, m):
    """Sizes whose metric spans several scratch chunks (the last one ragged): recompute equals
    stored over the whole vector in every arithmetic, and sampled entries match the oracle."""
    gr = fe.Mesh(m, p, deform_amp=0.1, geom_mode=fe.FE_GEOM_RECOMPUTE)
    gs = fe.Mesh(m, p, deform_amp=0.1)
    xg = S.primal_unique(m, p, seed=2)
    x = gr.gather(xg)
    for op in (fe.FE_LAPLACE, fe.FE_MASS):
        yr = gr.apply(x, op=op, flags=fe.FE_ASSEMBLE)
        ys = gs.apply(x, op=op, flags=fe.FE_ASSEMBLE)
        scale = ys.abs().max().item()
        assert (yr - ys).abs().max().item() <= TOL64 * scale, op
        yr32 = gr.apply(x.float(), op=op, prec=fe.FE_F32)
        ys32 = gs.apply(x.float(), op=op, prec=fe.FE_F32)
        s32 = ys32.abs().max().item()
        assert (yr32 - ys32).abs().max().item() <= TOL32 * s32, op
        del yr32, ys32
        om = oracle_mesh(m, p, amp=0.1)
        rng = np.random.default_rng(p)
        n3 = (p + 1) ** 3
        samples = [(int(c), int(l)) for c, l in zip(rng.integers(0, gr.n_cells, 8),
                                                    rng.integers(0, n3, 8))]
        samples += [(gr.n_cells - 1, n3 - 1)]
        got = np.array([yr[c * n3 + l].item() for c, l in samples])
        ref = sampled_assembled(om, op, xg, samples)
        assert np.abs(got - ref).max() <= TOL64 * scale, op


def test_recompute_cg_matches_stored(fe):
    """Jacobi-PCG on a recompute mesh takes the same path as on the stored mesh."""
    m, p = (5, 4, 3), 3
    bc = S.dual_cellwise(m, p, seed=21)
    out = {}
    for mode in (fe.FE_GEOM_STORED, fe.FE_GEOM_RECOMPUTE):
        gm = fe.Mesh(m, p, deform_amp=0.1, geom_mode=mode, dirichlet=True)
        x = torch.zeros(gm.cellwise_len, dtype=torch.float64, device="cuda")
        res, hist = gm.cg_solve(torch.from_numpy(bc).cuda(), x, rtol=1e-11, maxit=500,
                                history=True)
        assert res.status == fe.FE_OK
        out[mode] = (res, hist, to_host(x))
        xm = torch.zeros_like(x)
        rm = gm.cg_solve(torch.from_numpy(bc).cuda(), xm, rtol=1e-10, maxit=500,
                         mixed=fe.FE_F32, flexible=True)
        assert rm.status == fe.FE_OK and rm.rel_res <= 1e-10
    (rs, hs, xs), (rr, hr, xr) = out[fe.FE_GEOM_STORED], out[fe.FE_GEOM_RECOMPUTE]
    assert abs(rs.iters - rr.iters) <= 1
    k = min(rs.iters, rr.iters, 20)
    assert np.allclose(hs[:k, 0], hr[:k, 0], rtol=1e-9, atol=0)
    assert rel_max_err(xr, xs) <= 1e-9


def test_recompute_not_accepted_by_batched(fe):
    gm = fe.Mesh(2, 2, deform_amp=0.1, geom_mode=fe.FE_GEOM_RECOMPUTE)
    b = torch.ones(gm.cellwise_len, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(fe.FeError):
        fe.fe_cg_solve_batched([gm.handle], [b], [x], fe.fe_cg_opts(1e-8, 10, 0, 0, 1e-2, None))
