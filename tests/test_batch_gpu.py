"""Batched solves: one persistent launch applies every problem's operator per CG iteration.
Each result must be bitwise the same alone and in the mix, agree with the single-problem solver
to rounding, and reach the FP64 residual target (checked by the oracle)."""
import numpy as np
import pytest

import oracle as O
from paper_2607_02335_gb300 import synth as S
from tests.helpers import oracle_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPECS = [((4, 4, 4), 2, 0.05), ((5, 3, 4), 3, 0.12), ((2, 3, 2), 5, 0.0), ((2, 2, 2), 7, 0.1),
         ((6, 5, 3), 2, 0.15), ((3, 3, 3), 3, 0.08), ((1, 2, 3), 7, 0.02), ((4, 2, 5), 5, 0.1)]


@pytest.fixture(scope="module")
def fe():
    from paper_2607_02335_gb300 import fe as F
    return F


def build(fe):
    meshes, bs = [], []
    for i, (m, p, amp) in enumerate(SPECS):
        gm = fe.Mesh(m, p, deform_amp=amp, geom_mode=fe.FE_GEOM_AFFINE if amp == 0 else fe.FE_GEOM_STORED,
                     dirichlet=True)
        meshes.append(gm)
        bs.append(torch.from_numpy(S.dual_cellwise(m, p, seed=100 + i)).cuda())
    return meshes, bs


@pytest.mark.parametrize("mixed", [0, 1])
def test_batched_alone_equals_mix(fe, mixed):
    meshes, bs = build(fe)
    opts = fe.fe_cg_opts(1e-10, 5000, fe.FE_F32 if mixed else 0, 1 if mixed else 0, 1e-2, None)
    xs = [torch.zeros_like(b) for b in bs]
    res = fe.fe_cg_solve_batched([g.handle for g in meshes], bs, xs, opts)
    assert all(r.status == fe.FE_OK for r in res), [r.status for r in res]
    assert all(r.rel_res <= 1e-10 for r in res)
    for i, gm in enumerate(meshes):
        xa = torch.zeros_like(bs[i])
        ra = fe.fe_cg_solve_batched([gm.handle], [bs[i]], [xa], opts)[0]
        assert torch.equal(xa, xs[i]), i  # bitwise: same arithmetic alone and in the mix
        assert ra.iters == res[i].iters and ra.rel_res == res[i].rel_res
        # single-problem solver: same method, different reduction order
        xs1 = torch.zeros_like(bs[i])
        r1 = gm.cg_solve(bs[i], xs1, rtol=1e-10, maxit=5000, mixed=fe.FE_F32 if mixed else 0,
                         flexible=bool(mixed))
        assert r1.status == fe.FE_OK
        scale = float(xs1.abs().max())
        assert float((xs1 - xs[i]).abs().max()) <= 1e-8 * scale


def test_batched_residual_checked_by_oracle(fe):
    meshes, bs = build(fe)
    opts = fe.fe_cg_opts(1e-10, 5000, fe.FE_F32, 1, 1e-2, None)
    xs = [torch.zeros_like(b) for b in bs]
    res = fe.fe_cg_solve_batched([g.handle for g in meshes], bs, xs, opts)
    for i in (0, 3, 6):
        m, p, amp = SPECS[i]
        om = oracle_mesh(m, p, amp=amp, dirichlet=True)
        gidx = O.gather(om, np.arange(om.n_unique, dtype=np.float64)).astype(np.int64)
        xg = np.zeros(om.n_unique)
        xg[gidx] = xs[i].cpu().numpy()
        bg = O.scatter(om, bs[i].cpu().numpy())
        bg[O.boundary_global(om)] = 0.0
        r = bg - O.apply_dirichlet_csr(om, O.assemble_csr(om, O.LAPLACE), xg)
        assert np.linalg.norm(r) / np.linalg.norm(bg) <= 1.2e-10, i
        assert res[i].outer_iters >= 1


def test_batched_invalid(fe):
    meshes, bs = build(fe)
    opts = fe.fe_cg_opts(1e-10, 100, 0, 0, 1e-2, None)
    with pytest.raises(fe.FeError):
        fe.fe_cg_solve_batched([meshes[0].handle, meshes[0].handle], [bs[0], bs[0]],
                               [torch.zeros_like(bs[0])] * 2, opts)
    res = fe.fe_cg_solve_batched([meshes[0].handle], [bs[0]], [torch.zeros_like(bs[0])],
                                 fe.fe_cg_opts(1e-14, 2, 0, 0, 1e-2, None))
    assert res[0].status == fe.FE_ERR_NOT_CONVERGED and res[0].iters == 2
