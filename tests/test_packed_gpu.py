"""2^3-packed storage units (FE_LAYOUT_PACKED2, Sec. 2.2 and Table "tab:memory_overhead") through the
C ABI against the packed oracle (P^T A_K P over the structured oracle)."""
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


def to_host(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("p,m,dirichlet", [(1, (6, 4, 2), False), (1, (2, 2, 8), True),
                                           (2, (4, 2, 6), True), (2, (6, 4, 4), False),
                                           (3, (4, 4, 2), False), (3, (2, 6, 2), True)])
def test_packed_apply_and_dss_vs_oracle(fe, p, m, dirichlet):
    om = oracle_mesh(m, p, amp=0.1, dirichlet=dirichlet)
    pk = O.Packed(om)
    gm = fe.Mesh(m, p, deform_amp=0.1, dirichlet=dirichlet, layout=fe.FE_LAYOUT_PACKED2)
    lay = fe.fe_mesh_layout(gm.handle)
    assert lay.layout_id == fe.FE_LAYOUT_PACKED2 and lay.nodes_per_cell == (2 * p + 1) ** 3
    assert lay.n_cells == m[0] * m[1] * m[2] // 8 and gm.cellwise_len == pk.length
    xg = S.primal_unique(m, p, seed=9, dirichlet=dirichlet)
    xu = pk.gather(xg)
    x = torch.from_numpy(xu).cuda()
    for op in (fe.FE_LAPLACE, fe.FE_MASS):
        yref = pk.apply_local(op, xu)
        assert rel_max_err(to_host(gm.apply(x, op=op)), yref) <= 1e-12, (p, op)
        yasm = pk.dss(yref)
        assert rel_max_err(to_host(gm.apply(x, op=op, flags=fe.FE_ASSEMBLE)), yasm) <= 1e-12
        yn = to_host(gm.apply(x, op=op, flags=fe.FE_ASSEMBLE | fe.FE_NATIVE_F64))
        assert rel_max_err(yn, yasm) <= 1e-12
        y32 = to_host(gm.apply(x.float(), op=op, prec=fe.FE_F32, flags=fe.FE_ASSEMBLE))
        assert rel_max_err(y32, yasm) <= 2e-5
        y16 = to_host(gm.apply(x.float(), op=op, prec=fe.FE_F16_F32ACC))
        assert rel_max_err(y16, yref) <= 8e-3
    ones = torch.ones(gm.cellwise_len, dtype=torch.float64, device="cuda")
    assert np.array_equal(to_host(gm.dss(ones)), pk.multiplicity())
    r = np.random.default_rng(p).standard_normal(gm.cellwise_len)
    assert rel_max_err(to_host(gm.dss(torch.from_numpy(r).cuda())), pk.dss(r)) <= 1e-15


@pytest.mark.parametrize("p,m", [(2, 48), (3, 32)])
def test_packed_equals_cellwise_at_size(fe, p, m):
    """At benchmark-like sizes: the packed apply is the cell-wise apply summed into the units
    (P^T), and the assembled outputs agree entry by entry through the packing map."""
    om = oracle_mesh(m, p, amp=0.1)
    pk = O.Packed(om)
    gc = fe.Mesh(m, p, deform_amp=0.1)
    gp = fe.Mesh(m, p, deform_amp=0.1, layout=fe.FE_LAYOUT_PACKED2)
    xg = S.primal_unique(m, p, seed=0)
    xc = gc.gather(xg)
    xu = torch.from_numpy(pk.gather(xg)).cuda()
    P = torch.from_numpy(pk.P).cuda()
    for op in (fe.FE_LAPLACE, fe.FE_MASS):
        yc = gc.apply(xc, op=op)
        ref = torch.zeros(gp.cellwise_len, dtype=torch.float64, device="cuda").index_add_(0, P, yc)
        yp = gp.apply(xu, op=op)
        assert (yp - ref).abs().max().item() <= 1e-12 * ref.abs().max().item()
        ya = gp.apply(xu, op=op, flags=fe.FE_ASSEMBLE)
        yca = gc.apply(xc, op=op, flags=fe.FE_ASSEMBLE)
        assert (ya[P] - yca).abs().max().item() <= 1e-12 * yca.abs().max().item()


def test_packed_invalid(fe):
    for kw in (dict(m=(3, 2, 2), p=2), dict(m=(2, 2, 2), p=4)):
        with pytest.raises(fe.FeError) as e:
            fe.Mesh(kw["m"], kw["p"], layout=fe.FE_LAYOUT_PACKED2)
        assert e.value.status == fe.FE_ERR_INVALID
    with pytest.raises(fe.FeError):
        fe.Mesh((2, 2, 2), 2, geom_mode=fe.FE_GEOM_RECOMPUTE, layout=fe.FE_LAYOUT_PACKED2)
    gm = fe.Mesh((2, 2, 2), 2, layout=fe.FE_LAYOUT_PACKED2, dirichlet=True)
    with pytest.raises(fe.FeError):
        gm.diag()
    b = torch.zeros(gm.cellwise_len, dtype=torch.float64, device="cuda")
    with pytest.raises(fe.FeError):
        gm.cg_solve(b, torch.zeros_like(b))
    # affine packed mesh against its stored twin
    ga = fe.Mesh((4, 2, 2), 2, geom_mode=fe.FE_GEOM_AFFINE, layout=fe.FE_LAYOUT_PACKED2)
    gs = fe.Mesh((4, 2, 2), 2, layout=fe.FE_LAYOUT_PACKED2)
    x = torch.randn(ga.cellwise_len, dtype=torch.float64, device="cuda")
    ya, ys = ga.apply(x, flags=fe.FE_ASSEMBLE), gs.apply(x, flags=fe.FE_ASSEMBLE)
    assert (ya - ys).abs().max().item() <= 1e-12 * ys.abs().max().item()
