"""Hanging nodes through shadow cells (Appendix, Algorithm "Full DSS Operator with Hanging Node
Resolution") through the C ABI against the constrained oracle S = G_c G_c^T."""
import numpy as np
import pytest

import oracle as O
from tests.helpers import rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(4, (1, 1, 1), (3, 2, 3), 1), (4, (1, 1, 1), (3, 2, 3), 2), (4, (1, 1, 1), (2, 3, 3), 3),
         (5, (1, 2, 1), (3, 4, 3), 4), (3, (1, 1, 1), (2, 2, 2), 7)]


@pytest.fixture(scope="module")
def fe():
    from paper_2607_02335_gb300 import fe as F
    return F


def to_host(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("mc,lo,hi,p", CASES)
def test_hanging_node_dss_and_apply(fe, mc, lo, hi, p):
    ad = O.Adaptive(mc, lo, hi, p)
    gm = fe.AMRMesh(mc, lo, hi, p)
    assert gm.cellwise_len == ad.length and gm.unique_dofs == ad.n_unique
    rng = np.random.default_rng(p)
    r = rng.standard_normal(ad.length) * ad.active_entries
    z = to_host(gm.dss(torch.from_numpy(r).cuda()))
    assert rel_max_err(z, ad.dss(r)) <= 1e-13
    r32 = torch.from_numpy(r).float().cuda()
    gm.dss(r32, prec=fe.FE_F32, z=r32)
    assert rel_max_err(to_host(r32), ad.dss(r)) <= 1e-6
    if p == 7:
        return  # the oracle's Q7 element matrices on this mesh take too long for a unit test
    xc = ad.gather(rng.uniform(-1, 1, ad.n_unique))
    x = torch.from_numpy(xc).cuda()
    for op in (fe.FE_LAPLACE, fe.FE_MASS):
        yref = ad.apply_local(op, xc)
        assert rel_max_err(to_host(gm.apply(x, op=op)), yref) <= 1e-12, (p, op)
        yasm = ad.dss(yref)
        assert rel_max_err(to_host(gm.apply(x, op=op, flags=fe.FE_ASSEMBLE)), yasm) <= 1e-12
        y32 = to_host(gm.apply(x.float(), op=op, prec=fe.FE_F32, flags=fe.FE_ASSEMBLE))
        assert rel_max_err(y32, yasm) <= 2e-5, (p, op, "fp32")


def test_constant_in_the_kernel_across_the_interface(fe):
    """The assembled Laplacian of the constant field (constrained gather of ones) vanishes, also on
    the coarse and fine copies along the refinement interface."""
    ad = O.Adaptive(5, (1, 1, 2), (4, 3, 4), 3)
    gm = fe.AMRMesh(5, (1, 1, 2), (4, 3, 4), 3)
    one = torch.from_numpy(ad.gather(np.ones(ad.n_unique))).cuda()
    y = gm.apply(one, flags=fe.FE_ASSEMBLE)
    ym = gm.apply(one, op=fe.FE_MASS, flags=fe.FE_ASSEMBLE)
    assert y.abs().max().item() <= 1e-12 * ym.abs().max().item() * 1e3


def test_invalid_boxes(fe):
    for lo, hi in (((0, 1, 1), (2, 2, 2)), ((1, 1, 1), (4, 2, 2)), ((2, 1, 1), (2, 2, 2))):
        with pytest.raises(fe.FeError) as e:
            fe.AMRMesh(4, lo, hi, 2)
        assert e.value.status == fe.FE_ERR_INVALID
