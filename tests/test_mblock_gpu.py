"""Block-structured meshes (Sec. 4.2, Algorithm "Unstructured Inter-Block Summation") through the
C ABI against the block-structured oracle, whose numbering comes from node coordinates.

DSS sums the same copies in another order (rounding only); the FP64 apply meets the 1e-12 bar."""
import numpy as np
import pytest

import oracle as O
from paper_2607_02335_gb300 import synth as S
from tests.helpers import rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MESHES = {
    "cube_in_cube": lambda m, seed: S.mb_cube_in_cube(m, seed=seed),
    "star3": lambda m, seed: S.mb_star(3, m, 2, seed=seed),
    "star5": lambda m, seed: S.mb_star(5, m, 1, seed=seed),
}


@pytest.fixture(scope="module")
def fe():
    from paper_2607_02335_gb300 import fe as F
    return F


def to_host(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("p", [1, 2, 3, 4, 7])
def test_dss_and_multiplicity(fe, name, p):
    m = 2 if p < 7 else 1
    v, b, d = MESHES[name](m, p)
    om = O.MBMesh(v, b, d, p)
    gm = fe.MBMesh(v, b, d, p)
    assert gm.unique_dofs == om.n_unique  # topology count vs coordinate matching
    assert gm.cellwise_len == om.n_cellwise
    ones = torch.ones(gm.cellwise_len, dtype=torch.float64, device="cuda")
    assert np.array_equal(to_host(gm.dss(ones)), om.multiplicity())
    r = np.random.default_rng(p).standard_normal(gm.cellwise_len)
    z = to_host(gm.dss(torch.from_numpy(r).cuda()))
    assert rel_max_err(z, om.dss(r)) <= 1e-15
    r32 = torch.from_numpy(r).float().cuda()
    gm.dss(r32, prec=fe.FE_F32, z=r32)  # in place
    assert rel_max_err(to_host(r32), om.dss(r)) <= 1e-6


def test_interface_valences(fe):
    gm = fe.MBMesh(*S.mb_cube_in_cube(2, seed=0), 2)
    info = gm.info()
    # 6 inner faces + 12 side faces shared; corners of the inner cube meet 4 blocks
    assert info["face_pairs"] == 18 and info["max_valence"] == 4
    # nodes strictly inside the 12 inner + 8 radial + 12 outer edges (all shared), and the corners
    assert info["edge_entities"] == 32 * (2 * 2 - 1) and info["vertex_entities"] == 16
    gs = fe.MBMesh(*S.mb_star(5, 2, 1, seed=0), 2)
    assert gs.info()["max_valence"] == 5


@pytest.mark.parametrize("name,p", [("cube_in_cube", 2), ("cube_in_cube", 3), ("star5", 3),
                                    ("star3", 4), ("cube_in_cube", 5)])
def test_apply_local_and_assembled(fe, name, p):
    v, b, d = MESHES[name](2, 10 + p)
    om = O.MBMesh(v, b, d, p)
    gm = fe.MBMesh(v, b, d, p)
    xg = np.random.default_rng(p).uniform(-1, 1, om.n_unique)
    xc = om.gather(xg)
    x = torch.from_numpy(xc).cuda()
    for op in (fe.FE_LAPLACE, fe.FE_MASS):
        yref = om.apply_local(op, xc)
        assert rel_max_err(to_host(gm.apply(x, op=op)), yref) <= 1e-12, (name, p, op)
        yasm = om.gather(om.scatter(yref))
        y = to_host(gm.apply(x, op=op, flags=fe.FE_ASSEMBLE))
        assert rel_max_err(y, yasm) <= 1e-12, (name, p, op, "assembled")
        yn = to_host(gm.apply(x, op=op, flags=fe.FE_ASSEMBLE | fe.FE_NATIVE_F64))
        assert rel_max_err(yn, yasm) <= 1e-12, (name, p, op, "native")
        y32 = to_host(gm.apply(x.float(), op=op, prec=fe.FE_F32, flags=fe.FE_ASSEMBLE))
        assert rel_max_err(y32, yasm) <= 2e-5, (name, p, op, "fp32")
    # the assembled Laplacian annihilates constants across the block interfaces
    one = torch.ones(gm.cellwise_len, dtype=torch.float64, device="cuda")
    yl = gm.apply(one, op=fe.FE_LAPLACE, flags=fe.FE_ASSEMBLE)
    assert yl.abs().max().item() <= 1e-12 * to_host(gm.apply(x, flags=fe.FE_ASSEMBLE)).__abs__().max()


def test_invalid_block_meshes(fe):
    v, b, d = S.mb_cube_in_cube(2, seed=0)
    d2 = d.copy()
    d2[1] = [3, 3, 3]  # the first outer block no longer conforms with the inner cube
    with pytest.raises(fe.FeError) as e:
        fe.MBMesh(v, b, d2, 2)
    assert e.value.status == fe.FE_ERR_INVALID and "conform" in str(e.value)
    b2 = b.copy()
    b2[0] = b2[0][[1, 0, 3, 2, 5, 4, 7, 6]]  # mirror the inner cube's frame: left-handed
    with pytest.raises(fe.FeError) as e:
        fe.MBMesh(v, b2, d, 2)
    assert "left-handed" in str(e.value)
    gm = fe.MBMesh(v, b, d, 2)
    x = gm.empty()
    with pytest.raises(fe.FeError):
        fe.fe_mb_apply(gm.handle, fe.FE_LAPLACE, fe.FE_F64, x, x)  # overlap
