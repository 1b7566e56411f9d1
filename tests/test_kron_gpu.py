"""The 16-bit operators on the tensor cores (n = 2..4: one mma.sync product G x per 16 cells, the
metric in FP32, one product G^T t) against the FP64 oracle.

Error budget of these kernels: x, the Kronecker entries (formed in FP32, rounded once) and the
metric-scaled point values are each rounded to the 16-bit format, the metric is stored in it; with
FP32 accumulation that is about five roundings of unit roundoff u between x and y (bf16 u = 2^-9,
fp16 u = 2^-12), amplified by the cancellation of the Laplacian of a random field.  The bounds are
the ones the sum-factorized 16-bit kernels meet with their dozen roundings.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2607_02335_gb300 import synth as S
from tests.helpers import oracle_mesh, rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_LOWP = {"bf16": 6e-2, "fp16": 8e-3}


@pytest.fixture(scope="module")
def fe():
    from paper_2607_02335_gb300 import fe as F
    return F


def to_host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def precs(fe):
    return (("bf16", fe.FE_BF16_F32ACC), ("fp16", fe.FE_F16_F32ACC))


# cell counts that are not multiples of the 16 cells of a warp's task
SHAPES = {1: (5, 5, 5), 2: (5, 4, 3), 3: (7, 3, 3)}


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("dirichlet", [False, True])
def test_tensor_core_apply_vs_oracle(fe, p, dirichlet):
    m = SHAPES[p]
    om = oracle_mesh(m, p, amp=0.1, dirichlet=dirichlet)
    gm = fe.Mesh(m, p, deform_amp=0.1, dirichlet=dirichlet)
    xc = O.gather(om, S.primal_unique(m, p, seed=3))
    x32 = torch.from_numpy(xc).float().cuda()
    for name, prec in precs(fe):
        for op in (fe.FE_LAPLACE, fe.FE_MASS):
            yref = O.apply_local(om, op, xc)
            y = to_host(gm.apply(x32, op=op, prec=prec))
            assert rel_max_err(y, yref) <= TOL_LOWP[name], (p, op, name, rel_max_err(y, yref))
            if dirichlet:  # masked rows are exactly zero
                assert np.all(y[yref == 0.0] == 0.0)
            ya = to_host(gm.apply(x32, op=op, prec=prec, flags=fe.FE_ASSEMBLE))
            yd = to_host(gm.dss(gm.apply(x32, op=op, prec=prec), prec=fe.FE_F32))
            assert np.array_equal(ya, yd), (p, op, name)


def test_tensor_core_apply_large_mesh_sampled(fe):
    """Q3 on 41 x 40 x 39 cells (3998 warp tasks, more than one per resident warp, the last one
    ragged): sampled cell ranges against the oracle's element matrices."""
    m, p = (41, 40, 39), 3
    om = oracle_mesh(m, p, amp=0.1, dirichlet=True)
    gm = fe.Mesh(m, p, deform_amp=0.1, dirichlet=True)
    n3 = (p + 1) ** 3
    ncell = m[0] * m[1] * m[2]
    xc = S.dual_cellwise(m, p, seed=11)
    x32 = torch.from_numpy(xc).float().cuda()
    ranges = [(0, 24), (ncell // 2 - 7, 33), (ncell - 29, 29)]
    for name, prec in precs(fe):
        for op in (fe.FE_LAPLACE, fe.FE_MASS):
            y = to_host(gm.apply(x32, op=op, prec=prec))
            for c0, nc in ranges:
                mats = O.element_matrices(om, op, c0, nc)
                yref = O.apply_local_mats(om, c0, mats, xc[c0 * n3:(c0 + nc) * n3])
                got = y[c0 * n3:(c0 + nc) * n3]
                assert rel_max_err(got, yref) <= TOL_LOWP[name], (op, name, c0)


def test_tensor_core_and_fma_pipe_kernels_agree(fe, monkeypatch):
    """The tensor-core kernels and the sum-factorized FMA-pipe kernels (FE_LOWP_FMA=1) compute
    the same operator: both within their bound of the oracle, and of each other."""
    m, p = (6, 5, 4), 3
    om = oracle_mesh(m, p, amp=0.1)
    gm = fe.Mesh(m, p, deform_amp=0.1)
    xc = O.gather(om, S.primal_unique(m, p, seed=4))
    x32 = torch.from_numpy(xc).float().cuda()
    for name, prec in precs(fe):
        for op in (fe.FE_LAPLACE, fe.FE_MASS):
            yref = O.apply_local(om, op, xc)
            yt = to_host(gm.apply(x32, op=op, prec=prec))
            monkeypatch.setenv("FE_LOWP_FMA", "1")
            yf = to_host(gm.apply(x32, op=op, prec=prec))
            monkeypatch.delenv("FE_LOWP_FMA")
            et, ef = rel_max_err(yt, yref), rel_max_err(yf, yref)
            assert et <= TOL_LOWP[name] and ef <= TOL_LOWP[name], (op, name, et, ef)
            assert rel_max_err(yt, yf) <= 2 * TOL_LOWP[name]
            assert not np.array_equal(yt, yf)  # two different kernels really ran
    assert "FE_LOWP_FMA" not in os.environ
