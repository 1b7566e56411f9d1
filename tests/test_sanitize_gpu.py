"""Memory hygiene of the kernels without a sanitizer: every output buffer sits between two guard
regions filled with a canary bit pattern, and is poisoned with NaN before the call.  After the call
the guards must hold the canary bit for bit (no write outside the buffer) and no NaN may remain (no
entry left unwritten), on tiny meshes (1^3, 2^3, 3x1x2 cells) at every degree and on the placement
modes of the assembled apply (bricks, z-carry chunks, 2^3-packed units), with the values checked
against the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2607_02335_gb300 import synth as S
from tests.helpers import oracle_mesh, rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GUARD = 64
PAD = 4  # GUARD + PAD entries before the output: 16-byte aligned for float and double
CANARY = 0x7FF4DEADBEEF1234  # a signalling-NaN bit pattern no kernel produces


@pytest.fixture(scope="module")
def fe():
    from paper_2607_02335_gb300 import fe as F
    return F


def guarded(n, dtype=torch.float64):
    """(whole buffer, the n-entry output inside it): guards filled with the canary, output NaN."""
    buf = torch.empty(n + 2 * GUARD + PAD, dtype=dtype, device="cuda")
    bits = buf.view(torch.int64) if dtype == torch.float64 else buf.view(torch.int32)
    bits.fill_(CANARY if dtype == torch.float64 else 0x7FA0BEEF)
    out = buf[GUARD + PAD:GUARD + PAD + n]
    out.fill_(float("nan"))
    return buf, out


def check_guards(buf, n, dtype=torch.float64):
    torch.cuda.synchronize()
    bits = buf.view(torch.int64) if dtype == torch.float64 else buf.view(torch.int32)
    want = CANARY if dtype == torch.float64 else 0x7FA0BEEF
    head, tail = bits[:GUARD + PAD], bits[GUARD + PAD + n:]
    assert bool((head == want).all()) and bool((tail == want).all()), "write outside the output"


@pytest.mark.parametrize("p", range(1, 8))
@pytest.mark.parametrize("m", [(1, 1, 1), (2, 2, 2), (3, 1, 2)])
@pytest.mark.parametrize("dirichlet", [False, True])
def test_tiny_meshes_every_degree(fe, p, m, dirichlet):
    gm = fe.Mesh(m, p, deform_amp=0.1, dirichlet=dirichlet)
    om = oracle_mesh(m, p, amp=0.1, dirichlet=dirichlet)
    xg = S.primal_unique(m, p, seed=p, dirichlet=dirichlet)
    x = gm.gather(xg)
    for op in (fe.FE_LAPLACE, fe.FE_MASS):
        for flags in (0, fe.FE_ASSEMBLE):
            buf, y = guarded(gm.cellwise_len)
            fe.fe_apply(gm.handle, op, fe.FE_F64, x, y, flags)
            check_guards(buf, gm.cellwise_len)
            yh = y.cpu().numpy()
            assert not np.isnan(yh).any(), "entries left unwritten"
            if flags:
                ref = O.gather(om, O.apply_assembled(om, op, xg))
            else:  # the oracle masks Dirichlet rows and columns of the local operator too
                ref = O.apply_local(om, op, x.cpu().numpy())
            assert rel_max_err(yh, ref) <= 1e-12
    # the DSS alone
    r = torch.from_numpy(S.dual_cellwise(m, p, seed=3)).cuda()
    buf, z = guarded(gm.cellwise_len)
    fe.fe_dss(gm.handle, fe.FE_F64, r, z)
    check_guards(buf, gm.cellwise_len)
    assert rel_max_err(z.cpu().numpy(), O.dss(om, r.cpu().numpy())) <= 1e-14


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("prec", [0, 1])
def test_placement_modes(fe, monkeypatch, p, prec):
    dt = torch.float64 if prec == fe.FE_F64 else torch.float32
    m = (9, 5, 7)
    gm = fe.Mesh(m, p, deform_amp=0.1, dirichlet=True)
    x = gm.gather(S.primal_unique(m, p, seed=2, dirichlet=True)).to(dt)
    outs = []
    for chunk in ("0", "3"):  # one-layer bricks, then z-carry chunks of 3 layers
        monkeypatch.setenv("FE_ZCARRY_CHUNK", chunk)
        for op in (fe.FE_LAPLACE, fe.FE_MASS):
            buf, y = guarded(gm.cellwise_len, dt)
            fe.fe_apply(gm.handle, op, prec, x, y, fe.FE_ASSEMBLE)
            check_guards(buf, gm.cellwise_len, dt)
            assert not torch.isnan(y).any()
            outs.append(y.clone())
    assert torch.equal(outs[0], outs[2]) and torch.equal(outs[1], outs[3])
    # 2^3-packed storage units
    pm = (4, 2, 6)
    pk = fe.Mesh(pm, p, deform_amp=0.1, layout=fe.FE_LAYOUT_PACKED2)
    xp = torch.from_numpy(S.dual_cellwise((2, 1, 3), 2 * p, seed=4)).cuda().to(dt)[: pk.cellwise_len]
    for op in (fe.FE_LAPLACE, fe.FE_MASS):
        for flags in (0, fe.FE_ASSEMBLE):
            buf, y = guarded(pk.cellwise_len, dt)
            fe.fe_apply(pk.handle, op, prec, xp.contiguous(), y, flags)
            check_guards(buf, pk.cellwise_len, dt)
            assert not torch.isnan(y).any()
