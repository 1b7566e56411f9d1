"""Assembled applies whose kernel also sums the z-interfaces inside chunks of z-layers (the z-carry
brick placement; the launcher picks the chunk, or FE_ZCARRY_CHUNK forces it).  The result must be
bit for bit that of the one-layer brick kernel followed by the full z-pass (reached through a
one-slab mesh, whose assembled apply always takes that path), and match the oracle on sampled
nodes, including nodes on the interfaces between chunks (every layer boundary is sampled)."""
import numpy as np
import pytest

from paper_2607_02335_gb300 import synth as S
from tests.helpers import oracle_mesh, rel_max_err, sampled_assembled

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    from paper_2607_02335_gb300 import fe as F
    return F


# (p, m, dirichlet, prec): layer counts not divisible by the forced chunks
CASES = [(1, (64, 64, 66), True, 0), (2, (56, 32, 67), False, 0), (3, (32, 32, 130), True, 0),
         (3, (32, 32, 130), False, 1), (2, (56, 32, 67), True, 1)]


@pytest.fixture
def chunk(request, monkeypatch):
    """Layers per CTA forced through FE_ZCARRY_CHUNK (None: the launcher's own choice)."""
    if request.param is not None:
        monkeypatch.setenv("FE_ZCARRY_CHUNK", str(request.param))
    return request.param


@pytest.mark.parametrize("chunk", [2, 5, 16, None], indirect=True)
@pytest.mark.parametrize("p,m,dirichlet,prec", CASES)
@pytest.mark.parametrize("op", [0, 1])
def test_zcarry_is_bitwise_the_brick_path(fe, chunk, p, m, dirichlet, prec, op):
    from paper_2607_02335_gb300.slab import Slab, ThreadSlabGroup
    dt = torch.float64 if prec == fe.FE_F64 else torch.float32
    whole = fe.Mesh(m, p, deform_amp=0.1, dirichlet=dirichlet)
    xg = S.primal_unique(m, p, seed=12, dirichlet=dirichlet)
    x = whole.gather(xg).to(dt)
    y = whole.apply(x, op=op, prec=prec, flags=fe.FE_ASSEMBLE)
    one = Slab(m, p, 0, m[2], deform_amp=0.1, dirichlet=dirichlet)
    comm = ThreadSlabGroup(1).comm(0, one.plane_len, "cuda:0")
    y_ref = one.apply(x, op=op, prec=prec, flags=fe.FE_ASSEMBLE, comm=comm)
    torch.cuda.synchronize()
    assert torch.equal(y, y_ref)
    if prec == fe.FE_F64 and op == 0 and chunk == 5:
        om = oracle_mesh(m, p, amp=0.1, dirichlet=dirichlet)
        mx, my, mz = m
        n = p + 1
        rng = np.random.default_rng(3)
        samples = []
        for cz in range(mz):  # a node on the top face of every layer, and one inside
            cx, cy = int(rng.integers(mx)), int(rng.integers(my))
            cell = (cz * my + cy) * mx + cx
            samples.append((cell, ((n - 1) * n + int(rng.integers(n))) * n + int(rng.integers(n))))
            samples.append((cell, int(rng.integers(n ** 3))))
        ref = sampled_assembled(om, op, xg, samples)
        got = np.array([y[c * n ** 3 + l].item() for c, l in samples])
        scale = float(y.abs().max())
        assert np.max(np.abs(got - ref)) / scale <= 1e-12
