"""Parity of the CUDA operator path (through the C ABI) with the FP64 CPU oracle.

Bar (from the method's FP64 target): relative max-norm error <= 1e-12 for the FP64 path
(double-word arithmetic on the FP32 pipe, and the native FP64 variant); FP32 path <= 2e-5
(a few units of float rounding amplified by the ~n-term contractions and the metric).
"""
import numpy as np
import pytest

import oracle as O
from paper_2607_02335_gb300 import synth as S
from tests.helpers import oracle_mesh, rel_max_err, sampled_assembled

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


@pytest.fixture(scope="module")
def fe():
    from paper_2607_02335_gb300 import fe as F
    return F


def to_host(t):
    return t.detach().cpu().numpy().astype(np.float64)


# shapes chosen so that every degree spans several CTAs and ends on a ragged one
SHAPES = {1: (5, 5, 5), 2: (5, 4, 3), 3: (5, 4, 3), 4: (7, 3, 3), 5: (5, 4, 3), 6: (7, 3, 3),
          7: (3, 3, 2)}


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_local_apply_all_degrees(fe, p):
    m = SHAPES[p]
    amp = 0.1
    om = oracle_mesh(m, p, amp=amp)
    gm = fe.Mesh(m, p, deform_amp=amp)
    xg = S.primal_unique(m, p, seed=0)
    xc = O.gather(om, xg)
    x = torch.from_numpy(xc).cuda()
    for op in (fe.FE_LAPLACE, fe.FE_MASS):
        yref = O.apply_local(om, op, xc)
        y = to_host(gm.apply(x, op=op, prec=fe.FE_F64))
        assert rel_max_err(y, yref) <= TOL64, (p, op)
        if p in (2, 3, 7):
            yn = to_host(gm.apply(x, op=op, prec=fe.FE_F64, flags=fe.FE_NATIVE_F64))
            assert rel_max_err(yn, yref) <= TOL64, (p, op, "native")
            y32 = to_host(gm.apply(x.float(), op=op, prec=fe.FE_F32))
            assert rel_max_err(y32, yref) <= TOL32, (p, op, "fp32")


def test_pr1_q2_affine_assembled_dirichlet_vs_csr(fe):
    """8^3 affine Q2 Laplace, FP64, FE_ASSEMBLE + Dirichlet, x from seed 0 zeroed on the
    boundary, against the oracle's assembled sparse SpMV."""
    m, p = 8, 2
    om = oracle_mesh(m, p, dirichlet=True)
    csr = O.assemble_csr(om, O.LAPLACE)
    xg = S.primal_unique(m, p, seed=0, dirichlet=True)
    yg = O.apply_dirichlet_csr(om, csr, xg)
    yref = O.gather(om, yg)
    for mode in (fe.FE_GEOM_AFFINE, fe.FE_GEOM_STORED):
        gm = fe.Mesh(m, p, geom_mode=mode, dirichlet=True)
        x = gm.gather(xg)
        y = to_host(gm.apply(x, op=fe.FE_LAPLACE, prec=fe.FE_F64, flags=fe.FE_ASSEMBLE))
        assert rel_max_err(y, yref) <= TOL64, mode
        assert gm.cellwise_len == 13824 and gm.unique_dofs == 4913


@pytest.mark.parametrize("p,m", [(2, (4, 3, 5)), (3, (3, 4, 2)), (5, (2, 3, 2))])
def test_assembled_deformed_dirichlet_vs_csr(fe, p, m):
    om = oracle_mesh(m, p, amp=0.1, dirichlet=True)
    gm = fe.Mesh(m, p, deform_amp=0.1, dirichlet=True)
    xg = S.primal_unique(m, p, seed=3, dirichlet=True)
    x = gm.gather(xg)
    for op in (O.LAPLACE, O.MASS):
        csr = O.assemble_csr(om, op)
        yref = O.gather(om, O.apply_dirichlet_csr(om, csr, xg))
        y = to_host(gm.apply(x, op=op, prec=fe.FE_F64, flags=fe.FE_ASSEMBLE))
        assert rel_max_err(y, yref) <= TOL64, op
        # every copy of a node holds the same assembled value (bitwise)
        gidx = O.gather(om, np.arange(om.n_unique, dtype=np.float64)).astype(np.int64)
        hi = np.full(om.n_unique, -np.inf)
        lo = np.full(om.n_unique, np.inf)
        np.maximum.at(hi, gidx, y)
        np.minimum.at(lo, gidx, y)
        assert np.array_equal(hi, lo)


# (degree, mesh): several bricks along x and y with a ragged last brick, for every degree
FUSED = [(1, (17, 10, 3)), (2, (15, 9, 2)), (3, (9, 10, 3)), (4, (11, 5, 2)), (5, (7, 5, 2)),
         (6, (5, 5, 2)), (7, (5, 3, 2))]


@pytest.mark.parametrize("p,m", FUSED)
def test_fused_assembly_equals_apply_then_dss(fe, p, m):
    """FE_ASSEMBLE sums the x/y interfaces inside each CTA's brick of cells and leaves the rest to
    the DSS passes between bricks; the result must equal the unassembled apply followed by the
    full structured DSS (same sums in another order: rounding-level differences only)."""
    for dirichlet in (False, True):
        gm = fe.Mesh(m, p, deform_amp=0.1, dirichlet=dirichlet)
        x = gm.gather(S.primal_unique(m, p, seed=6, dirichlet=dirichlet))
        for op in (fe.FE_LAPLACE, fe.FE_MASS):
            yf = to_host(gm.apply(x, op=op, flags=fe.FE_ASSEMBLE))
            yr = to_host(gm.dss(gm.apply(x, op=op)))
            assert rel_max_err(yf, yr) <= 1e-14, (p, op, dirichlet)
            yf32 = to_host(gm.apply(x.float(), op=op, prec=fe.FE_F32, flags=fe.FE_ASSEMBLE))
            yr32 = to_host(gm.dss(gm.apply(x.float(), op=op, prec=fe.FE_F32), prec=fe.FE_F32))
            assert rel_max_err(yf32, yr32) <= 1e-6, (p, op, dirichlet, "fp32")
            yn = to_host(gm.apply(x, op=op, flags=fe.FE_ASSEMBLE | fe.FE_NATIVE_F64))
            assert rel_max_err(yn, yr) <= 1e-12, (p, op, dirichlet, "native")
    # against the oracle on the Dirichlet mesh
    om = oracle_mesh(m, p, amp=0.1, dirichlet=True)
    xg = S.primal_unique(m, p, seed=6, dirichlet=True)
    yref = O.gather(om, O.apply_dirichlet_csr(om, O.assemble_csr(om, O.LAPLACE), xg))
    gm = fe.Mesh(m, p, deform_amp=0.1, dirichlet=True)
    y = to_host(gm.apply(gm.gather(xg), flags=fe.FE_ASSEMBLE))
    assert rel_max_err(y, yref) <= TOL64


def test_dss_multiplicity_and_random(fe):
    m, p = (3, 4, 2), 3
    om = oracle_mesh(m, p)
    gm = fe.Mesh(m, p)
    ones = torch.ones(gm.cellwise_len, dtype=torch.float64, device="cuda")
    assert np.array_equal(to_host(gm.dss(ones)), O.multiplicity(om))
    r = S.dual_cellwise(m, p, seed=5)
    z = to_host(gm.dss(torch.from_numpy(r).cuda()))
    assert rel_max_err(z, O.dss(om, r)) <= 1e-15
    # in place, FP32
    r32 = torch.from_numpy(r).float().cuda()
    gm.dss(r32, prec=fe.FE_F32, z=r32)
    assert rel_max_err(to_host(r32), O.dss(om, r)) <= 1e-6


@pytest.mark.parametrize("p,amp,dirichlet", [(2, 0.1, True), (3, 0.1, False), (4, 0.0, True)])
def test_diag_vs_oracle(fe, p, amp, dirichlet):
    m = (3, 2, 4)
    om = oracle_mesh(m, p, amp=amp, dirichlet=dirichlet)
    for geom in ((fe.FE_GEOM_STORED, fe.FE_GEOM_AFFINE) if amp == 0 else (fe.FE_GEOM_STORED,)):
        gm = fe.Mesh(m, p, deform_amp=amp, geom_mode=geom, dirichlet=dirichlet)
        for op in (O.LAPLACE, O.MASS):
            dref = O.gather(om, O.diag_global(om, op))
            assert rel_max_err(to_host(gm.diag(op)), dref) <= TOL64


def test_pairing_and_lemma(fe):
    m, p = (4, 3, 3), 2
    om = oracle_mesh(m, p)
    gm = fe.Mesh(m, p)
    f = S.dual_cellwise(m, p, seed=7)
    u = S.primal_unique(m, p, seed=8)
    uc = O.gather(om, u)
    got = gm.pairing(torch.from_numpy(f).cuda(), torch.from_numpy(uc).cuda())
    ref = float(np.sum(f * uc))
    assert abs(got - ref) <= 1e-14 * np.abs(f * uc).sum()
    # Lemma (Duality Pairing Identity): <f, G u> = <G^T f, u>
    assert abs(got - O.scatter(om, f) @ u) <= 1e-13 * np.abs(f * uc).sum()
    # bitwise reproducible
    got2 = gm.pairing(torch.from_numpy(f).cuda(), torch.from_numpy(uc).cuda())
    assert got == got2


def test_edge_cases(fe):
    # single cell: no interfaces, DSS is the identity
    om = oracle_mesh(1, 4, amp=0.1)
    gm = fe.Mesh(1, 4, deform_amp=0.1)
    xc = S.dual_cellwise(1, 4, seed=1)
    x = torch.from_numpy(xc).cuda()
    y = to_host(gm.apply(x, flags=fe.FE_ASSEMBLE))
    assert rel_max_err(y, O.apply_local(om, O.LAPLACE, xc)) <= TOL64
    # thin meshes
    for m in ((1, 1, 5), (6, 1, 1), (1, 7, 1)):
        om = oracle_mesh(m, 2, amp=0.05, dirichlet=True)
        gm = fe.Mesh(m, 2, deform_amp=0.05, dirichlet=True)
        xg = S.primal_unique(m, 2, seed=2, dirichlet=True)
        y = to_host(gm.apply(gm.gather(xg), flags=fe.FE_ASSEMBLE))
        yref = O.gather(om, O.apply_dirichlet_csr(om, O.assemble_csr(om, O.LAPLACE), xg))
        assert rel_max_err(y, yref) <= TOL64, m
    # small input magnitudes keep their relative accuracy (the double-word range of the FP64
    # path is |x| >= ~1e-20, see fe_internal.h)
    om = oracle_mesh((2, 2, 2), 3, amp=0.1)
    gm = fe.Mesh((2, 2, 2), 3, deform_amp=0.1)
    xc = S.dual_cellwise((2, 2, 2), 3, seed=4) * 1e-20
    y = to_host(gm.apply(torch.from_numpy(xc).cuda()))
    assert rel_max_err(y, O.apply_local(om, O.LAPLACE, xc)) <= TOL64


def test_invalid_arguments(fe):
    d = fe.fe_mesh_desc(2, 2, 2, 8, 0.0, 0, 0, 0)
    with pytest.raises(fe.FeError) as e:
        fe.fe_mesh_create(d)
    assert e.value.status == fe.FE_ERR_INVALID and "degree" in str(e.value)
    gm = fe.Mesh(2, 2)
    x = gm.empty()
    with pytest.raises(fe.FeError):
        fe.fe_apply(gm.handle, fe.FE_LAPLACE, fe.FE_F64, x, x)  # overlap
    with pytest.raises(fe.FeError):
        fe.fe_apply(gm.handle, fe.FE_LAPLACE, 7, x, gm.empty())  # unknown precision
    with pytest.raises(fe.FeError):
        fe.fe_apply(gm.handle, fe.FE_LAPLACE, fe.FE_F64, 0, gm.empty())
    with pytest.raises(fe.FeError):
        fe.fe_apply(gm.handle, fe.FE_LAPLACE, fe.FE_F64, x.data_ptr() + 8, gm.empty())


FULL = [(2, 48), (3, 96), (7, 32)]


@pytest.mark.parametrize("p,m", FULL)
def test_full_size_sampled_parity(fe, p, m):
    """Sweep sizes of the throughput benchmark (deformed, stored geometry, FE_ASSEMBLE): sampled
    entries against the oracle's element rows, plus the constant-annihilation property."""
    amp = 0.1
    gm = fe.Mesh(m, p, deform_amp=amp)
    om = oracle_mesh(m, p, amp=amp)
    xg = S.primal_unique(m, p, seed=0)
    x = gm.gather(xg)
    rng = np.random.default_rng(p)
    ncell = gm.n_cells
    n3 = (p + 1) ** 3
    samples = [(int(c), int(l)) for c, l in zip(rng.integers(0, ncell, 24), rng.integers(0, n3, 24))]
    samples += [(0, 0), (ncell - 1, n3 - 1), (ncell // 2, n3 // 2)]
    for op in (fe.FE_LAPLACE, fe.FE_MASS):
        y = gm.apply(x, op=op, flags=fe.FE_ASSEMBLE)
        got = np.array([y[c * n3 + l].item() for c, l in samples])
        ref = sampled_assembled(om, op, xg, samples)
        scale = y.abs().max().item()
        assert np.abs(got - ref).max() <= TOL64 * scale, op
        del y
    ones = torch.ones(gm.cellwise_len, dtype=torch.float64, device="cuda")
    y1 = gm.apply(ones, op=fe.FE_LAPLACE, flags=fe.FE_ASSEMBLE)
    yx = gm.apply(x, op=fe.FE_LAPLACE, flags=fe.FE_ASSEMBLE)
    assert y1.abs().max().item() <= 1e-12 * yx.abs().max().item()


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_smooth_input_accuracy(fe, p):
    """Smooth inputs: the Laplacian of a smooth field is small against the intermediate gradients,
    so rounding before the derivative is amplified by about (p/h)^2 (~1e3 here).  The FP64 path
    forms every gradient component from differences of neighbouring binary64 inputs before any
    double-word rounding; both it and native FP64 sum factorization stay within 1e-12 of the
    oracle, unassembled and assembled (where the element contributions cancel further)."""
    m = SHAPES[p]
    om = oracle_mesh(m, p, amp=0.1)
    gm = fe.Mesh(m, p, deform_amp=0.1)
    xg = O.exact_nodal(om, O.RHS_SINE)
    xc = O.gather(om, xg)
    x = torch.from_numpy(xc).cuda()
    for op in (fe.FE_LAPLACE, fe.FE_MASS):
        yref = O.apply_local(om, op, xc)
        assert rel_max_err(to_host(gm.apply(x, op=op, flags=fe.FE_NATIVE_F64)), yref) <= TOL64
        assert rel_max_err(to_host(gm.apply(x, op=op)), yref) <= TOL64, (p, op)
        ya = O.gather(om, O.apply_assembled(om, op, xg))
        assert rel_max_err(to_host(gm.apply(x, op=op, flags=fe.FE_ASSEMBLE)), ya) <= TOL64, (p, op)


@pytest.mark.parametrize("p,m", [(3, 48), (7, 16)])
def test_smooth_input_at_larger_sizes(fe, p, m):
    """At finer meshes the local Laplacian of a smooth field amplifies input rounding by about
    p^4/h, and FP64 evaluations in different orders (native sum factorization, the oracle's
    element matrices) drift apart towards 1e-12.  The double-word path must stay as close to the
    oracle as native FP64 is (sampled cells against the oracle's element matrices)."""
    om = oracle_mesh(m, p, amp=0.1)
    gm = fe.Mesh(m, p, deform_amp=0.1)
    xc = O.gather(om, O.exact_nodal(om, O.RHS_SINE))
    n3, nc = (p + 1) ** 3, m ** 3
    x = torch.from_numpy(xc).cuda()
    for op in (fe.FE_LAPLACE, fe.FE_MASS):
        y = to_host(gm.apply(x, op=op))
        yn = to_host(gm.apply(x, op=op, flags=fe.FE_NATIVE_F64))
        den = np.abs(y).max()
        e_dw = e_nat = 0.0
        for c0 in (0, nc // 3, nc // 2 + m * m // 2 + m // 2, nc - 8):
            yr = O.apply_local_mats(om, c0, O.element_matrices(om, op, c0, 8),
                                    xc[c0 * n3:(c0 + 8) * n3])
            e_dw = max(e_dw, np.abs(y[c0 * n3:(c0 + 8) * n3] - yr).max() / den)
            e_nat = max(e_nat, np.abs(yn[c0 * n3:(c0 + 8) * n3] - yr).max() / den)
        assert e_nat <= 3e-12, (p, m, op, e_nat)
        assert e_dw <= max(1.5 * e_nat, TOL64), (p, m, op, e_dw, e_nat)


@pytest.mark.parametrize("scale", [1e-300, 1e-30, 1e30, 1e300])
def test_extreme_magnitudes(fe, scale):
    """The FP64 path scales each CTA's inputs by a power of two before the double-word arithmetic,
    so inputs far outside the float range keep their relative accuracy (unassembled and
    assembled, smooth and random inputs, both operators)."""
    m, p = (3, 2, 2), 3
    om = oracle_mesh(m, p, amp=0.1)
    gm = fe.Mesh(m, p, deform_amp=0.1)
    xg = O.exact_nodal(om, O.RHS_SINE)
    for xc in (O.gather(om, xg) * scale, S.dual_cellwise(m, p, seed=4) * scale):
        x = torch.from_numpy(xc).cuda()
        for op in (fe.FE_LAPLACE, fe.FE_MASS):
            yref = O.apply_local(om, op, xc)
            assert np.isfinite(yref).all()
            y = to_host(gm.apply(x, op=op))
            assert rel_max_err(y, yref) <= TOL64, (scale, op)
            yd = to_host(gm.dss(gm.apply(x, op=op)))
            ya = to_host(gm.apply(x, op=op, flags=fe.FE_ASSEMBLE))
            assert rel_max_err(ya, yd) <= 1e-14, (scale, op)


def test_mixed_magnitudes_within_a_cta(fe):
    """Cells of very different magnitude in one CTA: each keeps its accuracy relative to the
    largest output (the relative max-norm of the bar)."""
    m, p = (4, 3, 2), 2
    om = oracle_mesh(m, p, amp=0.1)
    gm = fe.Mesh(m, p, deform_amp=0.1)
    n3 = (p + 1) ** 3
    xc = S.dual_cellwise(m, p, seed=5)
    xc[: 3 * n3] *= 1e12
    xc[5 * n3: 7 * n3] *= 1e-9
    yref = O.apply_local(om, O.LAPLACE, xc)
    y = to_host(gm.apply(torch.from_numpy(xc).cuda()))
    assert rel_max_err(y, yref) <= TOL64


# 16-bit operands with FP32 accumulation: every stage output (interpolated values, gradients,
# metric products, even-odd sums) is rounded to the 16-bit format, about a dozen roundings of unit
# roundoff u on the way from x to y (bf16 u = 2^-9, fp16 u = 2^-12), amplified by the
# cancellation of the Laplacian of a random field; the bounds allow ~12 u x a factor of 2.5.
TOL_LOWP = {"bf16": 6e-2, "fp16": 8e-3}


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_lowp_apply_vs_oracle(fe, p):
    m = SHAPES[p]
    om = oracle_mesh(m, p, amp=0.1)
    gm = fe.Mesh(m, p, deform_amp=0.1)
    xc = O.gather(om, S.primal_unique(m, p, seed=0))
    x32 = torch.from_numpy(xc).float().cuda()
    for name, prec in (("bf16", fe.FE_BF16_F32ACC), ("fp16", fe.FE_F16_F32ACC)):
        for op in (fe.FE_LAPLACE, fe.FE_MASS):
            yref = O.apply_local(om, op, xc)
            y = to_host(gm.apply(x32, op=op, prec=prec))
            assert rel_max_err(y, yref) <= TOL_LOWP[name], (p, op, name, rel_max_err(y, yref))
            ya = to_host(gm.apply(x32, op=op, prec=prec, flags=fe.FE_ASSEMBLE))
            yd = to_host(gm.dss(gm.apply(x32, op=op, prec=prec), prec=fe.FE_F32))
            assert rel_max_err(ya, yd) <= 1e-6, (p, op, name)


def test_lowp_requires_stored_geometry(fe):
    for mode in (fe.FE_GEOM_AFFINE, fe.FE_GEOM_RECOMPUTE):
        gm = fe.Mesh(3, 2, geom_mode=mode)
        x = gm.empty(fe.FE_F32)
        with pytest.raises(fe.FeError) as e:
            fe.fe_apply(gm.handle, fe.FE_LAPLACE, fe.FE_BF16_F32ACC, x, gm.empty(fe.FE_F32))
        assert e.value.status == fe.FE_ERR_INVALID
