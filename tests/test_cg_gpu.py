"""Cell-wise CG (Algorithm "Communication-Free (Flexible) PCG") against the oracle's assembled
Jacobi-PCG: the Equivalence theorem says the iterates coincide, so alpha_k, beta_k and the
relative residuals must agree up to rounding; solutions, exact quadratic reproduction, mixed
precision to an FP64 residual of 1e-10 checked by the oracle."""
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


def unique_from_cellwise(om, xc):
    gidx = O.gather(om, np.arange(om.n_unique, dtype=np.float64)).astype(np.int64)
    xg = np.zeros(om.n_unique)
    xg[gidx] = xc
    return xg, gidx


def oracle_relres(om, b_cell, x_cell):
    """||G^T b - A_D x_glob|| / ||G^T b|| over free nodes, in FP64 on the CPU."""
    xg, _ = unique_from_cellwise(om, x_cell)
    bg = O.scatter(om, b_cell)
    bnd = O.boundary_global(om)
    bg[bnd] = 0.0
    csr = O.assemble_csr(om, O.LAPLACE)
    r = bg - O.apply_dirichlet_csr(om, csr, xg)
    return np.linalg.norm(r) / np.linalg.norm(bg)


@pytest.mark.parametrize("flexible", [False, True])
def test_equivalence_theorem_iterates(fe, flexible):
    m, p = (4, 3, 5), 3
    om = oracle_mesh(m, p, amp=0.1, dirichlet=True)
    gm = fe.Mesh(m, p, deform_amp=0.1, dirichlet=True)
    bc = S.dual_cellwise(m, p, seed=21)
    ref = O.cg(om, O.LAPLACE, O.scatter(om, bc), rtol=1e-12, maxit=500, flexible=flexible)
    assert ref["status"] == 0
    x = torch.zeros(gm.cellwise_len, dtype=torch.float64, device="cuda")
    res, hist = gm.cg_solve(torch.from_numpy(bc).cuda(), x, rtol=1e-12, maxit=500,
                            flexible=flexible, history=True)
    assert res.status == fe.FE_OK
    assert abs(res.iters - ref["iters"]) <= 1
    k = 25
    assert np.allclose(hist[:k, 0], ref["alpha"][:k], rtol=1e-9, atol=0)
    assert np.allclose(hist[:k - 1, 1], ref["beta"][:k - 1], rtol=1e-8, atol=0)
    assert np.allclose(hist[:k, 2], ref["relres"][1:k + 1], rtol=1e-9, atol=0)
    # the iterate is continuous and equals G x_glob of the assembled solve
    xc = x.cpu().numpy()
    xg, gidx = unique_from_cellwise(om, xc)
    assert np.array_equal(xc, xg[gidx])
    assert rel_max_err(xg, ref["x"]) <= 1e-9
    assert oracle_relres(om, bc, xc) <= 1.5e-12


def test_quadratic_solution_reproduced(fe):
    m, p = 4, 2
    om = oracle_mesh(m, p, dirichlet=True)
    for geom in (fe.FE_GEOM_AFFINE, fe.FE_GEOM_STORED):
        gm = fe.Mesh(m, p, geom_mode=geom, dirichlet=True)
        b = torch.from_numpy(O.rhs(om, O.RHS_QUADRATIC)).cuda()
        x = torch.zeros_like(b)
        res = gm.cg_solve(b, x, rtol=1e-13, maxit=1000)
        assert res.status == fe.FE_OK
        uex = O.gather(om, O.exact_nodal(om, O.RHS_QUADRATIC))
        assert np.abs(x.cpu().numpy() - uex).max() <= 1e-11


@pytest.mark.parametrize("p,m", [(2, (6, 5, 4)), (3, (4, 4, 3)), (5, (2, 3, 2))])
def test_mixed_precision_reaches_fp64_residual(fe, p, m):
    om = oracle_mesh(m, p, amp=0.1, dirichlet=True)
    gm = fe.Mesh(m, p, deform_amp=0.1, dirichlet=True)
    bc = O.rhs(om, O.RHS_SINE)
    b = torch.from_numpy(bc).cuda()
    x64 = torch.zeros_like(b)
    r64 = gm.cg_solve(b, x64, rtol=1e-10, maxit=3000)
    x32 = torch.zeros_like(b)
    r32 = gm.cg_solve(b, x32, rtol=1e-10, maxit=3000, mixed=fe.FE_F32)
    # a tight inner tolerance stalls near eps_32 * cond(A); the stagnation guard hands over
    xt = torch.zeros_like(b)
    rt = gm.cg_solve(b, xt, rtol=1e-10, maxit=3000, mixed=fe.FE_F32, inner_rtol=1e-6)
    # FP64 FCG with the FP32 PCG as variable preconditioner
    xf = torch.zeros_like(b)
    rf = gm.cg_solve(b, xf, rtol=1e-10, maxit=3000, mixed=fe.FE_F32, flexible=True)
    assert r64.status == fe.FE_OK and r32.status == fe.FE_OK and rt.status == fe.FE_OK
    assert rf.status == fe.FE_OK and rf.rel_res <= 1e-10
    assert oracle_relres(om, bc, xt.cpu().numpy()) <= 1.2e-10
    assert oracle_relres(om, bc, xf.cpu().numpy()) <= 1.2e-10
    assert r32.outer_iters >= 2 and r32.rel_res <= 1e-10
    assert oracle_relres(om, bc, x64.cpu().numpy()) <= 1.2e-10
    assert oracle_relres(om, bc, x32.cpu().numpy()) <= 1.2e-10
    e64 = O.l2_error(om, x64.cpu().numpy(), O.RHS_SINE)
    e32 = O.l2_error(om, x32.cpu().numpy(), O.RHS_SINE)
    assert abs(e64 - e32) <= 1e-6 * e64


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_mixed_16bit_inner_operator(fe, prec):
    """FP64 FCG preconditioned by an inner PCG whose operator has 16-bit operands and FP32
    accumulation, and FP64 iterative refinement around it: both reach an FP64 residual of 1e-10,
    checked by the oracle from the returned x."""
    m, p = (5, 4, 3), 3
    om = oracle_mesh(m, p, amp=0.1, dirichlet=True)
    gm = fe.Mesh(m, p, deform_amp=0.1, dirichlet=True)
    bc = O.rhs(om, O.RHS_SINE)
    b = torch.from_numpy(bc).cuda()
    code = fe.FE_BF16_F32ACC if prec == "bf16" else fe.FE_F16_F32ACC
    xf = torch.zeros_like(b)
    rf = gm.cg_solve(b, xf, rtol=1e-10, maxit=6000, mixed=code, flexible=True)
    assert rf.status == fe.FE_OK and rf.rel_res <= 1e-10
    assert oracle_relres(om, bc, xf.cpu().numpy()) <= 1.2e-10
    xi = torch.zeros_like(b)
    ri = gm.cg_solve(b, xi, rtol=1e-10, maxit=6000, mixed=code)
    assert ri.status == fe.FE_OK and oracle_relres(om, bc, xi.cpu().numpy()) <= 1.2e-10
    # the FP32 inner operator still works on the same mesh afterwards (inner graphs rebuilt)
    x32 = torch.zeros_like(b)
    r32 = gm.cg_solve(b, x32, rtol=1e-10, maxit=6000, mixed=fe.FE_F32, flexible=True)
    assert r32.status == fe.FE_OK and oracle_relres(om, bc, x32.cpu().numpy()) <= 1.2e-10


def test_cg_statuses(fe):
    m, p = (3, 3, 3), 2
    gm = fe.Mesh(m, p, deform_amp=0.05, dirichlet=True)
    b = torch.from_numpy(S.dual_cellwise(m, p, seed=3)).cuda()
    x = torch.zeros_like(b)
    res = gm.cg_solve(b, x, rtol=1e-14, maxit=3)
    assert res.status == fe.FE_ERR_NOT_CONVERGED and res.iters == 3
    z = torch.zeros_like(b)
    x.fill_(1.0)
    res = gm.cg_solve(z, x, rtol=1e-10, maxit=10)
    assert res.status == fe.FE_OK and res.iters == 0 and float(x.abs().max()) == 0.0
    with pytest.raises(fe.FeError):
        gm.cg_solve(b, x, rtol=1e-10, maxit=0)


def test_cg_reproducible_and_warm_start(fe):
    m, p = (5, 4, 3), 3
    gm = fe.Mesh(m, p, deform_amp=0.1, dirichlet=True)
    b = torch.from_numpy(S.dual_cellwise(m, p, seed=9)).cuda()
    x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
    r1 = gm.cg_solve(b, x1, rtol=1e-11, maxit=2000)
    r2 = gm.cg_solve(b, x2, rtol=1e-11, maxit=2000)
    assert r1.iters == r2.iters and torch.equal(x1, x2)
    r3 = gm.cg_solve(b, x1, rtol=1e-11, maxit=2000)  # already converged start
    assert r3.status == fe.FE_OK and r3.iters <= 2


@pytest.mark.parametrize("p,m,amp", [(1, (3, 2, 4), 0.1), (2, (3, 4, 2), 0.1), (3, (2, 3, 2), 0.0),
                                     (5, (2, 2, 1), 0.15), (7, (1, 2, 1), 0.1)])
def test_rhs_and_l2_error_vs_oracle(fe, p, m, amp):
    om = oracle_mesh(m, p, amp=amp, dirichlet=True)
    gm = fe.Mesh(m, p, deform_amp=amp, dirichlet=True)
    for kind in (O.RHS_SINE, O.RHS_QUADRATIC):
        bref = O.rhs(om, kind)
        b = gm.rhs(kind)
        assert rel_max_err(b.cpu().numpy(), bref) <= 1e-12, kind
        u = S.primal_unique(m, p, seed=4)
        uc = O.gather(om, u)
        e = gm.l2_error(torch.from_numpy(uc).cuda(), kind)
        assert abs(e - O.l2_error(om, uc, kind)) <= 1e-12 * abs(e)


def test_reliable_update_solve_at_48cubed(fe):
    """FP32 PCG with FP64 reliable updates on the deformed Q3 48^3 mesh (sine load): the FP64
    residual of the returned x (formed with the FP64 operator, itself parity-tested against the
    oracle) is below 1e-10, the solution agrees with FP64 PCG's to the solve's accuracy, and the
    FP32 iteration count stays within 1.5x of FP64 PCG's (the kept search direction)."""
    gm = fe.Mesh(48, 3, deform_amp=0.1, dirichlet=True)
    b = gm.rhs(fe.FE_RHS_SINE)
    x64 = torch.zeros_like(b)
    r64 = gm.cg_solve(b, x64, rtol=1e-10, maxit=5000)
    x32 = torch.zeros_like(b)
    r32 = gm.cg_solve(b, x32, rtol=1e-10, maxit=5000, mixed=fe.FE_F32, inner_rtol=0.1)
    assert r64.status == fe.FE_OK and r32.status == fe.FE_OK
    assert r32.rel_res <= 1e-10 and r32.outer_iters >= 2
    assert r32.iters <= 1.5 * r64.iters
    # FP64 residual of the mixed solution, recomputed here: ||G^T (b - A x)|| / ||G^T b|| over the
    # free nodes (the assembled mass of ones vanishes exactly on the Dirichlet nodes)
    free = gm.apply(torch.ones_like(b), op=fe.FE_MASS, flags=fe.FE_ASSEMBLE) != 0
    inv_mult = free / gm.dss(torch.ones_like(b))

    def gnorm(v):
        w = gm.dss(v)
        return float(torch.sqrt((w * w * inv_mult).sum()))

    res = b - gm.apply(x32, op=fe.FE_LAPLACE)
    assert gnorm(res) / gnorm(b) <= 1.05e-10
    assert float((x32 - x64).abs().max()) <= 1e-8 * float(x64.abs().max())
    e64, e32 = gm.l2_error(x64), gm.l2_error(x32)
    assert abs(e64 - e32) <= 1e-6 * e64


@pytest.mark.parametrize("scale", [1e-300, 1e-30, 1e30, 1e300])
@pytest.mark.parametrize("scheme", ["fp64", "mixed", "fcg"])
def test_badly_scaled_rhs(fe, scheme, scale):
    """A right-hand side far from unit size solves like the unscaled one (solution scaled, same
    iteration count up to a few): the solver scales the system by an exact power of two, so the
    double-word pairings (FP32's exponent range) neither overflow nor flush."""
    m, p = (6, 5, 4), 3
    gm = fe.Mesh(m, p, deform_amp=0.1, dirichlet=True)
    b = gm.rhs(fe.FE_RHS_SINE)
    mixed = 0 if scheme == "fp64" else fe.FE_F32
    out = {}
    for sc in (1.0, scale):
        x = torch.zeros_like(b)
        r = gm.cg_solve(b * sc, x, rtol=1e-10, maxit=2000, mixed=mixed,
                        flexible=(scheme == "fcg"), inner_rtol=0.1)
        assert r.status == fe.FE_OK and r.iters > 0 and r.rel_res <= 1e-10, (sc, r.iters)
        out[sc] = (r.iters, x.cpu().numpy() / sc)
    assert abs(out[scale][0] - out[1.0][0]) <= max(3, out[1.0][0] // 20)
    assert rel_max_err(out[scale][1], out[1.0][1]) <= 1e-8


def test_batched_badly_scaled_rhs(fe):
    """Each problem of a batch is scaled by its own power of two."""
    meshes = [fe.Mesh(5, 2, deform_amp=0.05, dirichlet=True), fe.Mesh(4, 3, dirichlet=True)]
    scales = [1e-200, 1e200]
    for mixed in (0, fe.FE_F32):
        opts = fe.fe_cg_opts(1e-10, 2000, mixed, 0, 0.1, None)
        bs = [m.rhs(fe.FE_RHS_SINE) for m in meshes]
        xs = [torch.zeros_like(b) for b in bs]
        ref = fe.fe_cg_solve_batched([m.handle for m in meshes], bs, xs, opts)
        xr = [x.cpu().numpy() for x in xs]
        bs2 = [b * s for b, s in zip(bs, scales)]
        xs2 = [torch.zeros_like(b) for b in bs2]
        res = fe.fe_cg_solve_batched([m.handle for m in meshes], bs2, xs2, opts)
        for r0, r1, x0, x1, s in zip(ref, res, xr, xs2, scales):
            assert r1.status == fe.FE_OK and r1.iters > 0, (mixed, s)
            assert abs(r1.iters - r0.iters) <= 3
            assert rel_max_err(x1.cpu().numpy() / s, x0) <= 1e-8


def test_nonfinite_rhs_is_rejected(fe):
    gm = fe.Mesh(3, 2, dirichlet=True)
    b = gm.rhs(fe.FE_RHS_SINE)
    b[5] = float("inf")
    with pytest.raises(fe.FeError) as e:
        gm.cg_solve(b, torch.zeros_like(b), rtol=1e-10)
    assert e.value.status == fe.FE_ERR_INVALID
