"""Request server with continuous batching: results are bitwise the same served alone and in a
mix, agree with the single-problem solver, memory budget and slot limits hold, and latency
statistics are reported."""
import time

import numpy as np
import pytest

import oracle as O
from paper_2607_02335_gb300 import synth as S
from tests.helpers import oracle_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (cells, degree, amplitude, mixed, explicit rhs)
REQS = [((4, 4, 4), 2, 0.1, 0, False), ((3, 3, 3), 3, 0.05, 1, False), ((2, 2, 2), 7, 0.1, 1, True),
        ((5, 4, 3), 2, 0.0, 0, True), ((3, 2, 2), 5, 0.12, 1, False), ((2, 3, 2), 3, 0.0, 0, False),
        ((6, 4, 4), 2, 0.08, 1, False)]


@pytest.fixture(scope="module")
def fe():
    from paper_2607_02335_gb300 import fe as F
    return F


def desc_of(fe, m, p, amp):
    mx, my, mz = m
    geom = fe.FE_GEOM_AFFINE if amp == 0 else fe.FE_GEOM_STORED
    return fe.fe_mesh_desc(mx, my, mz, p, amp, geom, 1, 0)


def rhs_of(i, m, p, explicit):
    return S.dual_cellwise(m, p, seed=200 + i) if explicit else None


def run_server(fe, idx, budget=8 << 30, slots=4):
    srv = fe.fe_serve_create(budget, slots, 0)
    tickets = {}
    for i in idx:
        m, p, amp, mixed, explicit = REQS[i]
        opts = fe.fe_cg_opts(1e-10, 4000, fe.FE_F32 if mixed else 0, 1 if mixed else 0, 1e-2, None)
        tickets[i] = fe.fe_serve_submit(srv, desc_of(fe, m, p, amp), rhs_of(i, m, p, explicit), opts)
    out = {}
    t0 = time.time()
    while len(out) < len(idx):
        for i, t in tickets.items():
            if i in out:
                continue
            m, p, amp, mixed, explicit = REQS[i]
            x = np.zeros(m[0] * m[1] * m[2] * (p + 1) ** 3)
            r = fe.fe_serve_poll(srv, t, x)
            if r is not None:
                out[i] = (r, x)
        assert time.time() - t0 < 120, "server did not finish"
        time.sleep(0.001)
    stats = fe.fe_serve_stats(srv)
    fe.fe_serve_destroy(srv)
    return out, stats


def test_serve_same_alone_and_in_mix(fe):
    idx = list(range(len(REQS)))
    mix, (p50, p99, sps) = run_server(fe, idx, slots=3)
    assert all(mix[i][0].status == fe.FE_OK for i in idx), [mix[i][0].status for i in idx]
    assert all(mix[i][0].rel_res <= 1e-10 for i in idx)
    assert 0 < p50 <= p99 and sps > 0
    for i in idx:
        alone, _ = run_server(fe, [i])
        assert np.array_equal(alone[i][1], mix[i][1]), i
        assert alone[i][0].iters == mix[i][0].iters


def test_serve_matches_single_solver_and_oracle(fe):
    idx = [0, 1, 2]
    mix, _ = run_server(fe, idx)
    for i in idx:
        m, p, amp, mixed, explicit = REQS[i]
        gm = fe.Mesh(m, p, deform_amp=amp, geom_mode=fe.FE_GEOM_AFFINE if amp == 0 else fe.FE_GEOM_STORED,
                     dirichlet=True)
        b = torch.from_numpy(rhs_of(i, m, p, explicit)).cuda() if explicit else gm.rhs(fe.FE_RHS_SINE)
        x = torch.zeros_like(b)
        r = gm.cg_solve(b, x, rtol=1e-10, maxit=4000, mixed=fe.FE_F32 if mixed else 0, flexible=bool(mixed))
        assert r.status == fe.FE_OK
        xs = x.cpu().numpy()
        assert np.abs(xs - mix[i][1]).max() <= 1e-8 * np.abs(xs).max()
        om = oracle_mesh(m, p, amp=amp, dirichlet=True)
        bc = b.cpu().numpy()
        gidx = O.gather(om, np.arange(om.n_unique, dtype=np.float64)).astype(np.int64)
        xg = np.zeros(om.n_unique)
        xg[gidx] = mix[i][1]
        bg = O.scatter(om, bc)
        bg[O.boundary_global(om)] = 0.0
        res = bg - O.apply_dirichlet_csr(om, O.assemble_csr(om, O.LAPLACE), xg)
        assert np.linalg.norm(res) / np.linalg.norm(bg) <= 1.2e-10


def test_serve_budget_slots_and_errors(fe):
    srv = fe.fe_serve_create(64 << 20, 1, 0)  # 64 MiB, one slot
    opts = fe.fe_cg_opts(1e-10, 4000, 0, 0, 1e-2, None)
    with pytest.raises(fe.FeError) as e:
        fe.fe_serve_submit(srv, fe.fe_mesh_desc(32, 32, 32, 3, 0.1, 0, 1, 0), None, opts)
    assert e.value.status == fe.FE_ERR_OOM
    with pytest.raises(fe.FeError):
        fe.fe_serve_poll(srv, 12345)
    ts = [fe.fe_serve_submit(srv, desc_of(fe, (3, 3, 3), 2, 0.1), None, opts) for _ in range(4)]
    done = {}
    t0 = time.time()
    while len(done) < len(ts):
        for t in ts:
            if t not in done:
                r = fe.fe_serve_poll(srv, t)
                if r is not None:
                    done[t] = r
        assert time.time() - t0 < 60
    assert all(r.status == fe.FE_OK for r in done.values())
    # identical requests give identical iteration counts
    assert len({r.iters for r in done.values()}) == 1
    fe.fe_serve_destroy(srv)
