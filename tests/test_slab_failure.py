"""Host logic of the slab communicators on CPU, failures included: thread-driven slabs exchange
planes and gather scalars exactly as include/fe.h specifies; a slab that never reaches the exchange
(a dead thread, a rank that left) turns into an error status of the waiting slabs' callbacks after
a bounded wait, never a hang.  The library maps a non-zero callback return to FE_ERR_COMM."""
import datetime
import os
import socket
import threading
import time

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _run_threads(n, fn):
    out, errs = [None] * n, [None] * n

    def body(r):
        try:
            out[r] = fn(r)
        except BaseException as e:  # noqa: BLE001
            errs[r] = e

    th = [threading.Thread(target=body, args=(r,)) for r in range(n)]
    for t in th:
        t.start()
    for t in th:
        t.join(60)
        assert not t.is_alive()
    return out, errs


def test_thread_slabs_exchange_and_gather_on_cpu():
    from paper_2607_02335_gb300.slab import ThreadSlabGroup
    n, plen = 4, 50
    g = ThreadSlabGroup(n, timeout=10)
    comms = [g.comm(r, plen, "cpu") for r in range(n)]

    def work(r):
        c = comms[r]
        for s in (0, 1):
            if c.has[s]:
                c.send[s].copy_(torch.arange(plen, dtype=torch.float64) + 1000 * r + 100 * s)
        sides = (1 if c.has[0] else 0) | (2 if c.has[1] else 0)
        assert c._exchange_cb(None, sides, 8, plen, None) == 0
        c.red_send[:3] = torch.tensor([r, 2.0 * r, -r], dtype=torch.float64)
        assert c._allgather_cb(None, 3, None) == 0
        return [c.recv[s].clone() if c.has[s] else None for s in (0, 1)], c.red_all[:3 * n].clone()

    out, errs = _run_threads(n, work)
    assert all(e is None for e in errs)
    base = torch.arange(plen, dtype=torch.float64)
    for r in range(n):
        recv, gathered = out[r]
        if r > 0:  # from below: the lower slab's top plane (its side 1)
            assert torch.equal(recv[0], base + 1000 * (r - 1) + 100)
        if r < n - 1:  # from above: the upper slab's bottom plane (its side 0)
            assert torch.equal(recv[1], base + 1000 * (r + 1))
        want = torch.tensor([v for k in range(n) for v in (k, 2.0 * k, -k)], dtype=torch.float64)
        assert torch.equal(gathered, want)


def test_thread_slab_that_never_arrives_is_an_error_not_a_hang():
    from paper_2607_02335_gb300.slab import ThreadSlabGroup
    g = ThreadSlabGroup(2, timeout=1.0)
    comms = [g.comm(r, 8, "cpu") for r in range(2)]
    t0 = time.time()
    # slab 1 has died before its exchange: slab 0 waits at most the barrier's timeout
    assert comms[0]._exchange_cb(None, 2, 8, 8, None) == 1
    assert comms[0].error is not None
    assert time.time() - t0 < 10
    # the group is broken for everyone afterwards: the next call fails at once
    assert comms[1]._allgather_cb(None, 3, None) == 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=2,
                                         timeout=datetime.timedelta(seconds=3))
    from paper_2607_02335_gb300.slab import DistSlabComm
    c = DistSlabComm(16, "cpu")
    if rank == 1:
        out[1] = "left"  # this rank leaves between steps, before the exchange
        os._exit(0)
    t0 = time.time()
    status = c._exchange_cb(None, 2, 8, 16, None)
    out[0] = (status, type(c.error).__name__ if c.error else None, time.time() - t0)
    os._exit(0)


def test_rank_that_left_surfaces_as_a_callback_error():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    status, err, waited = res[0]
    assert res[1] == "left"
    assert status == 1 and err is not None
    assert waited < 60
