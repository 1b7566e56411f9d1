"""Host logic of the multi-GPU bench path (replicas, weak scaling) on CPU ranks: two gloo
processes, the slowest rank's time sets the job time and the rate counts every rank's units."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    local_ms = 10.0 * (rank + 1)  # rank 1 is the slow one
    total_ms = b.max_over_ranks(local_ms, world, "cpu")
    rate = b.job_rate(1_000_000, 4, world, total_ms * 1e-3)
    out[rank] = (total_ms, rate)
    torch.distributed.barrier()
    torch.distributed.destroy_process_group()


def test_two_rank_timing_takes_the_slowest_and_counts_all_units():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    total_ms, rate = res[0]
    assert total_ms == 20.0
    assert rate == pytest.approx(1_000_000 * 2 * 4 / 0.020 / 1e9)


def test_single_rank_needs_no_process_group():
    b = _bench()
    assert b.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert b.job_rate(10, 2, 1, 1.0) == pytest.approx(2e-8)
