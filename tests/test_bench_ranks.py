"""Host logic of bench.py on CPU: the multi-GPU path (replicas, weak scaling) on two gloo
processes, where the slowest rank's time sets the job time and the rate counts every rank's units;
and the reference arm's JSON line."""
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


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the CPU oracle and prints one JSON line with the keys the
    contract names (no GPU involved)."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                       timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    for key in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "config", "dtype"):
        assert key in line, key
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_unknown_extra_blocks_are_rejected():
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--extras", "serving,bogus"],
                       capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert r.returncode != 0 and "bogus" in r.stderr


def test_committed_profile_belongs_to_the_committed_kernels():
    """profiles/traffic.txt was captured from the kernel sources in the tree (the bench reports
    its traffic and instruction figures only then), and the issue roofline built from it is a
    fraction of the issue peak for the kernel time the bench measures."""
    b = _bench()
    d = b.committed_profile()
    assert d, "profiles/traffic.txt is stale: recapture it for the current kernel sources"
    assert b.committed_traffic() == int(d["bytes_per_launch"])
    per_dof = float(d["warp_instructions_per_cellwise_dof"])
    assert per_dof == pytest.approx(float(d["warp_instructions"]) / 7077888, rel=1e-4)
    r = b.issue_roofline(1.385, 56623104)  # Q3 96^3 Laplace volumetric, its measured time
    assert r is not None and 0.5 < r["frac"] < 1.05
    assert r["achieved"] == pytest.approx(per_dof * 56623104 / 1.385e-3 / 1e12, rel=1e-3)


def test_profile_commands_run_with_the_committed_bench(monkeypatch):
    """Every profiler summary under profiles/ names the command that made it: an ncu run with
    --clock-control none over `python bench.py ...` arguments that the committed bench.py still
    accepts (a stale summary would cite a command that no longer runs)."""
    import glob
    import re
    import shlex
    import sys
    b = _bench()
    paths = sorted(glob.glob(os.path.join(ROOT, "profiles", "*")))
    assert paths
    checked = 0
    for path in paths:
        text = open(path).read().replace("\\\n", " ")
        cmds = [ln for ln in text.splitlines() if re.search(r"\bncu\s+-", ln) and "bench.py" in ln]
        assert cmds, f"{os.path.basename(path)} gives no ncu command over bench.py"
        for cmd in cmds:
            assert "--clock-control none" in cmd, (path, cmd)
            words = shlex.split(cmd[cmd.index("bench.py"):])
            monkeypatch.setattr(sys, "argv", words)
            args = b.parse()
            if args.profile_case:
                parts = args.profile_case.split(",")
                assert int(parts[0]) in range(1, 8) and int(parts[1]) > 0
                assert parts[2] in ("laplace", "mass")
                assert len(parts) < 4 or parts[3] == "vol"
                assert len(parts) < 5 or parts[4] in ("f64", "f32", "bf16", "fp16")
            checked += 1
    assert checked >= len(paths)
