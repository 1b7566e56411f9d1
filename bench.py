"""Throughput benchmark of the cell-wise matrix-free operator apply on GB300.

Workload (one "step"): the FP64 operator sweep on deformed unit-cube meshes
(x + 0.1 sin(pi x) sin(pi y) sin(pi z) per coordinate, stored per-quadrature-point geometry):
Laplace and mass at Q2 on 48^3 cells, Q3 on 96^3 cells and Q7 on 32^3 cells, each applied with
the shared-node summation (FE_ASSEMBLE), i.e. six assembled operator applications.  Inputs are
drawn per unique node (seed 0) and gathered to cell-wise storage.  value = unique DoFs processed
per second (GDoF/s) over the whole step.  L2 is flushed (a 512 MB write) before every timed step.

`python bench.py --gpus N --steps K --warmup W [--impl reference]`; N > 1 runs under torchrun,
one independent replica per GPU (weak scaling).  `--impl reference` times the FP64 CPU oracle on
the host cores on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# the oracle's OpenMP threads stay on their cores while it is timed (read when its runtime starts)
os.environ.setdefault("OMP_PROC_BIND", "close")
os.environ.setdefault("OMP_PLACES", "cores")

SWEEP = [(2, 48), (3, 96), (7, 32)]  # (degree, cells per direction)
AMP = 0.1
METRIC = "Operator-apply GDoF/s (unique DoFs, FP64, FE_ASSEMBLE) over the Q2/Q3/Q7 sweep"
UNIT = "GDoF/s"
GEO_BYTES = {0: 48, 1: 8}  # stored geometry bytes per cell-wise DoF: Laplace 6 doubles, mass 1
FP64_PIPE_TFLOPS = 0.98   # FP64 FMA rate probed on a pool GB300 (0.49 T FMA/s), for context


EXTRAS = ("geometry_recompute", "reduced_precision_apply", "block_structured_dss", "packed_storage",
          "hanging_node_dss", "slab_decomposition", "solve_mixed_vs_fp64", "batched", "serving")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--small", action="store_true", help="tiny sizes (plumbing check only)")
    ap.add_argument("--batch-count", type=int, default=256, help="problems of the batched solve")
    ap.add_argument("--serve-requests", type=int, default=200, help="requests per serving run")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrival rate (1/s)")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--serve-slots", type=int, default=256)
    ap.add_argument("--serve-cap-s", type=float, default=60.0, help="wall-time cap per serving run")
    ap.add_argument("--no-extras", action="store_true", help="operator sweep only")
    ap.add_argument("--extras", default="all",
                    help="comma list of extra blocks to run (default all): geometry_recompute, "
                         "reduced_precision_apply, block_structured_dss, packed_storage, "
                         "hanging_node_dss, slab_decomposition, solve_mixed_vs_fp64, batched, "
                         "serving")
    ap.add_argument("--profile-batched", type=int, default=0,
                    help="N: only run the batched mixed solve of the first N problems of the "
                         "batched workload, untimed (for profiler captures)")
    ap.add_argument("--profile-solve", default=None, choices=["fp64", "mixed"],
                    help="only run one solve of the Q3 64^3 Poisson problem of the "
                         "solve_mixed_vs_fp64 block (FP64 PCG, or FP32 PCG with FP64 reliable "
                         "updates), untimed (for profiler captures)")
    ap.add_argument("--profile-case", default=None,
                    help="p,m,op[,vol[,f64|f32|bf16|fp16]]: only run K+W applies of one case "
                         "(for profiler captures)")
    args = ap.parse_args()
    if args.extras != "all":
        unknown = set(args.extras.split(",")) - set(EXTRAS)
        if unknown:
            ap.error(f"unknown extra blocks: {', '.join(sorted(unknown))}")
    return args


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks sampling
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id, self.lines, self.proc = gpu_id, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle timing
SAMPLE_CELLS = {2: 8192, 3: 2048, 7: 16}


class OracleSampler:
    """The oracle's element-by-element FP64 apply (element matrices precomputed, OpenMP over
    cells) on a bounded sample of cells of every (op, degree) of the sweep."""

    def __init__(self, threads: int):
        import oracle as O
        from paper_2607_02335_gb300 import synth as S

        self.O, self.threads, self.items = O, threads, []
        for p, m in SWEEP:
            mesh = O.Mesh(m, p, amp=AMP)
            nc, n3 = SAMPLE_CELLS[p], (p + 1) ** 3
            xc = S.dual_cellwise(m, p, seed=0)[: nc * n3].copy()
            for op in (O.LAPLACE, O.MASS):
                mats = O.element_matrices(mesh, op, 0, nc, nthreads=threads)
                self.items.append(dict(op=op, p=p, mesh=mesh, mats=mats, xc=xc, ncw=nc * n3, ts=[]))

    def time_once(self):
        for it in self.items:
            t0 = time.perf_counter()
            self.O.apply_local_mats(it["mesh"], 0, it["mats"], it["xc"], nthreads=self.threads)
            it["ts"].append(time.perf_counter() - t0)

    def reset(self):
        for it in self.items:
            it["ts"] = []

    def sample_seconds(self):
        """Median time of one pass over the sample (every item once)."""
        return sum(float(np.median(it["ts"])) for it in self.items)

    def full_step_estimate(self):
        """(seconds, unique DoFs) of one full step extrapolated from the median per-cell-DoF rates."""
        t, nu = 0.0, 0
        for it in self.items:
            m = dict(SWEEP)[it["p"]]
            rate = float(np.median(it["ts"])) / it["ncw"]
            t += rate * m ** 3 * (it["p"] + 1) ** 3
            nu += (m * it["p"] + 1) ** 3
        return t, nu

    def describe(self):
        return (f"element-by-element FP64 apply with precomputed element matrices on the first "
                f"{SAMPLE_CELLS} cells (per degree) of each sweep mesh, Laplace and mass; median "
                f"of the timed passes per item, rates scaled to the full step (DSS not included); "
                f"OpenMP threads bound to cores")


def csr_spmv_baseline(threads, p=2, m=48, reps=10):
    """The oracle's assembled CSR matrix of the Q2 48^3 deformed Laplace (about 1.1e8 nonzeros)
    and its OpenMP SpMV on the host cores: the sparse-matrix baseline of the unique-DoF rate."""
    import oracle as O
    from paper_2607_02335_gb300 import synth as S
    mesh = O.Mesh(m, p, amp=AMP)
    t0 = time.perf_counter()
    csr = O.assemble_csr(mesh, O.LAPLACE, nthreads=threads)
    t_asm = time.perf_counter() - t0
    x = S.primal_unique(m, p, seed=0)
    O.csr_spmv(csr, x)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        O.csr_spmv(csr, x)
        ts.append(time.perf_counter() - t0)
    t = float(np.median(ts))
    return {"mesh": f"Q{p} {m}^3 deformed (amp {AMP}), Laplace A_CG in CSR (oracle assembly)",
            "nnz": int(len(csr[2])), "unique_dofs": mesh.n_unique, "assembly_s": round(t_asm, 3),
            "spmv_ms": round(t * 1e3, 3), "gdofs_unique": round(mesh.n_unique / t / 1e9, 4),
            "cores": threads}


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank):
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    t_all = time.perf_counter()
    smp = OracleSampler(threads)
    for _ in range(args.warmup):
        smp.time_once()
    smp.reset()
    for _ in range(args.steps):
        smp.time_once()
    t_step, nu = smp.full_step_estimate()
    value = nu / t_step / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        # a step here is one timed pass over the bounded sample; the full sweep's time is estimated
        "ms_per_step": round(smp.sample_seconds() * 1e3, 3),
        "full_step_estimate_ms": round(t_step * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "FP64 operator sweep, deformed unit cube (amp 0.1), stored geometry, "
                               "Laplace+mass at Q2/48^3, Q3/96^3, Q7/32^3, FE_ASSEMBLE",
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": smp.describe()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": round(time.perf_counter() - t_all, 2),
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("fe_apply_kernel.cuh", "fe_arith.h", "fe_apply_launch.cuh"):
        with open(os.path.join(ROOT, "paper_2607_02335_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_profile():
    """The committed ncu figures of the roofline kernel (profiles/traffic.txt), or {} when the
    kernel sources changed after the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return {}
    d = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                d[k.strip()] = v.strip()
    return d if d.get("source_sha") == kernel_source_sha() else {}


def committed_traffic():
    """dram read + write bytes per launch of the roofline kernel from the committed ncu summary,
    or None when the kernel sources changed after the capture."""
    d = committed_profile()
    return int(d["bytes_per_launch"]) if "bytes_per_launch" in d else None


def issue_roofline(kernel_ms, cellwise_dofs):
    """The roofline kernel against the SMs' instruction issue: warp instructions per cell-wise DoF
    from the committed ncu capture, times the DoFs of the timed launch, over the CUDA-event time,
    against 152 SMs x 4 schedulers x one warp instruction per clock at the maximum SM clock."""
    d = committed_profile()
    if "warp_instructions_per_cellwise_dof" not in d:
        return None
    per_dof = float(d["warp_instructions_per_cellwise_dof"])
    mhz = 2070.0
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    achieved = per_dof * cellwise_dofs / (kernel_ms * 1e-3) / 1e12
    peak = 152 * 4 * mhz * 1e6 / 1e12
    return {"unit": "T warp-instructions/s", "achieved": round(achieved, 4), "peak": round(peak, 4),
            "frac": round(achieved / peak, 4), "warp_instructions_per_cellwise_dof": per_dof,
            "note": "the kernel is bound by instruction issue (double-word FP64 arithmetic on the "
                    "FP32 pipe); frac is its share of the issue peak"}


def max_over_ranks(x, world, device):
    """The largest value of x over the ranks of the job (the slowest replica sets the time)."""
    if world <= 1:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank_step, steps, world, seconds):
    """Whole-job GDoF/s: every rank processes units_per_rank_step per step (weak scaling)."""
    return units_per_rank_step * world * steps / seconds / 1e9


def run_ours(args, rank, world):
    import torch

    from paper_2607_02335_gb300 import fe
    from paper_2607_02335_gb300 import synth as S

    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    sweep = [(2, 6), (3, 6), (7, 3)] if args.small else SWEEP
    cases = []  # (mesh, x, y, op, p, m)
    meshes = []
    for p, m in sweep:
        gm = fe.Mesh(m, p, deform_amp=AMP, device=dev)
        x = gm.gather(S.primal_unique(m, p, seed=0))
        meshes.append((gm, x, p, m))
        for op in (fe.FE_LAPLACE, fe.FE_MASS):
            cases.append((gm, x, gm.empty(fe.FE_F64), op, p, m))
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)

    def step():
        for gm, x, y, op, p, m in cases:
            fe.fe_apply(gm.handle, op, fe.FE_F64, x, y, fe.FE_ASSEMBLE, stream)

    units_per_step = sum(gm.unique_dofs for gm, _, _, _, _, _ in cases)
    launches_per_step = len(cases) * 4  # volumetric kernel + 3 DSS axis passes
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    gpu_id = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    sampler = ClockSampler(f"GPU-{gpu_id}" if gpu_id else str(dev))
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    value = job_rate(units_per_step, args.steps, world, total_ms * 1e-3)

    # per-case breakdown: assembled apply and the volumetric kernel alone; 5 warm-ups, then the
    # median of 20 reps with L2 flushed before each, and of 20 reps without the flush
    peak, peak_kind = load_peaks()
    reps = 20
    per_case = []

    def rep_median(gm, x, y, op, flags, flushed):
        for _ in range(5):
            fe.fe_apply(gm.handle, op, fe.FE_F64, x, y, flags, stream)
        ts = []
        for _ in range(reps):
            if flushed:
                flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fe.fe_apply(gm.handle, op, fe.FE_F64, x, y, flags, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    for gm, x, y, op, p, m in cases:
        res = {}
        for flags, key in ((fe.FE_ASSEMBLE, "assembled_ms"), (0, "volumetric_ms")):
            res[key] = rep_median(gm, x, y, op, flags, True)
            res[key + "_unflushed"] = rep_median(gm, x, y, op, flags, False)
        # the same operator on the FP64 pipe (the cross-check arithmetic, also within 1e-12)
        res["native_fp64_volumetric_ms"] = rep_median(gm, x, y, op, fe.FE_NATIVE_F64, True)
        ncw, n = gm.cellwise_len, p + 1
        alg_bytes = ncw * (16 + GEO_BYTES[op])
        vol_gbs = alg_bytes / (res["volumetric_ms"] * 1e-3) / 1e9
        # FP64 flops per cell-wise DoF of the plain formulation (no even-odd): Laplace 24n+17,
        # mass 12n+1; the FP64-equivalent rate against the FP64 pipe's measured FMA rate
        flops = ncw * ((24 * n + 17) if op == fe.FE_LAPLACE else (12 * n + 1))
        fp64_tf = flops / (res["volumetric_ms"] * 1e-3) / 1e12
        per_case.append({
            "op": "laplace" if op == fe.FE_LAPLACE else "mass", "degree": p, "cells": f"{m}^3",
            "cellwise_dofs": ncw, "unique_dofs": gm.unique_dofs,
            "assembled_ms": round(res["assembled_ms"], 4), "volumetric_ms": round(res["volumetric_ms"], 4),
            "assembled_ms_unflushed": round(res["assembled_ms_unflushed"], 4),
            "volumetric_ms_unflushed": round(res["volumetric_ms_unflushed"], 4),
            "gdofs_unique_assembled": round(gm.unique_dofs / (res["assembled_ms"] * 1e-3) / 1e9, 3),
            "gdofs_cellwise_assembled": round(ncw / (res["assembled_ms"] * 1e-3) / 1e9, 3),
            "gdofs_cellwise_volumetric": round(ncw / (res["volumetric_ms"] * 1e-3) / 1e9, 3),
            "volumetric_alg_bytes": alg_bytes, "volumetric_gbs": round(vol_gbs, 1),
            "volumetric_hbm_frac": round(vol_gbs / peak, 4),
            "fp64_equiv_tflops": round(fp64_tf, 3),
            "vs_fp64_pipe_peak": round(fp64_tf / FP64_PIPE_TFLOPS, 2),
            "native_fp64_volumetric_ms": round(res["native_fp64_volumetric_ms"], 4),
            "native_fp64_hbm_frac": round(alg_bytes / (res["native_fp64_volumetric_ms"] * 1e-3) / 1e9 / peak, 4),
        })
    dom = max(per_case, key=lambda c: c["volumetric_ms"])
    achieved = dom["volumetric_gbs"]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": committed_traffic(),
                "kernel": f"k_apply<{dom['degree'] + 1},dw,{dom['op']},stored>",
                "peak_source": f"{peak_kind} hbm_gbs (burst copy)",
                "alg_bytes_per_launch": dom["volumetric_alg_bytes"],
                "issue": issue_roofline(dom["volumetric_ms"], dom["cellwise_dofs"])}

    # end to end through the C ABI with host buffers: every step copies each mesh's input in and
    # both operators' outputs out, as unique-node vectors (fe_apply_host: the cell-wise expansion
    # and the selection of one copy per node run on the device).  One stream per mesh; the
    # read-backs of a call overlap its next apply and the other meshes' work.
    hx, hy = {}, {}
    for gm, x, p, m in meshes:
        hx[id(gm)] = torch.from_numpy(S.primal_unique(m, p, seed=0)).pin_memory()
        hy[id(gm)] = [torch.empty(gm.unique_dofs, dtype=torch.float64).pin_memory()
                      for _ in range(2)]
    h2d = sum(gm.unique_dofs * 8 for gm, *_ in meshes)
    d2h = sum(gm.unique_dofs * 8 for gm, *_ in cases)
    e2e_steps = max(3, min(args.steps, 20))
    e2e_streams = {id(gm): torch.cuda.Stream() for gm, *_ in meshes}
    # the small meshes first: the large Q3 input then arrives while they compute
    e2e_meshes = sorted(meshes, key=lambda t: t[0].unique_dofs)
    ops = [fe.FE_LAPLACE, fe.FE_MASS]
    for gm, *_ in e2e_meshes:  # first call allocates the staging
        fe.fe_apply_host(gm.handle, ops, hx[id(gm)], hy[id(gm)], 0, e2e_streams[id(gm)])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for gm, *_ in e2e_meshes:
            fe.fe_apply_host(gm.handle, ops, hx[id(gm)], hy[id(gm)], 0, e2e_streams[id(gm)])
        torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, dev)
    e2e_value = job_rate(units_per_step, 1, world, e2e_s)

    extras = {}
    if not args.small and not args.no_extras:
        for gm, *_ in meshes:
            gm.close()
        del cases, meshes
        torch.cuda.empty_cache()
        want = None if args.extras == "all" else set(args.extras.split(","))

        def run(name, fn):
            if want is None or name in want:
                extras[name] = fn()

        run("geometry_recompute",
            lambda: recompute_geometry(fe, torch, sweep, per_case, flush, stream, reps))
        run("reduced_precision_apply", lambda: reduced_precision_apply(fe, torch, flush, stream))
        run("block_structured_dss", lambda: multiblock_dss(fe, torch, flush, stream))
        run("packed_storage", lambda: packed_storage(fe, torch, flush, stream))
        run("hanging_node_dss", lambda: hanging_node_dss(fe, torch, flush, stream))
        run("slab_decomposition", lambda: slab_decomposition(fe, torch, flush, stream))
        run("solve_mixed_vs_fp64", lambda: mixed_vs_fp64_solve(fe, torch))
        run("batched", lambda: batched_solve(fe, torch, count=args.batch_count))
        run("serving", lambda: serving_block(fe, args))

    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "FP64 operator sweep, deformed unit cube (amp 0.1), stored geometry, "
                               "Laplace+mass at " + ", ".join(f"Q{p}/{m}^3" for p, m in sweep)
                               + ", FE_ASSEMBLE (volumetric apply + structured DSS)",
                   "l2": "flushed (512 MB write) before every timed step",
                   "arithmetic": "FP64 to 1e-12 of the oracle: double-word (hi+lo float) on the FP32 "
                                 "pipe, binary64 inputs differenced before any rounding, FP64 I/O",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "per_case": per_case,
        "roofline": roofline,
        "e2e": {"value": round(e2e_value, 4), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        **extras,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        smp = OracleSampler(threads)
        smp.time_once()
        smp.reset()
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 10.0 or len(smp.items[0]["ts"]) < 5:
            smp.time_once()
        t_cpu, nu = smp.full_step_estimate()
        line["cpu_baseline"] = {"value": round(nu / t_cpu / 1e9, 6), "unit": UNIT, "cores": threads,
                                "kind": "oracle", "sample": smp.describe(),
                                "passes": len(smp.items[0]["ts"])}
        smp.threads = 1  # the same sample on one core, one pass
        smp.reset()
        smp.time_once()
        t1, _ = smp.full_step_estimate()
        line["cpu_baseline"]["value_1core"] = round(nu / t1 / 1e9, 6)
        line["cpu_baseline"]["csr_spmv"] = csr_spmv_baseline(threads)
    if rank == 0:
        print(json.dumps(line), flush=True)


def recompute_geometry(fe, torch, sweep, per_case, flush, stream, reps):
    """The operator sweep with the metric recomputed from cell-wise nodal coordinates (double-word
    coordinates, 24 B per cell-wise DoF, instead of the stored metric): volumetric and assembled
    time per case, next to the stored-metric time of the same case."""
    from paper_2607_02335_gb300 import synth as S

    stored = {(c["degree"], c["op"]): c for c in per_case}
    out = []
    for p, m in sweep:
        gm = fe.Mesh(m, p, deform_amp=AMP, geom_mode=fe.FE_GEOM_RECOMPUTE)
        x = gm.gather(S.primal_unique(m, p, seed=0))
        y = gm.empty(fe.FE_F64)
        for op in (fe.FE_LAPLACE, fe.FE_MASS):
            name = "laplace" if op == fe.FE_LAPLACE else "mass"
            res = {}
            for flags, key in ((fe.FE_ASSEMBLE, "assembled_ms"), (0, "volumetric_ms")):
                fe.fe_apply(gm.handle, op, fe.FE_F64, x, y, flags, stream)
                tot = 0.0
                for _ in range(reps):
                    flush.fill_(1.0)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    fe.fe_apply(gm.handle, op, fe.FE_F64, x, y, flags, stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    tot += e0.elapsed_time(e1)
                res[key] = tot / reps
            ncw = gm.cellwise_len
            st = stored[(p, name)]
            out.append({
                "op": name, "degree": p, "cells": f"{m}^3",
                "assembled_ms": round(res["assembled_ms"], 4),
                "volumetric_ms": round(res["volumetric_ms"], 4),
                "gdofs_unique_assembled": round(gm.unique_dofs / (res["assembled_ms"] * 1e-3) / 1e9, 3),
                "volumetric_hbm_bytes_per_cellwise_dof": 16 + 24,
                "stored_volumetric_ms": st["volumetric_ms"],
                "time_vs_stored": round(res["volumetric_ms"] / st["volumetric_ms"], 3)})
        del x, y
        gm.close()
    return out


def hanging_node_dss(fe, torch, flush, stream, reps=20):
    """DSS with hanging nodes (shadow cells) on a 48^3 coarse grid whose central 24^3 cells are
    refined (48^3 fine cells), p = 1..5, per unique DoF of the conforming space, next to the
    structured DSS of the same number of cells (Appendix, Table "tab:dss_adaptive")."""
    out = {"workload": "coarse 48^3, box [12,36)^3 refined 2x2x2 (48^3 fine cells), FP64"}
    rows = []
    for p in (1, 2, 3, 4, 5):
        am = fe.AMRMesh(48, (12, 12, 12), (36, 36, 36), p)
        r = torch.randn(am.cellwise_len, dtype=torch.float64, device="cuda")
        z = am.empty()
        fe.fe_amr_dss(am.handle, fe.FE_F64, r, z, stream)
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fe.fe_amr_dss(am.handle, fe.FE_F64, r, z, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.median(ts))
        rows.append({"degree": p, "unique_dofs": am.unique_dofs, "stored": am.cellwise_len,
                     "dss_ms": round(ms, 4), "gdofs_unique": round(am.unique_dofs / ms / 1e6, 3)})
        del r, z
        am.close()
    out["rows"] = rows
    return out


def slab_decomposition(fe, torch, flush, stream, reps=20):
    """Slab decomposition measured on one GPU.  (1) The Q3 mesh 48 x 48 x 96 (deformed) against its
    upper slab of 48^3 cells: assembled apply inside the slab, and the pack / add kernels of its
    interface plane (the device work a slab adds per exchanged DSS; the transfer itself is the
    caller's).  (2) PCG on Q3 32^3 (Dirichlet, sine load, rtol 1e-10): the whole mesh against two
    slabs driven by two threads of this process on the same GPU, exchanging through host barriers
    and device copies, so the second figure carries that orchestration, not a link."""
    import threading
    from paper_2607_02335_gb300 import slab as SL

    def med(fn):
        fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    p, m = 3, (48, 48, 96)
    whole = fe.Mesh(m, p, deform_amp=AMP)
    x = torch.randn(whole.cellwise_len, dtype=torch.float64, device="cuda")
    y = whole.empty()
    t_whole = med(lambda: fe.fe_apply(whole.handle, fe.FE_LAPLACE, fe.FE_F64, x, y, fe.FE_ASSEMBLE,
                                      stream))
    del x, y
    whole.close()
    s = SL.Slab(m, p, 48, 96, deform_amp=AMP)
    x = torch.randn(s.cellwise_len, dtype=torch.float64, device="cuda")
    y = s.empty()
    plane = torch.empty(s.plane_len, dtype=torch.float64, device="cuda")
    t_slab = med(lambda: fe.fe_apply(s.handle, fe.FE_LAPLACE, fe.FE_F64, x, y, fe.FE_ASSEMBLE, stream))
    t_pack = med(lambda: fe.fe_slab_face_pack(s.handle, fe.FE_F64, y, 0, plane, stream))
    t_add = med(lambda: fe.fe_slab_face_add(s.handle, fe.FE_F64, y, 0, plane, stream))
    out = {"apply": {"mesh": "Q3 48x48x96, deformed, FP64, Laplace, FE_ASSEMBLE",
                     "whole_ms": round(t_whole, 4), "slab_48cubed_ms": round(t_slab, 4),
                     "plane_pack_ms": round(t_pack, 4), "plane_add_ms": round(t_add, 4),
                     "plane_bytes_per_neighbour": s.plane_len * 8,
                     "slab_gdofs_unique": round(s.unique_dofs / (t_slab + t_pack + t_add) / 1e6, 3)}}
    del x, y, plane
    s.close()

    mc = (32, 32, 32)
    whole = fe.Mesh(mc, p, deform_amp=AMP, dirichlet=True)
    b = whole.rhs()
    xw = torch.zeros(whole.cellwise_len, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rw = whole.cg_solve(b, xw, rtol=1e-10, maxit=5000)
    t_w = time.perf_counter() - t0
    whole.close()
    slabs = [SL.Slab(mc, p, z0, z1, deform_amp=AMP, dirichlet=True) for z0, z1 in
             SL.slab_ranges(mc[2], 2)]
    grp = SL.ThreadSlabGroup(2)
    comms = [grp.comm(r, slabs[r].plane_len, "cuda:0") for r in range(2)]
    bs = [sl_.rhs() for sl_ in slabs]
    xs = [torch.zeros(sl_.cellwise_len, dtype=torch.float64, device="cuda") for sl_ in slabs]
    res = [None, None]

    def body(r):
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            res[r] = slabs[r].cg_solve(bs[r], xs[r], comm=comms[r], rtol=1e-10, maxit=5000)
        st.synchronize()

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    th = [threading.Thread(target=body, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    t_s = time.perf_counter() - t0
    out["pcg"] = {"mesh": "Q3 32^3, deformed, Dirichlet, sine load, rtol 1e-10",
                  "whole": {"iters": rw.iters, "s": round(t_w, 4),
                            "ms_per_iter": round(1e3 * t_w / max(rw.iters, 1), 4)},
                  "two_thread_slabs_one_gpu": {
                      "iters": res[0].iters, "status": [int(r.status) for r in res],
                      "s": round(t_s, 4), "ms_per_iter": round(1e3 * t_s / max(res[0].iters, 1), 4)}}
    for sl_ in slabs:
        sl_.close()
    return out


def packed_storage(fe, torch, flush, stream, reps=20):
    """2^3-packed storage units against one cell per unit, FP64 Laplace and mass at Q2 48^3 and
    Q3 96^3 (deformed): volumetric and assembled time, stored values and bytes per unique DoF."""
    from paper_2607_02335_gb300 import synth as S

    def med(fn):
        fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    out = []
    for p, m in ((2, 48), (3, 96)):
        for layout, name in ((fe.FE_LAYOUT_CELLS, "cells"), (fe.FE_LAYOUT_PACKED2, "packed2")):
            gm = fe.Mesh(m, p, deform_amp=AMP, layout=layout)
            x = torch.randn(gm.cellwise_len, dtype=torch.float64, device="cuda")
            y = gm.empty()
            for op in (fe.FE_LAPLACE, fe.FE_MASS):
                tv = med(lambda: fe.fe_apply(gm.handle, op, fe.FE_F64, x, y, 0, stream))
                ta = med(lambda: fe.fe_apply(gm.handle, op, fe.FE_F64, x, y, fe.FE_ASSEMBLE, stream))
                out.append({"case": f"Q{p} {m}^3", "layout": name,
                            "op": "laplace" if op == fe.FE_LAPLACE else "mass",
                            "stored_per_unique": round(gm.cellwise_len / gm.unique_dofs, 3),
                            "volumetric_ms": round(tv, 4), "assembled_ms": round(ta, 4),
                            "gdofs_unique_assembled": round(gm.unique_dofs / ta / 1e6, 3)})
            del x, y
            gm.close()
    return out


def multiblock_dss(fe, torch, flush, stream, m=32, p=3, reps=20):
    """DSS and assembled apply of the seven-block cube-in-cube (m^3 cells of degree p per block,
    every block frame turned at random) next to one structured mesh with the same cell count
    (64 x 56 x 64 for m = 32): the cost of the inter-block summation (Sec. 4.2)."""
    from paper_2607_02335_gb300 import synth as S

    def med(fn):
        fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    out = {"workload": f"cube-in-cube, 7 blocks of {m}^3 cells, Q{p}, random block frames; "
                       f"structured reference mesh 64x56x64 cells, Q{p}"}
    mb = fe.MBMesh(*S.mb_cube_in_cube(m, seed=0), p)
    r = torch.randn(mb.cellwise_len, dtype=torch.float64, device="cuda")
    z = mb.empty()
    info = mb.info()
    t_dss = med(lambda: fe.fe_mb_dss(mb.handle, fe.FE_F64, r, z, stream))
    t_asm = med(lambda: fe.fe_mb_apply(mb.handle, fe.FE_LAPLACE, fe.FE_F64, r, z, fe.FE_ASSEMBLE,
                                        stream))
    out["block_structured"] = {"unique_dofs": mb.unique_dofs, "cellwise_dofs": mb.cellwise_len,
                               "interfaces": info, "dss_ms": round(t_dss, 4),
                               "dss_gdofs_unique": round(mb.unique_dofs / t_dss / 1e6, 3),
                               "laplace_assembled_ms": round(t_asm, 4),
                               "laplace_assembled_gdofs_unique": round(mb.unique_dofs / t_asm / 1e6, 3)}
    del r, z
    mb.close()
    gm = fe.Mesh((64, 56, 64), p)
    r = torch.randn(gm.cellwise_len, dtype=torch.float64, device="cuda")
    z = gm.empty()
    t_dss = med(lambda: fe.fe_dss(gm.handle, fe.FE_F64, r, z, stream))
    t_asm = med(lambda: fe.fe_apply(gm.handle, fe.FE_LAPLACE, fe.FE_F64, r, z, fe.FE_ASSEMBLE,
                                     stream))
    out["structured"] = {"unique_dofs": gm.unique_dofs, "cellwise_dofs": gm.cellwise_len,
                         "dss_ms": round(t_dss, 4),
                         "dss_gdofs_unique": round(gm.unique_dofs / t_dss / 1e6, 3),
                         "laplace_assembled_ms": round(t_asm, 4),
                         "laplace_assembled_gdofs_unique": round(gm.unique_dofs / t_asm / 1e6, 3)}
    del r, z
    gm.close()
    return out


def reduced_precision_apply(fe, torch, flush, stream, m=96, p=3, reps=10):
    """Volumetric apply of the Q3 96^3 deformed mesh in the reduced-precision arithmetics of the
    inner solves: FP32 (FMA pipe), and 16-bit operands with FP32 accumulation (16-bit metric) on
    the tensor cores (mma.sync, the default for n <= 4) and on the FMA pipe (FE_LOWP_FMA=1)."""
    from paper_2607_02335_gb300 import synth as S

    peak, _ = load_peaks()
    gm = fe.Mesh(m, p, deform_amp=AMP)
    x = gm.gather(S.primal_unique(m, p, seed=0)).float()
    y = gm.empty(fe.FE_F32)
    out = []
    cases = (("fp32", fe.FE_F32, 4, "fma_pipe"),
             ("bf16_f32acc", fe.FE_BF16_F32ACC, 2, "tensor_cores_mma_sync"),
             ("bf16_f32acc", fe.FE_BF16_F32ACC, 2, "fma_pipe"),
             ("fp16_f32acc", fe.FE_F16_F32ACC, 2, "tensor_cores_mma_sync"),
             ("fp16_f32acc", fe.FE_F16_F32ACC, 2, "fma_pipe"))
    for name, prec, gbytes, engine in cases:
        force_fma = engine == "fma_pipe" and prec != fe.FE_F32
        if force_fma:
            os.environ["FE_LOWP_FMA"] = "1"
        try:
            for op in (fe.FE_LAPLACE, fe.FE_MASS):
                fe.fe_apply(gm.handle, op, prec, x, y, 0, stream)
                ts = []
                for _ in range(reps):
                    flush.fill_(1.0)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    fe.fe_apply(gm.handle, op, prec, x, y, 0, stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                ms = float(np.median(ts))
                alg = gm.cellwise_len * (8 + (6 if op == fe.FE_LAPLACE else 1) * gbytes)
                out.append({"arith": name, "engine": engine,
                            "op": "laplace" if op == fe.FE_LAPLACE else "mass",
                            "case": f"Q{p} {m}^3", "volumetric_ms": round(ms, 4),
                            "alg_bytes_per_cellwise_dof": alg // gm.cellwise_len,
                            "hbm_frac": round(alg / (ms * 1e-3) / 1e9 / peak, 4)})
        finally:
            if force_fma:
                del os.environ["FE_LOWP_FMA"]
    del x, y
    gm.close()
    return out


def mixed_vs_fp64_solve(fe, torch, m=64, p=3, rtol=1e-10):
    """Poisson -Laplace u = f, u = sin sin sin, Q3 on the deformed 64^3 mesh: Jacobi-PCG in FP64
    against FP32 PCG with FP64 reliable updates (and FP64 FCG preconditioned by an FP32 PCG solve),
    all to a relative FP64 residual of 1e-10.  Each solve is run twice and the second run is timed
    (the first builds the CUDA graphs)."""
    gm = fe.Mesh(m, p, deform_amp=AMP, dirichlet=True)
    b = gm.rhs(fe.FE_RHS_SINE)
    out = {"workload": f"Q{p}, {m}^3 deformed (amp {AMP}), sine manufactured solution, "
                       f"Jacobi-PCG to rtol {rtol}", "unique_dofs": gm.unique_dofs,
           "cellwise_dofs": gm.cellwise_len}
    sols = {}
    variants = (("fp64", 0, False, 0.1), ("mixed_fp32_reliable_updates", fe.FE_F32, False, 0.1),
                ("mixed_fp64_fcg_fp32_pcg_precond", fe.FE_F32, True, 1e-2))
    for name, mixed, flex, inner in variants:
        for rep in range(2):
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = gm.cg_solve(b, x, rtol=rtol, maxit=20000, mixed=mixed, flexible=flex,
                              inner_rtol=inner)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        sols[name] = x
        out[name] = {"status": fe.STATUS_NAMES[res.status], "iters": res.iters,
                     "outer_iters": res.outer_iters, "rel_res_fp64": res.rel_res,
                     "seconds": round(dt, 4), "ms_per_iter": round(dt * 1e3 / max(res.iters, 1), 4),
                     "l2_error_vs_exact": gm.l2_error(x)}
    for name, *_ in variants[1:]:
        out[name]["max_abs_diff_vs_fp64"] = float((sols[name] - sols["fp64"]).abs().max())
        out[name]["speedup_over_fp64"] = round(out["fp64"]["seconds"] / out[name]["seconds"], 3)
    gm.close()
    return out


def batched_solve(fe, torch, count=256, seed=0, rtol=1e-10, seq_count=64):
    """256 independent Poisson problems (m ~ U{4..32}, p ~ U{2,3,5,7}, deformation amplitude
    ~ U[0, 0.15], random dual right-hand side per cell-wise entry, seed 0) solved together by the
    batched engine to rtol 1e-10: mixed (FP32 PCG with FP64 reliable updates, one persistent apply
    launch per iteration) and FP64 PCG.  Beside them, the first seq_count problems solved one
    after another with fe_cg_solve and batched, to show what the one-launch batching buys."""
    from paper_2607_02335_gb300 import synth as S

    probs = S.batched_problems(count, seed=seed)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    t0 = time.perf_counter()
    meshes, bs = [], []
    for pr in probs:
        gm = fe.Mesh(pr["m"], pr["p"], deform_amp=pr["amp"], dirichlet=True)
        meshes.append(gm)
        bs.append(torch.rand(gm.cellwise_len, dtype=torch.float64, device="cuda", generator=gen) * 2 - 1)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    ncw = sum(g.cellwise_len for g in meshes)
    out = {"workload": f"{count} problems, m~U{{4..32}}, p~U{{2,3,5,7}}, amp~U[0,0.15], random dual "
                       f"rhs, rtol {rtol}, one persistent apply launch per iteration",
           "cellwise_dofs_total": ncw, "setup_seconds": round(t_setup, 3)}

    def batched(idx, mixed):
        opts = fe.fe_cg_opts(rtol, 20000, fe.FE_F32 if mixed else 0, 0, 0.1, None)
        xs = [torch.zeros_like(bs[i]) for i in idx]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = fe.fe_cg_solve_batched([meshes[i].handle for i in idx], [bs[i] for i in idx], xs, opts)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, res, xs

    for name, mixed in (("mixed", True), ("fp64", False)):
        t, res, xs = batched(range(count), mixed)
        ok = sum(r.status == fe.FE_OK for r in res)
        blk = {"solve_seconds": round(t, 3), "solves_per_s": round(count / t, 3), "converged": ok,
               "max_rel_res": max(r.rel_res for r in res),
               "iters_max": max(r.iters for r in res), "outer_iters_max": max(r.outer_iters for r in res)}
        if mixed:
            # a sample of problems solved alone through the same engine: the mix must not change them
            sample = sorted(range(count), key=lambda i: meshes[i].cellwise_len)[: min(6, count)]
            diffs = []
            for i in sample:
                _, _, xa = batched([i], True)
                diffs.append(float((xa[0] - xs[i]).abs().max()))
            blk["alone_vs_mix_max_abs_diff"] = max(diffs) if diffs else None
            blk["alone_vs_mix_sample"] = len(sample)
        out[name] = blk
        del xs
    # batching against one solve after another (same scheme, same first seq_count problems)
    idx = list(range(min(seq_count, count)))
    t_b, _, _ = batched(idx, True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in idx:
        x = torch.zeros_like(bs[i])
        meshes[i].cg_solve(bs[i], x, rtol=rtol, maxit=20000, mixed=fe.FE_F32, inner_rtol=0.1)
    torch.cuda.synchronize()
    t_s = time.perf_counter() - t0
    out["batched_vs_sequential"] = {"problems": len(idx), "scheme": "mixed (reliable updates)",
                                    "batched_s": round(t_b, 3), "sequential_fe_cg_solve_s": round(t_s, 3),
                                    "speedup": round(t_s / t_b, 3)}
    out["mixed_speedup_over_fp64"] = round(out["fp64"]["solve_seconds"] / out["mixed"]["solve_seconds"], 3)
    for g in meshes:
        g.close()
    del bs
    torch.cuda.empty_cache()
    return out


def serving_block(fe, args):
    """The serving workload at the arrival rate of the benchmark (200/s, far above what one GPU
    solves, so latencies are queueing) and at about 70% of the FP64 capacity measured in that run
    (latencies of the engine), FP64 and mixed at each rate."""
    out = {"workload": f"Poisson arrivals, m lognormal (median 16, sigma 0.5, max 64), p in {{2,3,7}}, "
                       f"amp {AMP}, sine load, rtol 1e-10, budget {args.serve_budget_gb} GB, "
                       f"{args.serve_slots} slots"}
    base = {"rate_per_s": args.serve_rate, "requests": args.serve_requests}
    for name, mixed in (("fp64", False), ("mixed", True)):
        base[name] = serving_run(fe, mixed, args.serve_requests, args.serve_rate, args.serve_budget_gb,
                                 args.serve_slots, args.serve_cap_s)
    out["at_benchmark_rate"] = base
    cap = base["fp64"]["solves_per_s"]
    if cap > 0:
        rate = round(0.7 * cap, 3)
        n = max(20, min(args.serve_requests, int(rate * 25)))
        part = {"rate_per_s": rate, "requests": n, "basis": "0.7 x FP64 solves/s at the benchmark rate"}
        for name, mixed in (("fp64", False), ("mixed", True)):
            part[name] = serving_run(fe, mixed, n, rate, args.serve_budget_gb, args.serve_slots,
                                     args.serve_cap_s)
        out["at_70pct_fp64_capacity"] = part
    return out


def serving_run(fe, mixed, n_req, rate, budget_gb, slots, cap_s, seed=0):
    """Poisson arrivals at `rate`/s of Jacobi-CG solves (m lognormal, median 16, max 64; p in
    {2,3,7}; manufactured sine load; rtol 1e-10) submitted to one server; returns its stats."""
    from paper_2607_02335_gb300 import synth as S

    arrivals = S.poisson_arrivals(rate, n_req, seed=seed)
    reqs = S.serving_requests(n_req, seed=seed)
    opts = fe.fe_cg_opts(1e-10, 20000, fe.FE_F32 if mixed else 0, 0, 0.1, None)
    srv = fe.fe_serve_create(int(budget_gb * 2 ** 30), slots, 0)
    pending, done, submitted = {}, {}, 0
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while submitted < n_req and arrivals[submitted] <= now:
            rq = reqs[submitted]
            d = fe.fe_mesh_desc(rq["m"], rq["m"], rq["m"], rq["p"], AMP, fe.FE_GEOM_STORED, 1, 0)
            pending[fe.fe_serve_submit(srv, d, None, opts)] = submitted
            submitted += 1
        for t in list(pending):
            r = fe.fe_serve_poll(srv, t)
            if r is not None:
                done[pending.pop(t)] = r
        if submitted == n_req and not pending:
            break
        if now > cap_s:
            break
        time.sleep(0.0005)
    wall = time.perf_counter() - t0
    p50, p99, sps = fe.fe_serve_stats(srv)
    fe.fe_serve_destroy(srv)
    return {"submitted": submitted, "completed": len(done), "wall_s": round(wall, 3),
            "solves_per_s": round(sps, 3), "p50_s": round(p50, 4), "p99_s": round(p99, 4),
            "converged": sum(r.status == fe.FE_OK for r in done.values()),
            "max_rel_res": max((r.rel_res for r in done.values()), default=None)}


def run_profile_case(args):
    """One (degree, cells, operator[, vol[, arithmetic]]) case applied W+K times with FE_ASSEMBLE
    (vol: the volumetric apply alone; arithmetic f64 (default), f32, bf16 or fp16); no timing."""
    import torch

    from paper_2607_02335_gb300 import fe
    from paper_2607_02335_gb300 import synth as S

    parts = args.profile_case.split(",")
    p, m, opname = int(parts[0]), int(parts[1]), parts[2]
    flags = 0 if len(parts) > 3 and parts[3] == "vol" else fe.FE_ASSEMBLE
    arith = parts[4] if len(parts) > 4 else "f64"
    prec = {"f64": fe.FE_F64, "f32": fe.FE_F32, "bf16": fe.FE_BF16_F32ACC,
            "fp16": fe.FE_F16_F32ACC}[arith]
    op = fe.FE_LAPLACE if opname == "laplace" else fe.FE_MASS
    gm = fe.Mesh(m, p, deform_amp=AMP)
    x = gm.gather(S.primal_unique(m, p, seed=0))
    if prec != fe.FE_F64:
        x = x.float()
    y = gm.empty(fe.FE_F64 if prec == fe.FE_F64 else fe.FE_F32)
    for _ in range(args.warmup + args.steps):
        fe.fe_apply(gm.handle, op, prec, x, y, flags)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case, "launches": args.warmup + args.steps}))


def run_profile_batched(args):
    """The first N problems of the batched workload solved once by the batched engine (mixed,
    rtol 1e-10), untimed."""
    import torch

    from paper_2607_02335_gb300 import fe
    from paper_2607_02335_gb300 import synth as S

    probs = S.batched_problems(256, seed=0)[: args.profile_batched]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    meshes = [fe.Mesh(pr["m"], pr["p"], deform_amp=pr["amp"], dirichlet=True) for pr in probs]
    bs = [torch.rand(g.cellwise_len, dtype=torch.float64, device="cuda", generator=gen) * 2 - 1
          for g in meshes]
    xs = [torch.zeros_like(b) for b in bs]
    opts = fe.fe_cg_opts(1e-10, 20000, fe.FE_F32, 0, 0.1, None)
    res = fe.fe_cg_solve_batched([g.handle for g in meshes], bs, xs, opts)
    torch.cuda.synchronize()
    print(json.dumps({"profile_batched": len(meshes),
                      "converged": sum(r.status == fe.FE_OK for r in res),
                      "iters_max": max(r.iters for r in res)}))


def run_profile_solve(args):
    """One solve of the solve_mixed_vs_fp64 workload (Q3 64^3 deformed, sine load, rtol 1e-10):
    FP64 PCG or FP32 PCG with FP64 reliable updates, untimed."""
    import torch

    from paper_2607_02335_gb300 import fe

    gm = fe.Mesh(64, 3, deform_amp=AMP, dirichlet=True)
    b = gm.rhs(fe.FE_RHS_SINE)
    x = torch.zeros_like(b)
    mixed = fe.FE_F32 if args.profile_solve == "mixed" else 0
    res = gm.cg_solve(b, x, rtol=1e-10, maxit=20000, mixed=mixed, flexible=False, inner_rtol=0.1)
    torch.cuda.synchronize()
    print(json.dumps({"profile_solve": args.profile_solve, "status": fe.STATUS_NAMES[res.status],
                      "iters": res.iters, "outer_iters": res.outer_iters}))
    gm.close()


def main():
    args = parse()
    if args.profile_solve:
        run_profile_solve(args)
        return
    if args.profile_case:
        run_profile_case(args)
        return
    if args.profile_batched > 0:
        run_profile_batched(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    run_ours(args, rank, world)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
