"""Benchmark of the DTT-PSTD hot path: grid-point updates per second.

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

One bench step is one full configured simulation: the initial fields are
copied in from device-resident copies, u^{-1/2} is derived (init_velocity),
and the configured number of leapfrog steps runs (pstd_run, graph-replayed).
Grid-point updates = prod(N_i) cells x leapfrog steps.  L2 is flushed (a
256 MB write) before every timed bench step; the flush is not timed.

Under torchrun (N > 1) every rank runs an independent replica of the workload
on its own GPU (the path does not shard a single grid); value = all ranks'
updates / the slowest rank's time.

--impl reference times the FP64 CPU oracle (the only other implementation of
this method) on the host cores, each bench step a bounded sample of the same
workload (a fixed number of leapfrog steps of the full grid).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2005_00322_gb300 import inputs  # noqa: E402

METRIC = "PSTD grid-point updates/s vs plain FP32 path at ≤1e-4 rel L2 vs FP64 oracle"
UNIT = "grid-point updates/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
CSRC = os.path.join(ROOT, "paper_2005_00322_gb300", "csrc")

WORKLOADS = {
    "plane512_dx_ny": inputs.plane512_dx_ny,
    "line256_dd": inputs.line256_dd,
    "cube256_ddnndd": lambda: inputs.cube256(steps=200),
    "cube384_dnd": lambda: inputs.cube384_dnd(),
}


def cells(w) -> int:
    return int(np.prod(w.ncells))


def csrc_digest() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(CSRC, f), "rb").read())
    return h.hexdigest()[:16]


def host_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads") or 0) for i in threadpool_info())
        if n:
            return int(n)
    except Exception:
        pass
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(w, seconds: float, max_steps: int | None = None):
    """Time the FP64 oracle stepping the full grid of ``w`` for about ``seconds``."""
    from oracle import pstd
    desc = pstd.Desc(w.ncells, (w.dx,), w.bc, c0=w.c0, rho0=w.rho0,
                     dt=pstd.dt_from_cfl(w.cfl, w.dx, w.c0))
    sl = tuple(slice(j[0], j[-1] + 1) for j in (pstd.p_nodes(n, b) for n, b in zip(w.ncells, w.bc)))
    p0 = w.p0_full()[sl]
    s = pstd.State(p0, pstd.init_velocity(desc, p0, None))
    s = pstd.step(desc, s)                       # warm the BLAS pools
    n, t0 = 0, time.perf_counter()
    while True:
        s = pstd.step(desc, s)
        n += 1
        el = time.perf_counter() - t0
        if (max_steps and n >= max_steps) or (not max_steps and el >= seconds):
            break
    return n, el


class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = max((num(r[2]) or 0) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        load = [s for s in sm if s >= 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows)}


def reference_arm(args, w, rank: int) -> None:
    if rank != 0:
        return
    per_step = 20
    for _ in range(args.warmup):
        oracle_sample(w, 0, max_steps=per_step)
    t = 0.0
    for _ in range(args.steps):
        n, el = oracle_sample(w, 0, max_steps=per_step)
        t += el
    updates = cells(w) * per_step * args.steps
    value = updates / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "ncells": list(w.ncells), "cfl": w.cfl,
                   "leapfrog_steps_per_bench_step": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_threads(), "kind": "oracle",
                         "sample": f"{per_step} FP64 leapfrog steps of the full {w.name} grid per bench step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="plane512_dx_ny", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--leapfrog-steps", type=int, default=0, help="override the workload's step count")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    w = WORKLOADS[args.workload]()
    if args.leapfrog_steps:
        w.steps = args.leapfrog_steps
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        reference_arm(args, w, rank)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2005_00322_gb300 import Solver

    solver = Solver(w.ncells, w.dx, w.bc, c0=w.c0, rho0=w.rho0, cfl=w.cfl)
    st = solver.stream
    p0 = torch.tensor(np.asarray(solver.restrict(w.p0_full()), np.float32), device="cuda")
    p, us = solver.zeros()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    def one_step():
        p.copy_(p0)
        for u in us:
            u.zero_()
        solver.init_velocity(p, us)
        n = solver.last_launch_count()
        solver.run(p, us, w.steps)
        return n + solver.last_launch_count()

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    # device-resident timed region: CUDA events on the plan's stream per bench step
    launches = 0
    times = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            launches += one_step()
            e1.record(st)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t = sum(times)
    if dist:
        tt = torch.tensor([t], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    updates = cells(w) * w.steps * args.steps * world
    value = updates / t

    # dominant kernel: the fused axis pass (k_step); average launch duration
    # from events over direct launches of whole steps on the plan's stream
    nk = 64
    p.copy_(p0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(nk):
        solver.step(p, us)
    e1.record(st)
    e1.synchronize()
    per_launch = e0.elapsed_time(e1) / 1e3 / (nk * w.ndim)
    alg_bytes = 2 * (w.ndim + 1) * 4 * cells(w) / w.ndim     # per launch: one axis' share
    peaks = json.load(open(PEAKS)) if os.path.exists(PEAKS) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    traffic = None
    if os.path.exists(TRAFFIC):
        tr = json.load(open(TRAFFIC))
        ent = tr.get(w.name)
        if ent and ent.get("csrc_digest") == csrc_digest():
            traffic = ent.get("dram_bytes_per_launch")
    achieved = alg_bytes / per_launch / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": "k_step",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s",
                "alg_bytes_per_launch": alg_bytes}

    # end to end through the public API with host buffers
    ph = torch.from_numpy(np.asarray(solver.restrict(w.p0_full()), np.float32)).pin_memory()
    uh = [torch.zeros(s, dtype=torch.float32).pin_memory() for s in solver.shapes[1:]]
    po = torch.empty_like(ph).pin_memory()
    uo = [torch.empty_like(u).pin_memory() for u in uh]
    h2d = ph.numel() * 4 + sum(u.numel() * 4 for u in uh)
    d2h = h2d
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        p.copy_(ph, non_blocking=True)
        for u, h in zip(us, uh):
            u.copy_(h, non_blocking=True)
        solver.init_velocity(p, us)
        solver.run(p, us, w.steps)
        po.copy_(p, non_blocking=True)
        for h, u in zip(uo, us):
            h.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
    te = time.perf_counter() - t0
    if dist:
        tt = torch.tensor([te], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        te = float(tt.item())
    e2e = {"value": updates / te, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and world == 1:
        n, el = oracle_sample(w, args.cpu_seconds)
        cpu = {"value": cells(w) * n / el, "unit": UNIT, "cores": host_threads(), "kind": "oracle",
               "sample": f"{n} FP64 leapfrog steps of the full {w.name} grid ({el:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "ncells": list(w.ncells),
                       "bc": ["".join(b) for b in w.bc], "cfl": w.cfl,
                       "leapfrog_steps_per_bench_step": w.steps,
                       "l2": "flushed (256 MB write) before each timed bench step",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clk.summary(), "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
