"""Benchmark of the DTT-PSTD hot path: grid-point updates per second.

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]
                [--form fft|split|split-bf16|tensor|order2] [--persistent]
python bench.py --learned [--learned-iters I]

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
    # batched forms: leapfrog steps per bench step are reduced (the configured
    # runs are 1500 / 4000 steps); --leapfrog-steps overrides
    "cube256_r0.4": lambda: inputs.cube256_reflect(0.4, steps=32),
    "plane_batch": lambda: inputs.plane_batch(steps=200),
}


def members_of(w):
    """The independent runs of a workload: itself, its wall combinations or its batch."""
    if isinstance(w, list):
        return w
    return [w]


def cells(w) -> int:
    return int(np.prod(w.ncells))


def csrc_digest() -> str:
    """Digest of the sources that build and launch the axis-pass kernels
    (the register-FFT passes and the plan that schedules them)."""
    h = hashlib.sha256()
    for f in sorted(os.listdir(CSRC)):
        if f.startswith("pstd_w") or f in ("pstd_plan.cu", "pstd_internal.h", "pstd_ops.cuh"):
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


def oracle_sample(w, seconds: float, max_steps: int | None = None, order2: bool = False):
    """Time the FP64 oracle stepping the full grid of ``w`` for about ``seconds``
    (the coupled leapfrog, or the second-order form with ``order2``)."""
    from oracle import order2 as o2
    from oracle import pstd
    desc = pstd.Desc(w.ncells, (w.dx,), w.bc, c0=w.c0, rho0=w.rho0,
                     dt=pstd.dt_from_cfl(w.cfl, w.dx, w.c0))
    sl = tuple(slice(j[0], j[-1] + 1) for j in (pstd.p_nodes(n, b) for n, b in zip(w.ncells, w.bc)))
    p0 = w.p0_full()[sl]
    if order2:
        s = (p0, o2.init_prev(desc, p0))
        step = lambda st: o2.step(desc, *st)
    else:
        s = pstd.State(p0, pstd.init_velocity(desc, p0, None))
        step = lambda st: pstd.step(desc, st)
    s = step(s)                                  # warm the BLAS pools
    n, t0 = 0, time.perf_counter()
    while True:
        s = step(s)
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


def rank_max(x: float, dist, device) -> float:
    """The largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def modal_rel_l2(w, solver, p_final) -> float:
    """Relative L2 of the final pressure of one full run of ``w`` against the
    FP64 separable modal solution (the CPU leg: calls oracle/)."""
    from oracle import modal, pstd
    od = pstd.Desc(w.ncells, (w.dx,), w.bc, c0=w.c0, rho0=w.rho0, dt=solver.dt)
    facs = [[term[i][pstd.p_nodes(n, b)] for i, (n, b) in enumerate(zip(w.ncells, w.bc))]
            for term in w.factors()]
    ref = modal.separable_modal_pressure(od, facs, w.steps)
    got = np.asarray(p_final, np.float64)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def energy_drift(run) -> dict:
    """|E^n - E^0| / E^0 over one full run of the workload, the energies formed
    in FP64 on the GPU (pstd_energy) from p^n, u^{n-1/2} and u^{n+1/2}."""
    import torch
    s = run.solver
    p, us = run.p, run.us
    p.copy_(run.p0)
    for u in us:
        u.zero_()
    s.init_velocity(p, us)

    def energy_now():
        pn, uprev = p.clone(), [u.clone() for u in us]
        s.step(p, us)
        return s.energy(pn, uprev, us)
    e0 = energy_now()
    s.run(p, us, run.w.steps - 2)
    e1 = energy_now()
    torch.cuda.synchronize()
    return {"value": abs(e1 - e0) / e0, "steps": run.w.steps, "e0": e0,
            "how": "pstd_energy (FP64 on the GPU) after step 1 and after the last step"}


def hbm_case(peak: float, name: str = "cube256_ddnndd") -> dict:
    """The HBM-bound configuration: one plain FP32 256^3 grid (DD / NN / DD),
    axis passes timed from graph-replayed runs of 32 and 96 steps (events on
    the plan's stream; the 268 MB state exceeds L2)."""
    import torch
    w = WORKLOADS[name]()
    r = SingleRunner(w)
    r.p.copy_(r.p0)
    r.solver.init_velocity(r.p, r.us)
    st = r.stream

    def run_time(n):
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(st)
        r.leapfrog(n)
        a1.record(st)
        a1.synchronize()
        return a0.elapsed_time(a1) / 1e3
    run_time(32)
    step_s = (run_time(96) - run_time(32)) / 64
    alg_step = 2 * (w.ndim + 1) * 4 * cells(w)
    per_launch = step_s / w.ndim
    ach = alg_step / w.ndim / per_launch / 1e9
    r.close()
    return {"workload": name, "ms_per_step": step_s * 1e3, "updates_per_s": cells(w) / step_s,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "kernel": "k_wstep (fused axis pass)", "alg_bytes_per_launch": alg_step / w.ndim,
                         "launch_s": per_launch}}


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units processed by all ranks divided by the slowest rank's time."""
    return units_per_rank * world / seconds_max


class SingleRunner:
    """One grid through Solver (pstd_plan / pstd_run)."""

    def __init__(self, w, form="fft", persistent=False, autotune=True):
        import torch
        from paper_2005_00322_gb300 import Solver
        self.w = w
        # order2: the second-order pressure-only form (pstd_init_prev / pstd_run2)
        self.order2 = form == "order2"
        # the FFT form's axis-pass schedules are measured on the device
        # (pstd_plan_autotune) unless --no-autotune
        self.solver = Solver(w.ncells, w.dx, w.bc, c0=w.c0, rho0=w.rho0, cfl=w.cfl,
                             form="fft" if self.order2 else form, persistent=persistent,
                             autotune=autotune and not persistent)
        self.stream = self.solver.stream
        p0 = np.asarray(self.solver.restrict(w.p0_full()), np.float32)
        self.p0 = torch.tensor(p0, device="cuda")
        self.p, self.us = self.solver.zeros()
        if self.order2:
            self.us = [torch.zeros_like(self.p)]          # p^{n-1}
            self.host_in = [torch.from_numpy(p0).pin_memory()]
            self.host_out = [torch.empty_like(self.host_in[0]).pin_memory() for _ in range(2)]
        else:
            self.host_in = [torch.from_numpy(p0).pin_memory()] + \
                [torch.zeros(sh, dtype=torch.float32).pin_memory() for sh in self.solver.shapes[1:]]
            self.host_out = [torch.empty_like(h).pin_memory() for h in self.host_in]
        self.cells = cells(w)
        self.ndim = w.ndim
        self.launches_per_step = w.ndim
        # fields read and written once per step at the algorithmic minimum
        self.fields = 2 if self.order2 else w.ndim + 1

    def _start(self):
        if self.order2:
            self.solver.init_prev(self.p, self.us[0])
        else:
            self.solver.init_velocity(self.p, self.us)

    def _run(self, n):
        if self.order2:
            self.solver.run2(self.p, self.us[0], n)
        else:
            self.solver.run(self.p, self.us, n)

    def step(self):
        self.p.copy_(self.p0)
        for u in self.us:
            u.zero_()
        self._start()
        n = self.solver.last_launch_count()
        self._run(self.w.steps)
        return n + self.solver.last_launch_count()

    def step_e2e(self):
        for d, h in zip([self.p] + self.us, self.host_in):
            d.copy_(h, non_blocking=True)
        self._start()
        self._run(self.w.steps)
        for h, d in zip(self.host_out, [self.p] + self.us):
            h.copy_(d, non_blocking=True)

    def leapfrog(self, n):
        self._run(n)

    def close(self):
        self.solver.close()


class BatchRunner:
    """Independent grids in one batch (pstd_batch_*): wall combinations or a batch."""

    def __init__(self, w, persistent=False):
        import torch
        from paper_2005_00322_gb300.batch import Batch, reflection_combos
        self.w = w
        if isinstance(w, list):
            mem = w
            specs = [dict(ncells=m.ncells, dx=m.dx, bc=m.bc, cfl=m.cfl, c0=m.c0, rho0=m.rho0) for m in mem]
            p_full = [m.p0_full() for m in mem]
            self.weights = None
            self.steps = mem[0].steps
        else:
            bcs, self.weights = reflection_combos(w.ncells, w.dx, w.refl, w.c0, w.rho0, 1.0)
            specs = [dict(ncells=w.ncells, dx=w.dx, bc=b, cfl=w.cfl, c0=w.c0, rho0=w.rho0) for b in bcs]
            full = w.p0_full()
            p_full = [full] * len(specs)
            self.steps = w.steps
        self.batch = Batch(specs)
        if persistent:
            # every run as one cooperative kernel over all members
            self.batch.set_persistent()
        self.stream = self.batch.stream
        self.fields = self.batch.zeros()
        self.p0 = []
        self.host_in, self.host_out = [], []
        from paper_2005_00322_gb300.solver import stored_node_range
        for (p, us), spec, pf in zip(self.fields, specs, p_full):
            sl = tuple(slice(stored_node_range(n, b)[0], stored_node_range(n, b)[1] + 1)
                       for n, b in zip(spec["ncells"], spec["bc"]))
            q = np.ascontiguousarray(np.asarray(pf, np.float32)[sl])
            self.p0.append(torch.tensor(q, device="cuda"))
            hin = [torch.from_numpy(q).pin_memory()] + [torch.zeros(u.shape).pin_memory() for u in us]
            self.host_in.append(hin)
            self.host_out.append([torch.empty_like(h).pin_memory() for h in hin])
        self.cells = sum(int(np.prod(sp["ncells"])) for sp in specs)
        self.ndim = max(len(sp["ncells"]) for sp in specs)
        self.launches_per_step = sum(len(sp["ncells"]) for sp in specs)
        self.out = None
        if self.weights is not None:
            self.out = torch.empty(tuple(n + 1 for n in w.ncells), device="cuda")

    def step(self):
        for (p, us), q in zip(self.fields, self.p0):
            p.copy_(q)
            for u in us:
                u.zero_()
        self.batch.init_velocity(self.fields)
        n = self.batch.last_launch_count()
        self.batch.run(self.fields, self.steps)
        n += self.batch.last_launch_count()
        if self.weights is not None:
            self.batch.combine(self.weights, self.fields, self.out)
            n += self.batch.last_launch_count()
        return n

    def step_e2e(self):
        for (p, us), hin in zip(self.fields, self.host_in):
            for d, h in zip([p] + us, hin):
                d.copy_(h, non_blocking=True)
        self.batch.init_velocity(self.fields)
        self.batch.run(self.fields, self.steps)
        if self.weights is not None:
            self.batch.combine(self.weights, self.fields, self.out)
        for (p, us), hout in zip(self.fields, self.host_out):
            for h, d in zip(hout, [p] + us):
                h.copy_(d, non_blocking=True)

    def leapfrog(self, n):
        self.batch.run(self.fields, n)

    def close(self):
        self.batch.close()


LEARNED_METRIC = "learned-operator 200-step pressure predictions/s (128x128 NN/DD box)"


def learned_main(args) -> None:
    """--learned: the spectral neural operator against the solver it replaces.

    The configured workload: a 128^2 box, Neumann walls on x and Dirichlet on y,
    200 steps at CFL 0.3; inputs of 1-6 Gaussian blobs of sigma U[2, 8] dx
    (inputs.sno_initial_pressures); 20k training samples (seed 1), 1k test
    samples (seed 2) and 512 held-out samples (seed 3) that set the gate.  The
    network (4 layers, 32 channels, 16 modes per axis) trains on PSTD answers.
    The solver is the arbiter: requests whose content above the 16th mode is too
    large for the network (gate set on the held-out set at tolerance 1e-2
    relative L2) are answered by PSTD.  Reported: the network's error on the
    whole test set, the share of it the gate admits and their worst error, and
    the throughput of the network, of batched PSTD (64 members per graph) and
    of the gated pipeline on the test set (batches of 256, device-resident, L2
    flushed between timed calls).
    """
    import torch
    from paper_2005_00322_gb300.batch import Batch
    from paper_2005_00322_gb300.sno import SpectralOperator, Surrogate, pstd_reference
    from paper_2005_00322_gb300.solver import stored_node_range

    w = inputs.plane128_nn_dd()
    ncells, bc = w.ncells, w.bc
    ntr, nte, nho = args.learned_train, 1024, 512
    sl = tuple(slice(stored_node_range(k, b)[0], stored_node_range(k, b)[1] + 1) for k, b in zip(ncells, bc))

    def dataset(n, seed):
        full = inputs.sno_initial_pressures(n, seed=seed, ncells=ncells)
        p0 = torch.tensor(full[(slice(None),) + sl].astype(np.float32), device="cuda")
        return p0, pstd_reference(ncells, bc, w.dx, w.cfl, w.steps, p0)
    p_tr, t_tr = dataset(ntr, 1)
    p_te, t_te = dataset(nte, 2)
    p_ho, t_ho = dataset(nho, 3)
    net = SpectralOperator(ncells, bc, channels=32, modes=16, layers=4, seed=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = net.train(p_tr, t_tr, iters=args.learned_iters, batch=32, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    sur = Surrogate(net, w.dx, w.cfl, w.steps, tol=1e-2)
    ho_max = sur.validate(p_ho, t_ho)
    err = net.rel_err(net.predict(p_te), t_te).cpu().numpy()
    frac = net.high_mode_fraction(p_te).cpu().numpy()
    admitted = frac < sur.gate
    err16 = net.rel_err(net.predict(p_te, bf16=True), t_te).cpu().numpy()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def timed(fn, samples):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            tot += e0.elapsed_time(e1) / 1e3
        return samples * args.steps / tot

    xb = p_te[:256].contiguous()
    # the gated pipeline answers the whole test set; its error against PSTD
    outs = [sur(p_te[i:i + 256].contiguous()) for i in range(0, nte, 256)]
    pipe_err = net.rel_err(torch.cat(outs), t_te).cpu().numpy()
    with Clocks(0) as clk:
        net_rate = timed(lambda: net.predict(xb), 256)
        net16_rate = timed(lambda: net.predict(xb, bf16=True), 256)
        pipe_rate = timed(lambda: sur(xb), 256)
    # PSTD: one batch plan of 64 members, each bench call loads 64 initial
    # pressures, derives u^{-1/2} and runs the 200 steps
    bt = Batch([dict(ncells=ncells, dx=w.dx, bc=bc, cfl=w.cfl)] * 64)
    fields = bt.zeros()

    def pstd_call():
        for m, (p, us) in enumerate(fields):
            p.copy_(p_te[m])
            for u in us:
                u.zero_()
        bt.init_velocity(fields)
        bt.run(fields, w.steps)
    pstd_rate = timed(pstd_call, 64)
    bt.close()
    line = {
        "metric": LEARNED_METRIC, "value": pipe_rate, "unit": "samples/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "plane128_nn_dd_learned", "ncells": list(ncells), "bc": ["".join(b) for b in bc],
                   "cfl": w.cfl, "leapfrog_steps": w.steps, "channels": 32, "modes": 16, "layers": 4,
                   "inputs": "1-6 blobs, sigma U[2, 8] dx, amplitude U[-1, 1]",
                   "batch": 256, "l2": "flushed (256 MB write) before each timed call"},
        "pstd": {"value": pstd_rate, "unit": "samples/s", "batch": 64},
        "network": {"value": net_rate, "speedup_vs_pstd": net_rate / pstd_rate},
        "gated_pipeline": {"value": pipe_rate, "speedup_vs_pstd": pipe_rate / pstd_rate,
                           "max_rel_l2": float(pipe_err.max()), "share_by_network": float(admitted.mean())},
        "bf16_weights": {"value": net16_rate, "test_max_rel_l2": float(err16.max()),
                         "test_median_rel_l2": float(np.median(err16))},
        "accuracy": {"test": nte, "max_rel_l2": float(err.max()), "median_rel_l2": float(np.median(err)),
                     "share_within_tol": float((err <= 1e-2).mean()),
                     "admitted_max_rel_l2": float(err[admitted].max()) if admitted.any() else None,
                     "arbiter": "PSTD on the same inputs"},
        "gate": {"tol": sur.tol, "high_mode_fraction_below": sur.gate, "heldout": nho,
                 "heldout_max_rel_l2": ho_max, "heldout_share": sur.routed, "trusted": sur.trusted},
        "train": {"samples": ntr, "iters": args.learned_iters, "batch": 32, "seconds": t_train,
                  "final_loss": float(np.mean(losses[-50:]))},
        "clocks": clk.summary(),
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
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the plan's default axis-pass schedules (no pstd_plan_autotune)")
    ap.add_argument("--persistent", action="store_true",
                    help="pstd_run (a batch: pstd_batch_run over all members) as one cooperative kernel "
                         "with grid barriers")
    ap.add_argument("--form", default="fft", choices=["fft", "split", "split-bf16", "tensor", "order2"],
                    help="fft: spectral FFT route; split: FP16 hi/lo dense form (mma.sync); split-bf16: "
                         "BF16 three-way split dense form on tcgen05; tensor: TF32 hi/lo dense form on "
                         "tcgen05; order2: second-order pressure-only form on the FFT passes")
    ap.add_argument("--learned", action="store_true",
                    help="train and time the learned operator against 200 PSTD steps (prints its own line)")
    ap.add_argument("--learned-iters", type=int, default=12000)
    ap.add_argument("--learned-train", type=int, default=20000)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.learned:
        learned_main(args)
        return

    w = WORKLOADS[args.workload]()
    if args.leapfrog_steps:
        for m in members_of(w):
            m.steps = args.leapfrog_steps
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    single = not isinstance(w, list) and w.refl is None
    w0 = members_of(w)[0]

    if args.impl == "reference":
        reference_arm(args, w0 if single or isinstance(w, list) else
                      inputs.cube256(bc=(("N", "N"),) * 3, steps=w.steps), rank)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)

    run = (SingleRunner(w, args.form, args.persistent, not args.no_autotune) if single
           else BatchRunner(w, args.persistent))
    st = run.stream
    steps_per = members_of(w)[0].steps
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    for _ in range(args.warmup):
        run.step()
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
            launches += run.step()
            e1.record(st)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t = rank_max(sum(times), dist, "cuda")
    updates = run.cells * steps_per * args.steps * world
    value = whole_job_rate(run.cells * steps_per * args.steps, world, t)

    # dominant kernel: the fused axis pass.  Its mean duration inside a run
    # comes from events on the plan's stream around two graph-replayed runs
    # of 32 and 96 steps: the difference cancels the per-run velocity
    # conversions and launch set-up, leaving 64 steps of axis passes.
    def run_time(n):
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(st)
        run.leapfrog(n)
        a1.record(st)
        a1.synchronize()
        return a0.elapsed_time(a1) / 1e3
    run_time(32)
    step_s = (run_time(96) - run_time(32)) / 64
    nfields = (lambda m: run.fields) if single else (lambda m: len(m) + 1)
    alg_step = sum(2 * nfields(m) * 4 * int(np.prod(m)) for m in
                   ([mm.ncells for mm in members_of(w)] if single or isinstance(w, list)
                    else [w.ncells] * len(run.weights)))
    if single:
        per_launch = step_s / run.launches_per_step
        alg_bytes = alg_step / run.launches_per_step
    else:       # concurrent members: whole-step bandwidth
        per_launch = step_s
        alg_bytes = alg_step
    peaks = json.load(open(PEAKS)) if os.path.exists(PEAKS) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    traffic = None
    if os.path.exists(TRAFFIC):
        tr = json.load(open(TRAFFIC))
        # counters belong to the kernel that ran: the fused step pass, or the
        # kernel of another form (key "<workload>/<form>")
        variant = args.form if args.form != "fft" else ("persistent" if args.persistent else "")
        ent = tr.get(args.workload + ("/" + variant if variant else ""))
        if ent and ent.get("csrc_digest") == csrc_digest():
            traffic = ent.get("dram_bytes_per_launch")
    achieved = alg_bytes / per_launch / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": ("k_wgrad dir 4 (second-order axis pass)" if args.form == "order2"
                           else "k_wstep (fused axis pass)") if single
                else "every member's axis passes (k_wstep register passes, k_step generic / convolution "
                     "passes), concurrent graph branches",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s",
                "alg_bytes_per_launch": alg_bytes,
                "launch_s": per_launch if single else None, "step_s": step_s}
    if single and args.form in ("split", "split-bf16", "tensor"):
        # dense split forms: tensor-bound GEMMs.  Per axis and step two GEMMs
        # (N x lp and lp x N operators) over cells / lp lines, with three
        # split products each (FP16 and TF32 hi/lo: 12 N x cells flops) or six
        # (BF16 three-way split: 24 N x cells).  The TF32 and BF16 forms launch
        # two GEMMs per axis.
        cells_p = int(np.prod(run.solver.shapes[0]))
        prods = 6 if args.form == "split-bf16" else 3
        flops_step = sum(4.0 * prods * n * cells_p for n in w.ncells)
        nl = w.ndim * (1 if args.form == "split" else 2)
        sust = peaks.get("bf16_tflops_sustained", 1700.0)
        tpeak = sust * (1.1 / 2.25) if args.form == "tensor" else sust
        ach = flops_step / step_s / 1e12
        roofline = {"bound": "tensor", "achieved": ach, "peak": tpeak, "unit": "TFLOP/s", "frac": ach / tpeak,
                    "traffic": traffic,
                    "kernel": {"tensor": "k_tc_gemm<1> (tcgen05 kind::tf32)",
                               "split-bf16": "k_tc16 (tcgen05 kind::f16, BF16 three-way split, TMA-fed)",
                               "split": "k_gemm_step (mma.sync m16n8k16 f16)"}[args.form],
                    "peak_source": ("MEASURED_PEAKS.json bf16_tflops_sustained x 1.1/2.25 nominal tf32:bf16 "
                                    "(of measured)") if args.form == "tensor" else
                                   "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)",
                    "alg_flops_per_launch": flops_step / nl, "launch_s": step_s / nl, "step_s": step_s}

    # end to end through the public API with host buffers
    h2d = sum(h.numel() * 4 for h in (run.host_in if single else [x for m in run.host_in for x in m]))
    d2h = sum(h.numel() * 4 for h in (run.host_out if single else [x for m in run.host_out for x in m]))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run.step_e2e()
        torch.cuda.synchronize()
    te = rank_max(time.perf_counter() - t0, dist, "cuda")
    e2e = {"value": updates / te, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # accuracy of the benchmarked run: the final pressure of the last e2e run
    # (a full configured run from p0) against the FP64 modal solution, and the
    # FP64 energy drift over one full run (single coupled-leapfrog grids)
    acc = None
    drift = None
    if single and rank == 0:
        p_fin = run.host_out[0].numpy().copy()
        if not (args.form == "order2"):
            drift = energy_drift(run)
    hbm = None
    if rank == 0 and not (single and w0.ncells == WORKLOADS["cube256_ddnndd"]().ncells and args.form == "fft"):
        hbm = hbm_case(peak)

    cpu = None
    if rank == 0 and world == 1 and single and steps_per == w0.steps:
        acc = {"value": modal_rel_l2(w0, run.solver, p_fin), "unit": "rel L2 of p",
               "against": "FP64 separable modal solution (oracle/modal.py)",
               "steps": steps_per, "bar": 1e-4}
    if rank == 0 and world == 1:
        wc = w0 if single or isinstance(w, list) else inputs.cube256(bc=(("N", "N"),) * 3)
        o2 = args.form == "order2" and single
        n, el = oracle_sample(wc, args.cpu_seconds, order2=o2)
        cpu = {"value": cells(wc) * n / el, "unit": UNIT, "cores": host_threads(), "kind": "oracle",
               "sample": f"{n} FP64 {'second-order' if o2 else 'leapfrog'} steps of the full {wc.name} grid "
                         f"({el:.1f} s)"}

    if rank == 0:
        nmem = 1 if single else (len(w) if isinstance(w, list) else len(run.weights))
        cfg = {"workload": args.workload, "members": nmem,
               "ncells": list(w0.ncells) if single or not isinstance(w, list) else "seeded, see inputs.plane_batch",
               "cfl": w0.cfl, "leapfrog_steps_per_bench_step": steps_per,
               "l2": "flushed (256 MB write) before each timed bench step",
               "parallelism": "replicas" if world > 1 else "single GPU", "form": args.form,
               "persistent": bool(args.persistent)}
        if single:
            cfg["schedule"] = run.solver.schedule()
            cfg["autotune_us_per_step"] = run.solver.tune_us
        if single:
            cfg["bc"] = ["".join(b) for b in w.bc]
        elif not isinstance(w, list):
            cfg["reflection"] = w.refl
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": cfg, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clk.summary(), "gpu_launches": launches,
            "rel_l2_vs_fp64": acc, "energy_drift_fp64": drift, "hbm_case": hbm,
        }
        print(json.dumps(line), flush=True)
    run.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
