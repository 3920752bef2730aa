"""Throughput of the fused three-population lattice-Boltzmann step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: the sheared drop on a 2048 x 1024 grid (walls at +/-0.01, R = 160, Re = 1, Ca = 0.2,
Langmuir EOS E0 = 0.2, psi0 = 0.3), populations stored in FP32, synthetic seeded fields.  A step is
one lbm_step(1): one launch of the fused collide-stream kernel over the whole grid.  The metric is
MLUPS (million lattice updates per second; one update advances f, g and h of one cell).  The
populations (436 MB) exceed the 129 MB L2, so no flush is needed between steps.

Timing: after W untimed steps, windows of exactly K steps are timed with CUDA events on the
lattice's stream, back to back, until at least one second of steps has been timed; the value is
the median window.  nvidia-smi samples the SM clock and throttle reasons over all timed legs.

Printed (one JSON line on rank 0): the device-timed throughput, the end-to-end throughput through
the C ABI with host buffers, the roofline of the step kernel against the measured HBM bandwidth,
the FP64 CPU oracle on the host cores as a baseline (every configuration, all cores and one), the
other legs (square grid, 16-bit storage, prescribed velocity, density ratio, many lattices,
serving) and the storage errors against the oracle.  With --gpus N > 1 (under torchrun) every rank
runs its own replica; the value is the sum of the lattice updates of all ranks over the slowest
rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY = 2048, 1024
BYTES_PER_LUP = 26 * 4 * 2 + 2 * 4 * 2  # 26 live float populations and 2 history floats, read + written
# the survey's count, which also stores phi and psi of the previous level (this design recovers
# them from the cell's own post-collision pairs, which it reads anyway)
BYTES_PER_LUP_SURVEY = 26 * 4 * 2 + 4 * 4 * 2
BYTES_PER_LUP_16 = 26 * 2 * 2 + 2 * 4 * 2  # the same populations stored in 16 bits
BYTES_PER_LUP_FG = 18 * 2 * 2 + 8 * 4 * 2 + 2 * 4 * 2  # f, g in 16 bits, h in FP32
BYTES_PER_LUP_PRESCRIBED = {"fp32": 9 * 8 * 2 + 2 * 4 * 2, "fp16": 9 * 4 * 2 + 2 * 4 * 2}  # f, g and u only
HALF_MODES = {"fp16": BYTES_PER_LUP_16, "bf16": BYTES_PER_LUP_16, "fp16_fg": BYTES_PER_LUP_FG,
              "bf16_fg": BYTES_PER_LUP_FG}
# density ratio != 1: the same populations and u history plus the mass-flux history S (2 floats)
BYTES_PER_LUP_VAR_RHO = {"fp32": BYTES_PER_LUP + 2 * 4 * 2, "fp16": BYTES_PER_LUP_16 + 2 * 4 * 2}
METRIC = "MLUPS (3 lattices) and % HBM roofline, FP32 vs half-store; serving p50/p99"
WORKLOAD = "sheared drop 2048x1024 (R=160, Re=1, Ca=0.2, Langmuir E0=0.2, psi0=0.3), FP32 storage"
PROFILE = os.path.join(ROOT, "profiles", "step_kernel_2048x1024_fp32.json")
KERNEL_SRC = os.path.join(ROOT, "paper_2408_15654_gb300", "csrc", "lbm_kernels.cuh")
MIN_TIMED_S = 1.0        # each device-timed leg times K-step windows until this much has passed
SERVING_MARGIN = 8 << 30  # device memory left free beside the serving arena


def kernel_hash() -> str:
    """Hash of the kernel source without its // comments and blank lines (what the compiler sees)."""
    code = []
    with open(KERNEL_SRC) as f:
        for line in f:
            line = line.split("//", 1)[0].rstrip()
            if line:
                code.append(line)
    return hashlib.sha256("\n".join(code).encode()).hexdigest()[:16]


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this kernel source."""
    try:
        with open(PROFILE) as f:
            prof = json.load(f)
    except (OSError, ValueError):
        return None
    if prof.get("kernel_hash") != kernel_hash():
        return None
    return prof.get("dram_bytes_per_launch")


def sig(x, n=4):
    """x rounded to n significant digits (keeps the JSON line short)."""
    if x is None or isinstance(x, (bool, int)):
        return x
    return float(f"{x:.{n}g}")


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed legs run, plus one query when it
    starts and one when it stops, so that the record exists however short the legs are."""

    QUERY = ("index,utilization.gpu,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        # the samples go to LBM_RECORD_DIR if it is set, else to a temporary file
        rec = os.environ.get("LBM_RECORD_DIR") or tempfile.gettempdir()
        self.path = os.path.join(rec, f"clocks_bench_{os.getpid()}.csv")
        self.edges = [self.query()]
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def query(self):
        try:
            r = subprocess.run(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-i",
                                str(self.gpu)], capture_output=True, text=True, timeout=10)
            return r.stdout.strip()
        except (OSError, subprocess.SubprocessError):
            return ""

    @staticmethod
    def parse(lines):
        rows = []
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append(dict(util=float(parts[1]), sm=float(parts[2]), smmax=float(parts[3]),
                                 hw=parts[6], hwt=parts[7], swt=parts[8], pcap=parts[9]))
            except ValueError:
                continue
        return rows

    def stop(self):
        self.edges.append(self.query())
        rows = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()
            rows = self.parse(open(self.path))
        source = "samples every 200 ms during the timed legs"
        if not rows:
            rows = self.parse(self.edges)
            source = "one query before and one after the timed legs"
        if not rows:
            return None
        loaded = [r for r in rows if r["util"] >= 50] or rows
        reasons = set()
        for r in loaded:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                            ("pcap", "sw_power_cap")):
                if r[k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in loaded), "sm_max_mhz": max(r["smmax"] for r in loaded),
                "reasons": sorted(reasons), "samples": len(loaded), "source": source}


def dist_setup(n_gpus: int, backend: str = "nccl"):
    """Rank, world size and local rank from the launcher's environment; one process per GPU joins
    a process group (NCCL on the GPUs; gloo runs the same host logic on CPU).  Replicas exchange
    nothing on the data path: the group carries only barriers and the max of the timings."""
    import torch
    rank, world, local = 0, 1, 0
    if n_gpus > 1 or "WORLD_SIZE" in os.environ:
        import torch.distributed as dist
        rank = int(os.environ.get("RANK", 0))
        world = int(os.environ.get("WORLD_SIZE", 1))
        local = int(os.environ.get("LOCAL_RANK", 0))
        if world > 1:
            if backend == "nccl":
                torch.cuda.set_device(local)
                dist.init_process_group("nccl", device_id=torch.device("cuda", local))
            else:
                dist.init_process_group(backend)
    return rank, world, local


def barrier_max(value: float, world: int) -> float:
    """The maximum of value over the ranks (the slowest rank's time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(cells_per_rank: int, steps: int, world: int, ms_max: float) -> float:
    """Whole-job throughput of weak-scaled replicas: the updates of all ranks over the slowest
    rank's time."""
    return cells_per_rank * steps * world / (ms_max * 1e-3) / 1e6


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def timed_windows(torch, stream, advance, k: int, min_s: float = None, max_windows: int = 2000):
    """Device time of windows of exactly k steps (advance(k) enqueues them on `stream`), recorded
    back to back with CUDA events until about min_s of steps has been timed.  Returns the median
    window in ms and the number of windows."""
    min_s = MIN_TIMED_S if min_s is None else min_s
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    advance(k)
    e1.record(stream)
    torch.cuda.synchronize()
    first = e0.elapsed_time(e1)
    n = max(0, min(max_windows - 1, int(min_s * 1e3 / max(first, 1e-3)) - 1))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for a, b in ev:
        a.record(stream)
        advance(k)
        b.record(stream)
    torch.cuda.synchronize()
    times = [first] + [a.elapsed_time(b) for a, b in ev]
    return statistics.median(times), len(times)


def oracle_mlups(oracle, p, f, threads: int, budget_s: float, max_steps: int = 200):
    """The FP64 oracle on `threads` host threads: whole steps of one lattice (after 1 untimed step)
    until about budget_s seconds; returns (MLUPS, steps timed)."""
    oracle.set_threads(threads)
    s = oracle.Sim(p)
    s.init(**f)
    t0 = time.perf_counter()
    s.step(1)
    t1 = time.perf_counter() - t0
    n = max(1, min(max_steps, int(budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    s.step(n)
    dt = time.perf_counter() - t0
    s.close()
    return p["nx"] * p["ny"] * n / dt / 1e6, n


def cpu_baselines(budget_s: float = 4.0):
    """The FP64 oracle on the host cores for every configuration: all cores and one core, a bounded
    number of whole steps each; the 64-lattice set as one step of each member in turn until the
    budget is spent."""
    import oracle
    from paper_2408_15654_gb300 import workloads as W
    cores = oracle.set_threads(0)
    cfgs = {"stationary_drop_128x128": W.stationary_drop(), "surface_diffusion_256x256": W.surface_diffusion(),
            "shear_drop_512x256": W.shear_drop(), "shear_drop_2048x1024": W.shear_drop_large(NX, NY)}
    out = {"cores": cores, "unit": "MLUPS"}
    for name, (p, f) in cfgs.items():
        v, n = oracle_mlups(oracle, p, f, cores, budget_s * (3 if name.endswith("2048x1024") else 1))
        v1, n1 = oracle_mlups(oracle, p, f, 1, budget_s)
        out[name] = {"all_cores": sig(v), "steps": n, "one_core": sig(v1), "steps_one_core": n1}
    # the 64-lattice set: members stepped once each, in order, until the budget is spent
    for label, threads in (("all_cores", cores), ("one_core", 1)):
        oracle.set_threads(threads)
        cells, t_total, stepped = 0, 0.0, 0
        for p, f in W.batch_instances(64, seed=0):
            s = oracle.Sim(p)
            s.init(**f)
            t0 = time.perf_counter()
            s.step(1)
            t_total += time.perf_counter() - t0
            s.close()
            cells += p["nx"] * p["ny"]
            stepped += 1
            if t_total > budget_s:
                break
        out.setdefault("batch_mix64", {})[label] = sig(cells / t_total / 1e6)
        out["batch_mix64"]["members_" + label] = stepped
    oracle.set_threads(cores)
    return out


def batch_leg(torch, lbm, W, storage: str, steps: int, alone_steps: int = 0):
    """The 64-lattice mix (sizes 128^2 .. 1024x512, seed 0) advanced by one launch per step:
    autotuned schedule, then `steps` device-timed steps; optionally each lattice alone for
    `alone_steps` steps (one lbm_step launch per lattice and step) for comparison."""
    bstream = torch.cuda.Stream()
    inst = W.batch_instances(64, seed=0)
    lats = []
    for p, f in inst:
        g = lbm.Lattice(dict(p, storage=storage), stream=bstream)
        g.init(**f)
        lats.append(g)
    cells = sum(g.nx * g.ny for g in lats)
    b = lbm.Batch(lats, bstream)
    sched, k = b.autotune(trial_steps=32)
    torch.cuda.synchronize()
    n0 = b.launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(bstream)
    b.step(steps)
    e1.record(bstream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if any(g.status != lbm.LBM_OK for g in lats):
        raise RuntimeError(f"unstable member in the {storage} batch: {lbm.lbm_last_error()}")
    bpl = BYTES_PER_LUP if storage == "fp32" else HALF_MODES[storage]
    out = {"value": sig(cells * steps / (ms * 1e-3) / 1e6), "unit": "MLUPS", "storage": storage, "steps": steps,
           "ms_per_step": sig(ms / steps), "schedule": sched, "graph_steps": k, "gpu_launches": b.launches - n0,
           "achieved_gbs": sig(cells * bpl * steps / (ms * 1e-3) / 1e9),
           "frac_of_measured_hbm": sig(cells * bpl * steps / (ms * 1e-3) / 1e9 / measured_peak()[0])}
    if alone_steps:
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(bstream)
        for g in lats:
            g.step(alone_steps)
        a1.record(bstream)
        torch.cuda.synchronize()
        out["one_at_a_time"] = {"value": sig(cells * alone_steps / (a0.elapsed_time(a1) * 1e-3) / 1e6),
                                "unit": "MLUPS", "steps": alone_steps, "gpu_launches": 64 * alone_steps}
    b.close()
    for g in lats:
        g.close()
    return out, cells


def serving_leg(torch, lbm, W, reqs, jobs, policy: str, max_jobs: int, arena_bytes: int, force_fp32: bool = False):
    """Replay the request stream against a lattice server: each job is submitted at its arrival
    time; time to solution = final fields copied out - submission, on the server's clock.  Jobs
    are admitted while their workspaces fit the arena (sized from the device's free memory) and the
    job cap allows."""
    import numpy as np

    stream = torch.cuda.Stream()
    srv = lbm.Server(arena_bytes, stream, policy=policy, max_jobs=max_jobs, max_cells=1 << 40,
                     chunk_steps=200, graph_steps=16)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r, (p, f) in zip(reqs, jobs):
        delay = t0 + r["t"] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        srv.submit(dict(p, storage="fp32") if force_fp32 else p, f, r["steps"])
    res = []
    while len(res) < len(reqs):
        got = srv.poll(64, timeout=5.0)
        if not got and time.perf_counter() - t0 > 3600:
            raise RuntimeError("server made no progress")
        res += got
    st = srv.stats()
    srv.close()
    del srv
    torch.cuda.empty_cache()
    bad = [r for r in res if r["status"] != lbm.LBM_OK]
    if bad:
        raise RuntimeError(f"serving job failed: {bad[0]['message']}")
    tts = np.array([r["t_done"] - r["t_submit"] for r in res])
    makespan = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
    lup = sum(r["nx"] * r["ny"] * r["steps"] for r in res)
    return {"policy": policy, "max_jobs": max_jobs, "jobs": len(res),
            "storage": "fp32" if force_fp32 else "fp32/fp16 as requested",
            "p50_s": sig(float(np.percentile(tts, 50))), "p99_s": sig(float(np.percentile(tts, 99))),
            "mean_s": sig(float(tts.mean())), "makespan_s": sig(makespan), "value": sig(lup / makespan / 1e6),
            "unit": "MLUPS", "lattice_updates": lup, "gpu_launches": st["kernel_launches"], "rounds": st["rounds"]}


def lattice_leg(torch, lbm, p, f, args, stream, world, what: str, bytes_per_lup):
    """Warm-up, then median K-step windows of one lattice (CUDA events on its stream)."""
    sim = lbm.Lattice(p, stream=stream)
    sim.init(**f)
    sim.step(args.warmup)
    torch.cuda.synchronize()
    barrier(world)
    ms, nwin = timed_windows(torch, stream, sim.step, args.steps)
    ms_max = barrier_max(ms, world)
    if sim.status != lbm.LBM_OK:
        raise RuntimeError(f"unstable state in the {what} benchmark: {lbm.lbm_last_error()}")
    kernel = sim.kernel
    sim.close()
    cells = p["nx"] * p["ny"]
    out = {"value": sig(cells * args.steps * world / (ms_max * 1e-3) / 1e6), "unit": "MLUPS",
           "us_per_step": sig(ms_max / args.steps * 1e3), "windows": nwin, "kernel": kernel}
    if bytes_per_lup:
        ach = cells * bytes_per_lup / (ms / args.steps * 1e-3) / 1e9
        out.update({"achieved_gbs": sig(ach), "frac_of_measured_hbm": sig(ach / measured_peak()[0]),
                    "algorithmic_bytes_per_lup": bytes_per_lup})
    return out


GOLDEN = os.path.join(ROOT, "tests", "golden", "shear_drop_2048x1024_10000_samples.txt")


def precision_leg(torch, lbm, W, stream):
    """The precision configuration's errors: every storage mode after the oracle's 10 000 steps of
    the 2048 x 1024 sheared drop, against the oracle's FP64 values at its seeded sample cells (the
    golden file written by the oracle alone); relative L2 over the samples, u against the sampled
    speed.  Not part of any timed region."""
    if not os.path.exists(GOLDEN):
        return None
    head, rows = {}, []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#"):
                parts = line[1:].split()
                if len(parts) == 2:
                    try:
                        head[parts[0]] = float(parts[1])
                    except ValueError:
                        pass
            elif line.strip():
                rows.append([float(v) for v in line.split()])
    import numpy as np
    a = np.array(rows)
    xs, ys = a[:, 0].astype(int), a[:, 1].astype(int)
    steps = int(head["steps"])
    out = {"steps": steps, "cells": len(xs), "n_eps": head["n_eps"]}
    p, f = W.shear_drop_large(NX, NY)
    for st in ("fp32",) + tuple(HALF_MODES):
        sim = lbm.Lattice(dict(p, storage=st, n_eps=head["n_eps"]), stream=stream)
        sim.init(**f)
        sim.step(steps)
        m = sim.moments()
        rel = lambda g, o: float(np.linalg.norm(g - o) / np.linalg.norm(o))  # noqa: E731
        du = np.hypot(m["ux"][ys, xs] - a[:, 4], m["uy"][ys, xs] - a[:, 5])
        out[st] = {"phi": sig(rel(m["phi"][ys, xs], a[:, 2]), 2), "psi": sig(rel(m["psi"][ys, xs], a[:, 3]), 2),
                   "u": sig(float(np.linalg.norm(du) / np.linalg.norm(np.hypot(a[:, 4], a[:, 5]))), 2),
                   "sum_phi": sig(abs(sim.total("phi") - head["total_phi"]) / head["total_phi"], 2)}
        sim.close()
    return out


def run_reference(args):
    """--impl reference: the FP64 oracle as it stands on the host cores (rank 0 only), on the same
    workload; W untimed steps (at most 3, each takes seconds), then up to K timed steps bounded to
    about 90 s."""
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    import oracle
    from paper_2408_15654_gb300 import workloads as W
    p, f = W.shear_drop_large(NX, NY)
    cores = oracle.set_threads(0)
    s = oracle.Sim(p)
    s.init(**f)
    warm = max(1, min(args.warmup, 3))
    t0 = time.perf_counter()
    s.step(warm)
    t_step = (time.perf_counter() - t0) / warm
    budget = 90.0
    k = max(1, min(args.steps, int(budget / max(t_step, 1e-6))))
    t0 = time.perf_counter()
    s.step(k)
    dt = time.perf_counter() - t0
    value = NX * NY * k / dt / 1e6
    sample = (f"{k} of the {args.steps} requested FP64 oracle steps of the 2048x1024 sheared drop "
              f"(bounded to ~{budget:.0f} s) after {warm} untimed, {cores} OpenMP threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": k, "warmup": warm, "ms_per_step": dt / k * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "FP64 CPU oracle (the reference arm) on " + WORKLOAD.replace(", FP32 storage", ""),
                   "grid": [NX, NY], "parallelism": f"host cores (OpenMP, {cores} threads)"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    from paper_2408_15654_gb300 import lbm
    from paper_2408_15654_gb300 import workloads as W

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    lbm.load()
    p, f = W.shear_drop_large(NX, NY)
    stream = torch.cuda.current_stream()
    cells = NX * NY
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None

    # ---- headline: FP32 storage, 2048 x 1024, inputs resident in HBM ----
    sim = lbm.Lattice(p, stream=stream)
    sim.init(**f)
    sim.step(args.warmup)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ms, nwin = timed_windows(torch, stream, sim.step, args.steps)
    torch.cuda.synchronize()
    barrier(world)
    ms_max = barrier_max(ms, world)
    if sim.status != lbm.LBM_OK:
        raise RuntimeError(f"unstable state during the benchmark: {lbm.lbm_last_error()}")
    value = aggregate_mlups(cells, args.steps, world, ms_max)
    timed_steps = args.steps * nwin

    # ---- the same workload with 16-bit population storage (FP32 arithmetic) ----
    half = {}
    for st, bpl in HALF_MODES.items():
        r = lattice_leg(torch, lbm, dict(p, storage=st), f, args, stream, world, st, bpl)
        half[st] = {"MLUPS": r["value"], "x_fp32": sig(r["value"] / value, 3), "us": r["us_per_step"],
                    "hbm_frac": r["frac_of_measured_hbm"], "B_per_lup": bpl}

    # ---- the square 2048 x 2048 grid (the second roofline lattice), FP32 and FP16 ----
    sp, sf = W.shear_drop(NX, NX, R=160.0)
    square = {st: lattice_leg(torch, lbm, dict(sp, storage=st), sf, args, stream, world, f"2048^2 {st}",
                              BYTES_PER_LUP if st == "fp32" else BYTES_PER_LUP_16) for st in ("fp32", "fp16")}
    square["workload"] = "sheared drop 2048x2048 (walls +/-0.01, R=160, Re=1, Ca=0.2, Langmuir E0=0.2)"

    # ---- the small configurations, FP32 (L2-resident, launch-bound: MLUPS only) ----
    small = {}
    for name, (cp, cf) in {"stationary_drop_128x128": W.stationary_drop(),
                           "surface_diffusion_256x256": W.surface_diffusion(),
                           "shear_drop_512x256": W.shear_drop()}.items():
        small[name] = lattice_leg(torch, lbm, cp, cf, args, stream, world, name, None)

    # ---- prescribed velocity (f and g only): the convection test's drop at 2048 x 1024 ----
    prescribed = {}
    pp, pf = W.convected_drop(NX, NY, R=160.0)
    for st, bpl in BYTES_PER_LUP_PRESCRIBED.items():
        prescribed[st] = lattice_leg(torch, lbm, dict(pp, storage=st), pf, args, stream, world, f"prescribed {st}", bpl)
    prescribed["workload"] = ("drop R=160 carried by an imposed u = (0.05, 0) on 2048x1024, periodic, "
                              "M_phi=1, D=2 (the convection test of Sec. 4 scaled up); f, g only")

    # ---- density ratio 10: the rising bubble of Sec. 4 at R = 256 (1024 x 2048) ----
    var_rho = {}
    bp, bf = W.rising_bubble(256.0)
    for st, bpl in BYTES_PER_LUP_VAR_RHO.items():
        var_rho[st] = lattice_leg(torch, lbm, dict(bp, storage=st), bf, args, stream, world, f"density-ratio {st}", bpl)
    var_rho["workload"] = ("rising bubble R=256 on 1024x2048 (Sec. 4: rho and mu ratio 10, Re=35, Bo=10, Pe=10, "
                           "E0=0.5, linear EOS, walls below and above, gravity); mass-flux history included")

    # ---- many lattices at once: the 64-lattice mix, FP32 and FP16 storage ----
    batch = {}
    if args.batch_steps > 0:
        for st in ("fp32", "fp16"):
            batch[st], bcells = batch_leg(torch, lbm, W, st, args.batch_steps,
                                          alone_steps=args.batch_alone_steps if st == "fp32" else 0)
        batch["workload"] = (f"64 seeded drops (seed 0), sizes uniform over 128^2, 256^2, 512x256, 1024x512 "
                             f"({bcells} cells), walls at +/-U with U ~ U[0, 0.02], linear EOS")
    clocks = sampler.stop() if sampler else None

    # ---- errors of every storage mode against the oracle after 10 000 steps (untimed) ----
    precision = precision_leg(torch, lbm, W, stream) if (rank == 0 and not args.no_precision) else None

    # ---- roofline of the step kernel (one launch per step, so launch duration = step time) ----
    peak, peak_kind = measured_peak()
    launch_s = ms / args.steps * 1e-3
    achieved = cells * BYTES_PER_LUP / launch_s / 1e9
    achieved_survey = cells * BYTES_PER_LUP_SURVEY / launch_s / 1e9
    traffic = profiled_traffic()

    # ---- end to end through the C ABI with pinned host buffers: upload the fields, K steps, read back ----
    host_in = {k: torch.from_numpy(np.array(v, dtype=np.float64)).pin_memory().numpy() for k, v in f.items()}
    host_out = [torch.empty((NY, NX), dtype=torch.float64).pin_memory().numpy() for _ in range(5)]
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    lbm.lbm_init_fields(sim.handle, *[host_in[k] for k in lbm.FIELDS], mem=lbm.LBM_MEM_HOST)
    sim.step(args.steps)
    lbm.lbm_get_moments(sim.handle, 31, host_out, lbm.LBM_MEM_HOST)
    e2e_s = barrier_max(time.perf_counter() - t0, world)
    e2e = cells * args.steps * world / e2e_s / 1e6
    io_bytes = 5 * cells * 8
    sim.close()
    del sim, host_in, host_out
    torch.cuda.empty_cache()

    # ---- serving: a seeded Poisson stream of sheared-drop jobs against the lattice server ----
    serving = {}
    if args.serving_requests > 0:
        reqs = W.serving_requests(200, 20.0, seed=0)[:args.serving_requests]
        jobs = [W.serving_job(r) for r in reqs]
        free, total = torch.cuda.mem_get_info()
        arena = max(1 << 30, free - SERVING_MARGIN)
        serving = {"workload": (f"the first {len(reqs)} of 200 seeded requests (seed 0): Poisson arrivals at 20/s, "
                                f"sheared drops on square grids side ~ U{{256..2048 step 64}}, R = 40 side/512, "
                                f"steps ~ U[5000, 50000], storage FP32 or FP16 with p = 1/2"),
                   "admission": (f"job workspaces from an arena of {arena >> 20} MiB, the device's free memory at "
                                 f"start less {SERVING_MARGIN >> 30} GiB; at most 64 jobs at once")}
        for pol in args.serving_policies.split(","):
            serving[pol] = serving_leg(torch, lbm, W, reqs, jobs, pol, 64, arena)
        # one job at a time, on the first requests of the same stream: with the storage each job
        # asked for (what continuous batching adds) and all in FP32 (the plain path)
        n1 = min(len(reqs), args.serving_alone) if args.serving_alone > 0 else len(reqs)
        serving["one_at_a_time"] = serving_leg(torch, lbm, W, reqs[:n1], jobs[:n1], "fcfs", 1, arena)
        serving["one_at_a_time_fp32"] = serving_leg(torch, lbm, W, reqs[:n1], jobs[:n1], "fcfs", 1, arena,
                                                     force_fp32=True)
        del jobs

    if rank == 0:
        base = cpu_baselines() if (world == 1 and not args.no_cpu_baseline) else None
        head = base["shear_drop_2048x1024"] if base else None
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [NX, NY], "storage": "fp32",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (2 x 218 MB population buffers), no flush",
                       "timing": f"median of {nwin} back-to-back windows of {args.steps} steps ({timed_steps} steps)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                         "algorithmic_bytes_per_lup": BYTES_PER_LUP,
                         "survey_bytes_per_lup": BYTES_PER_LUP_SURVEY,
                         "frac_at_survey_bytes": achieved_survey / peak},
            "cpu_baseline": ({"value": head["all_cores"], "unit": "MLUPS", "cores": base["cores"], "kind": "oracle",
                              "sample": f"{head['steps']} FP64 oracle steps of the 2048x1024 sheared drop after 1 "
                                        f"untimed step, OpenMP over rows ({base['cores']} threads); every "
                                        f"configuration on all cores and one core in cpu_baselines"}
                             if base else None),
            "e2e": {"value": e2e, "unit": "MLUPS", "h2d_bytes_per_step": io_bytes / args.steps,
                    "d2h_bytes_per_step": io_bytes / args.steps,
                    "job": f"lbm_init_fields(host) + lbm_step({args.steps}) + lbm_get_moments(host, all 5)"},
            "gpu_launches": timed_steps,
            "serving": serving,
            "batch": batch,
            "density_ratio": var_rho,
            "prescribed_velocity": prescribed,
            "small_configs_fp32": small,
            "cpu_baselines": base,
            "square_2048x2048": square,
            "gpu_launches_half_store": len(HALF_MODES) * args.steps,
            "clocks": clocks,
            # last, so that a reader of the line's tail sees them: each 16-bit mode against FP32 at
            # 2048 x 1024, and every storage mode's error against the oracle after 10 000 steps
            "half_store": half,
            "precision_vs_oracle": precision,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--timed-seconds", type=float, default=1.0,
                    help="device time each timed leg spends in K-step windows (0: one window)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the untimed storage-error leg")
    ap.add_argument("--batch-steps", type=int, default=1000, help="steps of the 64-lattice batch legs (0: skip)")
    ap.add_argument("--batch-alone-steps", type=int, default=100,
                    help="steps of each batch lattice run alone, one launch per lattice and step (0: skip)")
    ap.add_argument("--serving-requests", type=int, default=100,
                    help="requests of the seeded serving stream to replay (at most 200; 0: skip)")
    ap.add_argument("--serving-policies", default="fcfs", help="comma-separated: fcfs, shortest_first")
    ap.add_argument("--serving-alone", type=int, default=24,
                    help="requests replayed one job at a time for comparison (0: all of them)")
    args = ap.parse_args()
    global MIN_TIMED_S
    MIN_TIMED_S = max(0.0, args.timed_seconds)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
