"""Throughput of the fused three-population lattice-Boltzmann step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: the sheared drop on a 2048 x 1024 grid (walls at +/-0.01, R = 160, Re = 1, Ca = 0.2,
Langmuir EOS E0 = 0.2, psi0 = 0.3), populations stored in FP32, synthetic seeded fields.  A step is
one lbm_step(1): one launch of the fused collide-stream kernel over the whole grid.  The metric is
MLUPS (million lattice updates per second; one update advances f, g and h of one cell).  The
populations (436 MB) exceed the 129 MB L2, so no flush is needed between steps.

Printed (one JSON line on rank 0): the device-timed throughput, the end-to-end throughput through
the C ABI with host buffers, the roofline of the step kernel against the measured HBM bandwidth,
the FP64 CPU oracle on the host cores as a baseline, and the SM clocks sampled during the run.
With --gpus N > 1 (under torchrun) every rank runs its own replica; the value is the sum of the
lattice updates of all ranks over the slowest rank's time.
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


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    QUERY = ("index,utilization.gpu,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        # the samples go to LBM_RECORD_DIR if it is set, else to a temporary file
        rec = os.environ.get("LBM_RECORD_DIR") or tempfile.gettempdir()
        self.path = os.path.join(rec, f"clocks_bench_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append(dict(util=float(parts[1]), sm=float(parts[2]), smmax=float(parts[3]),
                                 hw=parts[6], hwt=parts[7], swt=parts[8], pcap=parts[9]))
            except ValueError:
                continue
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
                "reasons": sorted(reasons), "samples": len(loaded)}


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


def cpu_baseline(budget_s: float = 12.0):
    """The FP64 oracle on the host cores, on a bounded sample of the same workload: whole steps of
    the 2048 x 1024 grid until about budget_s seconds of CPU time have been spent."""
    import oracle
    from paper_2408_15654_gb300 import workloads as W
    p, f = W.shear_drop_large(NX, NY)
    cores = oracle.set_threads(0)
    s = oracle.Sim(p)
    s.init(**f)
    t0 = time.perf_counter()
    s.step(1)
    t1 = time.perf_counter() - t0
    n = max(1, min(200, int(budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    s.step(n)
    dt = time.perf_counter() - t0
    # the same oracle on one core, a few steps of the same run
    oracle.set_threads(1)
    t0 = time.perf_counter()
    s.step(1)
    t1c = time.perf_counter() - t0
    n1 = max(1, min(20, int(budget_s / 2 / max(t1c, 1e-6))))
    t0 = time.perf_counter()
    s.step(n1)
    dt1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    s.close()
    return {"value": NX * NY * n / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{n} FP64 oracle steps of the 2048x1024 sheared drop after 1 untimed step, "
                      f"OpenMP over rows ({cores} threads)",
            "single_core": {"value": NX * NY * n1 / dt1 / 1e6, "unit": "MLUPS", "cores": 1,
                            "sample": f"{n1} further steps of the same run on one thread, after 1 untimed step"}}


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
    out = {"value": cells * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "storage": storage, "steps": steps,
           "ms_per_step": ms / steps, "schedule": sched, "graph_steps": k, "gpu_launches": b.launches - n0,
           "achieved_gbs": cells * bpl * steps / (ms * 1e-3) / 1e9,
           "frac_of_measured_hbm": cells * bpl * steps / (ms * 1e-3) / 1e9 / measured_peak()[0]}
    if alone_steps:
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(bstream)
        for g in lats:
            g.step(alone_steps)
        a1.record(bstream)
        torch.cuda.synchronize()
        out["one_at_a_time"] = {"value": cells * alone_steps / (a0.elapsed_time(a1) * 1e-3) / 1e6, "unit": "MLUPS",
                                "steps": alone_steps, "gpu_launches": 64 * alone_steps}
    b.close()
    for g in lats:
        g.close()
    return out, cells


def serving_leg(torch, lbm, W, reqs, jobs, policy: str, max_jobs: int, force_fp32: bool = False):
    """Replay the request stream against a lattice server: each job is submitted at its arrival
    time; time to solution = final fields copied out - submission, on the server's clock."""
    import numpy as np

    stream = torch.cuda.Stream()
    srv = lbm.Server(8 << 30 if max_jobs > 1 else 1 << 30, stream, policy=policy, max_jobs=max_jobs,
                     max_cells=8 << 20, chunk_steps=200, graph_steps=16)
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
    bad = [r for r in res if r["status"] != lbm.LBM_OK]
    if bad:
        raise RuntimeError(f"serving job failed: {bad[0]['message']}")
    tts = np.array([r["t_done"] - r["t_submit"] for r in res])
    makespan = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
    lup = sum(r["nx"] * r["ny"] * r["steps"] for r in res)
    return {"policy": policy, "max_jobs": max_jobs, "storage": "fp32" if force_fp32 else "fp32/fp16 as requested",
            "p50_s": float(np.percentile(tts, 50)), "p99_s": float(np.percentile(tts, 99)),
            "mean_s": float(tts.mean()), "makespan_s": makespan, "value": lup / makespan / 1e6, "unit": "MLUPS",
            "lattice_updates": lup, "gpu_launches": st["kernel_launches"], "rounds": st["rounds"]}


def timed_leg(torch, lbm, p, f, args, stream, world, what: str, bytes_per_lup: int):
    """Warm-up, then exactly args.steps steps of one lattice timed with CUDA events on its stream."""
    sim = lbm.Lattice(p, stream=stream)
    sim.init(**f)
    sim.step(args.warmup)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ms_max = barrier_max(ms, world)
    if sim.status != lbm.LBM_OK:
        raise RuntimeError(f"unstable state in the {what} benchmark: {lbm.lbm_last_error()}")
    sim.close()
    cells = p["nx"] * p["ny"]
    ach = cells * bytes_per_lup / (ms / args.steps * 1e-3) / 1e9
    return {"value": cells * args.steps * world / (ms_max * 1e-3) / 1e6, "unit": "MLUPS",
            "ms_per_step": ms_max / args.steps, "achieved_gbs": ach,
            "frac_of_measured_hbm": ach / measured_peak()[0], "algorithmic_bytes_per_lup": bytes_per_lup}


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
    out = {"steps": steps, "sample_cells": len(xs), "n_eps": head["n_eps"]}
    p, f = W.shear_drop_large(NX, NY)
    for st in ("fp32",) + tuple(HALF_MODES):
        sim = lbm.Lattice(dict(p, storage=st, n_eps=head["n_eps"]), stream=stream)
        sim.init(**f)
        sim.step(steps)
        m = sim.moments()
        rel = lambda g, o: float(np.linalg.norm(g - o) / np.linalg.norm(o))  # noqa: E731
        du = np.hypot(m["ux"][ys, xs] - a[:, 4], m["uy"][ys, xs] - a[:, 5])
        out[st] = {"phi": rel(m["phi"][ys, xs], a[:, 2]), "psi": rel(m["psi"][ys, xs], a[:, 3]),
                   "u": float(np.linalg.norm(du) / np.linalg.norm(np.hypot(a[:, 4], a[:, 5]))),
                   "total_phi": abs(sim.total("phi") - head["total_phi"]) / head["total_phi"]}
        sim.close()
    return out


def run_reference(args):
    """--impl reference: the FP64 oracle as it stands on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    import oracle
    from paper_2408_15654_gb300 import workloads as W
    p, f = W.shear_drop_large(NX, NY)
    cores = oracle.set_threads(0)
    s = oracle.Sim(p)
    s.init(**f)
    t0 = time.perf_counter()
    s.step(min(args.warmup, 1) or 1)
    t_step = time.perf_counter() - t0
    budget = 90.0
    k = max(1, min(args.steps, int(budget / max(t_step, 1e-6))))
    t0 = time.perf_counter()
    s.step(k)
    dt = time.perf_counter() - t0
    value = NX * NY * k / dt / 1e6
    sample = (f"{k} of the {args.steps} requested FP64 oracle steps of the 2048x1024 sheared drop "
              f"(bounded to ~{budget:.0f} s), {cores} OpenMP threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": k, "warmup": 1, "ms_per_step": dt / k * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [NX, NY], "parallelism": "host cores (OpenMP)"},
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
    sim = lbm.Lattice(p, stream=stream)
    sim.init(**f)
    cells = NX * NY

    # warm-up
    sim.step(args.warmup)
    torch.cuda.synchronize()

    # device-timed region: exactly K steps, inputs already resident in HBM
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    start.record(stream)
    sim.step(args.steps)
    stop.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop() if sampler else None
    ms = start.elapsed_time(stop)
    ms_max = barrier_max(ms, world)
    st = sim.status
    if st != lbm.LBM_OK:
        raise RuntimeError(f"unstable state during the benchmark: {lbm.lbm_last_error()}")
    value = aggregate_mlups(cells, args.steps, world, ms_max)

    # the same workload with 16-bit population storage (FP32 arithmetic)
    half = {}
    for st, bpl in HALF_MODES.items():
        hs = lbm.Lattice(dict(p, storage=st), stream=stream)
        hs.init(**f)
        hs.step(args.warmup)
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hs.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        hms = barrier_max(e0.elapsed_time(e1), world)
        if hs.status != lbm.LBM_OK:
            raise RuntimeError(f"unstable state in the {st} benchmark: {lbm.lbm_last_error()}")
        hv = cells * args.steps * world / (hms * 1e-3) / 1e6
        hach = cells * bpl / (e0.elapsed_time(e1) / args.steps * 1e-3) / 1e9
        half[st] = {"value": hv, "unit": "MLUPS", "ratio_vs_fp32": hv / (cells * args.steps * world / (ms_max * 1e-3) / 1e6),
                    "ms_per_step": hms / args.steps, "achieved_gbs": hach,
                    "frac_of_measured_hbm": hach / measured_peak()[0], "algorithmic_bytes_per_lup": bpl}
        hs.close()

    # prescribed velocity (f and g only): the convection test's drop at 2048 x 1024
    prescribed = {}
    pp, pf = W.convected_drop(NX, NY, R=160.0)
    for st, bpl in BYTES_PER_LUP_PRESCRIBED.items():
        prescribed[st] = timed_leg(torch, lbm, dict(pp, storage=st), pf, args, stream, world, f"prescribed {st}", bpl)
    prescribed["workload"] = ("drop R=160 carried by an imposed u = (0.05, 0) on 2048x1024, periodic, "
                              "M_phi=1, D=2 (the convection test of Sec. 4 scaled up); f, g only")

    # density ratio 10: the rising bubble of Sec. 4 at R = 256 (1024 x 2048, the same cell count)
    var_rho = {}
    bp, bf = W.rising_bubble(256.0)
    for st, bpl in BYTES_PER_LUP_VAR_RHO.items():
        var_rho[st] = timed_leg(torch, lbm, dict(bp, storage=st), bf, args, stream, world, f"density-ratio {st}", bpl)
    var_rho["workload"] = ("rising bubble R=256 on 1024x2048 (Sec. 4: rho and mu ratio 10, Re=35, Bo=10, Pe=10, "
                           "E0=0.5, linear EOS, walls below and above, gravity); mass-flux history included")

    # errors of every storage mode against the oracle after 10 000 steps (untimed)
    precision = precision_leg(torch, lbm, W, stream) if (rank == 0 and not args.no_precision) else None

    # many lattices at once: the 64-lattice mix, FP32 and FP16 storage
    batch = {}
    if args.batch_steps > 0:
        for st in ("fp32", "fp16"):
            batch[st], bcells = batch_leg(torch, lbm, W, st, args.batch_steps,
                                          alone_steps=100 if st == "fp32" else 0)
        batch["workload"] = (f"64 seeded drops (seed 0), sizes uniform over 128^2, 256^2, 512x256, 1024x512 "
                             f"({bcells} cells), walls at +/-U with U ~ U[0, 0.02], linear EOS")

    # serving: a seeded Poisson stream of sheared-drop jobs against the lattice server
    serving = {}
    if args.serving_requests > 0:
        reqs = W.serving_requests(200, 20.0, seed=0)[:args.serving_requests]
        jobs = [W.serving_job(r) for r in reqs]
        serving = {"workload": (f"the first {len(reqs)} of 200 seeded requests (seed 0): Poisson arrivals at 20/s, "
                                f"sheared drops nx = side ~ U{{256..2048 step 64}}, ny = side/2, R = 40 side/512, "
                                f"steps ~ U[5000, 50000], storage FP32 or FP16 with p = 1/2; p99 over "
                                f"{len(reqs)} jobs")}
        for pol in args.serving_policies.split(","):
            serving[pol] = serving_leg(torch, lbm, W, reqs, jobs, pol, max_jobs=64)
        serving["one_at_a_time_fp32"] = serving_leg(torch, lbm, W, reqs, jobs, "fcfs", max_jobs=1, force_fp32=True)
        del jobs

    # roofline of the step kernel (one launch per step, so launch duration = step time)
    peak, peak_kind = measured_peak()
    launch_s = ms / args.steps * 1e-3
    achieved = cells * BYTES_PER_LUP / launch_s / 1e9
    traffic = profiled_traffic()

    # end to end through the C ABI with pinned host buffers: upload the fields, K steps, read back
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

    if rank == 0:
        base = cpu_baseline() if (world == 1 and not args.no_cpu_baseline) else None
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [NX, NY], "storage": "fp32",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (2 x 218 MB population buffers), no flush"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                         "algorithmic_bytes_per_lup": BYTES_PER_LUP},
            "half_store": half,
            "precision_vs_oracle": precision,
            "prescribed_velocity": prescribed,
            "density_ratio": var_rho,
            "batch": batch,
            "serving": serving,
            "cpu_baseline": base,
            "e2e": {"value": e2e, "unit": "MLUPS", "h2d_bytes_per_step": io_bytes / args.steps,
                    "d2h_bytes_per_step": io_bytes / args.steps,
                    "job": f"lbm_init_fields(host) + lbm_step({args.steps}) + lbm_get_moments(host, all 5)"},
            "gpu_launches": args.steps,
            "gpu_launches_half_store": len(HALF_MODES) * args.steps,
            "gpu_launches_prescribed": len(BYTES_PER_LUP_PRESCRIBED) * args.steps,
            "gpu_launches_density_ratio": len(BYTES_PER_LUP_VAR_RHO) * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the untimed storage-error leg")
    ap.add_argument("--batch-steps", type=int, default=1000, help="steps of the 64-lattice batch legs (0: skip)")
    ap.add_argument("--serving-requests", type=int, default=24,
                    help="requests of the seeded serving stream to replay (at most 200; 0: skip)")
    ap.add_argument("--serving-policies", default="fcfs,shortest_first")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
