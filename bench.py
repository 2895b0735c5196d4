#!/usr/bin/env python
"""Benchmark of the DUWP per-time-step hot path on GB300: particle-updates/s and the fraction of
the measured HBM bandwidth the streaming kernel reaches, plus step-latency percentiles, the
graph-replayed step, the plain one-instance-at-a-time FP64 loop, an end-to-end number through
the C ABI with host buffers, and the CPU oracle as a reported baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload batch64|mach8|sod] [--impl reference]

A step is one DUWP time step (Sec. 3.4 of the paper) of every instance of the workload.  A
particle-update is one particle streamed through one step (counted after absorption and
re-sampling).  Algorithmic bytes per particle-update: one read and one write of the particle
record, 32 B for FP32 records (64 B for FP64).  Default workload: 64 uneven Mach 1.2-8 argon
shock instances (100-4000 cells, 100-1000 particles per cell, FP32 particles, FP64 cells) in one
batch; about 1.4e8 particles, so the 2.2 GB of particle records per buffer exceed the 129 MB L2
and every step streams them from HBM.  Under torchrun each rank runs its own copy of the batch
(independent seeds): weak scaling with no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DUWP particle-updates/s"
UNIT = "particle-updates/s"


# ---------------------------------------------------------------------------- workloads
def _one_gpu_workload(name: str):
    """The instances of one GPU's share of the workload and its description."""
    from paper_2305_12071_gb300 import workloads as W
    if name == "batch64":
        ps = W.config3_batch(64, precision="fp32")
        return ps, {"workload": "batch64_shock_fp32", "instances": 64, "mach": "U[1.2,8]",
                    "cells": "U[100,4000]", "ppc_ref": "U[100,1000]", "omega": 0.81, "records": "fp32",
                    "cell_state": "fp64"}
    if name == "mach8":
        return [W.config4("fp32")], {"workload": "mach8_shock_1e5cells_fp32", "instances": 1, "cells": 100_000,
                                     "Kn": 0.1, "ppc_ref": 415, "omega": 0.68, "records": "fp32",
                                     "cell_state": "fp64"}
    if name == "mach8_fp64":
        return [W.config4("fp64")], {"workload": "mach8_shock_1e5cells_fp64", "instances": 1, "cells": 100_000,
                                     "Kn": 0.1, "ppc_ref": 415, "omega": 0.68, "records": "fp64",
                                     "cell_state": "fp64"}
    if name == "mach3":
        return [W.config1("fp64")], {"workload": "mach3_shock_100cells_fp64", "instances": 1, "cells": 100,
                                     "ppc_ref": 200, "omega": 0.81, "records": "fp64", "cell_state": "fp64"}
    if name == "sod":
        return [W.config2(Kn=1e-4, precision="fp32")], {"workload": "sod_1000cells_kn1e-4_fp32", "instances": 1,
                                                        "cells": 1000, "ppc_ref": 500, "records": "fp32",
                                                        "cell_state": "fp64"}
    if name == "sod_kn":
        # the Sod tube's Kn range (1e-4 .. 1) as one batch: 5 Knudsen numbers x 5 seeds, 1000 cells each
        kns = (1e-4, 1e-3, 1e-2, 1e-1, 1.0)
        ps = [W.config2(Kn=kn, precision="fp32", seed=1 + s) for kn in kns for s in range(5)]
        return ps, {"workload": "sod_1000cells_kn1e-4..1_x5seeds_fp32", "instances": len(ps), "cells": 1000,
                    "ppc_ref": 500, "Kn": list(kns), "records": "fp32", "cell_state": "fp64"}
    if name == "sod_sweep":
        # the paper's Sod Kn sweep (Sec. 4.2, Fig. 5): 100 cells, Kn 1e-5 .. 1e-2, many seeds at once
        kns = (1e-5, 1e-4, 1e-3, 1e-2)
        ps = [W.sod(n_cells=100, Kn=kn, ppc_ref=500.0, precision="fp32", seed=1 + s)
              for kn in kns for s in range(16)]
        return ps, {"workload": "sod_sweep_100cells_kn1e-5..1e-2_x16_fp32", "instances": len(ps), "cells": 100,
                    "ppc_ref": 500, "Kn": list(kns), "records": "fp32", "cell_state": "fp64"}
    raise SystemExit(f"unknown workload {name}")


def job(name: str, world: int = 1):
    """The whole job on `world` GPUs: `world` copies of the one-GPU workload with independent seeds
    (weak scaling), and its description."""
    base, cfg = _one_gpu_workload(name)
    plist = []
    for c in range(world):
        for p in base:
            q = dict(p)
            q["seed"] = int(p["seed"]) + 100_000 * c
            plist.append(q)
    return plist, cfg


def workload(name: str, rank: int = 0, world: int = 1):
    """The instances rank `rank` of `world` runs: whole instances of the job placed on the ranks by
    their device-memory footprint (no exchange between ranks), and the job's description."""
    from paper_2305_12071_gb300 import placement
    plist, cfg = job(name, world)
    mine = placement.assign(plist, world)[rank]
    cfg = dict(cfg)
    if world > 1:
        cfg["placement"] = "whole instances by footprint (largest first, least-loaded rank)"
    return [plist[i] for i in mine], cfg


def shard(n_items: int, rank: int, world: int):
    """Items of one rank when a list is split across ranks (round robin)."""
    return list(range(rank, n_items, world))


def aggregate(updates_per_rank, seconds_per_rank):
    """Whole-job throughput: all updates over the slowest rank's time."""
    t = max(seconds_per_rank)
    return (sum(updates_per_rank) / t) if t > 0 else 0.0


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.p = None
        self.lines = []

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------- helpers
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    """sha256 (first 16 hex) of the streaming kernel's source: the fixed-point moment helpers it
    calls and the part of csrc/duwp_kernels.cu from its section header to the far-mover sort that
    follows it."""
    with open(os.path.join(ROOT, "paper_2305_12071_gb300", "csrc", "duwp_kernels.cu"), encoding="utf-8") as fh:
        src = fh.read()
    f0 = src.index("// Exact fixed-point sums of particle moments")
    f1 = src.index("// Prefetch of the 128-byte line", f0)
    a = src.index("// Streaming kernel: one warp per cell.")
    b = src.index("// Far movers: rank sort", a)
    return hashlib.sha256((src[f0:f1] + src[a:b]).encode()).hexdigest()[:16]


def profiled_traffic(workload_name: str, updates_per_launch: float):
    """DRAM bytes per launch of the streaming kernel from the committed ncu summary, when it was
    taken on the current kernel source and on this workload (the 64-instance batch, Eq. (p) split);
    scaled by the particle-updates of a launch."""
    if workload_name != "batch64":
        return None, None
    path = os.path.join(ROOT, "profiles", "k_stream_ncu.md")
    try:
        txt = open(path).read()
    except OSError:
        return None, None
    m = re.search(r"kernel source hash:\s*`?([0-9a-f]{16})", txt)
    b = re.search(r"dram bytes per particle-update:\s*([0-9.]+)", txt)
    if not m or not b or m.group(1) != kernel_source_hash():
        return None, None
    per = float(b.group(1))
    return per * updates_per_launch, per


def oracle_sample(params_list, sample_idx, min_steps: int = 2, budget_s: float = 10.0, warm: int = 1):
    """Time the CPU oracle (single thread) on a sample of the instances: rounds of one step of every
    sampled instance, at least min_steps rounds and until about budget_s seconds of oracle time.
    Returns (particle-updates, seconds, rounds)."""
    import oracle as O
    inst = [O.Oracle(params_list[i]) for i in sample_idx]
    for o in inst:
        o.step(warm)
    updates, rounds = 0, 0
    t0 = time.perf_counter()
    while rounds < min_steps or time.perf_counter() - t0 < budget_s:
        for o in inst:
            before = o.num_particles()
            o.step(1)
            c = o.counters()
            # particles streamed = arrived - absorbed + re-sampled (interior cells)
            updates += before - int(c["nabs"].sum()) + int(c["nnew"].sum())
        rounds += 1
    dt = time.perf_counter() - t0
    return updates, dt, rounds


def _oracle_worker(job):
    """One process of the all-cores oracle line: oracle_sample on one instance."""
    params, budget_s = job
    ups, secs, rounds = oracle_sample([params], [0], budget_s=budget_s)
    return ups, secs, rounds


def oracle_all_cores(params_list, budget_s: float = 10.0):
    """The oracle on every host core at once: one process per instance (the oracle itself is
    single-threaded and instances are independent), each timed like oracle_sample.  Processes
    are spawned (this process already uses the GPU).  Returns (updates, seconds, processes):
    seconds the longest worker's timed span."""
    import multiprocessing as mp
    ncores = max(1, min(os.cpu_count() or 1, len(params_list)))
    step = max(1, len(params_list) // ncores)
    jobs = [(params_list[i], budget_s) for i in range(0, len(params_list), step)][:ncores]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(_oracle_worker, jobs)
    return sum(r[0] for r in res), max(r[1] for r in res), len(jobs)


# ---------------------------------------------------------------------------- serving
def serving_run(serve_seconds: float, device: int = 0, lanes: int = 1, long_steps: int = 2000,
                steps_per_launch: int = 32) -> dict:
    """Continuous batching under Poisson arrivals (50 requests/s of shock and Sod problems, cells
    log-uniform in [100, 1e4], 100-1000 particles per cell, Kn log-uniform in [1e-4, 1]): arrivals
    are replayed in real time for serve_seconds, then the server drains.  Returns the p50/p99 solve
    latency (arrival -> result) and the aggregate particle-updates/s."""
    from paper_2305_12071_gb300 import build as B
    from paper_2305_12071_gb300 import duwp
    from paper_2305_12071_gb300 import workloads as W
    B.build()
    reqs = W.serving_mix(duration_s=serve_seconds, rate_hz=50.0, precision="fp32")
    srv = duwp.Server(hbm_budget_bytes=96 << 30, max_slots=128, max_cells=1_000_000, steps_per_launch=steps_per_launch,
                      precision="fp32", device=device, lanes=lanes, long_steps=long_steps)
    pending, lat, queue_ms, run_ms = {}, [], [], []
    updates, i, failed = 0, 0, 0
    t0 = time.perf_counter()
    limit = 20.0 * serve_seconds + 60.0
    while (i < len(reqs) or pending) and time.perf_counter() - t0 < limit:
        now = time.perf_counter() - t0
        while i < len(reqs) and reqs[i][0] <= now:
            pending[srv.submit(reqs[i][1], reqs[i][2])] = reqs[i][0]
            i += 1
        for rid in list(pending):
            r = srv.poll(rid)
            if r is None:
                continue
            lat.append(time.perf_counter() - t0 - pending.pop(rid))
            updates += int(r["particle_updates"])
            queue_ms.append(r["queue_ms"])
            run_ms.append(r["run_ms"])
            failed += int(r["status"] != 0)
        time.sleep(0.001)
    wall = time.perf_counter() - t0
    srv.close()
    lat_s = sorted(lat)

    def pct(v, q):
        return v[min(len(v) - 1, int(math.ceil(q * len(v))) - 1)] if v else None

    return {"metric": "serving solve latency (arrival -> result)", "value": pct(lat_s, 0.5), "unit": "s",
            "p50_s": pct(lat_s, 0.5), "p99_s": pct(lat_s, 0.99), "higher_is_better": False,
            "requests": len(reqs), "completed": len(lat), "failed": failed,
            "unfinished": len(pending), "wall_s": wall,
            "particle_updates_per_s": updates / wall if wall > 0 else None,
            "queue_ms_p50": pct(sorted(queue_ms), 0.5), "run_ms_p50": pct(sorted(run_ms), 0.5),
            "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving_poisson50_mixed_fp32", "arrivals_s": serve_seconds,
                       "rate_hz": 50, "cells": "log-U[100,1e4]", "ppc_ref": "U[100,1000]",
                       "Kn": "log-U[1e-4,1]", "shock_steps": 500, "sod_steps": "to t = 0.15 at CFL 0.5",
                       "steps_per_launch": steps_per_launch, "max_slots": 128, "lanes": lanes,
                       "long_steps": long_steps if lanes > 1 else None}}


def run_serving(args, rank: int, world: int):
    if rank != 0:
        return
    print(json.dumps(serving_run(args.serve_seconds, int(os.environ.get("LOCAL_RANK", 0)))), flush=True)


# ---------------------------------------------------------------------------- the other configurations
# (key, workload, timed steps, warm-up steps): the configurations beside the headline batch, each as
# the step count it is specified with (configs 1, 2, 4; config 5 is the serving run)
SECONDARY = (
    ("config1_mach3_shock_100cells_fp64", "mach3", 500, 5),
    ("config2_sod_1000cells_kn1e-4..1_fp32", "sod_kn", 2000, 5),
    ("config2_sod_1000cells_kn1e-4_fp32", "sod", 2000, 5),
    ("sod_sweep_fig5_100cells_kn1e-5..1e-2_fp32", "sod_sweep", 2000, 5),
    ("config4_mach8_shock_1e5cells_fp32", "mach8", 200, 3),
    ("config4_mach8_shock_1e5cells_fp64", "mach8_fp64", 200, 3),
)


def secondary_run(name: str, steps: int, warmup: int, device: int, peak: float, oracle_budget_s: float = 3.0):
    """One configuration on one GPU: K steps timed as the library runs them (events per step), the
    kernels timed one by one over up to 20 steps (the streaming kernel's roofline), and the oracle
    on a bounded sample of the same instances when they are small enough."""
    import torch
    from paper_2305_12071_gb300 import autotune, duwp
    plist, cfg = workload(name)
    rec_bytes = 16 if plist[0].get("precision", "fp64") == "fp32" else 32
    sol = duwp.Solver(plist, device=device)
    sol.step(warmup)
    sol.sync()
    (t_best, r_best, g_best), _ = autotune.tune(sol)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.synchronize()
    u0 = sol.particle_updates()
    with torch.cuda.stream(sol.stream):
        evs[0].record()
    for j in range(steps):
        sol.step(1)
        with torch.cuda.stream(sol.stream):
            evs[j + 1].record()
    sol.sync()
    upd = sol.particle_updates() - u0
    step_ms = sorted(evs[j].elapsed_time(evs[j + 1]) for j in range(steps))
    span = evs[0].elapsed_time(evs[-1]) / 1e3
    kt = min(steps, 20)
    u2 = sol.particle_updates()
    kms, _ = sol.step_timed(kt)
    upl = (sol.particle_updates() - u2) / kt
    slots = duwp.Solver.KERNEL_SLOTS
    k_ms = kms[slots["k_stream"]] / kt
    achieved = rec_bytes * 2 * upl / (k_ms * 1e-3) / 1e9
    out = {"value": upd / span, "unit": UNIT, "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * span / steps,
           "step_ms_p50": step_ms[len(step_ms) // 2],
           "step_ms_p99": step_ms[min(len(step_ms) - 1, int(math.ceil(0.99 * len(step_ms))) - 1)],
           "dtype": "f32" if rec_bytes == 16 else "f64", "config": dict(cfg, launch={"threads": t_best, "reg_capped": r_best, "groups": g_best}),
           "particles": int(sum(sol.num_particles(i) for i in range(sol.n))),
           "kernel_ms_per_step": {n: float(kms[i] / kt) for n, i in slots.items()},
           "roofline": {"bound": "hbm", "kernel": "k_stream", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "algorithmic_bytes_per_update": rec_bytes * 2,
                        "updates_per_launch": upl, "launch_ms": k_ms}}
    sol.close()
    del sol
    torch.cuda.empty_cache()
    # the oracle (one host core) on a bounded sample: one instance per distinct problem, rounds of
    # one step each until about oracle_budget_s seconds
    est = sum(int(p["n_cells"]) * float(p["ppc_ref"]) for p in plist[:1])
    if est <= 2e6:
        idx = list(range(0, len(plist), max(1, len(plist) // 5)))[:5]
        ups, secs, rounds = oracle_sample(plist, idx, min_steps=1, budget_s=oracle_budget_s)
        out["cpu_baseline"] = {"value": ups / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"instances {idx}, 1 untimed + {rounds} timed steps each"}
    else:
        out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": "not run: the instance exceeds a bounded oracle sample"}
    return out


# ---------------------------------------------------------------------------- reference arm
def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    plist, cfg = workload(args.workload, 0)
    n = len(plist)
    sample = list(range(0, n, max(1, n // 4)))[:4] if n > 1 else [0]
    import oracle as O
    inst = [O.Oracle(plist[i]) for i in sample]
    if args.workload == "mach8":
        # one instance of 1e8 particles: the oracle takes a bounded piece of it per step
        raise SystemExit(json.dumps({"impl": "reference", "unavailable": "oracle sample of the 1e8-particle "
                                     "instance exceeds the few-minute bound of the reference arm"}))
    for _ in range(args.warmup):
        for o in inst:
            o.step(1)
    times, ups = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for o in inst:
            before = o.num_particles()
            o.step(1)
            c = o.counters()
            ups += before - int(c["nabs"].sum()) + int(c["nnew"].sum())
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = ups / tot
    cfg = dict(cfg)
    cfg["sample"] = f"instances {sample} of the batch (oracle, one thread)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": cfg["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- our arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch64",
                    choices=["batch64", "mach8", "mach8_fp64", "mach3", "sod", "sod_kn", "sod_sweep", "serve"])
    ap.add_argument("--split", default="p", choices=["p", "qmc"],
                    help="split fraction: Eq. (p) (default) or the QMC variant 1 - exp(-dt/tau)")
    ap.add_argument("--recon", default="first", choices=["first", "vanleer"],
                    help="wave-flux interface states: first order (default) or van Leer reconstruction")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="arrival window of --workload serve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configurations (Mach-3, Sod, Mach-8 FP32/FP64, serving) beside the headline")
    ap.add_argument("--latency-seconds", type=float, default=1.0,
                    help="steps run after the timed region for the step-latency percentiles")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--launch", default="", help="streaming-kernel launch shape threads,reg_capped[,groups] "
                                                 "(skips the autotuner)")
    ap.add_argument("--instances", type=int, default=0, help="use only the first N instances of the batch")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.workload == "serve" and args.impl != "reference":
        run_serving(args, rank, world)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2305_12071_gb300 import build as B
    B.build()
    from paper_2305_12071_gb300 import duwp

    torch.cuda.set_device(local)
    plist, cfg = workload(args.workload, rank, world)
    if args.split != "p":
        plist = [dict(q, split_mode=args.split) for q in plist]
        cfg = dict(cfg, split_mode=args.split)
    if args.recon != "first":
        plist = [dict(q, recon_mode=args.recon) for q in plist]
        cfg = dict(cfg, recon_mode=args.recon)
    if args.instances:
        plist = plist[:args.instances]
        cfg = dict(cfg, instances=len(plist), workload=cfg["workload"] + f"_first{len(plist)}")
    fp32 = plist[0].get("precision", "fp64") == "fp32"
    rec_bytes = 16 if fp32 else 32

    sol = duwp.Solver(plist, device=local)
    sol.step(args.warmup)
    sol.sync()
    tuned = None
    if args.launch:
        knobs = [int(x) for x in args.launch.split(",")]
        t_l, r_l, g_l = (knobs + [0, 2])[:3] if len(knobs) < 3 else knobs[:3]
        sol.set_launch(t_l, r_l, g_l)
        tuned = {"threads": t_l, "reg_capped": r_l, "groups": g_l, "candidates_ms": None}
    elif not args.no_tune:
        from paper_2305_12071_gb300 import autotune
        (t_best, r_best, g_best), tune_ms = autotune.tune(sol)
        tuned = {"threads": t_best, "reg_capped": r_best, "groups": g_best, "candidates_ms": tune_ms}

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ------------------------------------------------ timed region: K steps as the library runs them
    # (one CUDA graph per step: the collision kernel with the free cells streaming beside it, then the
    # other cells), an event on the library's stream after every step
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    barrier()
    u0 = sol.particle_updates()
    with torch.cuda.stream(sol.stream):
        evs[0].record()
    for j in range(args.steps):
        sol.step(1)
        with torch.cuda.stream(sol.stream):
            evs[j + 1].record()
    sol.sync()
    u1 = sol.particle_updates()
    barrier()
    clocks = clk.stop()
    step_ms = [evs[j].elapsed_time(evs[j + 1]) for j in range(args.steps)]
    span_s = evs[0].elapsed_time(evs[-1]) / 1e3
    updates = u1 - u0
    if dist is not None:
        t = torch.tensor([span_s, float(updates)], dtype=torch.float64, device="cuda")
        tmax = t.clone()
        dist.all_reduce(tmax[0:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:2], op=dist.ReduceOp.SUM)
        span_all, updates_all = float(tmax[0]), float(t[1])
    else:
        span_all, updates_all = span_s, float(updates)
    value = updates_all / span_all

    # ------------------------------------------------ step latency: further steps, one event each, for
    # about latency_seconds (p50/p99 over many steps; the throughput above is the K timed steps alone)
    lat_ms = []
    t_lat = time.perf_counter()
    while time.perf_counter() - t_lat < args.latency_seconds and len(lat_ms) < 100_000:
        chunk = [torch.cuda.Event(enable_timing=True) for _ in range(51)]
        with torch.cuda.stream(sol.stream):
            chunk[0].record()
        for j in range(50):
            sol.step(1)
            with torch.cuda.stream(sol.stream):
                chunk[j + 1].record()
        sol.sync()
        lat_ms += [chunk[j].elapsed_time(chunk[j + 1]) for j in range(50)]
    lat_ms.sort()

    # ------------------------------------------------ the same number of steps kernel by kernel, events
    # around each kernel (no overlap): per-kernel times and the streaming kernel's roofline
    u2 = sol.particle_updates()
    kms, _ = sol.step_timed(args.steps)
    upd_timed = sol.particle_updates() - u2
    serial_ms = kms[5] / args.steps

    # ------------------------------------------------ the stress / heat-flux read-out (Eq. gkt_moment1; not
    # part of the step): one pass over every particle record of the batch, events around 3 passes
    n_part = int(sum(sol.num_particles(i) for i in range(sol.n)))
    sol.stress_heat_accumulate()                      # the first call allocates its scratch
    sol.sync()
    ro_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(sol.stream):
        ro_ev[0].record()
    for _ in range(3):
        sol.stress_heat_accumulate()
    with torch.cuda.stream(sol.stream):
        ro_ev[1].record()
    sol.sync()
    ro_ms = ro_ev[0].elapsed_time(ro_ev[1]) / 3

    out = None
    if rank == 0:
        steps_sorted = sorted(step_ms)
        p50 = steps_sorted[len(steps_sorted) // 2]
        p99 = steps_sorted[min(len(steps_sorted) - 1, int(math.ceil(0.99 * len(steps_sorted))) - 1)]
        upl = upd_timed / args.steps                   # particle-updates per launch of the streaming kernel
        k_ms = kms[1] / args.steps
        peak, peak_kind = measured_peaks()
        achieved = rec_bytes * 2 * upl / (k_ms * 1e-3) / 1e9
        traffic, per_upd = profiled_traffic(args.workload if (args.split, args.recon) == ("p", "first") else "", upl)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "k_stream",
                "algorithmic_bytes_per_update": rec_bytes * 2, "updates_per_launch": upl,
                "launch_ms": k_ms, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}
        slots = duwp.Solver.KERNEL_SLOTS
        ksum = max(sum(kms[i] for i in slots.values()), 1e-30)
        kernel_share = {n: float(kms[i] / ksum) for n, i in slots.items()}
        cfg = dict(cfg)
        info0 = sol.info(0)
        cfg.update({"particles": int(sum(sol.num_particles(i) for i in range(sol.n))),
                    "cells_total": int(sum(p["n_cells"] for p in plist)),
                    "capacity_per_buffer": int(info0["capacity"]),
                    "l2": "inputs larger than L2 (particle records exceed 129 MB)",
                    "graphs": "one graph per step (eight kernels); the block kernel runs beside the collision kernel, the wave flux beside the particle kernels",
                    "launch": tuned})
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * span_all / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64",
               "data": "synthetic (seeded shock/Sod problems shaped like the paper's test cases)",
               "config": cfg, "clocks": clocks, "gpu_launches": 8 * args.steps,
               "step_ms_p50": p50, "step_ms_p99": p99, "serial_ms_per_step": serial_ms,
               "step_latency": {"steps": len(lat_ms), "p50_ms": lat_ms[len(lat_ms) // 2] if lat_ms else None,
                                "p99_ms": lat_ms[min(len(lat_ms) - 1, int(math.ceil(0.99 * len(lat_ms))) - 1)]
                                if lat_ms else None,
                                "note": "steps after the timed region, one event each, for about "
                                        f"{args.latency_seconds} s"},
               "kernel_ms_per_step": {n: float(kms[i] / args.steps) for n, i in slots.items()},
               "kernel_times": "from the same number of steps run kernel by kernel with events around each",
               "kernel_share": kernel_share, "roofline": roof,
               "readout": {"kernel": "k_sh_split + k_sh_sums + k_sh_finish", "what": "normal stress and heat flux of every cell",
                           "ms": ro_ms, "particles": n_part, "bytes_per_particle": rec_bytes,
                           "achieved_gbs": n_part * rec_bytes / (ro_ms * 1e-3) / 1e9,
                           "frac": n_part * rec_bytes / (ro_ms * 1e-3) / 1e9 / peak}}
    sol.close()
    del sol
    torch.cuda.empty_cache()

    # ------------------------------------------------ plain FP64 loop: one instance at a time, no graphs
    if rank == 0 and not args.no_plain and world == 1:
        pl_updates, pl_ms = 0, 0.0
        kplain = max(3, min(args.steps, 10))
        for p in plist:
            q = dict(p)
            q["precision"] = "fp64"
            s = duwp.Solver(q, device=local, graphs=False)
            s.step(3)
            s.sync()
            a = s.particle_updates()
            k, _ = s.step_timed(kplain)
            pl_updates += s.particle_updates() - a
            pl_ms += k[5]
            s.close()
            del s
        torch.cuda.empty_cache()
        plain = pl_updates / (pl_ms / 1e3)
        out["plain_fp64_loop"] = {"value": plain, "unit": UNIT, "steps": kplain,
                                  "note": "same instances, FP64 records, one instance per launch sequence, no graphs"}
        out["speedup_vs_plain_fp64_loop"] = value / plain

    # ------------------------------------------------ end to end through the C ABI with host buffers
    import numpy as np
    if rank == 0:
        total_cells = sum(int(p["n_cells"]) for p in plist)
        pinned = [{k: torch.empty(total_cells, dtype=torch.float64, pin_memory=True).numpy()
                   for k in ("rho", "u", "T", "wave_frac")} for _ in range(2)]
        t0 = time.perf_counter()
        s = duwp.Solver(plist, device=local)           # host params -> device (init)
        t_init = time.perf_counter()
        u_start = 0
        d2h = 0
        t_first = None
        for j in range(args.steps):
            s.step(1)                                   # step j enqueued
            if j > 0:
                s.moments_wait()                        # step j-1's profiles are on the host (step j runs)
                if t_first is None:
                    t_first = time.perf_counter()
            m = s.moments_all_async(pinned[j % 2])      # every instance's profiles into pinned host arrays
            d2h += sum(a.nbytes for a in m.values())
        s.moments_wait()
        if t_first is None:
            t_first = time.perf_counter()
        u_e2e = s.particle_updates() - u_start
        e2e_s = time.perf_counter() - t0
        t_end = time.perf_counter()
        import ctypes
        h2d = ctypes.sizeof(duwp.Params) * len(plist)
        out["e2e"] = {"value": u_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
                      "d2h_bytes_per_step": d2h / args.steps,
                      "note": "duwp_init_batch from host parameters, then per step duwp_step + "
                              "duwp_moments_all_async (profiles of every instance into pinned host arrays, "
                              "copied while the next step runs; each step's profiles are waited for); includes "
                              "the set-up and the first (all-sampling) step",
                      "breakdown_s": {"setup": t_init - t0, "first_step": t_first - t_init,
                                      "later_steps": t_end - t_first, "steps": args.steps}}
        s.close()
        del s

    # ------------------------------------------------ CPU oracle on a bounded sample
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n = len(plist)
        if n > 1:
            idx = list(range(0, n, 8))
            ups, secs, rounds = oracle_sample(plist, idx)
            sample = (f"instances {idx} of the batch, 1 untimed + {rounds} timed steps each "
                      f"(about 10 s of oracle time)")
        else:
            ups, secs = None, None
            sample = "not run: a single instance too large for a bounded oracle sample"
        if ups is not None:
            out["cpu_baseline"] = {"value": ups / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "sample": sample, "seconds": secs}
            # second line: the same oracle on every host core, one process per instance
            aups, asecs, nproc = oracle_all_cores(plist)
            out["cpu_baseline_all_cores"] = {
                "value": aups / asecs, "unit": UNIT, "cores": nproc, "kind": "oracle",
                "sample": f"{nproc} instances of the batch, one single-threaded oracle process each, "
                          f"1 untimed + at least 2 timed steps and about 10 s each; value = all their "
                          f"particle-updates / the longest process's timed span",
                "seconds": asecs}
        else:
            out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
    # ------------------------------------------------ the other configurations, on this GPU, after the rest
    if rank == 0 and world == 1 and not args.no_configs and args.workload == "batch64" and args.split == "p" \
            and args.recon == "first" and not args.instances:
        peak, _ = measured_peaks()
        configs = {}
        for key, name, steps, warm in SECONDARY:
            try:
                configs[key] = secondary_run(name, steps, warm, local, peak)
            except Exception as e:          # a configuration that cannot run is reported, not hidden
                configs[key] = {"error": f"{type(e).__name__}: {e}"}
        try:
            configs["config5_serving_poisson50"] = serving_run(args.serve_seconds, local)
        except Exception as e:
            configs["config5_serving_poisson50"] = {"error": f"{type(e).__name__}: {e}"}
        out["configs"] = configs
    if out is not None:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
