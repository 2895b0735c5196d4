"""Autotuner of the streaming kernel's launch shape.

Three knobs of the streaming kernel: threads per block (one warp per cell), the register budget
(up to 128, 64 or 40 registers per thread) -- together they fix the warps resident per SM -- and
the particles each lane has in flight (2 or 3 groups of 32 records per warp).  The tuner times a
few steps of the caller's own workload for every candidate with CUDA events (duwp_step_timed:
collision + streaming kernels) and keeps the fastest.  Results do not depend on the launch shape (the per-cell
moment sums are exact fixed-point integers and the partition order is defined by the method), so
tuning changes speed only.  Choices are cached in a JSON file keyed by device, precision and
workload size buckets.
"""
from __future__ import annotations

import json
import math
import os

_VERSION = 3          # layout of the launch knobs (entries of other versions are re-tuned)
_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune_cache.json")

CANDIDATES_FP32 = [(t, r, g) for g in (2, 3) for r in (0, 1, 2) for t in (64, 128, 256, 512)]
CANDIDATES_FP64 = CANDIDATES_FP32


def _key(solver) -> str:
    import torch
    name = torch.cuda.get_device_name()
    prec = solver.params[0].get("precision", "fp64")
    cells = sum(int(p["n_cells"]) for p in solver.params)
    parts = sum(solver.num_particles(i) for i in range(solver.n))
    ppc = parts / max(cells, 1)
    return f"{name}|{prec}|cells2^{int(math.log2(max(cells, 1)))}|ppc2^{int(math.log2(max(ppc, 1)))}"


def _load():
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d):
    os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
    tmp = _CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1)
    os.replace(tmp, _CACHE)


def tune(solver, steps: int = 3, use_cache: bool = True, candidates=None):
    """Pick and apply the fastest (threads, reg_capped) for this solver's workload.  The solver
    advances by len(candidates) * steps steps.  Returns (choice, timings)."""
    key = _key(solver)
    cache = _load() if use_cache else {}
    if use_cache and key in cache and cache[key].get("version") == _VERSION:
        t, r, g = cache[key]["threads"], cache[key].get("reg_capped", 0), cache[key].get("groups", 2)
        solver.set_launch(t, r, g)
        return (t, r, g), cache[key].get("timings", {})
    fp32 = solver.params[0].get("precision", "fp64") == "fp32"
    cands = candidates or (CANDIDATES_FP32 if fp32 else CANDIDATES_FP64)
    timings = {}
    best = None
    for t, r, g in cands:
        try:
            solver.set_launch(t, r, g)
        except Exception:
            continue
        solver.step_timed(1)                     # first launch of a shape: not timed
        k, _ = solver.step_timed(steps)
        ms = float(k[0] + k[1]) / steps
        timings[f"{t}r{r}g{g}"] = ms
        if best is None or ms < best[0]:
            best = (ms, t, r, g)
    if best is None:
        raise RuntimeError("no launch shape could be configured")
    solver.set_launch(best[1], best[2], best[3])
    cache[key] = {"threads": best[1], "reg_capped": best[2], "groups": best[3], "ms": best[0], "timings": timings,
                  "version": _VERSION}
    _save(cache)
    return (best[1], best[2], best[3]), timings
