"""Placement of whole DUWP instances on GPUs (ranks) by their device-memory footprint.

Instances never exchange data, so a batch or a serving pool spreads over several GPUs as
independent replicas: each GPU takes a set of whole instances.  The footprint of an instance is
dominated by its particle records (two buffers, each cell's output block twice its slot bound) and
grows with its expected particle count, the initial mass over the particle mass:
  N ~ (ppc_ref / rho_ref) * sum over cells of rho(cell centre),
so instances are placed greedily, largest first, each on the GPU with the least footprint so far
(longest-processing-time list scheduling: the loads differ by at most one instance's footprint).
"""
from __future__ import annotations


def expected_particles(p: dict) -> float:
    """Expected simulated particles of a problem dict: its initial mass over the particle mass."""
    n = int(p["n_cells"])
    dx = (p["x_max"] - p["x_min"]) / n
    mass = 0.0
    for i in range(n):
        xc = p["x_min"] + (i + 0.5) * dx
        mass += (p["left"][0] if xc < p.get("x_split", 0.5 * (p["x_min"] + p["x_max"])) else p["right"][0])
    return mass * float(p["ppc_ref"]) / float(p.get("rho_ref", 1.0))


def footprint_bytes(p: dict) -> float:
    """Device bytes of one instance: two particle buffers of four times the expected particles
    (16-byte FP32 or 32-byte FP64 records) plus about 512 bytes of per-cell arrays."""
    rec = 16 if p.get("precision", "fp64") == "fp32" else 32
    return 2.0 * 4.0 * expected_particles(p) * rec + 512.0 * (int(p["n_cells"]) + 2)


def assign(params: list, world: int) -> list:
    """Indices of the instances each of `world` ranks takes (each index exactly once; every rank's
    list in increasing order).  Greedy by footprint, largest first; ties go to the lower rank."""
    if world < 1:
        raise ValueError("world must be at least 1")
    order = sorted(range(len(params)), key=lambda i: (-footprint_bytes(params[i]), i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda j: (load[j], j))
        out[r].append(i)
        load[r] += footprint_bytes(params[i])
    return [sorted(x) for x in out]
