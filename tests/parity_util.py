"""Helpers of the GPU parity tests: run the CUDA library and the oracle on the same problem dict
and compare element by element."""
import numpy as np


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def solver(params, **kw):
    from paper_2305_12071_gb300 import build as B
    from paper_2305_12071_gb300 import duwp
    B.build()
    return duwp.Solver(params, **kw)


def compare_particles(gp: dict, op: dict, rel: float, what: str = ""):
    """Identical cell assignment and order (the stable sort permutation) and state within rel,
    relative to max(|value|, 1): positions in units of the cell width, velocities in units of the
    reference thermal scale."""
    assert len(gp["cell"]) == len(op["cell"]), f"{what}: particle count {len(gp['cell'])} vs {len(op['cell'])}"
    assert np.array_equal(gp["cell"], op["cell"]), f"{what}: cell assignment differs"
    for k in ("xl", "u", "v", "w"):
        a, b = gp[k], op[k]
        scale = np.maximum(np.abs(b), 1.0)
        err = np.abs(a - b) / scale
        bad = np.argmax(err) if len(err) else 0
        assert len(err) == 0 or err.max() <= rel, f"{what}: {k} max rel err {err.max():.3e} at {bad}: {a[bad]!r} vs {b[bad]!r}"


def compare_fields(gpsi: np.ndarray, opsi: np.ndarray, rel: float, what: str = ""):
    """|gpu - oracle| <= rel * (largest magnitude of that component over the cells)."""
    for k in range(5):
        scale = max(np.abs(opsi[:, k]).max(), 1e-300)
        err = np.abs(gpsi[:, k] - opsi[:, k]).max() / scale
        assert err <= rel, f"{what}: Psi component {k} rel err {err:.3e}"


def compare_counters(gc: dict, oc: dict, what: str = ""):
    for k in ("ncand", "nacc", "nabs", "nnew"):
        assert np.array_equal(gc[k], oc[k]), f"{what}: counter {k} differs at cells {np.nonzero(gc[k] != oc[k])[0][:10]}"
