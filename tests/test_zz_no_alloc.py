"""duwp_get_particles_noalloc: the allocation-free particle inspection for callers that cannot
allocate device memory at that point (inside stream capture, or with a fixed arena handed over at
set-up).  Through the C ABI it must give exactly what duwp_get_particles gives, on two calls in a
row (the second call reuses the library's static start table left by the first)."""
import numpy as np
import pytest

from paper_2305_12071_gb300 import workloads as W
from parity_util import solver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_particles_equal_get_particles(precision):
    import torch
    p = W.sod(n_cells=150, Kn=3e-4, ppc_ref=80, precision=precision, seed=21)
    s = solver(p)
    s.step(4)
    for call in range(2):
        ref = s.particles()                      # the existing entry point, host arrays
        n = len(ref["cell"])
        assert n > 0
        torch.cuda.synchronize()
        out = {"cell": torch.empty(n, dtype=torch.int32, device="cuda")}
        for k in ("xl", "u", "v", "w"):
            out[k] = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        s.particles_noalloc(out)
        s.sync()
        for k in ref:
            got = out[k].cpu().numpy()
            assert np.array_equal(got, ref[k]), f"call {call}: {k} differs"
        if call == 0:
            s.step(3)                            # different counts for the second call
    s.close()


def test_noalloc_rejects_wrong_size():
    import torch
    from paper_2305_12071_gb300 import duwp
    s = solver(W.config1("fp32"))
    s.step(2)
    n = s.num_particles()
    out = {"cell": torch.empty(n + 5, dtype=torch.int32, device="cuda")}
    for k in ("xl", "u", "v", "w"):
        out[k] = torch.empty(n + 5, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    s.particles_noalloc(out)
    with pytest.raises(duwp.DuwpError):
        s.sync()
    s.close()
