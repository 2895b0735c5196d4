"""Long-run statistics across precisions on the GPU: 128 seeds of the Mach-3 argon shock with FP32
particle records, run as one batch (500 steps, averages over the states after step 100), against
the stored FP64 oracle ensemble of 128 runs (tests/golden/shock_mach3_average.txt): relative L2
distance of the mean profiles at most 1%, and at most 3 of the 100 cells beyond 3 sigma of the
difference of the means, for density, velocity and temperature."""
import pytest

import stat_util as S
from parity_util import solver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_long_run_profiles_match_oracle_ensemble(precision):
    seeds = range(7000, 7128)
    plist = [S.problem(precision, s) for s in seeds]
    g = solver(plist)
    g.step(S.STEPS)
    runs = []
    for b in range(len(plist)):
        a, n = g.fields(inst=b, which=1)
        assert n == S.STEPS - S.AVG_START
        runs.append(S.profiles(a, n))
    g.close()
    v = S.verdict(S.summarize(runs), S.load_golden())
    assert S.agrees(v, with_l2=True), v
