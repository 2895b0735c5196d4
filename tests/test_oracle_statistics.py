"""The long-run statistical criterion on CPU, against the stored FP64 oracle ensemble (128 runs,
tests/golden/shock_mach3_average.txt): another FP64 ensemble and the oracle's FP32-record mode
(single-precision storage of the particle state at the points the GPU stores it) agree with it,
and the criterion rejects an ensemble whose viscosity is 5% too large.  64 runs per ensemble
(noise in the difference of the means ~0.55% of the temperature profile in L2)."""
import pytest

import stat_util as S


@pytest.fixture(scope="module")
def golden():
    return S.load_golden()


def test_stored_ensemble_reproduces(golden):
    v = S.verdict(S.oracle_ensemble("fp64", tuple(range(4000, 4064))), golden)
    assert S.agrees(v, with_l2=True), v


def test_fp32_records_agree_with_fp64_ensemble(golden):
    v = S.verdict(S.oracle_ensemble("fp32", tuple(range(5000, 5064))), golden)
    assert S.agrees(v, with_l2=True), v


def test_criterion_rejects_a_wrong_viscosity(golden):
    kn = S.problem("fp64", 1)["Kn"] * 1.05      # mean free path, hence mu_ref, 5% too large
    v = S.verdict(S.oracle_ensemble("fp64", tuple(range(6000, 6064)), Kn=kn), golden)
    assert not S.agrees(v, with_l2=True), v
