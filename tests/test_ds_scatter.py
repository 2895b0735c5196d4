"""The double-single arithmetic of single-precision records (host builds of the device header):
whenever the scattering (Appendix A) or the Maxwellian sampling (Eq. maxsample) reports success,
the stored floats are exactly the single-precision rounding of the double-precision evaluation of
the same formula, and the double-precision fallback stays rare."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2305_12071_gb300", "csrc")


def _nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p if os.path.exists(p) else None


def test_ds_scatter_matches_double_precision(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "ds_scatter_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-Xcompiler", "-ffp-contract=off", "-I", CSRC,
                    os.path.join(HERE, "ds_scatter_check.cu"), "-o", exe], check=True, capture_output=True)
    r = subprocess.run([exe, "400000"], capture_output=True, text=True)
    n, nfail, nfail_generic, nbad = map(int, r.stdout.split()[-4:])
    assert r.returncode == 0 and nbad == 0, r.stdout
    assert nfail_generic < 0.002 * n, r.stdout
    assert nfail >= n // 17 - 1, r.stdout       # the near-pole cases always take the fallback
    # the error bounds the rounding window rests on: double-single error below 2^-45.5 (c_r + |m|),
    # double-precision deviation within its stated bound
    line = [x for x in r.stdout.splitlines() if x.startswith("ds-error")][0]
    ds_exp = float(line.split("max 2^")[1].split(";")[0])
    fp_ratio = float(line.split("bound max ")[1])
    assert ds_exp < -45.5 and fp_ratio < 1.0, line


def test_ds_maxwell_matches_double_precision(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "ds_maxwell_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-Xcompiler", "-ffp-contract=off", "-I", CSRC,
                    os.path.join(HERE, "ds_maxwell_check.cu"), "-o", exe], check=True, capture_output=True)
    r = subprocess.run([exe, "300000"], capture_output=True, text=True)
    n, nfail, nbad, log_rel = r.stdout.split()[-4:]
    assert r.returncode == 0 and int(nbad) == 0, r.stdout
    assert int(nfail) < 0.001 * int(n), r.stdout
    line = [x for x in r.stdout.splitlines() if x.startswith("ds-error")][0]
    ds_exp = float(line.split("max 2^")[1].split(";")[0])
    fp_exp = float(line.split("max 2^")[2])
    assert ds_exp < -44.0 and fp_exp < -48.0, line
    assert float(log_rel) < 2.0 ** -44, r.stdout      # -log(1 - u) against long double


def test_fixed_to_double_is_the_rounded_conversion(tmp_path):
    # the exact fixed-point particle sums reach the cell update through fixed_to_double: it must be
    # bit for bit the double-precision conversion (round to nearest even) times the power of two
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "fixed_to_double_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, os.path.join(HERE, "fixed_to_double_check.cu"), "-o", exe],
                   check=True, capture_output=True)
    r = subprocess.run([exe, "2000000"], capture_output=True, text=True)
    tot, bad = map(int, r.stdout.split()[-2:])
    assert r.returncode == 0 and bad == 0 and tot > 2000000, r.stdout

