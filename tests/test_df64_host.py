"""The double-float power of the spring kernel (csrc/df64.cuh), compiled for the host
with the library's tables and checked against long-double powl over the range the
spring law meets: normalised stresses x = tau/(G0 gamma_ref) from 1e-8 to 200 and
exponents beta from 0.5 to 1.8 (h_max up to 0.3).  The device runs the same IEEE
single-precision operations (no contraction, explicit fma)."""
import os
import shutil
import subprocess

import pytest

from paper_2604_02755_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    lib = build.build()
    exe = str(tmp_path_factory.mktemp("df64") / "df64_check")
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", os.path.join(ROOT, "tests", "native", "df64_check.cpp"),
           "-o", exe, lib, "-Wl,-rpath," + os.path.dirname(lib)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("df64_check build failed:\n" + r.stderr)
    return exe


def run(exe, lx0, lx1, n):
    out = subprocess.run([exe, str(lx0), str(lx1), str(n)], capture_output=True, text=True, check=True).stdout
    worst, worst_w, declined = out.split()
    return float(worst), float(worst_w), int(declined)


def test_power_accuracy_over_the_spring_range(checker):
    worst, worst_w, declined = run(checker, -18.4, 5.3, 400000)
    assert declined == 0
    assert worst < 2e-13        # x^beta itself (~2^-42 at the extremes of ln x)
    assert worst_w < 1e-13      # as it enters the stress root and the tangent


def test_out_of_range_inputs_are_declined(checker):
    # x below 2^-100 is left to the FP64 path
    _, _, declined = run(checker, -75.0, -72.0, 1000)
    assert declined == 1000
