"""The double-float arithmetic of the spring kernel (csrc/df64.cuh), compiled for the
host with the library's tables: the power x^beta against long-double powl, and one
Halley step of the skeleton root from an FP32 seed (with the tangent at the new root)
against the root and tangent solved in long double -- over the range the spring law
meets: normalised stresses tau/(G0 gamma_ref) from 1e-8 to 200, exponents beta from 0.5
to 1.8 (h_max up to 0.3).  The device runs the same IEEE single-precision operations
(no contraction, explicit fma)."""
import os
import shutil
import subprocess

import pytest

from paper_2604_02755_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def compile_check(tmp_path_factory, name):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    lib = build.build()
    exe = str(tmp_path_factory.mktemp("df64") / name)
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", os.path.join(ROOT, "tests", "native", name + ".cpp"),
           "-o", exe, lib, "-Wl,-rpath," + os.path.dirname(lib)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(name + " build failed:\n" + r.stderr)
    return exe


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    return compile_check(tmp_path_factory, "df64_check")


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


def test_halley_step_root_and_tangent(tmp_path_factory):
    exe = compile_check(tmp_path_factory, "ro_check")
    out = subprocess.run([exe, "100000"], capture_output=True, text=True, check=True).stdout
    err_tau, err_G, max_step, declined = out.split()
    assert int(declined) == 0
    assert float(max_step) <= 2e-5        # within the step bound the kernel accepts
    assert float(err_tau) < 1e-13         # root of the skeleton equation
    assert float(err_G) < 1e-13           # tangent 1/g'(tau) at it


@pytest.mark.parametrize("S", [10, 17, 50, 150, 256])
def test_tensor_core_tangent_assembly_digits(tmp_path_factory, S):
    """The tensor-core assembly of D = sum_k G_k T_k (csrc/k_spring.cu) emulated on the
    host with the library's digit tables and the kernel's digit cut: the fragment table
    holds every (spring, column) once and zeros in the padding, every digit is exact in
    bf16, the digits of T reproduce T to 2^-49 of its column scale and those of G
    reproduce G to 2^-49 of 2^eG, every per-pair sum stays far below 2^24 (so FP32 holds it
    exactly), and the recombined D agrees with long double to 5e-14 of sum_k |G_k T_k| for
    tangents spread over four decades below G0 (5e-13 below 50 springs)."""
    exe = compile_check(tmp_path_factory, "tc_check")
    out = subprocess.run([exe, str(S), "200"], capture_output=True, text=True, check=True).stdout
    worst, cmax, mism, worst_t, worst_g, amax = out.split()
    assert int(mism) == 0
    assert float(worst_t) <= 2.0 ** -49
    assert float(worst_g) <= 2.0 ** -49
    assert int(amax) <= 128
    assert float(cmax) < 0.25
    assert float(worst) <= (5e-14 if S >= 50 else 5e-13)
