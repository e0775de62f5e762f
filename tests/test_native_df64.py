"""The double-float arithmetic of the mixed-precision update (kh_df64.cuh,
host build of the same header) against long double: two-sum and the
FMA product are exact; FP64 -> double-float loses at most 2^-48 (relative),
double-float -> FP64 and FP32 -> FP64 (subnormals included) are exact; the
pair operations stay within small multiples of 2^-48 (addition relative to
|a| + |b|, the others relative to the result)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_double_float_arithmetic(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "df64_check"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-x", "c++", "-D__host__=", "-D__device__=",
                           "-I", os.path.join(ROOT, "paper_2408_01361_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "native", "df64_check.cpp"), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).split()
    e = [float(t) for t in out[:11]]
    bad_norm, bad_f32 = int(out[11]), int(out[12])
    e_sum, e_prod, e_conv, e_back, e_add, e_addf, e_mul, e_mulf, e_div, e_rcp, e_sqrt = e
    assert e_sum == 0.0 and e_prod == 0.0 and e_back == 0.0 and bad_f32 == 0 and bad_norm == 0
    assert e_conv <= 1.01
    assert e_add <= 4 and e_addf <= 2 and e_mul <= 6 and e_mulf <= 3
    assert e_div <= 16 and e_rcp <= 8 and e_sqrt <= 6, e
