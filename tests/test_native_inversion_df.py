"""The mixed update's double-float inversion (noble2d_df: double-float
invariants, FP32 Newton, one double-float refinement) against the FP64
inversion (noble2d) on 2e5 seeded magnetised states in Minkowski and in the
funky-MKS Kerr metric (points from the oracle), sigma up to 50, |u~| from
3e-5 to 3, guesses 1e-3 off: no state fails, fewer than 0.1% are handed
back to FP64, and its error against the state is the FP64 inversion's (the
problems' conditioning sets both; host build of the same header). The
floors' FP32 inputs (b^2, the Lorentz factor, u_mu) formed from the metric's
leading parts agree with the FP64 fluid state to FP32 accuracy."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_double_float_inversion_matches_fp64(orc, tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    libdir = os.path.join(ROOT, "oracle")
    exe = tmp_path / "inversion_df_check"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-x", "c++", "-D__host__=", "-D__device__=", "-D__forceinline__=",
                           "-I", os.path.join(ROOT, "paper_2408_01361_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "native", "inversion_df_check.cpp"), "-o", str(exe),
                           "-L", libdir, "-loracle", "-Wl,-rpath," + libdir])
    out = subprocess.check_output([str(exe)]).split()
    worst_df, worst_64, worst_d = (float(t) for t in out[:3])
    need, fails, n = (int(t) for t in out[3:6])
    worst_fl = float(out[6])
    assert fails == 0 and n > 150000
    assert need < 1e-3 * n, need
    assert worst_df <= 1.5 * worst_64 + 1e-12, (worst_df, worst_64)
    assert worst_d < 1e-8, worst_d
    # the floors' FP32 b^2, gamma^2 and u_mu from the double-float metric's
    # leading parts: FP32 accuracy
    assert worst_fl < 2e-6, worst_fl
