"""The FP32-seeded FP64 square root and reciprocal of the mixed-precision
inversion (Newton's iteration applied once to an FP32 seed) against the C
library's correctly rounded results: relative error below 1e-14 over the
ranges the inversion feeds them (host build of the same header)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_refined_sqrt_and_reciprocal(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "refine_check"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-x", "c++", "-D__host__=", "-D__device__=",
                           "-I", os.path.join(ROOT, "paper_2408_01361_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "native", "refine_check.cpp"), "-o", str(exe)])
    es, er = (float(t) for t in subprocess.check_output([str(exe)]).split())
    assert es < 1e-14 and er < 1e-14, (es, er)
