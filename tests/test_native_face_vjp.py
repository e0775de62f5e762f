"""The adjoint's hand-written reverse sweep of one face side (fluid state,
fluxes, conserved vector, active signal speed) against the dual-number
evaluation of the same gradient, on seeded magnetised states in the Kerr
funky-MKS metric (from the oracle) and in Minkowski: agreement to round-off
(host build of the same header)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reverse_face_gradient_matches_dual_numbers(orc, tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    libdir = os.path.join(ROOT, "oracle")
    exe = tmp_path / "face_vjp_check"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-x", "c++", "-D__host__=", "-D__device__=",
                           "-I", os.path.join(ROOT, "paper_2408_01361_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "native", "face_vjp_check.cpp"), "-o", str(exe),
                           "-L", libdir, "-loracle", "-Wl,-rpath," + libdir])
    worst = float(subprocess.check_output([str(exe)]).split()[0])
    assert worst < 1e-11, worst
