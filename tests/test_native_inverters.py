"""The update's three FP64 primitive-recovery solvers (host build of the
same header): Noble et al.'s two-unknown Newton iteration, their one-unknown
1D_W scheme and Kastaun, Kalinani & Ciolfi's bracketed scheme. On 6e4
seeded magnetised states (Minkowski and funky-MKS Kerr, sigma to 50, |u~|
to 3, guesses 1e-3 off) every solver recovers every state, to the same
error (the problems' conditioning sets it). On a stress set (sigma to 1e4,
|u~| to 50, an unrelated state as the guess) the bracketed scheme and 1D_W
recover every state, with the error of the states' conditioning; the
two-unknown Newton iteration loses some (they go to the fixup)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_inverters_recover_states(orc, tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    libdir = os.path.join(ROOT, "oracle")
    exe = tmp_path / "inverters_check"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-x", "c++", "-D__host__=", "-D__device__=", "-D__forceinline__=",
                           "-I", os.path.join(ROOT, "paper_2408_01361_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "native", "inverters_check.cpp"), "-o", str(exe),
                           "-L", libdir, "-loracle", "-Wl,-rpath," + libdir])
    out = subprocess.check_output([str(exe)]).split()
    res = {}
    for q, name in enumerate(("noble2d", "1dw", "kastaun")):
        w, fa, fb, wb = out[4 * q: 4 * q + 4]
        res[name] = (float(w), int(fa), int(fb), float(wb))
    nA, nB = int(out[12]), int(out[13])
    assert nA > 50000 and nB == 60000
    base = res["noble2d"][0]
    for name, (w, fa, fb, wb) in res.items():
        assert fa == 0, (name, res)
        assert w <= 1.5 * base + 1e-12 and w < 1e-8, (name, res)
        assert wb < 1e-6, (name, res)
    assert res["kastaun"][2] == 0 and res["1dw"][2] == 0, res
    assert res["noble2d"][2] < 0.2 * nB, res
